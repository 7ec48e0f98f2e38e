"""tsu_grid_step_noalloc: stepping a grid that lives in the caller's device
memory without the library allocating anything.

Callers whose GPU memory is managed entirely by their own allocator, or who
cannot risk a cudaMalloc inside a latency-critical loop, use this entry point
instead of a context.  Here the test itself owns the device buffer (a torch
tensor); the library only launches kernels into it, with its scratch in a
static device array.  Two calls in a row must reproduce two steps of the
context-based path (tsu_step) on the same grid with the same time step.
"""
import numpy as np
import pytest

from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _context_run(w, prec, dt, steps):
    from paper_1901_06798_gb300 import binding
    cfg = dict(w["cfg"], dt_max=dt)
    ctx = W.load(binding.Tsunami(cfg, precision=prec), dict(w, cfg=cfg, gauges=np.zeros((0, 2))))
    (box, a0), = ctx.patches(0, 1)
    ctx.step(steps)
    (box, a2), = ctx.patches(0, 1)
    assert ctx.stats()["dt"] == dt
    ctx.close()
    return a0, a2


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_two_steps_match_context_path(prec):
    import torch
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=200, dx=2000.0)
    nx, ny = w["cfg"]["nx"], w["cfg"]["ny"]
    dt = 1.5
    a0, a2 = _context_run(w, prec, dt, 2)

    pitch = nx + 7                       # any pitch >= nx + 4
    fs = pitch * (ny + 4) + 5            # any field stride >= pitch * (ny + 4)
    dtype = np.float64 if prec == 0 else np.float32
    host = np.zeros(7 * fs, dtype=dtype)

    def field(k):
        return host[k * fs:k * fs + pitch * (ny + 4)].reshape(ny + 4, pitch)[2:ny + 2, 2:nx + 2]
    q0 = a0["h"] if prec == 0 else (a0["h"] + a0["B"])
    field(0)[:] = q0
    field(1)[:] = a0["hu"]
    field(2)[:] = a0["hv"]
    field(6)[:] = a0["B"]
    dev = torch.from_numpy(host).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    c = w["cfg"]
    for cur in (0, 1):
        rc, speeds = binding.tsu_grid_step_noalloc(prec, dev.data_ptr(), nx, ny, pitch, fs, cur, c["dx"], c["dy"],
                                                   dt, c["g"], c["drytol"], c["bc"], stream)
        assert rc == binding.TSU_OK
        assert 150.0 < max(speeds) < 250.0     # deep-water gravity-wave speed, sqrt(g * 4000 m) ~ 198 m/s
    out = dev.cpu().numpy()
    host[:] = out
    B = field(6).astype(np.float64)
    h = field(0).astype(np.float64) - (B if prec == 1 else 0.0)
    hu, hv = field(1).astype(np.float64), field(2).astype(np.float64)
    if prec == 0:
        for mine, ref in ((h, a2["h"]), (hu, a2["hu"]), (hv, a2["hv"])):
            assert np.abs(mine - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        assert np.abs((h + B) - (a2["h"] + a2["B"])).max() <= 1e-4
        assert np.abs(hu - a2["hu"]).max() <= 1e-4 * max(1.0, np.abs(a2["hu"]).max())
        # the context runs the split FP32 update (x and y kernels through a Q*
        # scratch), this entry point the fused kernel: the same operations, the same bits
        for mine, ref in ((h, a2["h"]), (hu, a2["hu"]), (hv, a2["hv"])):
            assert np.array_equal(mine, ref)


def test_noalloc_rejects_oversize_and_bad_layout():
    import torch
    from paper_1901_06798_gb300 import binding
    dev = torch.zeros(1024, dtype=torch.float64, device="cuda")
    big = 16384 + 1
    rc, _ = binding.tsu_grid_step_noalloc(0, dev.data_ptr(), big, 8, big + 4, (big + 4) * 12, 0, 1.0, 1.0, 0.1,
                                          9.81, 1e-3, [0, 0, 0, 0])
    assert rc == binding.TSU_ERR_ARG
    rc, _ = binding.tsu_grid_step_noalloc(0, dev.data_ptr(), 8, 8, 10, 200, 0, 1.0, 1.0, 0.1, 9.81, 1e-3,
                                          [0, 0, 0, 0])
    assert rc == binding.TSU_ERR_ARG
