"""The device side of the halo exchange of a level split over ranks, on one
GPU through the C ABI: tsu_halo_pack copies the boxes of a halo schedule out
of the sources' interiors into one device buffer, tsu_halo_unpack writes them
into the destinations' ghost rings.  The schedule's definition
(ranks.halo_schedule, ranks.exchange_halos: each message is the source
patch's interior block that lies in the destination's ghost ring) is checked
element by element: the packed buffer equals those interior blocks as read
back from the patches, and after unpacking, packing the destination ghost
boxes gives the same buffer bit for bit.  Both precisions (FP32: q0 is the
surface eta').  Malformed messages are rejected before any launch.
"""
import numpy as np
import pytest

from paper_1901_06798_gb300 import ranks
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_pack_unpack_move_the_schedule_boxes(prec):
    torch = pytest.importorskip("torch")
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=96, dx=2000.0)
    cfg = dict(w["cfg"], level1_tile=20)                 # 5 x 5 tiles, the last row and column 16 wide
    g = W.load(binding.Tsunami(cfg, precision=prec), dict(w, cfg=cfg))
    g.step(5)
    boxes = [tuple(int(v) for v in b) for b in g.boxes(0, 1)]
    owner = ranks.partition_patches(boxes, 2)
    sched = ranks.halo_schedule(boxes, owner, 96, 96)
    assert len(sched) > 0
    send = np.array([(q, *box) for (_, _, q, _, box) in sched], dtype=np.int32)
    recv = np.array([(p, *box) for (_, _, _, p, box) in sched], dtype=np.int32)
    n = 3 * sum((b[2] - b[0]) * (b[3] - b[1]) for *_, b in sched)
    dt = torch.float64 if prec == 0 else torch.float32
    buf = torch.full((n,), float("nan"), dtype=dt, device="cuda")
    g.halo_pack(0, 1, send, buf.data_ptr(), n)
    # expected: the sources' interior blocks (q0 = h, or eta' = h + B in FP32)
    pats = [a for _, a in g.patches(0, 1)]
    exp, off = np.empty(n), 0
    for (_, _, q, _, (i0, j0, i1, j1)) in sched:
        qi, qj = boxes[q][0], boxes[q][1]
        blk = (slice(j0 - qj, j1 - qj), slice(i0 - qi, i1 - qi))
        a = pats[q]
        q0 = a["h"] if prec == 0 else a["h"] + a["B"]
        for f in (q0, a["hu"], a["hv"]):
            m = (i1 - i0) * (j1 - j0)
            exp[off:off + m] = f[blk].ravel()
            off += m
    got = buf.double().cpu().numpy()
    if prec == 0:
        assert np.array_equal(got, exp)
    else:
        # h comes back as eta' - B in double; h + B recovers eta' only to the
        # rounding of |B| (eta' of 1e-6 m under 4000 m of water needs 56 bits)
        tol = np.empty(n)
        off = 0
        for (_, _, q, _, (i0, j0, i1, j1)) in sched:
            qi, qj = boxes[q][0], boxes[q][1]
            Bb = np.abs(pats[q]["B"][j0 - qj:j1 - qj, i0 - qi:i1 - qi]).ravel()
            m = Bb.size
            tol[off:off + m] = 2.0 ** -52 * np.maximum(Bb, 1.0) * 2
            tol[off + m:off + 3 * m] = 0.0                      # momenta are exact
            off += 3 * m
        assert np.all(np.abs(got - exp) <= tol)
    # into the destinations' ghost rings, and back out of them
    g.halo_unpack(0, 1, recv, buf.data_ptr(), n)
    back = torch.full((n,), float("nan"), dtype=dt, device="cuda")
    g.halo_pack(0, 1, recv, back.data_ptr(), n)
    assert torch.equal(buf, back)
    # malformed messages: a box outside the patch's storage, no such patch, a short buffer
    bad = [np.array([[0, -5, 0, 3, 3]]), np.array([[len(boxes), 0, 0, 1, 1]])]
    for m in bad:
        with pytest.raises(binding.TsuError) as e:
            g.halo_pack(0, 1, m, buf.data_ptr(), n)
        assert e.value.code == binding.TSU_ERR_ARG
    with pytest.raises(binding.TsuError) as e:
        g.halo_pack(0, 1, send, buf.data_ptr(), n - 1)
    assert e.value.code == binding.TSU_ERR_ARG
