#!/usr/bin/env python3
"""Benchmark: cell updates per second of the shallow-water wave-propagation
update on one GB300, FP32 surface-perturbation form (headline) and FP64.

Workload (the 4096^2 uniform run): 4096 x 4096 cells, dx = 500 m, synthetic
shelf bathymetry (4000 m abyssal plain, slope to a 200 m shelf, beach rising
to +50 m dry land along one edge), 2 m elliptical Gaussian seafloor uplift at
t = 0, extrapolating boundaries.  The state (537 MB in FP32, 1.07 GB in FP64
per buffer pair) is larger than the 129 MB L2, so no flush is needed between
steps.

One JSON line on rank 0.  Under torchrun every rank runs an independent
replica (the uniform grid is not sharded: replicas only) and `value` is the
cell updates of all ranks over the slowest rank's time.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell updates/sec (all AMR levels) FP32-pert vs FP64 on 1 GB300; % HBM roofline"
UNIT = "cell updates/s"
BYTES_PER_CELL = {"f32p": 28, "f64": 56}   # read q0,q1,q2,B + write q0,q1,q2 per interior cell update
# algorithmic floating-point operations (add/sub, mul, div, sqrt) per interior cell update of the
# split step with every edge active, counted on the oracle compiled with a counting scalar type
# (tests/test_oracle_flops.py, the all-wet 200^2 hump; comparisons and min/max not included)
FLOPS_PER_CELL = 365.5
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2.07 GHz;
# FP64: GB300's nominal dense FP64 rate
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def measured_alu_peaks(torch):
    """FP64 and FP32 dense arithmetic rates of this GPU, measured with library
    GEMMs (torch.matmul of 4096^2 FP64 -- cuBLAS runs it on the FP64 tensor
    path -- and of 8192^2 FP32 with TF32 off, on the FMA pipes), best of 5
    timed with CUDA events after a warm-up.  They are the denominators of the
    update's compute roofs."""
    out = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    torch.cuda.empty_cache()
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("step_kernel.cuh", "step_f32x2.cuh", "step_split_f32.cuh", "step_f32p.cu", "step_f64.cu", "tsu_device.h"):
        h.update(open(os.path.join(ROOT, "paper_1901_06798_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(prec):
    """DRAM bytes of one patch update (the x- and y-sweep kernels of the FP32
    split update together) from the committed ncu summary, only if it was taken
    on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(prec)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class Busy:
    """Device- and host-busy fractions of a timed region (the paper's P1/P2
    style metrics): the mean of nvidia-smi's utilization.gpu -- the share of
    each sample period in which a kernel was running -- and this process's
    CPU time over wall time."""

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        self.t0, self.c0 = time.perf_counter(), os.times()
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=utilization.gpu",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        wall = time.perf_counter() - self.t0
        c1 = os.times()
        host = ((c1.user - self.c0.user) + (c1.system - self.c0.system)) / wall if wall > 0 else None
        gpu = None
        if self.p:
            self.p.terminate()
            out, _ = self.p.communicate(timeout=10)
            v = []
            for line in out.strip().splitlines():
                try:
                    v.append(float(line.strip()))
                except ValueError:
                    pass
            gpu = statistics.mean(v) / 100.0 if v else None
        return {"gpu_busy_frac": gpu, "host_busy_frac": host}


def amr_level3_traffic():
    """DRAM bytes per cell of one level-3 update (x + y launches over all the
    level's patches) on the 3-level AMR workload, from the committed ncu
    summary, only if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("f32p_amr3_level3")
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e["dram_bytes_per_launch"] / e["cells"]


def update_roofline(lt, prec, steps):
    """Per-level and summed cost of the batched patch update from
    tsu_level_update_times: device ms per coarse step, interior cell updates,
    algorithmic bytes (BYTES_PER_CELL per interior cell update) over the
    update's event-timed duration, and that bandwidth over the measured HBM
    copy peak.  The batched patch update of the finer levels (2 and up, all
    patches of a level in one launch) is summed separately: it is where the
    AMR workloads spend their update time."""
    peak, how = peaks()
    bpc = BYTES_PER_CELL[prec]
    per = {}
    for lev, v in lt.items():
        if v["steps"] == 0:
            continue
        gbs = bpc * v["cells"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else None
        per[str(lev)] = {"ms_per_coarse_step": v["ms"] / steps, "cell_updates_per_coarse_step": v["cells"] / steps,
                         "level_steps_per_coarse_step": v["steps"] / steps, "kernels": v["kernels"],
                         "achieved_gbs": gbs, "frac": gbs / peak if gbs else None,
                         "device_cell_rate": v["cells"] / (v["ms"] * 1e-3) if v["ms"] > 0 else None}
    fine = [v for lev, v in lt.items() if lev >= 2 and v["steps"] > 0]
    allv = [v for v in lt.values() if v["steps"] > 0]
    out = {"per_level": per, "steps": steps, "bytes_per_cell": bpc,
           "device_cell_rate_all_levels": sum(v["cells"] for v in allv) / (sum(v["ms"] for v in allv) * 1e-3)}
    if fine:
        ms, cells = sum(v["ms"] for v in fine), sum(v["cells"] for v in fine)
        ach = bpc * cells / (ms * 1e-3) / 1e9
        tpc = amr_level3_traffic() if prec == "f32p" else None
        top = max((lev for lev, v in lt.items() if v["steps"] > 0), default=None)
        cells_launch = lt[top]["cells"] / lt[top]["steps"] if top else 0.0
        out["roofline"] = {"bound": "hbm", "what": "patch update of levels >= 2 (batched, one launch per level step)",
                           "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                           "peak_source": how,
                           # DRAM bytes of one update of the finest level (x + y launches), from ncu
                           "traffic": tpc * cells_launch if tpc else None,
                           "bytes_per_launch": bpc * cells_launch,
                           "traffic_bytes_per_cell": tpc}
    return out


def load_workload(prec_name, stream, transverse=0):
    from paper_1901_06798_gb300 import binding
    from paper_1901_06798_gb300 import workloads as W
    w = W.shelf(n=4096, dx=500.0)
    w = dict(w, cfg=dict(w["cfg"], transverse=transverse))
    prec = binding.TSU_F32P if prec_name == "f32p" else binding.TSU_F64
    ctx = binding.Tsunami(w["cfg"], precision=prec, stream=stream)
    W.load(ctx, w)
    return ctx, w


def run_ours(args, rank, world, dist, torch):
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream().cuda_stream
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    results = {}
    clocks.start()
    sel = set(args.legs.split(","))
    legs = []
    if "uniform" in sel:
        legs += [("f32p", 0, args.steps), ("f64", 0, max(1, min(args.steps, args.fp64_steps)))]
    if args.transverse_steps > 0 and "unsplit" in sel:
        kt = max(1, min(args.steps, args.transverse_steps))
        legs += [("f32p", 1, kt), ("f64", 1, max(1, kt // 5))]
    for prec, tr, K in legs:
        ctx, w = load_workload(prec, stream, tr)
        cells = w["cfg"]["nx"] * w["cfg"]["ny"]
        if args.shape:                                     # fixed launch shape (profiling runs)
            thr, seg = (int(v) for v in args.shape.split(","))
            if thr < 64 and (prec == "f64" or tr):         # 32 threads exist only in the split FP32 kernel
                thr = 64
            ctx.set_tuning(thr, seg)
            tune = (thr, seg)
        else:
            tune = ctx.autotune(3)                          # launch shape (untimed set-up)
        ctx.step(args.warmup)
        l0 = ctx.stats()["kernel_launches"]
        barrier()
        torch.cuda.synchronize()
        kernel_ms, step_ms = ctx.time_level1_steps(0, K)   # CUDA events on this stream
        torch.cuda.synchronize()
        barrier()
        launches = ctx.stats()["kernel_launches"] - l0
        elapsed = max_over_ranks(step_ms * K / 1000.0)
        kern = max_over_ranks(kernel_ms)
        # the same K-step measurement repeated (spread of the headline)
        reps = []
        if prec == "f32p" and not tr and args.repeats > 0:
            for _ in range(args.repeats):
                km, sm = ctx.time_level1_steps(0, K)
                reps.append((km, world * cells / (max_over_ranks(sm) / 1000.0)))
        results[prec + ("_unsplit" if tr else "")] = dict(K=K, cells=cells, elapsed=elapsed, kernel_ms=kern, launches=launches,
                             value=world * cells * K / elapsed, tune={"threads": tune[0], "seg_rows": tune[1]},
                             repeats=reps)
        ctx.close()
        del ctx
        torch.cuda.synchronize()
    clk = clocks.stop()

    # the 3-level AMR workload and the 64-scenario ensemble: cell updates of all
    # levels (and scenarios) over wall time, regrids (host clustering) included
    extra = {}
    if args.amr_steps > 0:
        from paper_1901_06798_gb300 import binding as B
        from paper_1901_06798_gb300 import workloads as W2
        amr_legs = [(n, f) for n, f in (("amr3", lambda: W2.amr3()),
                                        ("ensemble64", lambda: W2.ensemble(n_scen=64, n=1024, dx=2000.0, ratio=4)))
                    if n in sel]
        from paper_1901_06798_gb300 import ranks as RK
        for name, wf in amr_legs:
            w = wf()
            # the ensemble's scenarios are independent: with several ranks each
            # advances its own block of them (no collective on the data path);
            # the single-scenario AMR workload runs as a replica per rank
            sharded = name.startswith("ensemble") and world > 1
            if sharded:
                w, _, _ = RK.shard_workload(w, rank, world)
            w = dict(w, gauges=w["gauges"])
            legs_x = {}
            gauges = {}
            for prec in ("f32p", "f64"):
                K = args.amr_steps if prec == "f32p" else max(1, args.amr_steps // 4)
                ctx = B.Tsunami(w["cfg"], precision=B.TSU_F32P if prec == "f32p" else B.TSU_F64, stream=stream)
                W2.load(ctx, w)
                ctx.step(args.warmup)
                if args.shape:                                  # fixed launch shape (profiling runs)
                    thr, seg = (int(v) for v in args.shape.split(","))
                    if thr < 64 and prec == "f64":
                        thr = 64
                    ctx.set_tuning(thr, seg)
                    tune = (thr, seg)
                else:
                    tune = ctx.autotune(2)
                nscen = w["cfg"]["n_scenarios"]
                s0 = [ctx.stats(s) for s in range(nscen)]
                barrier()
                torch.cuda.synchronize()
                busy = Busy(int(os.environ.get("LOCAL_RANK", 0)))
                busy.start()
                t0 = time.perf_counter()
                ctx.step(K)
                torch.cuda.synchronize()
                el = max_over_ranks(time.perf_counter() - t0)
                bz = busy.stop()
                s1 = [ctx.stats(s) for s in range(nscen)]
                cu = sum(b["cell_updates"] - a["cell_updates"] for a, b in zip(s0, s1))
                cu_job = sum_over_ranks(cu) if sharded else world * cu
                legs_x[prec] = {"value": cu_job / el, "steps": K, "ms_per_step": el / K * 1e3,
                                "parallelism": (f"scenarios sharded over {world} ranks" if sharded
                                                else (f"replicas x{world}" if world > 1 else "1 GPU")),
                                "cell_updates_per_step": cu / K, "patches_per_level": s1[0]["patches"],
                                "regrid_host_ms_per_step": (s1[0]["regrid_host_ms"] - s0[0]["regrid_host_ms"]) / K,
                                "regrid_wait_ms_per_step": (s1[0]["regrid_wait_ms"] - s0[0]["regrid_wait_ms"]) / K,
                                "cluster_ms_per_step": (s1[0]["cluster_ms"] - s0[0]["cluster_ms"]) / K,
                                "patches_renewed_per_step": (s1[0]["patches_renewed"] - s0[0]["patches_renewed"]) / K,
                                "patches_reused_per_step": (s1[0]["patches_reused"] - s0[0]["patches_reused"]) / K,
                                **bz,
                                "launch_shape": {"threads": tune[0], "seg_rows": tune[1]}}
                # the batched patch update alone: CUDA events around each level
                # step's update launches, over a separate profiled run of Kp
                # coarse steps (the wall-time run above is not instrumented)
                Kp = max(1, min(K, 8))
                ctx.profile_levels(True)
                ctx.step(Kp)
                lt = ctx.level_update_times()
                ctx.profile_levels(False)
                legs_x[prec]["update"] = update_roofline(lt, prec, Kp)
                gauges[prec] = ctx.read_gauges()
                ctx.close()
                torch.cuda.synchronize()
            n = min(len(gauges["f32p"][0]), len(gauges["f64"][0]))
            ea, eb = gauges["f32p"][1][:n], gauges["f64"][1][:n]
            legs_x["gauge_max_abs_f32p_vs_f64_m"] = float(np.abs(ea - eb).max()) if n else None
            legs_x["f32p_over_f64"] = legs_x["f32p"]["value"] / legs_x["f64"]["value"]
            extra[name] = legs_x

    # end to end through the C ABI with host buffers: inputs uploaded from host
    # arrays, every step returns the simulated time to the host, and the final
    # surface field comes back to the host (at least 100 steps, so that the
    # per-run costs -- create, upload, init, final read -- do not stand in for
    # the stepping)
    if "e2e" not in sel:
        return results, clk, None, extra
    from paper_1901_06798_gb300 import binding
    from paper_1901_06798_gb300 import workloads as W
    w = W.shelf(n=4096, dx=500.0)
    Ke = max(args.steps, 100)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = binding.Tsunami(w["cfg"], precision=binding.TSU_F32P, stream=stream)
    W.load(ctx, dict(w, gauges=np.zeros((0, 2))))
    for _ in range(Ke):
        ctx.step(1)
    n = 4096
    eta = ctx.read_field(0, 1, "eta", n, n, 250.0, 250.0, 500.0, 500.0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ctx.close()
    e2e_elapsed = max_over_ranks(t1 - t0)
    h2d = sum(g[0].nbytes for g in w["topo"]) + sum(u[1].nbytes for u in w["uplift"])
    e2e = {"value": world * n * n * Ke / e2e_elapsed, "unit": UNIT, "h2d_bytes_per_step": h2d / Ke,
           "d2h_bytes_per_step": 8 + eta.nbytes / Ke, "steps": Ke,
           "note": "create + upload inputs + init + K tsu_step calls each returning t + final eta read"}
    return results, clk, e2e, extra


def run_config4(args, stream, torch):
    """The 4-level bay workload with plain flagging and with the learned
    flag predictor.  The flags follow the wave (|eta| > 0.01 m; the depth
    criterion is off, so the refined area is not a static shelf band and the
    buffer the predictor trims is a real share of it); the bay box is forced
    to the finest level as in the workload.  The predictor is trained on the
    GPU on (features, flags one regrid later) pairs logged from the uniform
    shelf workload (the same bathymetry and uplift at 2 km, 128^2 windows
    around flagged cells, the same criterion)."""
    from paper_1901_06798_gb300 import binding as B
    from paper_1901_06798_gb300 import workloads as W
    t_start = time.perf_counter()
    w2 = W.shelf(n=1024, dx=2000.0)
    cfg2 = dict(w2["cfg"], flag_eta_tol=0.01, flag_depth_below=0.0, regrid_interval=4)
    g = W.load(B.Tsunami(cfg2, precision=B.TSU_F32P, stream=stream), dict(w2, cfg=cfg2, gauges=np.zeros((0, 2))))
    rng = np.random.Generator(np.random.PCG64(4))
    X, T, prev, win = [], [], None, 128
    for _ in range(args.config4_train_regrids):
        f, fl = g.cnn_features(0, 1)
        if prev is not None:
            js, is_ = np.nonzero(fl)
            for _ in range(6):
                k = rng.integers(len(js))
                j0 = int(np.clip(js[k] - win // 2, 0, fl.shape[0] - win))
                i0 = int(np.clip(is_[k] - win // 2, 0, fl.shape[1] - win))
                X.append(prev[:, j0:j0 + win, i0:i0 + win])
                T.append(fl[j0:j0 + win, i0:i0 + win].astype(np.float32))
        prev = f
        g.step(4)
    g.close()
    X, T = np.stack(X), np.stack(T)
    theta, l0, l1 = B.cnn_train(W.cnn_init_params(0), X, T, np.ones_like(T), steps=600, batch=8, lr=2e-3, seed=1)
    train = {"samples": int(len(X)), "window": win, "loss_first": l0, "loss_last": l1,
             "seconds": time.perf_counter() - t_start}
    w = W.amr4_bay(depth_below=0.0)
    runs = {}
    k64 = max(1, min(args.config4_steps, 40))
    for name, use, prec in (("plain", 0, B.TSU_F32P), ("cnn", 1, B.TSU_F32P), ("f64_plain", 0, B.TSU_F64)):
        cfg = dict(w["cfg"], use_cnn=use, cnn_buffer=1)
        ctx = B.Tsunami(cfg, precision=prec, stream=stream)
        if use:
            ctx.cnn_set_weights(theta)
        W.load(ctx, dict(w, cfg=cfg))
        ctx.set_tuning(64 if prec == B.TSU_F64 else 32, 32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        misses, checked, done = 0, 0, 0
        nsteps = k64 if prec == B.TSU_F64 else args.config4_steps
        while done < nsteps:
            n = min(8, nsteps - done)
            ctx.step(n)
            done += n
            _, fl = ctx.cnn_features(0, 1)             # level-1 criterion flags now
            cov = np.zeros_like(fl, dtype=bool)
            r = w["cfg"]["ratios"][0]
            for (i0, j0, nx, ny) in ctx.boxes(0, 2):
                cov[j0 // r:(j0 + ny) // r, i0 // r:(i0 + nx) // r] = True
            misses += int(((fl > 0) & ~cov).sum())
            checked += int((fl > 0).sum())
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        st = ctx.stats()
        runs[name] = {"steps": nsteps, "wall_s": el, "cell_updates": st["cell_updates"],
                      "rate": st["cell_updates"] / el, "patches_per_level": st["patches"],
                      "missed_flags": misses, "checked_flags": checked, "t_end_s": st["t"],
                      "gauges": ctx.read_gauges()}
        ctx.close()
    ea, eb = runs["plain"].pop("gauges")[1], runs["cnn"].pop("gauges")[1]
    e64 = runs["f64_plain"].pop("gauges")[1]
    n = min(len(ea), len(eb))
    n64 = min(len(eb), len(e64))
    return {"workload": "amr4_bay: 3000 km, dx 4 km -> 31.25 m (ratios 4, 4, 8), bay radius 5 km, 10 gauges; "
                        "flags |eta| > 0.01 m (no depth criterion), bay box forced to level 4",
            "train": train, "plain": runs["plain"], "cnn": runs["cnn"], "f64_plain": runs["f64_plain"],
            "rate_ratio_f32p_cnn_over_f64_plain": runs["cnn"]["rate"] / runs["f64_plain"]["rate"],
            "gauge_max_abs_f32p_cnn_vs_f64_plain_m": float(np.abs(eb[:n64] - e64[:n64]).max()) if n64 else None,
            "cell_update_ratio_cnn_over_plain": runs["cnn"]["cell_updates"] / runs["plain"]["cell_updates"],
            "wall_ratio_cnn_over_plain": runs["cnn"]["wall_s"] / runs["plain"]["wall_s"],
            "gauge_max_abs_cnn_vs_plain_m": float(np.abs(ea[:n] - eb[:n]).max()) if n else None}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_rate(args):
    """Cell updates/s of the FP64 oracle (timing build) on the full 4096^2
    shelf workload, `steps` steps, in this process (OMP_NUM_THREADS set by
    the caller before the library loads)."""
    steps, = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1901_06798_gb300 import workloads as W
    w = W.shelf(n=4096, dx=500.0)
    o = W.load(oracle.Oracle(w["cfg"], variant="fast"), dict(w, gauges=np.zeros((0, 2))))
    t0 = time.perf_counter()
    o.step(steps)
    return 4096 * 4096 * steps / (time.perf_counter() - t0)


def _oracle_rate_with_threads(threads, steps):
    """_oracle_rate in a fresh spawned process with `threads` OpenMP threads."""
    import multiprocessing as mp
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = str(threads)
    try:
        with mp.get_context("spawn").Pool(1) as pool:
            return pool.map(_oracle_rate, [(steps,)])[0]
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old


def cpu_baseline():
    """The FP64 oracle as it stands, timed on the host on the full 4096^2
    workload: with OpenMP over the rows and columns of the sweeps on all host
    cores (the reported value), and on one core."""
    import oracle
    oracle.build("fast")
    cores = os.cpu_count() or 1
    v_all = _oracle_rate_with_threads(cores, 8)
    v_one = _oracle_rate_with_threads(1, 2)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "single_core_value": v_one,
            "sample": f"full 4096x4096 shelf workload: 8 steps on {cores} OpenMP threads (rows of the x sweep, "
                      "columns of the y sweep), and 2 steps on 1 thread; FP64 oracle built -O3 -ffp-contract=off"}


def _ref_worker(a):
    """One host core: the oracle on a 512 x 512 window of the 4096^2 workload."""
    steps, seed = a
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1901_06798_gb300 import workloads as W
    w = W.shelf(n=4096, dx=500.0)
    n = 512
    i0 = 4096 - 1200 - n // 2 + (seed % 4) * 8
    j0 = 2048 - n // 2 + (seed // 4) * 8
    cfg = dict(w["cfg"], nx=n, ny=n, x0=i0 * 500.0, y0=j0 * 500.0)
    o = W.load(oracle.Oracle(cfg, variant="fast"), dict(w, cfg=cfg, gauges=np.zeros((0, 2))))
    t0 = time.perf_counter()
    o.step(steps)
    return n * n * steps, time.perf_counter() - t0


def run_reference(args):
    import multiprocessing as mp
    import oracle
    oracle.build("fast")
    os.environ["OMP_NUM_THREADS"] = "1"   # one window per worker process and core
    cores = min(os.cpu_count() or 1, 16)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_ref_worker, [(args.warmup, k) for k in range(cores)])
        t0 = time.perf_counter()
        res = pool.map(_ref_worker, [(args.steps, k) for k in range(cores)])
        wall = time.perf_counter() - t0
    cells = sum(r[0] for r in res)
    v = cells / wall
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "shelf4096: 512x512 windows of the 4096x4096 dx=500 m shelf/uplift workload, "
                                   f"one per host core ({cores})"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} x 512x512 windows of the 4096^2 workload, {args.steps} steps each"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--amr-steps", type=int, default=16,
                    help="coarse steps of the 3-level AMR and 64-scenario ensemble legs (FP64: a quarter); 0 skips")
    ap.add_argument("--config4-steps", type=int, default=0,
                    help="coarse steps of the 4-level bay workload, plain vs learned flagging (0: skip)")
    ap.add_argument("--config4-train-regrids", type=int, default=40,
                    help="regrid intervals of the uniform shelf run that supply predictor training pairs")
    ap.add_argument("--transverse-steps", type=int, default=100,
                    help="steps of the unsplit (transverse-correction) legs; 0 skips them")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default="", help="threads,seg_rows of the patch update instead of autotuning")
    ap.add_argument("--legs", default="uniform,unsplit,amr3,ensemble64,e2e",
                    help="comma list of legs to run (a line without the uniform leg is marked partial)")
    ap.add_argument("--repeats", type=int, default=5, help="extra K-step timings of the headline leg (median)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    results, clk, e2e, extra = run_ours(args, rank, world, dist, torch)
    config4 = None
    if args.config4_steps > 0 and rank == 0:
        config4 = run_config4(args, torch.cuda.current_stream().cuda_stream, torch)
    alu = measured_alu_peaks(torch) if rank == 0 and "f32p" in results else {}
    if rank == 0 and "f32p" not in results:
        # a subset of the legs (profiling runs): no headline line
        print(json.dumps({"partial": True, "legs": args.legs, "amr": extra, "e2e": e2e, "clocks": clk,
                          **({"config4": config4} if config4 else {})}))
    elif rank == 0:
        hbm, src = peaks()
        r = results["f32p"]
        bpl = BYTES_PER_CELL["f32p"] * r["cells"]
        achieved = bpl / (r["kernel_ms"] / 1e3) / 1e9
        traffic = ncu_traffic("f32p")
        r64 = results["f64"]
        b64 = BYTES_PER_CELL["f64"] * r64["cells"]
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": r["K"],
            "warmup": args.warmup, "ms_per_step": r["elapsed"] / r["K"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "shelf4096: 4096x4096 cells, dx=500 m, shelf bathymetry with beach and dry land, "
                                   "2 m Gaussian uplift (25x50 km sigma) at t=0, extrapolating boundaries",
                       "precision": "FP32 surface-perturbation form (eta', hu, hv, B in FP32)",
                       "l2": "inputs larger than L2 (state 537 MB FP32 / 1.07 GB FP64); no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "launch_shape": r["tune"],
                       "step": "the kernels tsu_step runs per coarse step: dt, boundaries, the patch update, "
                               "the CFL check, the level-1 retake launch and its check, gauge sampling"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": "patch update = step_x_f32x2 + step_y_f32x2 (one launch each per step)",
                         "kernel_ms": r["kernel_ms"],
                         "bytes_per_launch": bpl, "peak_source": src},
            # the other roof of the same update: algorithmic flops against the FP32 pipes; neither
            # binds -- the update is bound by instruction issue (see the design notes)
            "roofline_fp32": {"bound": "alu", "achieved": FLOPS_PER_CELL * r["cells"] / (r["kernel_ms"] / 1e3) / 1e12,
                              "peak": alu.get("fp32", FP32_PEAK_TFLOPS), "unit": "TFLOP/s",
                              "frac": FLOPS_PER_CELL * r["cells"] / (r["kernel_ms"] / 1e3) / 1e12
                                      / alu.get("fp32", FP32_PEAK_TFLOPS),
                              "flops_per_cell": FLOPS_PER_CELL,
                              "peak_source": ("measured: FP32 GEMM 8192^3, TF32 off (FMA pipes)" if "fp32" in alu
                                              else "derived: 152 SMs x 128 lanes x 2 x 2.07 GHz"),
                              "peak_derived": FP32_PEAK_TFLOPS},
            "fp64": {"value": r64["value"], "steps": r64["K"], "ms_per_step": r64["elapsed"] / r64["K"] * 1e3,
                     "kernel_ms": r64["kernel_ms"],
                     "hbm_frac": (b64 / (r64["kernel_ms"] / 1e3) / 1e9) / hbm,
                     "fp64_frac": FLOPS_PER_CELL * r64["cells"] / (r64["kernel_ms"] / 1e3) / 1e12
                                  / alu.get("fp64", FP64_PEAK_TFLOPS),
                     "fp64_peak_tflops": alu.get("fp64", FP64_PEAK_TFLOPS),
                     "fp64_peak": ("measured: FP64 GEMM 4096^3 (cuBLAS, FP64 tensor path)" if "fp64" in alu
                                   else "nominal 1.25 TFLOP/s")},
            "fp32p_over_fp64": r["value"] / r64["value"],
            "repeats": {"n": len(r["repeats"]), "steps_each": r["K"],
                        "value_median": statistics.median(v for _, v in r["repeats"]) if r["repeats"] else None,
                        "value_min": min(v for _, v in r["repeats"]) if r["repeats"] else None,
                        "value_max": max(v for _, v in r["repeats"]) if r["repeats"] else None,
                        "kernel_ms_median": statistics.median(k for k, _ in r["repeats"]) if r["repeats"] else None},
            "unsplit": {k.split("_")[0]: {"value": u["value"], "steps": u["K"],
                                           "ms_per_step": u["elapsed"] / u["K"] * 1e3, "kernel_ms": u["kernel_ms"],
                                           "hbm_frac": (BYTES_PER_CELL[k.split("_")[0]] * u["cells"]
                                                        / (u["kernel_ms"] / 1e3) / 1e9) / hbm,
                                           "launch_shape": u["tune"]}
                        for k, u in results.items() if k.endswith("_unsplit")},
            "amr": extra,
            **({"config4": config4} if config4 else {}),
            "gpu_launches": results["f32p"]["launches"],
            "clocks": clk,
            "e2e": e2e,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
