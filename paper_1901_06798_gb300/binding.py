"""Thin ctypes binding of the C ABI declared in ``include/tsunami.h``.

Every function here only marshals arguments; all computation happens in the
CUDA library ``_build/libtsunami.so``.  Loading fails loudly (RuntimeError)
when the library has not been built -- there is no fallback path.

Module-level functions carry the C names (``tsu_create``, ``tsu_step``, ...);
the ``Tsunami`` class wraps a context with the same methods as the test
oracle so the two can be driven from one workload description.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtsunami.so")

MAX_LEVELS = 8
MAX_REGIONS = 8
TSU_OK, TSU_ERR_ARG, TSU_ERR_CUDA, TSU_ERR_CFL, TSU_ERR_NESTING, TSU_ERR_OOM, TSU_ERR_NOT_BUILT = 0, -1, -2, -3, -4, -5, -6
TSU_ERR_NAN = -7
TSU_ERR_TIMEOUT = -8
TSU_ERR_NEGDEPTH = -9
TSU_F64, TSU_F32P = 0, 1
FIELDS = {"h": 0, "hu": 1, "hv": 2, "eta": 3, "zeta": 4, "B": 5}

# every symbol include/tsunami.h declares
SYMBOLS = ["tsu_create", "tsu_destroy", "tsu_last_error", "tsu_add_topo", "tsu_set_eta", "tsu_add_uplift",
           "tsu_init", "tsu_step", "tsu_step_level", "tsu_regrid", "tsu_num_patches", "tsu_get_patches", "tsu_get_patch",
           "tsu_read_field", "tsu_add_gauges", "tsu_read_gauges", "tsu_get_stats", "tsu_sync",
           "tsu_level1_buffers", "tsu_time_level1_steps", "tsu_set_tuning",
           "tsu_grid_step_noalloc", "tsu_autotune", "tsu_cnn_num_params", "tsu_cnn_forward",
           "tsu_cnn_loss_grad", "tsu_cnn_train", "tsu_cnn_set_weights", "tsu_cnn_features", "tsu_cluster_flags", "tsu_set_velocity",
           "tsu_checkpoint_save", "tsu_checkpoint_restore", "tsu_profile_levels", "tsu_level_update_times",
           "tsu_halo_pack", "tsu_halo_unpack", "tsu_set_bulk_copies"]


class tsu_config(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("num_levels", C.c_int), ("ratios", C.c_int * MAX_LEVELS), ("bc", C.c_int * 4),
        ("g", C.c_double), ("drytol", C.c_double), ("cfl_desired", C.c_double), ("cfl_max", C.c_double),
        ("dt_max", C.c_double), ("regrid_interval", C.c_int), ("flag_eta_tol", C.c_double),
        ("flag_depth_below", C.c_double), ("patch_max", C.c_int), ("level1_tile", C.c_int),
        ("n_regions", C.c_int), ("regions", (C.c_double * 6) * MAX_REGIONS), ("n_scenarios", C.c_int),
        ("transverse", C.c_int), ("cluster_eff", C.c_double), ("use_graphs", C.c_int),
        ("use_cnn", C.c_int), ("cnn_buffer", C.c_int), ("manning_n", C.c_double),
        ("spherical", C.c_int), ("earth_radius", C.c_double), ("cfl_retake", C.c_int),
    ]


class tsu_stats(C.Structure):
    _fields_ = [("dt", C.c_double), ("t", C.c_double), ("mass", C.c_double), ("cell_updates", C.c_double),
                ("cfl_violations", C.c_longlong), ("patches", C.c_int * MAX_LEVELS),
                ("kernel_launches", C.c_longlong), ("regrids", C.c_longlong), ("regrid_host_ms", C.c_double),
                ("cluster_ms", C.c_double), ("cfl_retakes", C.c_longlong), ("regrid_wait_ms", C.c_double),
                ("patches_renewed", C.c_longlong), ("patches_reused", C.c_longlong)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path) or os.environ.get("TSU_REBUILD"):
        from . import build as _b
        _b.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built (run paper_1901_06798_gb300.build)")
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    fp = C.POINTER(C.c_float)
    sig = {
        "tsu_create": ([C.POINTER(tsu_config), P, C.POINTER(P)], I),
        "tsu_destroy": ([P], I),
        "tsu_last_error": ([P], C.c_char_p),
        "tsu_add_topo": ([P, dp, I, I, D, D, D, D], I),
        "tsu_set_eta": ([P, I, dp, I, I, D, D, D, D], I),
        "tsu_add_uplift": ([P, I, dp, I, I, D, D, D, D], I),
        "tsu_init": ([P], I),
        "tsu_step": ([P, I, dp], I),
        "tsu_step_level": ([P, I, dp], I),
        "tsu_profile_levels": ([P, I], I),
        "tsu_halo_pack": ([P, I, I, ip, I, P, C.c_longlong], I),
        "tsu_halo_unpack": ([P, I, I, ip, I, P, C.c_longlong], I),
        "tsu_level_update_times": ([P, dp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), I], I),
        "tsu_regrid": ([P, I, I], I),
        "tsu_num_patches": ([P, I, I, ip], I),
        "tsu_get_patches": ([P, I, I, ip, I, ip], I),
        "tsu_get_patch": ([P, I, I, I, dp, dp, dp, dp], I),
        "tsu_read_field": ([P, I, I, I, dp, I, I, D, D, D, D], I),
        "tsu_add_gauges": ([P, dp, I], I),
        "tsu_read_gauges": ([P, dp, dp, I, ip], I),
        "tsu_get_stats": ([P, I, C.POINTER(tsu_stats)], I),
        "tsu_sync": ([P], I),
        "tsu_level1_buffers": ([P, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(P), ip], I),
        "tsu_time_level1_steps": ([P, I, I, dp, dp], I),
        "tsu_set_tuning": ([P, I, I], I),
        "tsu_set_bulk_copies": ([P, I, C.c_longlong], I),
        "tsu_autotune": ([P, I, ip, ip, dp], I),
        "tsu_cnn_num_params": ([], I),
        "tsu_cluster_flags": ([P, P, I, I, D, I, I, ip, I, ip], I),
        "tsu_set_velocity": ([P, I, dp, dp, I, I, D, D, D, D], I),
        "tsu_checkpoint_save": ([P, P, C.c_size_t, C.POINTER(C.c_size_t)], I),
        "tsu_checkpoint_restore": ([P, P, C.c_size_t], I),
        "tsu_cnn_forward": ([fp, fp, I, I, I, I, fp], I),
        "tsu_cnn_loss_grad": ([fp, fp, fp, fp, I, I, I, dp, fp], I),
        "tsu_cnn_train": ([fp, fp, fp, fp, I, I, I, I, I, C.c_float, C.c_uint, dp, dp], I),
        "tsu_cnn_set_weights": ([P, fp, I], I),
        "tsu_cnn_features": ([P, I, I, fp, C.POINTER(C.c_ubyte)], I),
        "tsu_grid_step_noalloc": ([I, P, I, I, I, C.c_longlong, I, D, D, D, D, D, ip, dp, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class TsuError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def make_config(cfg: dict, precision: int = TSU_F64, use_graphs: bool = True) -> tsu_config:
    c = tsu_config()
    c.precision = precision
    c.nx, c.ny = cfg["nx"], cfg["ny"]
    c.x0, c.y0, c.dx, c.dy = cfg.get("x0", 0.0), cfg.get("y0", 0.0), cfg["dx"], cfg.get("dy", cfg["dx"])
    c.num_levels = cfg.get("num_levels", 1)
    for k, r in enumerate(cfg.get("ratios", [])):
        c.ratios[k] = r
    for k, b in enumerate(cfg.get("bc", [0] * 4)):
        c.bc[k] = b
    c.g = cfg.get("g", 9.81)
    c.drytol = cfg.get("drytol", 1e-3)
    c.cfl_desired = cfg.get("cfl_desired", 0.9)
    c.cfl_max = cfg.get("cfl_max", 1.0)
    c.dt_max = cfg.get("dt_max", 1e9)
    c.regrid_interval = cfg.get("regrid_interval", 0)
    c.flag_eta_tol = cfg.get("flag_eta_tol", 0.0)
    c.flag_depth_below = cfg.get("flag_depth_below", 0.0)
    c.patch_max = cfg.get("patch_max", 64)
    c.level1_tile = cfg.get("level1_tile", 0)
    regs = cfg.get("regions", [])
    c.n_regions = len(regs)
    for k, rg in enumerate(regs):
        for m in range(6):
            c.regions[k][m] = rg[m]
    c.n_scenarios = cfg.get("n_scenarios", 1)
    c.transverse = cfg.get("transverse", 0)
    c.cluster_eff = cfg.get("cluster_eff", 0.7)
    c.use_graphs = 1 if use_graphs else 0
    c.use_cnn = cfg.get("use_cnn", 0)
    c.cnn_buffer = cfg.get("cnn_buffer", 1)
    c.manning_n = cfg.get("manning_n", 0.0)
    c.spherical = cfg.get("spherical", 0)
    c.earth_radius = cfg.get("earth_radius", 0.0)
    c.cfl_retake = cfg.get("cfl_retake", 1)
    return c


class Tsunami:
    """One library context (the C ABI's tsu_ctx)."""

    def __init__(self, cfg: dict, precision: int = TSU_F64, stream=None, use_graphs: bool = True):
        self._L = load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg, precision, use_graphs)
        self.precision = precision
        h = C.c_void_p()
        rc = self._L.tsu_create(C.byref(self._c), C.c_void_p(stream) if stream else None, C.byref(h))
        if rc != 0:
            raise TsuError(rc, "tsu_create failed")
        self._h = h
        self.num_levels = self._c.num_levels
        self.n_scenarios = self._c.n_scenarios
        self.ngauges = 0

    def _check(self, rc, what, allow=()):
        if rc != 0 and rc not in allow:
            msg = self._L.tsu_last_error(self._h)
            raise TsuError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._L.tsu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _grid(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    def add_topo(self, B, x0, y0, dx, dy):
        B = self._grid(B)
        self._check(self._L.tsu_add_topo(self._h, _dp(B), B.shape[1], B.shape[0], x0, y0, dx, dy), "tsu_add_topo")

    def set_eta(self, scen, eta, x0, y0, dx, dy):
        e = self._grid(eta)
        self._check(self._L.tsu_set_eta(self._h, scen, _dp(e), e.shape[1], e.shape[0], x0, y0, dx, dy), "tsu_set_eta")

    def set_velocity(self, scen, u, v, x0, y0, dx, dy):
        uu, vv = self._grid(u), self._grid(v)
        self._check(self._L.tsu_set_velocity(self._h, scen, _dp(uu), _dp(vv), uu.shape[1], uu.shape[0], x0, y0, dx,
                                             dy), "tsu_set_velocity")

    def add_uplift(self, scen, dB, x0, y0, dx, dy):
        d = self._grid(dB)
        self._check(self._L.tsu_add_uplift(self._h, scen, _dp(d), d.shape[1], d.shape[0], x0, y0, dx, dy),
                    "tsu_add_uplift")

    def init(self):
        self._check(self._L.tsu_init(self._h), "tsu_init")

    def step(self, n: int = 1, allow_cfl: bool = False):
        t = np.zeros(self.n_scenarios)
        rc = self._check(self._L.tsu_step(self._h, n, _dp(t)), "tsu_step", allow=(TSU_ERR_CFL,) if allow_cfl else ())
        self.last_rc = rc
        return t

    def step_level(self, level: int, allow_cfl: bool = False):
        """One step of one level in the recursion's order (tsu_step_level)."""
        t = np.zeros(self.n_scenarios)
        rc = self._check(self._L.tsu_step_level(self._h, level, _dp(t)), "tsu_step_level",
                         allow=(TSU_ERR_CFL,) if allow_cfl else ())
        self.last_rc = rc
        return t

    def halo_pack(self, scen: int, level: int, msgs, dev_ptr: int, n_elems: int):
        """Copy halo boxes (rows of k, i0, j0, i1, j1) out of the level's patches
        into device memory at dev_ptr (tsu_halo_pack)."""
        m = np.ascontiguousarray(np.asarray(msgs, dtype=np.int32).reshape(-1, 5))
        self._check(self._L.tsu_halo_pack(self._h, scen, level, m.ctypes.data_as(C.POINTER(C.c_int)), len(m),
                                          C.c_void_p(dev_ptr), n_elems), "tsu_halo_pack")

    def halo_unpack(self, scen: int, level: int, msgs, dev_ptr: int, n_elems: int):
        """Copy halo boxes from device memory at dev_ptr into the level's
        patches (tsu_halo_unpack)."""
        m = np.ascontiguousarray(np.asarray(msgs, dtype=np.int32).reshape(-1, 5))
        self._check(self._L.tsu_halo_unpack(self._h, scen, level, m.ctypes.data_as(C.POINTER(C.c_int)), len(m),
                                            C.c_void_p(dev_ptr), n_elems), "tsu_halo_unpack")

    def profile_levels(self, enable: bool = True):
        """Start (or stop) recording per-level update times (tsu_profile_levels)."""
        self._check(self._L.tsu_profile_levels(self._h, 1 if enable else 0), "tsu_profile_levels")

    def level_update_times(self):
        """Per level (1-based keys): update milliseconds, interior cells, level
        steps and kernels since profiling started or was last read."""
        n = self.num_levels
        ms, cells = np.zeros(n), np.zeros(n)
        steps, kern = (C.c_longlong * n)(), (C.c_longlong * n)()
        self._check(self._L.tsu_level_update_times(self._h, _dp(ms), _dp(cells), steps, kern, n),
                    "tsu_level_update_times")
        return {l + 1: {"ms": float(ms[l]), "cells": float(cells[l]), "steps": int(steps[l]), "kernels": int(kern[l])}
                for l in range(n)}

    def regrid(self, scen: int, level: int):
        self._check(self._L.tsu_regrid(self._h, scen, level), "tsu_regrid")

    def num_patches(self, scen: int, level: int) -> int:
        n = C.c_int()
        self._check(self._L.tsu_num_patches(self._h, scen, level, C.byref(n)), "tsu_num_patches")
        return n.value

    def boxes(self, scen: int, level: int) -> np.ndarray:
        n = self.num_patches(scen, level)
        b = np.zeros(4 * max(n, 1), dtype=np.int32)
        m = C.c_int()
        self._check(self._L.tsu_get_patches(self._h, scen, level, b.ctypes.data_as(C.POINTER(C.c_int)), n,
                                            C.byref(m)), "tsu_get_patches")
        return b[: 4 * n].reshape(n, 4)

    def patches(self, scen: int, level: int):
        out = []
        for k, (i0, j0, nx, ny) in enumerate(self.boxes(scen, level)):
            a = {f: np.zeros((ny, nx)) for f in ("h", "hu", "hv", "B")}
            self._check(self._L.tsu_get_patch(self._h, scen, level, k, _dp(a["h"]), _dp(a["hu"]), _dp(a["hv"]),
                                              _dp(a["B"])), "tsu_get_patch")
            out.append(((int(i0), int(j0), int(nx), int(ny)), a))
        return out

    def level_array(self, scen: int, level: int, field: str, fill=np.nan):
        R = 1
        for k in range(level - 1):
            R *= self.cfg["ratios"][k]
        A = np.full((self.cfg["ny"] * R, self.cfg["nx"] * R), fill)
        for (i0, j0, nx, ny), a in self.patches(scen, level):
            A[j0:j0 + ny, i0:i0 + nx] = a[field] if field in a else a["h"] + a["B"]
        return A

    def read_field(self, scen, level, field, nx, ny, x0, y0, dx, dy):
        out = np.zeros((ny, nx))
        self._check(self._L.tsu_read_field(self._h, scen, level, FIELDS[field], _dp(out), nx, ny, x0, y0, dx, dy),
                    "tsu_read_field")
        return out

    def add_gauges(self, xy):
        xy = self._grid(xy)
        self._check(self._L.tsu_add_gauges(self._h, _dp(xy), xy.shape[0]), "tsu_add_gauges")
        self.ngauges += xy.shape[0]

    def read_gauges(self, max_samples: int = 1 << 16):
        ns, ng = self.n_scenarios, self.ngauges
        t = np.zeros(max_samples * ns)
        e = np.zeros(max_samples * ns * max(ng, 1))
        n = C.c_int()
        self._check(self._L.tsu_read_gauges(self._h, _dp(t), _dp(e), max_samples, C.byref(n)), "tsu_read_gauges")
        k = n.value
        return t[: k * ns].reshape(k, ns), e[: k * ns * ng].reshape(k, ns, ng)

    def stats(self, scen: int = 0) -> dict:
        s = tsu_stats()
        self._check(self._L.tsu_get_stats(self._h, scen, C.byref(s)), "tsu_get_stats")
        return {"dt": s.dt, "t": s.t, "mass": s.mass, "cell_updates": s.cell_updates,
                "cfl_violations": s.cfl_violations, "patches": list(s.patches)[: self.num_levels],
                "kernel_launches": s.kernel_launches, "regrids": s.regrids, "regrid_host_ms": s.regrid_host_ms,
                "cluster_ms": s.cluster_ms, "cfl_retakes": s.cfl_retakes, "regrid_wait_ms": s.regrid_wait_ms,
                "patches_renewed": s.patches_renewed, "patches_reused": s.patches_reused}

    def checkpoint(self) -> bytes:
        """The whole simulation state between steps (tsu_checkpoint_save)."""
        n = C.c_size_t()
        self._check(self._L.tsu_checkpoint_save(self._h, None, 0, C.byref(n)), "tsu_checkpoint_save")
        buf = C.create_string_buffer(n.value)
        self._check(self._L.tsu_checkpoint_save(self._h, buf, n.value, C.byref(n)), "tsu_checkpoint_save")
        return buf.raw[: n.value]

    def restore(self, data: bytes):
        """Continue from a checkpoint (tsu_checkpoint_restore); the context
        needs the same configuration and inputs and must be initialised."""
        self._check(self._L.tsu_checkpoint_restore(self._h, data, len(data)), "tsu_checkpoint_restore")

    def set_tuning(self, step_threads: int = 0, seg_rows: int = 0):
        self._check(self._L.tsu_set_tuning(self._h, step_threads, seg_rows), "tsu_set_tuning")

    def set_bulk_copies(self, enable: int, polls: int = 1 << 22):
        """x-sweep rows by bulk copies on mbarriers, each wait at most `polls` polls (0: give up at once)."""
        self._check(self._L.tsu_set_bulk_copies(self._h, enable, C.c_longlong(polls)), "tsu_set_bulk_copies")

    def autotune(self, reps: int = 3):
        """Pick the fastest launch shape of the patch update; returns (threads, seg_rows, ms)."""
        a, b, m = C.c_int(), C.c_int(), C.c_double()
        self._check(self._L.tsu_autotune(self._h, reps, C.byref(a), C.byref(b), C.byref(m)), "tsu_autotune")
        return a.value, b.value, m.value

    def cnn_set_weights(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(self._L.tsu_cnn_set_weights(self._h, th.ctypes.data_as(C.POINTER(C.c_float)), th.size),
                    "tsu_cnn_set_weights")

    def cnn_features(self, scen: int, level: int):
        """(features (5, ny_l, nx_l) float32, criterion flags (ny_l, nx_l) uint8) of a level."""
        R = 1
        for k in range(level - 1):
            R *= self.cfg["ratios"][k]
        ny, nx = self.cfg["ny"] * R, self.cfg["nx"] * R
        f = np.zeros((5, ny, nx), dtype=np.float32)
        g = np.zeros((ny, nx), dtype=np.uint8)
        self._check(self._L.tsu_cnn_features(self._h, scen, level, f.ctypes.data_as(C.POINTER(C.c_float)),
                                             g.ctypes.data_as(C.POINTER(C.c_ubyte))), "tsu_cnn_features")
        return f, g

    def sync(self):
        self._check(self._L.tsu_sync(self._h), "tsu_sync")

    def time_level1_steps(self, warmup: int, n: int):
        k = C.c_double()
        s = C.c_double()
        self._check(self._L.tsu_time_level1_steps(self._h, warmup, n, C.byref(k), C.byref(s)),
                    "tsu_time_level1_steps")
        return k.value, s.value

    def level1_buffers(self):
        ptrs = [C.c_void_p() for _ in range(4)]
        pitch = C.c_int()
        self._check(self._L.tsu_level1_buffers(self._h, *[C.byref(p) for p in ptrs], C.byref(pitch)),
                    "tsu_level1_buffers")
        return [p.value for p in ptrs], pitch.value


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def cluster_flags(flags, nestable=None, eff: float = 0.7, ratio: int = 1, patch_max: int = 1 << 30):
    """The library's clustering of a (ny, nx) 0/1 mask (host code, no GPU):
    boxes (i0, j0, w, h) as an (n, 4) int array."""
    L = load()
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    nst = None if nestable is None else np.ascontiguousarray(nestable, dtype=np.uint8)
    ny, nx = f.shape
    cap = 1024
    while True:
        out = np.zeros(4 * cap, dtype=np.int32)
        n = C.c_int()
        rc = L.tsu_cluster_flags(f.ctypes.data, None if nst is None else nst.ctypes.data, nx, ny, eff, ratio,
                                 patch_max, out.ctypes.data_as(C.POINTER(C.c_int)), cap, C.byref(n))
        if rc == 0:
            return out[: 4 * n.value].reshape(n.value, 4).copy()
        if n.value <= cap:
            raise TsuError(rc, "tsu_cluster_flags: bad arguments")
        cap = n.value


def cnn_num_params() -> int:
    return load().tsu_cnn_num_params()


def cnn_forward(theta, x, fp16: bool = False):
    """Logits (n, h, w) of inputs x (n, 5, h, w) on the GPU."""
    L = load()
    th, xx = _f32(theta), _f32(x)
    n, _, h, w = xx.shape
    out = np.zeros((n, h, w), dtype=np.float32)
    rc = L.tsu_cnn_forward(_fptr(th), _fptr(xx), n, h, w, 1 if fp16 else 0, _fptr(out))
    if rc:
        raise TsuError(rc, "tsu_cnn_forward")
    return out


def cnn_loss_grad(theta, x, t, m):
    L = load()
    th, xx, tt, mm = _f32(theta), _f32(x), _f32(t), _f32(m)
    n, _, h, w = xx.shape
    g = np.zeros(th.size, dtype=np.float32)
    loss = C.c_double()
    rc = L.tsu_cnn_loss_grad(_fptr(th), _fptr(xx), _fptr(tt), _fptr(mm), n, h, w, C.byref(loss), _fptr(g))
    if rc:
        raise TsuError(rc, "tsu_cnn_loss_grad")
    return loss.value, g


def cnn_train(theta, x, t, m, steps: int, batch: int = 4, lr: float = 1e-3, seed: int = 0):
    """Adam on the GPU; returns (trained theta, first-batch loss, last-batch loss)."""
    L = load()
    th = _f32(theta).copy()
    xx, tt, mm = _f32(x), _f32(t), _f32(m)
    n, _, h, w = xx.shape
    l0, l1 = C.c_double(), C.c_double()
    rc = L.tsu_cnn_train(_fptr(th), _fptr(xx), _fptr(tt), _fptr(mm), n, h, w, steps, batch, lr, seed,
                         C.byref(l0), C.byref(l1))
    if rc:
        raise TsuError(rc, "tsu_cnn_train")
    return th, l0.value, l1.value


def tsu_grid_step_noalloc(precision: int, block_ptr: int, nx: int, ny: int, pitch: int, field_stride: int,
                          cur: int, dx: float, dy: float, dt: float, g: float, drytol: float, bc, stream=None):
    """One step of a uniform grid in caller-owned device memory, allocating
    nothing (see include/tsunami.h).  Returns (rc, (max x speed, max y speed))."""
    L = load()
    bcv = (C.c_int * 4)(*bc)
    sp = (C.c_double * 2)()
    rc = L.tsu_grid_step_noalloc(precision, C.c_void_p(block_ptr), nx, ny, pitch, field_stride, cur, dx, dy, dt, g,
                                 drytol, bcv, sp, C.c_void_p(stream) if stream else None)
    return rc, (sp[0], sp[1])


# C-named module functions (argument marshalling only)
def tsu_create(cfg: dict, precision: int = TSU_F64, stream=None, use_graphs: bool = True) -> Tsunami:
    return Tsunami(cfg, precision, stream, use_graphs)


def tsu_destroy(ctx: Tsunami):
    ctx.close()
