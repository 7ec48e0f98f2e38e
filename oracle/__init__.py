"""FP64 CPU oracle for the shallow-water AMR wave-propagation update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_1901_06798_gb300``) and imports nothing from it.

The C sources (``swe.c``, ``amr.c``) follow the paper's Sec. 2-3 step by step;
this module only compiles them with ``-O2 -ffp-contract=off`` and marshals
arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRCS = ["swe.c", "amr.c"]
_HDRS = ["oracle.h", "ora_internal.h"]
_LIB = None
_LOCK = threading.Lock()

MAX_LEVELS = 8
MAX_REGIONS = 8
BC_WALL, BC_EXTRAP = 0, 1
FIELDS = {"h": 0, "hu": 1, "hv": 2, "eta": 3, "zeta": 4, "B": 5}


def build(variant: str = "parity", force: bool = False) -> str:
    """Compile the oracle.  ``parity``: -O2 -ffp-contract=off (the arithmetic
    exactly as written, one thread); ``fast``: the same source with -O3 and
    OpenMP over the rows and columns of a patch's sweeps, still without
    contraction (used only to time the CPU baseline; the same results)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, f"liboracle_{variant}.so")
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDRS]
    if not force and os.path.exists(out):
        mt = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= mt for d in deps):
            return out
    # the timing build shares a patch's row and column sweeps over OpenMP threads
    # (OMP_NUM_THREADS, default all cores); the parity build has no threads
    opt = ["-O2"] if variant == "parity" else ["-O3", "-fopenmp"]
    cmd = ["gcc", *opt, "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           *srcs, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build_flopcount(force: bool = False) -> str:
    """Compile ``flopcount.cpp``: ``swe.c`` with a counting scalar type, for the
    algorithmic operation count of one cell update (no contraction, as the oracle)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libora_flopcount.so")
    deps = [os.path.join(_HERE, s) for s in ("flopcount.cpp", "swe.c", *_HDRS)]
    if not force and os.path.exists(out):
        mt = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= mt for d in deps):
            return out
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fPIC", "-shared",
           "-Wno-class-memaccess", os.path.join(_HERE, "flopcount.cpp"), "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


FLOP_KINDS = ("add", "mul", "div", "sqrt", "cmp", "minmax", "abs", "neg")


def count_step_flops(h, hu, hv, B, g, drytol, dt, dx, dy):
    """Operation counts of one split step (``ora_step_patch``) of a patch given
    as (ny + 4, nx + 4) arrays with their ghost cells filled.  Returns a dict
    over FLOP_KINDS, and the updated (h, hu, hv)."""
    L = C.CDLL(build_flopcount())
    dp = C.POINTER(C.c_double)
    L.flop_count_step.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp] + [C.c_double] * 5 + [C.POINTER(C.c_longlong)]
    L.flop_count_step.restype = C.c_int
    ny4, nx4 = h.shape
    a = [np.ascontiguousarray(x, dtype=np.float64).copy() for x in (h, hu, hv, B)]
    out = (C.c_longlong * 8)()
    rc = L.flop_count_step(nx4 - 4, ny4 - 4, *[x.ctypes.data_as(dp) for x in a], g, drytol, dt, dx, dy, out)
    if rc != 0:
        raise ValueError(f"flop_count_step failed ({rc})")
    return dict(zip(FLOP_KINDS, list(out))), tuple(a[:3])


class ora_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("num_levels", C.c_int), ("ratios", C.c_int * MAX_LEVELS), ("bc", C.c_int * 4),
        ("g", C.c_double), ("drytol", C.c_double), ("cfl_desired", C.c_double),
        ("cfl_max", C.c_double), ("dt_max", C.c_double),
        ("regrid_interval", C.c_int),
        ("flag_eta_tol", C.c_double), ("flag_depth_below", C.c_double),
        ("patch_max", C.c_int), ("level1_tile", C.c_int),
        ("n_regions", C.c_int), ("regions", (C.c_double * 6) * MAX_REGIONS),
        ("n_scenarios", C.c_int), ("transverse", C.c_int), ("cluster_eff", C.c_double),
        ("manning_n", C.c_double), ("spherical", C.c_int), ("earth_radius", C.c_double), ("reflux", C.c_int),
        ("cfl_retake", C.c_int),
    ]


class ora_rp(C.Structure):
    _fields_ = [("Z", (C.c_double * 3) * 3), ("s", C.c_double * 3), ("wallL", C.c_int), ("wallR", C.c_int)]


def lib(variant: str = "parity"):
    global _LIB
    with _LOCK:
        if _LIB is None or _LIB[0] != variant:
            L = C.CDLL(build(variant))
            D, I, P = C.c_double, C.c_int, C.c_void_p
            dp = C.POINTER(C.c_double)
            L.ora_riemann.argtypes = [D, D, D, D, D, D, D, D, D, D, C.POINTER(ora_rp)]
            L.ora_riemann.restype = None
            L.ora_mc_limiter.argtypes = [D]
            L.ora_mc_limiter.restype = D
            L.ora_cluster.argtypes = [P, P, I, I, D, I, I, C.POINTER(C.c_int), I]
            L.ora_cluster.restype = I
            L.ora_create.argtypes = [C.POINTER(ora_config)]
            L.ora_create.restype = P
            L.ora_destroy.argtypes = [P]
            L.ora_destroy.restype = None
            for name in ("ora_add_topo",):
                getattr(L, name).argtypes = [P, dp, I, I, D, D, D, D]
                getattr(L, name).restype = I
            L.ora_set_velocity.argtypes = [P, I, dp, dp, I, I, D, D, D, D]
            L.ora_set_velocity.restype = I
            for name in ("ora_set_eta", "ora_add_uplift"):
                getattr(L, name).argtypes = [P, I, dp, I, I, D, D, D, D]
                getattr(L, name).restype = I
            L.ora_init.argtypes = [P]
            L.ora_init.restype = I
            L.ora_step.argtypes = [P, I, dp]
            L.ora_step.restype = I
            L.ora_regrid.argtypes = [P, I, I]
            L.ora_regrid.restype = I
            L.ora_num_patches.argtypes = [P, I, I]
            L.ora_num_patches.restype = I
            L.ora_get_patch.argtypes = [P, I, I, I, C.POINTER(C.c_int), dp, dp, dp, dp]
            L.ora_get_patch.restype = I
            L.ora_read_field.argtypes = [P, I, I, I, dp, I, I, D, D, D, D]
            L.ora_read_field.restype = I
            L.ora_add_gauges.argtypes = [P, dp, I]
            L.ora_add_gauges.restype = I
            L.ora_read_gauges.argtypes = [P, dp, dp, I, C.POINTER(C.c_int)]
            L.ora_read_gauges.restype = I
            L.ora_stats.argtypes = [P, I, dp]
            L.ora_stats.restype = I
            _LIB = (variant, L)
        return _LIB[1]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def riemann(hL, hnL, htL, BL, hR, hnR, htR, BR, g=9.81, drytol=1e-3):
    """Solve one normal-direction Riemann problem; returns (Z[3,3], s[3], wallL, wallR)."""
    r = ora_rp()
    lib().ora_riemann(g, drytol, hL, hnL, htL, BL, hR, hnR, htR, BR, C.byref(r))
    Z = np.array([[r.Z[p][m] for m in range(3)] for p in range(3)])
    return Z, np.array(list(r.s)), r.wallL, r.wallR


def mc_limiter(theta: float) -> float:
    return lib().ora_mc_limiter(theta)


def cluster(flags: np.ndarray, nestable: np.ndarray | None = None, eff=0.7, ratio=1, patch_max=1 << 30):
    """Berger-Rigoutsos clustering of a (ny, nx) 0/1 mask; returns boxes (i0, j0, w, h)."""
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    n = np.ones_like(f) if nestable is None else np.ascontiguousarray(nestable, dtype=np.uint8)
    ny, nx = f.shape
    maxb = nx * ny + 1
    out = np.zeros(4 * maxb, dtype=np.int32)
    nb = lib().ora_cluster(f.ctypes.data, n.ctypes.data, nx, ny, eff, ratio, patch_max,
                           out.ctypes.data_as(C.POINTER(C.c_int)), maxb)
    if nb < 0:
        raise RuntimeError("cluster overflow")
    return out[: 4 * nb].reshape(nb, 4).copy()


def make_config(cfg: dict) -> ora_config:
    c = ora_config()
    c.nx, c.ny = cfg["nx"], cfg["ny"]
    c.x0, c.y0, c.dx, c.dy = cfg.get("x0", 0.0), cfg.get("y0", 0.0), cfg["dx"], cfg.get("dy", cfg["dx"])
    c.num_levels = cfg.get("num_levels", 1)
    for k, r in enumerate(cfg.get("ratios", [])):
        c.ratios[k] = r
    for k, b in enumerate(cfg.get("bc", [BC_WALL] * 4)):
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
    c.manning_n = cfg.get("manning_n", 0.0)
    c.spherical = cfg.get("spherical", 0)
    c.earth_radius = cfg.get("earth_radius", 0.0)
    c.reflux = cfg.get("reflux", 0)
    c.cfl_retake = cfg.get("cfl_retake", 1)
    return c


class Oracle:
    """The whole method on the CPU: create, add topography/state/uplift, init,
    step, regrid, read patches/fields/gauges."""

    def __init__(self, cfg: dict, variant: str = "parity"):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self._L = lib(variant)
        self._h = self._L.ora_create(C.byref(self._c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.num_levels = self._c.num_levels
        self.n_scenarios = self._c.n_scenarios

    def close(self):
        if self._h:
            self._L.ora_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _grid(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"oracle {what} failed ({rc})")

    def add_topo(self, B, x0, y0, dx, dy):
        B = self._grid(B)
        self._check(self._L.ora_add_topo(self._h, _dp(B), B.shape[1], B.shape[0], x0, y0, dx, dy), "add_topo")

    def set_eta(self, scen, eta, x0, y0, dx, dy):
        e = self._grid(eta)
        self._check(self._L.ora_set_eta(self._h, scen, _dp(e), e.shape[1], e.shape[0], x0, y0, dx, dy), "set_eta")

    def set_velocity(self, scen, u, v, x0, y0, dx, dy):
        uu, vv = self._grid(u), self._grid(v)
        self._check(self._L.ora_set_velocity(self._h, scen, _dp(uu), _dp(vv), uu.shape[1], uu.shape[0], x0, y0, dx,
                                             dy), "set_velocity")

    def add_uplift(self, scen, dB, x0, y0, dx, dy):
        d = self._grid(dB)
        self._check(self._L.ora_add_uplift(self._h, scen, _dp(d), d.shape[1], d.shape[0], x0, y0, dx, dy),
                    "add_uplift")

    def init(self):
        self._check(self._L.ora_init(self._h), "init")

    def step(self, n: int = 1):
        t = np.zeros(self.n_scenarios)
        self._check(self._L.ora_step(self._h, n, _dp(t)), "step")
        return t

    def regrid(self, scen: int, level: int):
        self._check(self._L.ora_regrid(self._h, scen, level), "regrid")

    def num_patches(self, scen: int, level: int) -> int:
        return self._L.ora_num_patches(self._h, scen, level)

    def patches(self, scen: int, level: int):
        """List of (box, dict(h, hu, hv, B)) for the level's patches, interior only."""
        out = []
        for k in range(self.num_patches(scen, level)):
            box = (C.c_int * 4)()
            self._L.ora_get_patch(self._h, scen, level, k, box, None, None, None, None)
            nx, ny = box[2], box[3]
            a = {f: np.zeros((ny, nx)) for f in ("h", "hu", "hv", "B")}
            self._check(self._L.ora_get_patch(self._h, scen, level, k, box, _dp(a["h"]), _dp(a["hu"]),
                                              _dp(a["hv"]), _dp(a["B"])), "get_patch")
            out.append((tuple(box), a))
        return out

    def level_array(self, scen: int, level: int, field: str, fill=np.nan):
        """Assemble a level into a dense (ny_l, nx_l) array (tests on small grids)."""
        R = 1
        for k in range(level - 1):
            R *= self.cfg["ratios"][k]
        A = np.full((self.cfg["ny"] * R, self.cfg["nx"] * R), fill)
        for (i0, j0, nx, ny), a in self.patches(scen, level):
            v = a[field] if field in a else (a["h"] + a["B"])
            A[j0:j0 + ny, i0:i0 + nx] = v
        return A

    def read_field(self, scen, level, field, nx, ny, x0, y0, dx, dy):
        out = np.zeros((ny, nx))
        self._check(self._L.ora_read_field(self._h, scen, level, FIELDS[field], _dp(out), nx, ny, x0, y0, dx, dy),
                    "read_field")
        return out

    def add_gauges(self, xy):
        xy = self._grid(xy)
        self._check(self._L.ora_add_gauges(self._h, _dp(xy), xy.shape[0]), "add_gauges")
        self.ngauges = xy.shape[0]

    def read_gauges(self, max_samples=1 << 20):
        ns = self.n_scenarios
        ng = getattr(self, "ngauges", 0)
        t = np.zeros(max_samples * ns) if max_samples < 4096 else None
        n = C.c_int(0)
        # query size first with a small buffer
        cap = 4096
        while True:
            t = np.zeros(cap * ns)
            e = np.zeros(cap * ns * max(ng, 1))
            self._check(self._L.ora_read_gauges(self._h, _dp(t), _dp(e), cap, C.byref(n)), "read_gauges")
            if n.value < cap:
                break
            cap *= 4
        k = n.value
        return t[: k * ns].reshape(k, ns), e[: k * ns * ng].reshape(k, ns, ng)

    def stats(self, scen: int = 0) -> dict:
        out = np.zeros(7 + MAX_LEVELS)
        self._check(self._L.ora_stats(self._h, scen, _dp(out)), "stats")
        return {"dt": out[0], "t": out[1], "mass": out[2], "cfl_violations": int(out[3]),
                "cell_updates": out[4], "patches": [int(v) for v in out[5:5 + self.num_levels]],
                "cfl_retakes": int(out[5 + MAX_LEVELS]), "neg_clips": int(out[6 + MAX_LEVELS])}
