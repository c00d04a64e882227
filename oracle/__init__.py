"""FP64 CPU oracle of the coupled lattice Boltzmann aqueous-humor model
(arXiv 2102.12663, Sec. 2.3, Eqs. 6-17).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(the CUDA library and its Python binding) never imports, links or runs it, and
this package imports nothing from the product.

The arithmetic lives in ``lbm_oracle.c`` (plain C, fp64, built with
``-ffp-contract=off``); this module compiles it on demand with gcc and wraps it
with ctypes on numpy arrays.

Array conventions: a mask is ``uint8[ny, nx]`` of cell types; populations are
``float64[9, ny*nx]`` (flow, i = 0..8) and ``float64[4, ny*nx]`` (heat,
i = 1..4), cell (x, y) at flat index ``y*nx + x``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

FLUID, POROUS, COLD, HOT, ADIABATIC, INLET, OUTLET = range(7)


class Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("inlet_dir_x", ctypes.c_int32), ("inlet_dir_y", ctypes.c_int32),
        ("inlet_profile", ctypes.c_int32),
        ("inlet_lo", ctypes.c_int32), ("inlet_width", ctypes.c_int32),
        ("eye_normals", ctypes.c_int32), ("outlet_axis", ctypes.c_int32),
        ("arc_xc", ctypes.c_double), ("arc_yc", ctypes.c_double),
        ("arc_r", ctypes.c_double),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("tau_T", ctypes.c_double),
        ("g_beta", ctypes.c_double), ("g_dir", ctypes.c_double * 2),
        ("T_cold", ctypes.c_double), ("T_hot", ctypes.c_double),
        ("T0", ctypes.c_double), ("T_in", ctypes.c_double),
        ("u_in_max", ctypes.c_double), ("K", ctypes.c_double),
        ("p_out", ctypes.c_double), ("drive", ctypes.c_double * 2),
        ("noise_amp", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("tm_model", ctypes.c_int32), ("bouzidi", ctypes.c_int32), ("u_seep", ctypes.c_double),
    ]


class Obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "iop", "q_in", "q_out", "mass", "peak", "wss_cornea", "wss_iris",
        "residual", "n_fluid", "n_cornea", "n_iris")]


class VortexOut(ctypes.Structure):
    _fields_ = [("intensity", ctypes.c_double), ("intensity_abs", ctypes.c_double),
                ("psi_max", ctypes.c_double), ("psi_min", ctypes.c_double),
                ("max_x", ctypes.c_int32), ("max_y", ctypes.c_int32),
                ("min_x", ctypes.c_int32), ("min_y", ctypes.c_int32),
                ("n_fluid", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liblbm_oracle.so (gcc, -O2,
    -ffp-contract=off, OpenMP over rows)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-fopenmp", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_eye_mask.restype = ctypes.c_int
        L.orc_eye_mask.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, u8p, ctypes.POINTER(Geom)]
        L.orc_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        L.orc_moments.argtypes = [dp, dp, dp, dp]
        L.orc_collide.argtypes = [ctypes.POINTER(Params), ctypes.c_int, dp, dp, dp, dp]
        L.orc_init.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), u8p, dp, dp]
        L.orc_step.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), u8p,
                               dp, dp, dp, dp, dp, dp]
        L.orc_observe.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), u8p,
                                  dp, dp, dp, ctypes.POINTER(Obs)]
        L.orc_fields.argtypes = [ctypes.POINTER(Geom), u8p, dp, dp, dp, dp, dp]
        L.orc_run.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), u8p,
                              dp, dp, dp, dp, ctypes.c_int64]
        L.orc_seepage_velocity.restype = ctypes.c_double
        L.orc_seepage_velocity.argtypes = [ctypes.POINTER(Params), ctypes.c_double, ctypes.c_double]
        L.orc_set_threads.argtypes = [ctypes.c_int32]
        L.orc_link_q.argtypes = [ctypes.POINTER(Geom), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.orc_link_q.restype = ctypes.c_double
        L.orc_vortex.argtypes = [ctypes.POINTER(Geom), u8p, dp, ctypes.POINTER(VortexOut)]
        L.orc_get_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(state & (2**64 - 1))))


def make_params(**kw) -> Params:
    """Build the oracle's parameter struct from keyword values (lattice units).
    Unset fields default to a quiescent, isothermal, unforced state."""
    P = Params()
    P.tau = kw.get("tau", 1.0)
    P.tau_T = kw.get("tau_T", 1.0)
    P.g_beta = kw.get("g_beta", 0.0)
    gd = kw.get("g_dir", (0.0, -1.0))
    P.g_dir[0], P.g_dir[1] = float(gd[0]), float(gd[1])
    P.T_cold = kw.get("T_cold", 0.0)
    P.T_hot = kw.get("T_hot", 0.0)
    P.T0 = kw.get("T0", 0.0)
    P.T_in = kw.get("T_in", 0.0)
    P.u_in_max = kw.get("u_in_max", 0.0)
    P.K = kw.get("K_tm", kw.get("K", 1.0))
    P.p_out = kw.get("p_out", 0.0)
    dr = kw.get("drive", (0.0, 0.0))
    P.drive[0], P.drive[1] = float(dr[0]), float(dr[1])
    P.noise_amp = kw.get("noise_amp", 0.0)
    P.seed = int(kw.get("seed", 0)) & (2**64 - 1)
    P.tm_model = int(kw.get("tm_model", 0))
    P.bouzidi = int(kw.get("bouzidi", 0))
    P.u_seep = float(kw.get("u_seep", 0.0))
    return P


def eye_mask(nx: int, ny: int, angle_deg: float = 45.0, band: int = 0,
             inlet_cells: int = 0, tm_w: int = 0, tm_h: int = 0):
    """The analytic eye; returns (mask uint8[ny, nx], Geom)."""
    m = np.zeros((ny, nx), dtype=np.uint8)
    g = Geom()
    rc = lib().orc_eye_mask(nx, ny, float(angle_deg), band, inlet_cells, tm_w, tm_h,
                            _u8(m), ctypes.byref(g))
    if rc != 0:
        raise ValueError(f"eye geometry does not fit a {nx}x{ny} grid")
    return m, g


def mask_geom(nx: int, ny: int, periodic_x: int = 0, periodic_y: int = 0,
              inlet_dir=(0, 1), inlet_profile: int = 0, inlet_lo: int = 0,
              inlet_width: int = 1, outlet_axis: int | None = None, arc=None) -> Geom:
    """Geometry of a caller mask; arc = (xc, yc, r) makes the cold cells' wall
    the circle of that centre and radius (interpolated bounce-back)."""
    g = Geom()
    if arc is not None:
        g.arc_xc, g.arc_yc, g.arc_r = (float(v) for v in arc)
    g.outlet_axis = (0 if inlet_dir[0] != 0 else 1) if outlet_axis is None else outlet_axis
    g.nx, g.ny = nx, ny
    g.periodic_x, g.periodic_y = periodic_x, periodic_y
    g.inlet_dir_x, g.inlet_dir_y = int(inlet_dir[0]), int(inlet_dir[1])
    g.inlet_profile = inlet_profile
    g.inlet_lo, g.inlet_width = inlet_lo, inlet_width
    g.eye_normals = 0
    return g


def link_q(geom: Geom, x: int, y: int, i: int) -> float:
    """Fraction of link i from cell (x, y) at which it meets the cold wall's circle."""
    return float(lib().orc_link_q(ctypes.byref(geom), int(x), int(y), int(i)))


def seepage_velocity(params: Params, iop: float, h_tm: float) -> float:
    """Lumped TM (Sec. 2.3): seepage speed for the current IOP."""
    return float(lib().orc_seepage_velocity(ctypes.byref(params), float(iop), float(h_tm)))


def vortex(geom: Geom, mask: np.ndarray, u: np.ndarray) -> dict:
    """Vortex measures (Eq. 18, Tab. 3) of the velocity field u[2, ny, nx]."""
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(2, -1)
    assert m.size == geom.nx * geom.ny == uu.shape[1]
    o = VortexOut()
    lib().orc_vortex(ctypes.byref(geom), _u8(m), _dp(uu), ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in VortexOut._fields_}


def feq(p: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(p, ux, uy, _dp(out))
    return out


def moments(f9: np.ndarray):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    p, ux, uy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_moments(_dp(f9), ctypes.byref(p), ctypes.byref(ux), ctypes.byref(uy))
    return p.value, ux.value, uy.value


def collide(params: Params, porous: bool, f9: np.ndarray, g4: np.ndarray):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    g4 = np.ascontiguousarray(g4, dtype=np.float64)
    fs, gs = np.zeros(9), np.zeros(4)
    lib().orc_collide(ctypes.byref(params), int(bool(porous)), _dp(f9), _dp(g4), _dp(fs), _dp(gs))
    return fs, gs


class State:
    """Two-lattice oracle state: populations f[9, N], T[4, N] plus scratch."""

    def __init__(self, geom: Geom, params: Params, mask: np.ndarray):
        self.geom, self.params = geom, params
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert self.mask.size == geom.nx * geom.ny
        N = self.mask.size
        self.f = np.zeros((9, N))
        self.T = np.zeros((4, N))
        self._f2 = np.zeros((9, N))
        self._T2 = np.zeros((4, N))
        self.step_count = 0
        lib().orc_init(ctypes.byref(geom), ctypes.byref(params), _u8(self.mask),
                       _dp(self.f), _dp(self.T))

    @property
    def N(self) -> int:
        return self.mask.size

    def step(self):
        """One step; returns (q_in, q_out) of the step's boundary links."""
        qi, qo = ctypes.c_double(), ctypes.c_double()
        self._f2[:] = self.f
        self._T2[:] = self.T
        lib().orc_step(ctypes.byref(self.geom), ctypes.byref(self.params), _u8(self.mask),
                       _dp(self.f), _dp(self.T), _dp(self._f2), _dp(self._T2),
                       ctypes.byref(qi), ctypes.byref(qo))
        self.f, self._f2 = self._f2, self.f
        self.T, self._T2 = self._T2, self.T
        self.step_count += 1
        return qi.value, qo.value

    def run(self, nsteps: int):
        if nsteps <= 0:
            return
        lib().orc_run(ctypes.byref(self.geom), ctypes.byref(self.params), _u8(self.mask),
                      _dp(self.f), _dp(self.T), _dp(self._f2), _dp(self._T2), int(nsteps))
        self.step_count += int(nsteps)

    def observe(self, u_snap: np.ndarray | None = None) -> dict:
        o = Obs()
        snap = None
        if u_snap is not None:
            snap = np.ascontiguousarray(u_snap, dtype=np.float64).reshape(2, -1)
        lib().orc_observe(ctypes.byref(self.geom), ctypes.byref(self.params), _u8(self.mask),
                          _dp(self.f), _dp(self.T), _dp(snap) if snap is not None else None,
                          ctypes.byref(o))
        return {k: getattr(o, k) for k, _ in Obs._fields_}

    def fields(self):
        """Returns u[2, N], p[N], T[N] (zero outside active cells)."""
        N = self.N
        u, p, Tf = np.zeros((2, N)), np.zeros(N), np.zeros(N)
        lib().orc_fields(ctypes.byref(self.geom), _u8(self.mask), _dp(self.f), _dp(self.T),
                         _dp(u), _dp(p), _dp(Tf))
        return u, p, Tf
