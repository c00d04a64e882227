"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/liblbm.so``; this
module only builds the C structs, allocates the caller-owned device buffers
with PyTorch and passes the current CUDA stream.  There is no CPU fallback:
if the library is not built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
PRECISIONS = {"f64": F64, "f32": F32, "f16": F16DEV, "bf16": BF16DEV,
              "f16dev": F16DEV, "bf16dev": BF16DEV}
GEOM_EYE, GEOM_MASK = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, EUNSTABLE, EBUSY = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONVERGED", "EUNSTABLE", "EBUSY"]


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")
        self.status = status


class GeometryDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("kind", ctypes.c_int32),
        ("band_cells", ctypes.c_int32), ("inlet_cells", ctypes.c_int32),
        ("tm_w", ctypes.c_int32), ("tm_h", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("inlet_dir_x", ctypes.c_int32), ("inlet_dir_y", ctypes.c_int32),
        ("inlet_profile", ctypes.c_int32), ("inlet_lo", ctypes.c_int32),
        ("inlet_width", ctypes.c_int32),
        ("chamber_angle_deg", ctypes.c_double),
        ("host_mask", ctypes.POINTER(ctypes.c_uint8)),
    ]


class GeometryInfo(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int64), ("n_active", ctypes.c_int64), ("n_fluid", ctypes.c_int64),
        ("n_porous", ctypes.c_int64), ("n_inlet", ctypes.c_int64), ("n_outlet", ctypes.c_int64),
        ("inlet_dir_x", ctypes.c_int32), ("inlet_dir_y", ctypes.c_int32),
        ("inlet_profile", ctypes.c_int32), ("inlet_lo", ctypes.c_int32),
        ("inlet_width", ctypes.c_int32), ("eye_normals", ctypes.c_int32),
        ("outlet_axis", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("arc_xc", ctypes.c_double), ("arc_yc", ctypes.c_double), ("arc_r", ctypes.c_double),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("tau_T", ctypes.c_double), ("g_beta", ctypes.c_double),
        ("g_dir", ctypes.c_double * 2),
        ("T_cold", ctypes.c_double), ("T_hot", ctypes.c_double), ("T0", ctypes.c_double),
        ("T_in", ctypes.c_double), ("u_in_max", ctypes.c_double), ("K_tm", ctypes.c_double),
        ("porosity", ctypes.c_double), ("p_out", ctypes.c_double),
        ("drive", ctypes.c_double * 2), ("noise_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("dx_m", ctypes.c_double), ("dt_s", ctypes.c_double), ("rho0", ctypes.c_double),
        ("p_sc_pa", ctypes.c_double),
        ("tm_model", ctypes.c_int32), ("bouzidi", ctypes.c_int32), ("h_tm", ctypes.c_double),
    ]


class Observables(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("iop", ctypes.c_double), ("iop_pa", ctypes.c_double),
        ("q_in", ctypes.c_double), ("q_out", ctypes.c_double), ("mass", ctypes.c_double),
        ("peak_speed", ctypes.c_double), ("wss_cornea", ctypes.c_double),
        ("wss_iris", ctypes.c_double), ("wss_cornea_pa", ctypes.c_double),
        ("wss_iris_pa", ctypes.c_double), ("residual", ctypes.c_double),
        ("n_fluid", ctypes.c_int64), ("n_cornea", ctypes.c_int64), ("n_iris", ctypes.c_int64),
        ("nan_flag", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("u_seep", ctypes.c_double),
    ]


class VortexInfo(ctypes.Structure):
    _fields_ = [("intensity", ctypes.c_double), ("intensity_abs", ctypes.c_double),
                ("intensity_phys", ctypes.c_double), ("intensity_abs_phys", ctypes.c_double),
                ("psi_max", ctypes.c_double), ("psi_min", ctypes.c_double),
                ("max_x", ctypes.c_int32), ("max_y", ctypes.c_int32),
                ("min_x", ctypes.c_int32), ("min_y", ctypes.c_int32),
                ("max_mm", ctypes.c_double * 2), ("min_mm", ctypes.c_double * 2),
                ("n_fluid", ctypes.c_int64)]


# lbm_launch.stepping
STEP_PER_LAUNCH = 0    # one launch per step (CUDA-graph replay); the default
STEP_FLOW = 1          # one cooperative dataflow launch for many steps


class Launch(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("block_rows", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("stepping", ctypes.c_int32), ("sweep_steps", ctypes.c_int32),
                ("sweep_lag", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load liblbm.so.  Raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError("liblbm.so is not built: call __graft_entry__.build() "
                               "(or paper_2102_12663_gb300._build.build()) first")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    dom = ctypes.c_void_p
    P = ctypes.POINTER
    sigs = {
        "lbm_build_mask": (i32, [P(GeometryDesc), P(ctypes.c_uint8), P(GeometryInfo)]),
        "lbm_domain_bytes": (sz, [P(GeometryDesc), i32]),
        "lbm_create_domain": (i32, [P(GeometryDesc), i32, vp, sz, vp, P(dom)]),
        "lbm_set_params": (i32, [dom, P(Params)]),
        "lbm_reset_state": (i32, [dom]),
        "lbm_step": (i32, [dom, i64]),
        "lbm_run_to_steady": (i32, [dom, dbl, i32, i64, P(i64)]),
        "lbm_read_observables": (i32, [dom, P(Observables)]),
        "lbm_read_observables_noalloc": (i32, [dom, P(Observables)]),
        "lbm_read_field": (i32, [dom, vp, vp, vp]),
        "lbm_vortex": (i32, [dom, vp, P(VortexInfo)]),
        "lbm_read_populations": (i32, [dom, vp, vp]),
        "lbm_write_populations": (i32, [dom, vp, vp]),
        "lbm_state_bytes": (sz, [dom]),
        "lbm_save_state": (i32, [dom, vp, sz]),
        "lbm_load_state": (i32, [dom, vp, sz]),
        "lbm_set_launch": (i32, [dom, P(Launch)]),
        "lbm_get_launch": (i32, [dom, P(Launch)]),
        "lbm_get_step": (i64, [dom]),
        "lbm_debug_stall_tile": (i32, [dom, i32]),
        "lbm_get_info": (i32, [dom, P(GeometryInfo)]),
        "lbm_get_tile_count": (i64, [dom]),
        "lbm_get_edge_cell_count": (i64, [dom]),
        "lbm_step_bytes": (dbl, [dom]),
        "lbm_destroy_domain": (None, [dom]),
        "lbm_batch_bytes": (sz, [i32, i64]),
        "lbm_batch_create": (i32, [i32, i32, i64, P(Launch), vp, sz, vp, P(vp)]),
        "lbm_batch_add": (i32, [vp, dom]),
        "lbm_batch_remove": (i32, [vp, dom]),
        "lbm_batch_size": (i32, [vp]),
        "lbm_batch_step": (i32, [vp, i64]),
        "lbm_batch_check": (i32, [vp, i32]),
        "lbm_last_observables": (i32, [dom, P(Observables)]),
        "lbm_batch_set_launch": (i32, [vp, P(Launch)]),
        "lbm_batch_get_launch": (i32, [vp, P(Launch)]),
        "lbm_batch_tune": (i32, [vp, i32, P(Launch)]),
        "lbm_batch_step_bytes": (dbl, [vp]),
        "lbm_batch_active_cells": (i64, [vp]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int) -> None:
    if status != OK:
        raise LBMError(status, load().lbm_last_error().decode())


def _u8ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def geometry_desc(geometry: dict):
    """Build a GeometryDesc from a dict.  Keys: either ``kind='eye'`` with nx,
    ny, angle_deg (and optional band_cells, inlet_cells, tm_w, tm_h), or
    ``mask`` (uint8[ny, nx]) with periodic_x, periodic_y, inlet_dir,
    inlet_profile, inlet_lo, inlet_width.  Returns (desc, keepalive)."""
    g = GeometryDesc()
    keep = None
    if "mask" in geometry:
        m = np.ascontiguousarray(geometry["mask"], dtype=np.uint8)
        ny, nx = m.shape
        g.nx, g.ny, g.kind = nx, ny, GEOM_MASK
        g.periodic_x = int(geometry.get("periodic_x", 0))
        g.periodic_y = int(geometry.get("periodic_y", 0))
        d = geometry.get("inlet_dir", (0, 1))
        g.inlet_dir_x, g.inlet_dir_y = int(d[0]), int(d[1])
        g.inlet_profile = int(geometry.get("inlet_profile", 0))
        g.inlet_lo = int(geometry.get("inlet_lo", 0))
        g.inlet_width = int(geometry.get("inlet_width", 1))
        g.host_mask = _u8ptr(m)
        keep = m
    else:
        g.nx, g.ny, g.kind = int(geometry["nx"]), int(geometry["ny"]), GEOM_EYE
        g.chamber_angle_deg = float(geometry.get("angle_deg", 45.0))
        g.band_cells = int(geometry.get("band_cells", 0))
        g.inlet_cells = int(geometry.get("inlet_cells", 0))
        g.tm_w = int(geometry.get("tm_w", 0))
        g.tm_h = int(geometry.get("tm_h", 0))
    return g, keep


def build_mask(geometry: dict):
    """Host-only mask builder: returns (mask uint8[ny, nx], info dict)."""
    L = load()
    g, keep = geometry_desc(geometry)
    out = np.zeros((g.ny, g.nx), dtype=np.uint8)
    info = GeometryInfo()
    check(L.lbm_build_mask(ctypes.byref(g), _u8ptr(out), ctypes.byref(info)))
    return out, {k: getattr(info, k) for k, _ in GeometryInfo._fields_}


def make_params(p: dict) -> Params:
    P = Params()
    P.tau = p.get("tau", 1.0)
    P.tau_T = p.get("tau_T", 1.0)
    P.g_beta = p.get("g_beta", 0.0)
    gd = p.get("g_dir", (0.0, -1.0))
    P.g_dir[0], P.g_dir[1] = float(gd[0]), float(gd[1])
    P.T_cold = p.get("T_cold", 0.0)
    P.T_hot = p.get("T_hot", 0.0)
    P.T0 = p.get("T0", 0.0)
    P.T_in = p.get("T_in", 0.0)
    P.u_in_max = p.get("u_in_max", 0.0)
    P.K_tm = p.get("K_tm", p.get("K", 1.0))
    P.porosity = p.get("porosity", 0.3)
    P.p_out = p.get("p_out", 0.0)
    dr = p.get("drive", (0.0, 0.0))
    P.drive[0], P.drive[1] = float(dr[0]), float(dr[1])
    P.noise_amp = p.get("noise_amp", 0.0)
    P.seed = int(p.get("seed", 0)) & (2**64 - 1)
    P.dx_m = p.get("dx_m", 0.0)
    P.dt_s = p.get("dt_s", 0.0)
    P.rho0 = p.get("rho0", 0.0)
    P.p_sc_pa = p.get("p_sc_pa", 0.0)
    P.tm_model = int(p.get("tm_model", 0))
    P.bouzidi = int(p.get("bouzidi", 0))
    P.h_tm = float(p.get("h_tm", 0.0))
    return P


def _torch():
    import torch
    return torch


class Domain:
    """One problem instance whose state lives in a caller-owned torch buffer."""

    def __init__(self, geometry: dict, precision="f32", device=None, stream=None):
        torch = _torch()
        L = load()
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = torch.device(device if device is not None else "cuda")
        g, keep = geometry_desc(geometry)
        self.nx, self.ny = g.nx, g.ny
        nbytes = L.lbm_domain_bytes(ctypes.byref(g), self.precision)
        if nbytes == 0:
            raise LBMError(EINVAL, "invalid geometry or precision")
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        check(L.lbm_create_domain(ctypes.byref(g), self.precision,
                                  ctypes.c_void_p(self.buf.data_ptr()), self.nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        del keep
        self._h = h
        self._L = L

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.lbm_destroy_domain(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- parameters and stepping ------------------------------------------
    def set_params(self, params: dict):
        self._params = dict(params)
        check(self._L.lbm_set_params(self._h, ctypes.byref(make_params(params))))

    def reset(self):
        check(self._L.lbm_reset_state(self._h))

    def step(self, n: int = 1):
        check(self._L.lbm_step(self._h, int(n)))

    def run_to_steady(self, tol: float, check_every: int = 100, max_steps: int = 10**6):
        """Returns (status, steps); status OK or ENOTCONVERGED (others raise)."""
        steps = ctypes.c_int64()
        st = self._L.lbm_run_to_steady(self._h, float(tol), int(check_every), int(max_steps),
                                       ctypes.byref(steps))
        if st not in (OK, ENOTCONVERGED):
            check(st)
        return st, steps.value

    @property
    def step_count(self) -> int:
        return int(self._L.lbm_get_step(self._h))

    # -- read-back ----------------------------------------------------------
    def observables(self) -> dict:
        o = Observables()
        check(self._L.lbm_read_observables(self._h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Observables._fields_}

    def observables_noalloc(self) -> dict:
        """Same as observables(), with the library's own reduction scratch."""
        o = Observables()
        check(self._L.lbm_read_observables_noalloc(self._h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Observables._fields_}

    def last_observables(self) -> dict:
        """Observables of the last steady-state check of this domain
        (run_to_steady or a batch check): a host copy, no device work."""
        o = Observables()
        check(self._L.lbm_last_observables(self._h, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Observables._fields_}

    def fields(self):
        """(u[2, ny, nx], p[ny, nx], T[ny, nx]) float64 device tensors."""
        torch = _torch()
        u = torch.empty((2, self.ny, self.nx), dtype=torch.float64, device=self.device)
        p = torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
        T = torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
        check(self._L.lbm_read_field(self._h, ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(T.data_ptr())))
        return u, p, T

    def vortex(self, u=None) -> dict:
        """Vortex intensity and centres (Eq. 18, Tab. 3) of the device velocity
        field u[2, ny, nx] (float64; default: the current state's, from
        fields())."""
        if u is None:
            u = self.fields()[0]
        torch = _torch()
        assert u.dtype == torch.float64 and u.is_cuda and u.is_contiguous()
        assert tuple(u.shape) == (2, self.ny, self.nx)
        o = VortexInfo()
        check(self._L.lbm_vortex(self._h, ctypes.c_void_p(u.data_ptr()), ctypes.byref(o)))
        out = {k: getattr(o, k) for k, _ in VortexInfo._fields_}
        out["max_mm"] = tuple(o.max_mm)
        out["min_mm"] = tuple(o.min_mm)
        return out

    def populations(self):
        """(f[9, ny, nx], g[4, ny, nx]) float64 device tensors, natural order."""
        torch = _torch()
        f = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
        g = torch.empty((4, self.ny, self.nx), dtype=torch.float64, device=self.device)
        check(self._L.lbm_read_populations(self._h, ctypes.c_void_p(f.data_ptr()),
                                           ctypes.c_void_p(g.data_ptr())))
        return f, g

    def write_populations(self, f, g):
        torch = _torch()
        f = torch.as_tensor(f, dtype=torch.float64, device=self.device).contiguous()
        g = torch.as_tensor(g, dtype=torch.float64, device=self.device).contiguous()
        check(self._L.lbm_write_populations(self._h, ctypes.c_void_p(f.data_ptr()),
                                            ctypes.c_void_p(g.data_ptr())))
        self.stream.synchronize()

    def save_state(self) -> bytes:
        n = int(self._L.lbm_state_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        check(self._L.lbm_save_state(self._h, ctypes.cast(buf, ctypes.c_void_p), n))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(self._L.lbm_load_state(self._h, ctypes.cast(buf, ctypes.c_void_p), len(blob)))

    # -- launch shape and introspection -----------------------------------
    def set_launch(self, tile_w=128, block_rows=2, rows_per_thread=1, blocks_per_sm=0,
                   stepping=STEP_PER_LAUNCH, sweep_steps=1, sweep_lag=0):
        check(self._L.lbm_set_launch(self._h, ctypes.byref(
            Launch(tile_w, block_rows, rows_per_thread, blocks_per_sm, stepping, sweep_steps,
                   sweep_lag))))

    def get_launch(self) -> dict:
        l = Launch()
        check(self._L.lbm_get_launch(self._h, ctypes.byref(l)))
        return {k: getattr(l, k) for k, _ in Launch._fields_}

    def debug_stall_tile(self, tile: int):
        """Test hook: dataflow launches never report `tile` complete (-1: off)."""
        check(self._L.lbm_debug_stall_tile(self._h, int(tile)))

    def info(self) -> dict:
        i = GeometryInfo()
        check(self._L.lbm_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in GeometryInfo._fields_}

    def tile_count(self) -> int:
        return int(self._L.lbm_get_tile_count(self._h))

    def edge_cell_count(self) -> int:
        """Cells that plain steps update in edge-cell blocks (0: none)."""
        return int(self._L.lbm_get_edge_cell_count(self._h))

    def step_bytes(self) -> float:
        return float(self._L.lbm_step_bytes(self._h))


def _launch_dict(l: Launch) -> dict:
    return {k: getattr(l, k) for k, _ in Launch._fields_}


class Batch:
    """Many domains of one precision advanced by one launch per time step."""

    def __init__(self, precision="f32", max_instances=64, max_tiles=1 << 20, launch=None,
                 device=None, stream=None):
        torch = _torch()
        L = load()
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = int(L.lbm_batch_bytes(int(max_instances), int(max_tiles)))
        if nbytes == 0:
            raise LBMError(EINVAL, "invalid batch capacity")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        lp = ctypes.byref(Launch(**launch)) if launch else None
        h = ctypes.c_void_p()
        check(L.lbm_batch_create(self.precision, int(max_instances), int(max_tiles), lp,
                                 ctypes.c_void_p(self.buf.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h, self._L = h, L
        self.members = []

    def add(self, dom: Domain):
        check(self._L.lbm_batch_add(self._h, dom.handle))
        self.members.append(dom)

    def remove(self, dom: Domain):
        check(self._L.lbm_batch_remove(self._h, dom.handle))
        self.members.remove(dom)

    def __len__(self):
        return int(self._L.lbm_batch_size(self._h))

    def step(self, n: int = 1):
        check(self._L.lbm_batch_step(self._h, int(n)))

    def check(self, check_every: int = 100):
        check(self._L.lbm_batch_check(self._h, int(check_every)))

    def set_launch(self, **launch):
        check(self._L.lbm_batch_set_launch(self._h, ctypes.byref(Launch(**launch))))

    def get_launch(self) -> dict:
        l = Launch()
        check(self._L.lbm_batch_get_launch(self._h, ctypes.byref(l)))
        return _launch_dict(l)

    def tune(self, steps_per_candidate: int = 20) -> dict:
        l = Launch()
        check(self._L.lbm_batch_tune(self._h, int(steps_per_candidate), ctypes.byref(l)))
        return _launch_dict(l)

    def step_bytes(self) -> float:
        return float(self._L.lbm_batch_step_bytes(self._h))

    def active_cells(self) -> int:
        return int(self._L.lbm_batch_active_cells(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.lbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
