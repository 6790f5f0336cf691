"""Python binding of liblagflux (include/lagflux.h).

Argument marshalling only: every step of the scheme runs in the CUDA library.
The functions below carry the C names; `LagrangeFlux` wraps one context for
torch users (device tensors are passed by data_ptr on torch's current stream).
There is no CPU fallback: if the library is missing, importing raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LAGFLUX_LIB selects another build of the same library (e.g. a tuning variant).
LIB_PATH = os.environ.get("LAGFLUX_LIB") or os.path.join(_HERE, "liblagflux.so")

LF_OK, LF_ERR_ARG, LF_ERR_CUDA, LF_ERR_OOM, LF_ERR_NONPHYSICAL, LF_ERR_TIMEOUT, LF_ERR_STATE = range(7)
MAX_SPECIES = 2  # LF_MAX_SPECIES
LIMITERS = {"minmod": 0, "sweby": 1, "vanleer": 2}
BCS = {"transmissive": 0, "periodic": 1}
PRECISIONS = {"fp64": 0, "fp32": 1}
RIEMANN = {"maxc": 0, "per_side": 1}


class lf_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("riemann", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("time_order", ctypes.c_int32),
        ("nspecies", ctypes.c_int32),
        ("xmin", ctypes.c_double),
        ("xmax", ctypes.c_double),
        ("ymin", ctypes.c_double),
        ("ymax", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("nz", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("zmin", ctypes.c_double),
        ("zmax", ctypes.c_double),
    ]


_vp, _i32, _i64, _d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER

# name -> (restype, argtypes); mirrors include/lagflux.h
SIGNATURES = {
    "lf_init": (ctypes.c_int, [_P(lf_config), _vp, _P(_vp)]),
    "lf_destroy": (None, [_vp]),
    "lf_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_set_primitive": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_get_primitive": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_set_conservative": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_get_conservative": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_set_primitives": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_get_primitives": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_set_partial_densities": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_get_partial_densities": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_set_mass_fractions": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_get_mass_fractions": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lf_step": (ctypes.c_int, [_vp, _P(_d)]),
    "lf_step_fixed": (ctypes.c_int, [_vp, _d]),
    "lf_run": (ctypes.c_int, [_vp, _d, _i32, _P(_i32), _P(_d)]),
    "lf_get_time": (ctypes.c_int, [_vp, _P(_d), _P(_i64)]),
    "lf_conservation_sums": (ctypes.c_int, [_vp, _P(_d)]),
    "lf_sync": (ctypes.c_int, [_vp]),
    "lf_set_tile_rows": (ctypes.c_int, [_vp, _i32]),
    "lf_get_tile_rows": (ctypes.c_int, [_vp, _P(_i32)]),
    "lf_autotune": (ctypes.c_int, [_vp, _i32, _P(_i32)]),
    "lf_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lf_profile_read": (ctypes.c_int, [_vp, _P(_d), _P(_i64)]),
    "lf_step_noalloc": (ctypes.c_int, [_P(lf_config), _vp, _vp, _d, _P(_d), _vp]),
    "lf_adjoint_forward": (ctypes.c_int, [_vp, _i32, _P(_d)]),
    "lf_adjoint_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_adjoint": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _P(_d), ctypes.c_int]),
    "lf_adjoint_set_passes": (ctypes.c_int, [_vp, _i32]),
    "lf_batch_init": (ctypes.c_int, [_P(lf_config), _i32, _vp, _P(_vp)]),
    "lf_batch_destroy": (None, [_vp]),
    "lf_batch_set_primitive": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_batch_get_state": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lf_batch_run": (ctypes.c_int, [_vp, _i32, _i32]),
    "lf_batch_autotune": (ctypes.c_int, [_vp, _i32, _P(_i32)]),
    "lf_batch_set_rows": (ctypes.c_int, [_vp, _i32]),
    "lf_batch_get_times": (ctypes.c_int, [_vp, _P(_d), _P(_i64)]),
    "lf_batch_profile": (ctypes.c_int, [_vp, _i32, _P(_d)]),
    "lf_batch_last_error": (ctypes.c_char_p, [_vp]),
    "lf_measure_peak": (ctypes.c_int, [_i32, _i32, _d, _P(_d)]),
    "lf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lf_last_error": (ctypes.c_char_p, [_vp]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"liblagflux.so not built at {path}; run paper_1607_08710_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()
globals().update({name: getattr(_lib, name) for name in SIGNATURES})


class LagrangeFluxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.lf_status_string(status).decode()}: {message}")
        self.status = status


@dataclass
class Config:
    nx: int
    ny: int = 1
    dim: int = 2
    limiter: str = "vanleer"
    bc: str = "transmissive"
    precision: str = "fp64"
    riemann: str = "maxc"
    gamma: float = 1.4
    cfl: float = 0.45
    beta: float = 1.5
    xmin: float = 0.0
    xmax: float = 1.0
    ymin: float = 0.0
    ymax: float = 1.0
    device: int = 0
    time_order: int = 2  # 2: Heun (Sec. 4), 3: SSP-RK3
    nspecies: int = 0  # transported mass fractions (Sec. 5), 0 .. MAX_SPECIES
    nz: int = 1
    zmin: float = 0.0
    zmax: float = 1.0
    tile_rows: int = 0  # rows per tile of the 2D stage kernels; 0: chosen from the mesh and the GPU

    def to_c(self) -> lf_config:
        return lf_config(self.dim, self.nx, self.ny if self.dim >= 2 else 1, LIMITERS[self.limiter], BCS[self.bc],
                         PRECISIONS[self.precision], RIEMANN[self.riemann], self.device, self.time_order,
                         self.nspecies, self.xmin, self.xmax, self.ymin, self.ymax, self.gamma, self.cfl, self.beta,
                         self.nz if self.dim == 3 else 1, self.tile_rows, self.zmin, self.zmax)

    @property
    def nfields(self) -> int:
        """Planes of a whole state: 4 (5 in 3D) + nspecies."""
        return (5 if self.dim == 3 else 4) + self.nspecies

    @property
    def shape(self) -> tuple:
        """Shape of one plane: (ny, nx), or (nz, ny, nx) in 3D."""
        ny = self.ny if self.dim >= 2 else 1
        return (self.nz, ny, self.nx) if self.dim == 3 else (ny, self.nx)

    @property
    def np_dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32


def _ptr_and_kind(a):
    """(pointer, on_device) for a torch tensor or numpy array; None passes NULL."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(a)}")


class LagrangeFlux:
    """One mesh and its state on the GPU, advanced by the Lagrange-flux scheme."""

    def __init__(self, cfg: Config, stream=None):
        self.cfg = cfg
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream(cfg.device).cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        self._stream = stream
        c = cfg.to_c()
        h = ctypes.c_void_p()
        st = _lib.lf_init(ctypes.byref(c), ctypes.c_void_p(stream), ctypes.byref(h))
        if st != LF_OK:
            raise LagrangeFluxError(st, _lib.lf_last_error(None).decode())
        self._h = h

    # -- helpers ---------------------------------------------------------
    def _check(self, st: int):
        if st != LF_OK:
            raise LagrangeFluxError(st, _lib.lf_last_error(self._h).decode())

    def _planes(self, planes, expect_device=None):
        ptrs, kinds = [], set()
        n = self.cfg.nx * (self.cfg.ny if self.cfg.dim == 2 else 1)
        for a in planes:
            p, k = _ptr_and_kind(a)
            if a is not None:
                if int(np.prod(a.shape)) != n:
                    raise ValueError(f"plane has {int(np.prod(a.shape))} elements, expected {n}")
                kinds.add(k)
                self._check_dtype(a)
            ptrs.append(p)
        if len(kinds) != 1:
            raise ValueError("all planes must be on the same side (all host or all device)")
        return ptrs, kinds.pop()

    def _check_dtype(self, a):
        want = self.cfg.np_dtype
        if isinstance(a, np.ndarray):
            ok = a.dtype == want
        else:
            import torch

            ok = a.dtype == (torch.float64 if want == np.float64 else torch.float32)
        if not ok:
            raise TypeError(f"buffer dtype {a.dtype} does not match precision {self.cfg.precision}")

    # -- API -------------------------------------------------------------
    def set_state(self, rho, rhou, rhov, rhoE):
        p, k = self._planes([rho, rhou, rhov, rhoE])
        self._check(_lib.lf_set_state(self._h, *p, k))

    def set_primitive(self, rho, u, v, p):
        ptrs, k = self._planes([rho, u, v, p])
        self._check(_lib.lf_set_primitive(self._h, *ptrs, k))

    def get_state(self, out=None):
        """Conservative state as (4, ny, nx); `out` may be a torch CUDA tensor or numpy array."""
        if out is None:
            ny = self.cfg.ny if self.cfg.dim == 2 else 1
            out = np.empty((4, ny, self.cfg.nx), dtype=self.cfg.np_dtype)
        ptrs, k = self._planes([out[0], out[1], out[2], out[3]])
        self._check(_lib.lf_get_state(self._h, *ptrs, k))
        return out

    def get_primitive(self, out=None):
        if out is None:
            ny = self.cfg.ny if self.cfg.dim == 2 else 1
            out = np.empty((4, ny, self.cfg.nx), dtype=self.cfg.np_dtype)
        ptrs, k = self._planes([out[0], out[1], out[2], out[3]])
        self._check(_lib.lf_get_primitive(self._h, *ptrs, k))
        return out

    # -- whole-state transfers (any dim, species included) ---------------
    def _state_buffer(self, a):
        n = self.cfg.nfields * int(np.prod(self.cfg.shape))
        p, k = _ptr_and_kind(a)
        if int(np.prod(a.shape)) != n:
            raise ValueError(f"state buffer has {int(np.prod(a.shape))} elements, expected {n}")
        self._check_dtype(a)
        return p, k

    def _state_out(self, out):
        return np.empty((self.cfg.nfields,) + self.cfg.shape, dtype=self.cfg.np_dtype) if out is None else out

    def set_conservative(self, U):
        """U: (nfields,) + shape conservative planes (rho, rho u, rho v, [rho w,] rho E, rho y_k)."""
        p, k = self._state_buffer(U)
        self._check(_lib.lf_set_conservative(self._h, p, k))

    def get_conservative(self, out=None):
        out = self._state_out(out)
        p, k = self._state_buffer(out)
        self._check(_lib.lf_get_conservative(self._h, p, k))
        return out

    def set_primitives(self, q):
        """q: (nfields,) + shape primitive planes (rho, u, v, [w,] p, y_k)."""
        p, k = self._state_buffer(q)
        self._check(_lib.lf_set_primitives(self._h, p, k))

    def get_primitives(self, out=None):
        out = self._state_out(out)
        p, k = self._state_buffer(out)
        self._check(_lib.lf_get_primitives(self._h, p, k))
        return out

    # -- species (Sec. 5) -------------------------------------------------
    def _species_buffer(self, a):
        n = self.cfg.nspecies * int(np.prod(self.cfg.shape))
        p, k = _ptr_and_kind(a)
        if int(np.prod(a.shape)) != n:
            raise ValueError(f"species buffer has {int(np.prod(a.shape))} elements, expected {n}")
        self._check_dtype(a)
        return p, k

    def _species_out(self, out):
        if out is None:
            out = np.empty((self.cfg.nspecies,) + self.cfg.shape, dtype=self.cfg.np_dtype)
        return out

    def set_partial_densities(self, rho_y):
        """rho_y: (nspecies,) + shape partial densities rho y_k."""
        p, k = self._species_buffer(rho_y)
        self._check(_lib.lf_set_partial_densities(self._h, p, k))

    def get_partial_densities(self, out=None):
        out = self._species_out(out)
        p, k = self._species_buffer(out)
        self._check(_lib.lf_get_partial_densities(self._h, p, k))
        return out

    def set_mass_fractions(self, y):
        """y: (nspecies,) + shape mass fractions; rho y_k uses the current density."""
        p, k = self._species_buffer(y)
        self._check(_lib.lf_set_mass_fractions(self._h, p, k))

    def get_mass_fractions(self, out=None):
        out = self._species_out(out)
        p, k = self._species_buffer(out)
        self._check(_lib.lf_get_mass_fractions(self._h, p, k))
        return out

    def step(self, return_dt: bool = False):
        if return_dt:
            dt = ctypes.c_double()
            self._check(_lib.lf_step(self._h, ctypes.byref(dt)))
            return dt.value
        self._check(_lib.lf_step(self._h, None))
        return None

    def step_fixed(self, dt: float):
        self._check(_lib.lf_step_fixed(self._h, float(dt)))

    def run(self, t_end: float = 0.0, max_steps: int = 2**31 - 1):
        n = ctypes.c_int32()
        t = ctypes.c_double()
        self._check(_lib.lf_run(self._h, float(t_end), int(max_steps), ctypes.byref(n), ctypes.byref(t)))
        return n.value, t.value

    def time(self):
        t, s = ctypes.c_double(), ctypes.c_int64()
        self._check(_lib.lf_get_time(self._h, ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def conservation_sums(self) -> np.ndarray:
        """FP64 sums of the nfields conservative fields."""
        out = (ctypes.c_double * self.cfg.nfields)()
        self._check(_lib.lf_conservation_sums(self._h, out))
        return np.array(out[:])

    def profile(self, enable: bool = True):
        """Start (or stop) per-stage event timing; enabling resets the totals."""
        self._check(_lib.lf_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """((ms_predictor, ms_corrector), (launches_predictor, launches_corrector))."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_int64 * 2)()
        self._check(_lib.lf_profile_read(self._h, ms, n))
        return (ms[0], ms[1]), (n[0], n[1])

    def sync(self):
        self._check(_lib.lf_sync(self._h))

    # -- launch shape ------------------------------------------------------
    @property
    def tile_rows(self) -> int:
        """Rows per tile of the y-march (2D) or planes per z-tile (3D); 0 in 1D."""
        r = ctypes.c_int32()
        self._check(_lib.lf_get_tile_rows(self._h, ctypes.byref(r)))
        return r.value

    @tile_rows.setter
    def tile_rows(self, rows: int):
        self._check(_lib.lf_set_tile_rows(self._h, int(rows)))

    def autotune(self, trial_steps: int = 3) -> int:
        """Times the candidate tile heights on the current state (which is left
        unchanged), keeps the fastest and returns it."""
        r = ctypes.c_int32()
        self._check(_lib.lf_autotune(self._h, int(trial_steps), ctypes.byref(r)))
        return r.value

    # -- discrete adjoint ------------------------------------------------
    def adjoint_forward(self, nsteps: int) -> np.ndarray:
        """nsteps CFL steps with sqrt(N) checkpoints; returns the frozen dt sequence."""
        dts = np.zeros(nsteps)
        self._check(_lib.lf_adjoint_forward(self._h, int(nsteps), dts.ctypes.data_as(_P(_d))))
        return dts

    def _adjoint_buffers(self, bufs):
        """Pointers and the common side (host/device) of the adjoint buffers,
        each 4 * nx * ny values of the configured precision."""
        n = 4 * self.cfg.nx * self.cfg.ny
        ptrs, kinds = [], set()
        for a in bufs:
            p, k = _ptr_and_kind(a)
            if a is not None:
                if int(np.prod(a.shape)) != n:
                    raise ValueError(f"adjoint buffer has {int(np.prod(a.shape))} elements, expected {n}")
                self._check_dtype(a)
                kinds.add(k)
            ptrs.append(p)
        if len(kinds) != 1:
            raise ValueError("adjoint buffers must all be on the host or all on the device")
        return ptrs, kinds.pop()

    def adjoint_backward(self, lambda_T, grad_U0=None, grad_q0=None):
        """lambda_T: (4, ny, nx) dJ/dU(T), a contiguous CUDA tensor or host
        array.  Fills the given buffers (on the same side) with dJ/dU(0)
        and/or dJ/d(rho, u, v, p)(0)."""
        (pl, pu, pq), k = self._adjoint_buffers([lambda_T, grad_U0, grad_q0])
        self._check(_lib.lf_adjoint_backward(self._h, pl, pu, pq, k))

    def adjoint(self, nsteps: int, lambda_T, grad_U0=None, grad_q0=None) -> np.ndarray:
        """Forward run of nsteps with checkpoints, then the reverse sweep from
        the given lambda_T, in one call (lf_adjoint); returns the dt sequence."""
        (pl, pu, pq), k = self._adjoint_buffers([lambda_T, grad_U0, grad_q0])
        dts = np.zeros(nsteps)
        self._check(_lib.lf_adjoint(self._h, int(nsteps), pl, pu, pq, dts.ctypes.data_as(_P(_d)), k))
        return dts

    ADJOINT_PASSES = {"auto": 0, "tables": 1, "direct": 2}

    def set_adjoint_passes(self, passes: str):
        """'tables', 'direct' or 'auto' (tables in FP64, direct in FP32)."""
        self._check(_lib.lf_adjoint_set_passes(self._h, self.ADJOINT_PASSES[passes]))

    def close(self):
        if getattr(self, "_h", None):
            _lib.lf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class LagrangeFluxBatch:
    """Many independent 2D meshes advanced together (one persistent launch per stage)."""

    def __init__(self, cfgs, stream=None):
        if not cfgs:
            raise ValueError("need at least one problem")
        self.cfgs = list(cfgs)
        if stream is None:
            try:
                import torch

                stream = torch.cuda.current_stream(cfgs[0].device).cuda_stream if torch.cuda.is_available() else 0
            except ImportError:
                stream = 0
        arr = (lf_config * len(self.cfgs))(*[c.to_c() for c in self.cfgs])
        h = ctypes.c_void_p()
        st = _lib.lf_batch_init(arr, len(self.cfgs), ctypes.c_void_p(stream), ctypes.byref(h))
        if st != LF_OK:
            raise LagrangeFluxError(st, _lib.lf_batch_last_error(None).decode())
        self._h = h

    def _check(self, st: int):
        if st != LF_OK:
            raise LagrangeFluxError(st, _lib.lf_batch_last_error(self._h).decode())

    def _planes(self, p, planes):
        c = self.cfgs[p]
        n = c.nx * c.ny
        ptrs, kinds = [], set()
        for a in planes:
            ptr, k = _ptr_and_kind(a)
            if int(np.prod(a.shape)) != n:
                raise ValueError(f"problem {p}: plane has {int(np.prod(a.shape))} elements, expected {n}")
            ptrs.append(ptr)
            kinds.add(k)
        if len(kinds) != 1:
            raise ValueError("all planes must be on the same side (all host or all device)")
        return ptrs, kinds.pop()

    def set_primitive(self, p, rho, u, v, pr):
        ptrs, k = self._planes(p, [rho, u, v, pr])
        self._check(_lib.lf_batch_set_primitive(self._h, p, *ptrs, k))

    def get_state(self, p, out=None):
        c = self.cfgs[p]
        if out is None:
            out = np.empty((4, c.ny, c.nx), dtype=c.np_dtype)
        ptrs, k = self._planes(p, [out[0], out[1], out[2], out[3]])
        self._check(_lib.lf_batch_get_state(self._h, p, *ptrs, k))
        return out

    def run(self, nsteps: int, use_graph: bool = True):
        self._check(_lib.lf_batch_run(self._h, int(nsteps), 1 if use_graph else 0))

    def autotune(self, trial_steps: int = 3) -> int:
        rows = ctypes.c_int32()
        self._check(_lib.lf_batch_autotune(self._h, int(trial_steps), ctypes.byref(rows)))
        return rows.value

    def set_rows(self, rows: int):
        self._check(_lib.lf_batch_set_rows(self._h, int(rows)))

    def times(self):
        n = len(self.cfgs)
        t = (ctypes.c_double * n)()
        s = (ctypes.c_int64 * n)()
        self._check(_lib.lf_batch_get_times(self._h, t, s))
        return np.array(t[:]), np.array(s[:])

    def profile(self, nsteps: int):
        """nsteps direct-launch steps with per-stage CUDA events; returns the
        summed (predictor, corrector) device times in ms (lf_batch_profile)."""
        ms = (ctypes.c_double * 2)()
        self._check(_lib.lf_batch_profile(self._h, int(nsteps), ms))
        return ms[0], ms[1]

    def close(self):
        if getattr(self, "_h", None):
            _lib.lf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PEAK_KINDS = {"fp64": 0, "fp32": 1, "fp32_paired": 2}


def measure_peak(kind: str, device: int = 0, target_ms: float = 30.0) -> float:
    """Measured fused multiply-add throughput (TFLOP/s) of `kind` ('fp64',
    'fp32' or 'fp32_paired') on `device` (lf_measure_peak)."""
    r = ctypes.c_double()
    st = _lib.lf_measure_peak(int(device), PEAK_KINDS[kind], float(target_ms), ctypes.byref(r))
    if st != LF_OK:
        raise LagrangeFluxError(st, _lib.lf_last_error(None).decode())
    return r.value


def _autograd_function():
    import torch

    class LagrangeFluxRun(torch.autograd.Function):
        """(rho0, u0, v0, p0) -> conservative state after `nsteps` CFL steps.

        The forward records the dt sequence and sqrt(N) checkpoints; the
        backward is the discrete adjoint with that dt sequence frozen."""

        @staticmethod
        def forward(ctx, rho0, u0, v0, p0, solver, nsteps):
            solver.set_primitive(rho0.contiguous(), u0.contiguous(), v0.contiguous(), p0.contiguous())
            solver.adjoint_forward(nsteps)
            c = solver.cfg
            U = torch.empty((4, c.ny, c.nx), dtype=rho0.dtype, device=rho0.device)
            solver.get_state(U)
            ctx.solver = solver
            return U

        @staticmethod
        def backward(ctx, gU):
            s = ctx.solver
            gq = torch.empty_like(gU)
            s.adjoint_backward(gU.contiguous(), grad_q0=gq)
            return gq[0], gq[1], gq[2], gq[3], None, None

    return LagrangeFluxRun


def run_differentiable(solver: "LagrangeFlux", rho0, u0, v0, p0, nsteps: int):
    """Differentiable run: returns the (4, ny, nx) conservative state after
    nsteps steps; gradients flow back to the primitive initial fields."""
    return _autograd_function().apply(rho0, u0, v0, p0, solver, nsteps)
