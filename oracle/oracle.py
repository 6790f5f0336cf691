"""ctypes front end of the FP64 CPU oracle (lagflux_oracle.cpp).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain reference of the
Lagrange-flux scheme (arXiv:1607.08710, Sec. 4 and 4.1) that the CUDA path is
checked against.  Only tests, the smoke check and the CPU-baseline leg of the
benchmark may import this module; the product package never does.

Arrays use the oracle's own layout: a state is a float64 array of shape
(4 + nspecies, ny, nx) holding (rho, rho u, rho v, rho E, rho y_1 ..) -- or
(rho, u, v, p, y_1 ..) for primitive states -- with x fastest.  1D problems
have ny == 1.  3D states have shape (5 + nspecies, nz, ny, nx) and hold
(rho, rho u, rho v, rho w, rho E, rho y_1 ..) or (rho, u, v, w, p, y_1 ..).

Parity status of each function (see the pins in tests/test_oracle_*.py):
  limiter, interface_solve, face_flux, prim/cons, dt, residual, run,
  run_tangent -- all pinned (closed forms, invariants, exact Riemann
  solutions, convergence order, finite differences).  Species transport
  (nspecies > 0, Sec. 5) is pinned by the constant-fraction and
  complementary-fraction invariants, bitwise independence of the gas
  dynamics, second-order convergence of uniform-flow advection to the exact
  translation and the maximum principle (tests/test_oracle_species.py).  The scheme's exact
  numerical values on the paper's shock tubes are not printed in the paper
  (figures lost), so no stored value pins them; the invariants above do.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lagflux_oracle.cpp")
_LIB = os.path.join(_HERE, "liblagflux_oracle.so")
_lock = threading.Lock()
_lib = None

LIMITERS = {"minmod": 0, "sweby": 1, "vanleer": 2}
BCS = {"transmissive": 0, "periodic": 1}
RIEMANN = {"maxc": 0, "per_side": 1}
OK, NONPHYSICAL, ARG = 0, 1, 2


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("riemann", ctypes.c_int32),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("time_order", ctypes.c_int32),
        ("nspecies", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("dz", ctypes.c_double),
    ]


@dataclass
class OracleConfig:
    """Problem description for the oracle (unit square / unit interval by default)."""

    nx: int
    ny: int = 1
    dim: int = 2
    limiter: str = "vanleer"
    bc: str = "transmissive"
    riemann: str = "maxc"
    gamma: float = 1.4
    cfl: float = 0.45
    beta: float = 1.5
    lx: float = 1.0
    ly: float = 1.0
    time_order: int = 2  # 2: Heun (Sec. 4), 3: third-order SSP Runge-Kutta
    nspecies: int = 0  # transported mass fractions y_k (Sec. 5)
    nz: int = 1
    lz: float = 1.0

    @property
    def nfields(self) -> int:
        return (5 if self.dim == 3 else 4) + self.nspecies

    @property
    def shape(self) -> tuple:
        """Shape of one plane: (ny, nx), or (nz, ny, nx) in 3D."""
        ny = self.ny if self.dim >= 2 else 1
        return (self.nz, ny, self.nx) if self.dim == 3 else (ny, self.nx)

    def to_c(self) -> _Cfg:
        ny = self.ny if self.dim >= 2 else 1
        nz = self.nz if self.dim == 3 else 1
        return _Cfg(
            self.dim, self.nx, ny, LIMITERS[self.limiter], BCS[self.bc], RIEMANN[self.riemann],
            self.lx / self.nx, self.ly / ny if self.dim >= 2 else 1.0, self.gamma, self.cfl, self.beta,
            self.time_order, self.nspecies, nz, 0, self.lz / nz if self.dim == 3 else 1.0,
        )


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


_LIB_OMP = os.path.join(_HERE, "liblagflux_oracle_omp.so")


def build_omp(force: bool = False) -> str:
    """The same source compiled with -fopenmp: the timing build that runs the
    oracle's cell and face loops on all host cores (same bits as build())."""
    with _lock:
        if not force and os.path.exists(_LIB_OMP) and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC):
            return _LIB_OMP
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_OMP)
        return _LIB_OMP


def threads(n: int = 0) -> int:
    """Sets (n > 0) and returns the thread count of the loaded oracle build."""
    return int(_load().oracle_threads(int(n)))


def _declare(lib):
    P = ctypes.POINTER
    d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    pd = P(d)
    lib.oracle_limiter.argtypes = [P(_Cfg), i64, pd, pd, pd]
    lib.oracle_interface_solve.argtypes = [P(_Cfg), i64, pd, pd, pd, pd]
    lib.oracle_face_flux.argtypes = [P(_Cfg), ctypes.c_int, i64, pd, pd, pd]
    lib.oracle_prim_to_cons.argtypes = [P(_Cfg), pd, pd]
    lib.oracle_cons_to_prim.argtypes = [P(_Cfg), pd, pd]
    lib.oracle_dt.argtypes = [P(_Cfg), pd, pd]
    lib.oracle_residual.argtypes = [P(_Cfg), pd, pd]
    lib.oracle_run.argtypes = [P(_Cfg), pd, i32, d, d, pd, pd, P(i32), pd]
    lib.oracle_run_tangent.argtypes = [P(_Cfg), pd, pd, i32, pd, pd, pd]
    lib.oracle_threads.argtypes = [ctypes.c_int]
    lib.oracle_count_ops.argtypes = [P(_Cfg), pd, pd]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def compile_variant(source_text: str, out_path: str, opt: str = "-O1") -> str:
    """Compiles an edited copy of the oracle source (used by the mutation tests)."""
    src = out_path[:-3] + ".cpp"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["g++", opt, "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", out_path, src],
                   check=True, capture_output=True)
    return out_path


class use_library:
    """Context manager: route every call of this module to another oracle build."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _declare(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(rc: int, allow_nonphysical: bool = False) -> int:
    if rc == ARG:
        raise OracleError("oracle: invalid argument")
    if rc == NONPHYSICAL and not allow_nonphysical:
        raise OracleError("oracle: non-positive density or pressure")
    return rc


# ---------------------------------------------------------------------------
# Face-level building blocks (for pins)
# ---------------------------------------------------------------------------
def limiter(cfg: OracleConfig, a, b) -> np.ndarray:
    a, b = _f64(a).ravel(), _f64(b).ravel()
    out = np.empty_like(a)
    c = cfg.to_c()
    _check(_load().oracle_limiter(ctypes.byref(c), a.size, _ptr(a), _ptr(b), _ptr(out)))
    return out


def interface_solve(cfg: OracleConfig, L, R):
    """L, R: (..., 3) arrays of (rho, u_normal, p).  Returns (p*, u*)."""
    L, R = _f64(L).reshape(-1, 3), _f64(R).reshape(-1, 3)
    ps, us = np.empty(len(L)), np.empty(len(L))
    c = cfg.to_c()
    _check(_load().oracle_interface_solve(ctypes.byref(c), len(L), _ptr(L), _ptr(R), _ptr(ps), _ptr(us)))
    return ps, us


def face_flux(cfg: OracleConfig, direction: int, qL, qR) -> np.ndarray:
    """qL, qR: (..., nfields) primitive face states (rho, u, v, p, y_1 ..).
    Returns (..., nfields) fluxes."""
    nf = cfg.nfields
    qL, qR = _f64(qL).reshape(-1, nf), _f64(qR).reshape(-1, nf)
    F = np.empty_like(qL)
    c = cfg.to_c()
    _check(_load().oracle_face_flux(ctypes.byref(c), direction, len(qL), _ptr(qL), _ptr(qR), _ptr(F)))
    return F


# ---------------------------------------------------------------------------
# Whole-mesh operations
# ---------------------------------------------------------------------------
def _state(cfg: OracleConfig, U) -> np.ndarray:
    U = _f64(U)
    shape = (cfg.nfields,) + cfg.shape
    if U.shape != shape:
        U = U.reshape(shape)
    return np.ascontiguousarray(U)


def prim_to_cons(cfg: OracleConfig, q) -> np.ndarray:
    q = _state(cfg, q)
    U = np.empty_like(q)
    c = cfg.to_c()
    _check(_load().oracle_prim_to_cons(ctypes.byref(c), _ptr(q), _ptr(U)))
    return U


def cons_to_prim(cfg: OracleConfig, U) -> np.ndarray:
    U = _state(cfg, U)
    q = np.empty_like(U)
    c = cfg.to_c()
    _check(_load().oracle_cons_to_prim(ctypes.byref(c), _ptr(U), _ptr(q)))
    return q


def cfl_dt(cfg: OracleConfig, U) -> float:
    U = _state(cfg, U)
    dt = np.zeros(1)
    c = cfg.to_c()
    _check(_load().oracle_dt(ctypes.byref(c), _ptr(U), _ptr(dt)))
    return float(dt[0])


def residual(cfg: OracleConfig, U) -> np.ndarray:
    """L(U) = -(1/|K|) sum_A |A| Phi_A for every cell."""
    U = _state(cfg, U)
    LU = np.empty_like(U)
    c = cfg.to_c()
    _check(_load().oracle_residual(ctypes.byref(c), _ptr(U), _ptr(LU)))
    return LU


@dataclass
class RunResult:
    U: np.ndarray
    steps: int
    t: float
    dts: np.ndarray
    status: int


def run(cfg: OracleConfig, U0, max_steps: int, t_end: float = 0.0, t0: float = 0.0,
        dts=None, allow_nonphysical: bool = False) -> RunResult:
    """Lagrange-flux steps (Sec. 4): Heun/RK2, or SSP-RK3 if cfg.time_order == 3.
    dts freezes the dt sequence."""
    U = _state(cfg, U0).copy()
    dts_in = None if dts is None else _f64(dts)
    if dts_in is not None and dts_in.size < max_steps:
        raise ValueError("dts shorter than max_steps")
    dts_out = np.zeros(max(max_steps, 1))
    steps = ctypes.c_int32(0)
    t = ctypes.c_double(0.0)
    c = cfg.to_c()
    rc = _load().oracle_run(ctypes.byref(c), _ptr(U), int(max_steps), float(t0), float(t_end),
                            _ptr(dts_in), _ptr(dts_out), ctypes.byref(steps), ctypes.byref(t))
    _check(rc, allow_nonphysical)
    return RunResult(U, steps.value, t.value, dts_out[: steps.value].copy(), rc)


def run_tangent(cfg: OracleConfig, q0, dq0, dts):
    """Forward-mode (dual number) derivative of len(dts) steps with frozen dt.

    q0, dq0: primitive initial planes (rho, u, v, p, y_1 ..) and a tangent direction.
    Returns (U_T, dU_T): final conservative state and its directional derivative.
    """
    q0, dq0 = _state(cfg, q0), _state(cfg, dq0)
    dts = _f64(dts).ravel()
    U, dU = np.empty_like(q0), np.empty_like(q0)
    c = cfg.to_c()
    _check(_load().oracle_run_tangent(ctypes.byref(c), _ptr(q0), _ptr(dq0), len(dts), _ptr(dts),
                                      _ptr(U), _ptr(dU)))
    return U, dU


COUNT_PARTS = ("primitives", "slopes", "faces", "balances", "predictor_update", "corrector_update", "wave_speed")
COUNT_KINDS = ("add", "mul", "div", "sqrt")


def count_ops(cfg: OracleConfig, U) -> dict:
    """Operations per cell of the method on state U, part by part (minimal
    schedule: every primitive state, slope, face flux and flux balance formed
    once; see count_stage_ops in the C++ source): {part: {kind: count}}."""
    U = _state(cfg, U)
    out = np.zeros(4 * len(COUNT_PARTS))
    c = cfg.to_c()
    _check(_load().oracle_count_ops(ctypes.byref(c), _ptr(U), _ptr(out)))
    return {p: dict(zip(COUNT_KINDS, out[4 * i:4 * i + 4].tolist())) for i, p in enumerate(COUNT_PARTS)}


def flops_per_cell(counts: dict) -> dict:
    """Flops per cell of the predictor, the corrector (with the CFL wave-speed
    sum of the next step) and the whole Heun step, each operation counted as
    one flop; `div_sqrt` is how many of them are divisions or square roots."""
    tot = {p: sum(v.values()) for p, v in counts.items()}
    ds = {p: v["div"] + v["sqrt"] for p, v in counts.items()}
    stage = ("primitives", "slopes", "faces", "balances")
    pred = sum(tot[p] for p in stage) + tot["predictor_update"]
    corr = sum(tot[p] for p in stage) + tot["corrector_update"] + tot["wave_speed"]
    pred_ds = sum(ds[p] for p in stage) + ds["predictor_update"]
    corr_ds = sum(ds[p] for p in stage) + ds["corrector_update"] + ds["wave_speed"]
    return {"predictor": pred, "corrector": corr, "step": pred + corr,
            "div_sqrt": {"predictor": pred_ds, "corrector": corr_ds, "step": pred_ds + corr_ds}}
