"""The allocation-free step (lf_step_noalloc) against the ordinary context path.

lf_step_noalloc exists for callers that must not allocate device memory
(code inside another framework's memory manager, time-critical loops where
cudaMalloc/cudaFree would synchronise the device, hosts that reserve all GPU
memory up front).  It keeps its scratch in a static device array of the
library.  Here it is called through the C ABI twice in a row -- the second
call starting from the first call's output, so stale scratch from the first
call must not leak into the second -- and compared with lf_init + lf_step on
the same input.  Both paths run the same stage kernels on the same values, so
the comparison is bit for bit.  The file is named so that pytest collects it
last.
"""
import ctypes

import pytest

from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300 import lagflux as L  # noqa: E402

def noalloc(cfg_c, U_in, U_out, dt, dt_used=None):
    """One lf_step_noalloc call through the C ABI on torch's current stream."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.lf_step_noalloc(ctypes.byref(cfg_c), ctypes.c_void_p(U_in.data_ptr()), ctypes.c_void_p(U_out.data_ptr()),
                             dt, None if dt_used is None else ctypes.byref(dt_used), stream)


def context_steps(cfg, prim, nsteps, fixed_dt):
    """U0 and the state after nsteps steps of the ordinary context path, with the dts used."""
    tdt = torch.float64 if cfg.precision == "fp64" else torch.float32
    ctx = L.LagrangeFlux(cfg)
    q = torch.from_numpy(prim).to("cuda", tdt)
    ctx.set_primitive(q[0], q[1], q[2], q[3])
    U0 = torch.empty((4,) + prim.shape[1:], dtype=tdt, device="cuda")
    ctx.get_state(U0)
    dts = []
    for _ in range(nsteps):
        if fixed_dt:
            ctx.step_fixed(fixed_dt)
            dts.append(fixed_dt)
        else:
            dts.append(ctx.step(return_dt=True))
    ref = torch.empty_like(U0)
    ctx.get_state(ref)
    ctx.close()
    return U0, ref, dts


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("fixed_dt", [0.0, 1.5e-4])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
@pytest.mark.parametrize("nx,ny", [(200, 150), (201, 151)])
def test_noalloc_matches_context_path_twice(precision, fixed_dt, bc, nx, ny):
    """Two calls in a row (the second in place, from the first call's output)
    equal two lf_step calls of a context bit for bit, state and dt: both run
    the same stage kernels on the same values, so stale scratch from the
    first call would show as a difference.  Odd nx: dense rows start on odd
    cells, so the FP32 kernels take per-cell copies instead of lane vectors."""
    prim = inputs.quadrant(nx, ny, seed=21).stack()
    cfg = L.Config(nx=nx, ny=ny, precision=precision, limiter="vanleer", bc=bc, cfl=0.45)
    U0, ref, dts_ref = context_steps(cfg, prim, 2, fixed_dt)
    c = cfg.to_c()
    A = U0.clone()
    B = torch.empty_like(U0)
    dt_used = ctypes.c_double()
    assert noalloc(c, A, B, fixed_dt, dt_used) == L.LF_OK, L.lf_last_error(None)
    assert dt_used.value == dts_ref[0]
    assert noalloc(c, B, B, fixed_dt, dt_used) == L.LF_OK, L.lf_last_error(None)
    assert dt_used.value == dts_ref[1]
    torch.cuda.synchronize()
    assert torch.equal(B, ref)
    assert torch.equal(A, U0)  # the input of the first call is untouched


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("fixed_dt", [0.0, 2e-4])
def test_noalloc_1d_sod_in_place(precision, fixed_dt):
    """The 1D branch: Sod's tube on 1000 cells (Sec. 4.2), every call in place
    (U_in == U_out) from the first one, against lf_init + lf_step after three
    steps.  Bit for bit, except one case: in 1D FP32 with the CFL dt, lf_step
    takes the wave-speed maximum of a step's result from the corrector's
    epilogue (paired-FP32 arithmetic on the lane's two cells) while
    lf_step_noalloc forms it in the separate wave-speed pass (scalar FP32), and
    the two compiled forms of the same formula have been measured to round
    the maximum one FP32 ulp apart (dt 3.05874752e-4 against 3.05874774e-4 on
    this tube).  That case checks dt to 2.4e-7 (two FP32 ulps) and the state
    to the FP32 parity bound."""
    prim = inputs.named_shock_tube("sod", 1000).stack()
    cfg = L.Config(nx=1000, ny=1, dim=1, precision=precision, limiter="minmod", bc="transmissive", cfl=0.5)
    U0, ref, dts_ref = context_steps(cfg, prim, 3, fixed_dt)
    c = cfg.to_c()
    U = U0.clone()
    dt_used = ctypes.c_double()
    loose = precision == "fp32" and fixed_dt == 0.0
    for k in range(3):
        assert noalloc(c, U, U, fixed_dt, dt_used) == L.LF_OK, L.lf_last_error(None)
        if loose:
            assert dt_used.value == pytest.approx(dts_ref[k], rel=2.4e-7)
        else:
            assert dt_used.value == dts_ref[k]
    torch.cuda.synchronize()
    if loose:
        for l in range(4):
            err = float((U[l].double() - ref[l].double()).abs().sum() / ref[l].double().abs().sum().clamp_min(1e-300))
            assert err <= 2e-5, (l, err)
    else:
        assert torch.equal(U, ref)


def test_noalloc_rejects_oversized_mesh_and_bad_arguments():
    cfg = L.Config(nx=1024, ny=1024).to_c()  # 2^20 cells > 2^18
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = L.lf_step_noalloc(ctypes.byref(cfg), p, p, 0.0, None, None)
    assert st == L.LF_ERR_ARG
    assert b"LF_NOALLOC_MAX_CELLS" in L.lf_last_error(None)
    ok = L.Config(nx=16, ny=16).to_c()
    assert L.lf_step_noalloc(ctypes.byref(ok), None, p, 0.0, None, None) == L.LF_ERR_ARG
    assert L.lf_step_noalloc(ctypes.byref(ok), p, p, float("nan"), None, None) == L.LF_ERR_ARG


def test_noalloc_reports_nonphysical_state():
    nx = ny = 64
    prim = inputs.quadrant(nx, ny, seed=2).stack()
    prim[3, 5, 5] = -1.0
    cfg = L.Config(nx=nx, ny=ny, precision="fp64")
    ctx = L.LagrangeFlux(cfg)
    q = torch.from_numpy(prim).cuda()
    ctx.set_primitive(q[0], q[1], q[2], q[3])
    U = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    ctx.get_state(U)
    ctx.close()
    out = torch.empty_like(U)
    c = cfg.to_c()
    dt_used = ctypes.c_double()
    st = L.lf_step_noalloc(ctypes.byref(c), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1e-4,
                           ctypes.byref(dt_used), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.LF_ERR_NONPHYSICAL
