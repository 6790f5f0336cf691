"""The allocation-free step (lf_step_noalloc) against the ordinary context path.

lf_step_noalloc exists for callers that must not allocate device memory
(code inside another framework's memory manager, time-critical loops where
cudaMalloc/cudaFree would synchronise the device, hosts that reserve all GPU
memory up front).  It keeps its scratch in a static device array of the
library.  Here it is called through the C ABI twice in a row -- the second
call starting from the first call's output, so stale scratch from the first
call must not leak into the second -- and compared with lf_init + lf_step on
the same input, within the FP64 tolerance of the parity tests.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300 import lagflux as L  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def rel_l1(a, b):
    return float((a.double() - b.double()).abs().sum() / b.double().abs().sum())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("fixed_dt", [False, True])
@pytest.mark.parametrize("nx,ny", [(200, 150), (201, 151)])
def test_noalloc_matches_context_path_twice(precision, fixed_dt, nx, ny):
    # odd nx: dense rows start on odd cells, so the kernels must use per-cell access
    prim = inputs.quadrant(nx, ny, seed=21).stack()
    cfg = L.Config(nx=nx, ny=ny, precision=precision, limiter="vanleer", bc="transmissive", cfl=0.45)
    tdt = torch.float64 if precision == "fp64" else torch.float32

    # ordinary path: context, CFL (or fixed) steps
    ctx = L.LagrangeFlux(cfg)
    q = torch.from_numpy(prim).to("cuda", tdt)
    ctx.set_primitive(q[0], q[1], q[2], q[3])
    U0 = torch.empty((4, ny, nx), dtype=tdt, device="cuda")
    ctx.get_state(U0)
    dts_ref = []
    for _ in range(2):
        if fixed_dt:
            ctx.step_fixed(1.5e-4)
            dts_ref.append(1.5e-4)
        else:
            dts_ref.append(ctx.step(return_dt=True))
    ref = torch.empty_like(U0)
    ctx.get_state(ref)
    ctx.close()

    # allocation-free path, two calls in a row through the C ABI
    c = cfg.to_c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = U0.clone()
    B = torch.empty_like(U0)
    dt_used = ctypes.c_double()
    st = L.lf_step_noalloc(ctypes.byref(c), ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                           1.5e-4 if fixed_dt else 0.0, ctypes.byref(dt_used), stream)
    assert st == L.LF_OK, L.lf_last_error(None)
    assert dt_used.value == pytest.approx(dts_ref[0], rel=1e-15 if precision == "fp64" else 1e-6)
    st = L.lf_step_noalloc(ctypes.byref(c), ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                           1.5e-4 if fixed_dt else 0.0, ctypes.byref(dt_used), stream)
    assert st == L.LF_OK, L.lf_last_error(None)
    assert dt_used.value == pytest.approx(dts_ref[1], rel=1e-15 if precision == "fp64" else 1e-6)
    torch.cuda.synchronize()
    for l in range(4):
        assert rel_l1(B[l], ref[l]) <= TOL[precision]
    # the input of the first call is untouched
    torch.testing.assert_close(A, U0, rtol=0, atol=0)


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
