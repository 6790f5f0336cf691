"""The benchmark's full meshes -- the 8192^2 periodic Kelvin-Helmholtz layer
(ten CFL steps) and the 384^3 periodic 3D shear layer (five) -- on the GPU,
against the FP64 oracle run on the whole mesh by its OpenMP build on the
host's cores (the same bits as the plain build, test_oracle_openmp.py): every
cell of every field is compared, not samples.

Bars: FP64 relative L1 <= 1e-12 per conservative field and the oracle's own
CFL dt sequence to 1e-14; FP32 (state in FP32, dt from an FP64 reduction)
relative L1 <= 2e-5 per field against its own norm, on the GPU's dt sequence.
One exception, in both precisions: the 3D layer's rho w.  w starts at zero
and the initial flow is divergence-free, so after five steps rho w holds
only what the scheme generates at the density contacts, orders of magnitude
below the other momentum components; rounding-level differences are large
against its own norm (FP64 1.4e-8 measured), so it is measured against the
momentum magnitude |rho u| + |rho v| + |rho w| (its own-norm error is
printed beside it).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux  # noqa: E402

N, STEPS = 8192, 10
KW = dict(limiter="vanleer", bc="periodic", cfl=0.45)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


@pytest.fixture(scope="module")
def prim():
    return inputs.kelvin_helmholtz(N, N, seed=0).stack()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_whole_8192_mesh_ten_steps_against_openmp_oracle(prim, precision):
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(Config(nx=N, ny=N, precision=precision, **KW))
    q = torch.from_numpy(prim).to("cuda", tdt)
    s.set_primitive(q[0], q[1], q[2], q[3])
    del q
    U = torch.empty((4, N, N), dtype=tdt, device="cuda")
    s.get_state(U)
    U0 = U.double().cpu().numpy()  # the oracle starts from the GPU's conservative state
    dts = [s.step(return_dt=True) for _ in range(STEPS)]
    s.get_state(U)
    got = U.double().cpu().numpy()
    del U
    s.close()

    oc = O.OracleConfig(nx=N, ny=N, **KW)
    with O.use_library(O.build_omp()):
        O.threads(host_cores())
        ref = O.run(oc, U0, STEPS) if precision == "fp64" else O.run(oc, U0, STEPS, dts=dts)
    assert ref.steps == STEPS
    if precision == "fp64":
        np.testing.assert_allclose(dts, ref.dts, rtol=1e-14, atol=0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for field in range(4):
        err = np.abs(got[field] - ref.U[field]).sum() / np.abs(ref.U[field]).sum()
        print(f"8192^2 {precision} field {field}: relative L1 {err:.3e}")
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"


N3, STEPS3 = 384, 5


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_whole_384_cube_five_steps_against_openmp_oracle(precision):
    tdt = torch.float64 if precision == "fp64" else torch.float32
    q = inputs.shear_layer_3d(N3, seed=0).stack()
    s = LagrangeFlux(Config(nx=N3, ny=N3, nz=N3, dim=3, precision=precision, **KW))
    s.set_primitives(torch.from_numpy(q).to("cuda", tdt))
    del q
    U0 = s.get_conservative().astype(np.float64)
    dts = [s.step(return_dt=True) for _ in range(STEPS3)]
    got = s.get_conservative().astype(np.float64)
    s.close()

    oc = O.OracleConfig(nx=N3, ny=N3, nz=N3, dim=3, **KW)
    with O.use_library(O.build_omp()):
        O.threads(host_cores())
        ref = O.run(oc, U0, STEPS3) if precision == "fp64" else O.run(oc, U0, STEPS3, dts=dts)
    assert ref.steps == STEPS3
    if precision == "fp64":
        np.testing.assert_allclose(dts, ref.dts, rtol=1e-14, atol=0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    momentum = sum(np.abs(ref.U[m]).sum() for m in (1, 2, 3))
    for field in range(5):
        diff = np.abs(got[field] - ref.U[field]).sum()
        own = diff / np.abs(ref.U[field]).sum()
        err = diff / momentum if field == 3 else own
        print(f"384^3 {precision} field {field}: relative L1 {err:.3e} (against its own norm {own:.3e})")
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"
