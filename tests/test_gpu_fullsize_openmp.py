"""The benchmark's full 8192^2 periodic Kelvin-Helmholtz mesh, ten CFL steps
on the GPU, against the FP64 oracle run on the whole mesh by its OpenMP build
on the host's cores (the same bits as the plain build, test_oracle_openmp.py):
every cell of every field is compared, not samples.

Bars: FP64 relative L1 <= 1e-12 per conservative field and the oracle's own
CFL dt sequence to 1e-14; FP32 (state in FP32, dt from an FP64 reduction)
relative L1 <= 2e-5 per field against its own norm, on the GPU's dt sequence.
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
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"
