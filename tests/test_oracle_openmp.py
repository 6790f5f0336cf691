"""The OpenMP timing build of the oracle returns the same bits as the plain
single-threaded build (its parallel loops write each element from one
iteration; its reductions are a logical AND and an exact maximum)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs


@pytest.fixture(scope="module")
def omp_lib():
    return O.build_omp()


@pytest.mark.parametrize("case", ["quadrant", "kh", "octant"])
def test_openmp_build_is_bitwise_equal(omp_lib, case):
    if case == "quadrant":
        oc = O.OracleConfig(nx=67, ny=45, limiter="vanleer", bc="transmissive", cfl=0.45)
        q = inputs.quadrant(67, 45, seed=3).stack()
    elif case == "kh":
        oc = O.OracleConfig(nx=64, ny=64, limiter="sweby", beta=1.5, bc="periodic", cfl=0.45)
        q = inputs.kelvin_helmholtz(64, 64, seed=1).stack()
    else:
        oc = O.OracleConfig(nx=13, ny=11, nz=9, dim=3, limiter="minmod", bc="periodic", cfl=0.4)
        q = inputs.octant(13, 11, 9, seed=2).stack()
    U0 = O.prim_to_cons(oc, q)
    plain = O.run(oc, U0, 7)
    assert O.threads() == 1
    with O.use_library(omp_lib):
        n = O.threads(4)
        assert n == 4
        par = O.run(oc, U0, 7)
    np.testing.assert_array_equal(par.U, plain.U)
    assert par.t == plain.t and par.steps == plain.steps
