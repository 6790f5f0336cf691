"""The op-counting scalar of the oracle (count_ops) against operation counts
written out by hand from the formulas it runs.  These counts are the
algorithmic flops per cell that the FP64 roofline divides by."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs


def uniform_state(oc, n):
    q = np.ones((4, n, n))
    q[1] *= 0.3
    q[2] *= -0.2
    return O.prim_to_cons(oc, q)


def test_counts_of_a_uniform_2d_state():
    """Free stream: no limiter is active, so every part has a fixed count.
    Primitives (eq. 1): u, v, E by three divisions; |u|^2 by two products and
    two sums (from 0); p = (gamma-1) rho (E - |u|^2/2) by three products and a
    difference.  Slopes: two differences per field and axis, 4 x 2 x 2 = 16.
    One face: face states 2 x 4 x (product, sum); eqs. 13-14: two sound speeds
    (product, division, root each), rho_L + rho_R, p* (5 products, 3 sums,
    2 divisions), u* (3 products, 3 sums, 2 divisions); the upwind
    conservative state (6 products, 3 sums, 1 division); eq. 12 (4 products,
    then p* and p* u*: 1 product, 2 sums): 20 sums, 29 products, 7 divisions,
    2 roots, and two faces per cell in 2D.  Flux balance per field: per axis
    two products and two sums, then one division by |K|.  Predictor per field:
    U - dt b; corrector per field: U - dt (b + b)/2.  Wave speed: c (product,
    division, root), then per axis (|u| + c)/h added to the sum."""
    oc = O.OracleConfig(nx=24, ny=24, limiter="vanleer", bc="periodic", cfl=0.45)
    c = O.count_ops(oc, uniform_state(oc, 24))
    as_list = lambda p: [c[p][k] for k in O.COUNT_KINDS]
    assert as_list("primitives") == [3, 5, 3, 0]
    assert as_list("slopes") == [16, 0, 0, 0]
    assert as_list("faces") == [40, 58, 14, 4]
    assert as_list("balances") == [16, 16, 4, 0]
    assert as_list("predictor_update") == [4, 4, 0, 0]
    assert as_list("corrector_update") == [8, 4, 4, 0]
    assert as_list("wave_speed") == [4, 1, 3, 1]
    f = O.flops_per_cell(c)
    assert f["predictor"] == 11 + 16 + 116 + 36 + 8
    assert f["corrector"] == 11 + 16 + 116 + 36 + 16 + 9
    assert f["step"] == f["predictor"] + f["corrector"]


def test_counts_scale_with_dimension():
    """The face part of a 1D mesh is one face per cell with the same count as
    a 2D face (four fields either way), and the 3D wave speed adds one axis."""
    o1 = O.OracleConfig(nx=40, dim=1, limiter="minmod", bc="periodic", cfl=0.45)
    q1 = np.ones((4, 1, 40))
    q1[1] *= 0.3
    c1 = O.count_ops(o1, O.prim_to_cons(o1, q1))
    assert [c1["faces"][k] for k in O.COUNT_KINDS] == [20, 29, 7, 2]
    assert [c1["slopes"][k] for k in O.COUNT_KINDS] == [8, 0, 0, 0]
    o3 = O.OracleConfig(nx=6, ny=5, nz=4, dim=3, limiter="minmod", bc="periodic", cfl=0.45)
    q3 = np.ones((5, 4, 5, 6))
    c3 = O.count_ops(o3, O.prim_to_cons(o3, q3))
    assert [c3["wave_speed"][k] for k in O.COUNT_KINDS] == [6, 1, 4, 1]


def test_active_van_leer_limiters_add_their_formula():
    """Each active van Leer limiter 2ab/(a+b) adds two products, one sum and
    one division to the two differences: on a state with a known number of
    active limiters the slope part says so.  A periodic row of n cells whose
    u rises by one unit per cell over k cells and falls back at once has
    k - 1 cells with both differences positive (ab > 0)."""
    n, k = 20, 7
    oc = O.OracleConfig(nx=n, dim=1, limiter="vanleer", bc="periodic", cfl=0.45)
    q = np.ones((4, 1, n))
    q[1, 0, :] = 0.0
    q[1, 0, :k] = 0.01 * np.arange(k)  # cells 1 .. k-2 sit inside the ramp; cell k-1 is its top
    c = O.count_ops(oc, O.prim_to_cons(oc, q))
    active = (k - 2) / n  # cells 1 .. k-2: both differences 0.01 > 0
    assert c["slopes"]["mul"] == pytest.approx(2 * active)
    assert c["slopes"]["div"] == pytest.approx(active)
    assert c["slopes"]["add"] == pytest.approx(8 + active)


def test_counts_on_the_shear_layer():
    """On the benchmark's shear layer only a few limiters are active (the
    layer is constant along x except for v): the count stays near the
    free-stream one, about 399 flops per cell-update, 60 of them divisions
    or roots."""
    oc = O.OracleConfig(nx=256, ny=256, limiter="vanleer", bc="periodic", cfl=0.45)
    U = O.prim_to_cons(oc, inputs.kelvin_helmholtz(256, 256, seed=0).stack())
    f = O.flops_per_cell(O.count_ops(oc, U))
    assert 390 < f["step"] < 410
    assert 55 < f["div_sqrt"]["step"] < 65


def test_openmp_build_refuses_to_count():
    oc = O.OracleConfig(nx=8, ny=8)
    U = uniform_state(oc, 8)
    with O.use_library(O.build_omp()):
        with pytest.raises(O.OracleError):
            O.count_ops(oc, U)
