"""Pins of the oracle's three-dimensional step (the finite-volume form of
Sec. 4 with a third flux direction).

Checks that do not retype the oracle: a problem varying along one axis only
equals the 1D scheme (pinned against exact Riemann solutions) with the
velocity components permuted; a 2D problem extruded along the third axis
equals the 2D scheme; axis permutations commute with the step; free streams
are preserved exactly; mass, momentum, energy and species are conserved on a
periodic mesh; the smooth diagonal wave converges at second order to its exact
translation; and the CFL time step matches a hand computation.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs


def cfg3(nx, ny, nz, **kw):
    return O.OracleConfig(nx=nx, ny=ny, nz=nz, dim=3, **kw)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("limiter,bc", [("minmod", "transmissive"), ("vanleer", "periodic"), ("sweby", "transmissive")])
def test_one_axis_problem_equals_1d(axis, limiter, bc):
    n = 40
    tube = inputs.named_shock_tube("sod", n).stack()[:, 0, :]  # (4, n): rho, u, v(=0), p
    c1 = O.OracleConfig(nx=n, dim=1, limiter=limiter, bc=bc, beta=1.5)
    dts = [2.5e-3] * 12
    r1 = O.run(c1, O.prim_to_cons(c1, tube[:, None, :]), 12, dts=dts).U[:, 0, :]  # rho, rho u, rho v, rho E
    shape = [1, 1, 1]
    shape[2 - axis] = n  # array axes are (z, y, x)
    q = np.zeros((5,) + tuple(shape))
    line = [slice(None) if a == 2 - axis else 0 for a in range(3)]
    q[(0,) + tuple(line)] = tube[0]
    q[(1 + axis,) + tuple(line)] = tube[1]  # the tube's velocity along `axis`
    q[(4,) + tuple(line)] = tube[3]
    nz, ny, nx = shape
    c3 = cfg3(nx, ny, nz, limiter=limiter, bc=bc, beta=1.5)
    r3 = O.run(c3, O.prim_to_cons(c3, q), 12, dts=dts).U.reshape(5, n)
    np.testing.assert_allclose(r3[0], r1[0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r3[1 + axis], r1[1], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r3[4], r1[3], rtol=1e-14, atol=1e-15)
    for d in range(3):
        if d != axis:
            assert np.all(r3[1 + d] == 0.0)


def permute_axes(U, perm):
    """Relabels the spatial axes of a 3D state (fields, z, y, x): new axis d
    is old axis perm[d] (0 = x, 1 = y, 2 = z), velocity components included."""
    order = [0] + [1 + (2 - perm[2 - p]) for p in range(3)]
    out = np.transpose(U, order).copy()
    for d in range(3):
        out[1 + d] = np.transpose(U[1 + perm[d]], [2 - perm[2 - p] for p in range(3)])
    return np.ascontiguousarray(out)


@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_extruded_2d_problem_equals_2d(plane):
    """The 2D quadrant problem laid in a coordinate plane and extruded along
    the third axis (4 cells, periodic) equals the 2D scheme in every layer."""
    nx2, ny2, ext = 14, 11, 4
    q2 = inputs.quadrant(nx2, ny2, seed=4).stack()  # rho, u, v, p on (ny2, nx2)
    c2 = O.OracleConfig(nx=nx2, ny=ny2, limiter="vanleer", bc="periodic")
    dts = [2e-3] * 8
    r2 = O.run(c2, O.prim_to_cons(c2, q2), 8, dts=dts).U
    # build it in the xy plane (extruded along z), then relabel the axes
    q3 = np.zeros((5, ext, ny2, nx2))
    for f2, f3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
        q3[f3] = q2[f2][None]
    perm = {"xy": [0, 1, 2], "xz": [0, 2, 1], "yz": [2, 0, 1]}[plane]  # new axis d = old axis perm[d]
    qp = permute_axes(q3, perm)
    n_old = [nx2, ny2, ext]
    n_new = [n_old[perm[d]] for d in range(3)]
    c3 = cfg3(n_new[0], n_new[1], n_new[2], limiter="vanleer", bc="periodic")
    r3 = O.run(c3, O.prim_to_cons(c3, qp), 8, dts=dts).U
    inv = [perm.index(d) for d in range(3)]
    back = permute_axes(r3, inv)  # (5, ext, ny2, nx2) in the xy layout
    for layer in range(ext):
        for f2, f3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
            np.testing.assert_allclose(back[f3, layer], r2[f2], rtol=1e-13, atol=1e-14)
    assert np.abs(back[3]).max() <= 1e-15


@pytest.mark.parametrize("perm", [[2, 1, 0], [1, 2, 0], [2, 0, 1]])
def test_axis_permutation_commutes_with_the_step(perm):
    nx, ny, nz = 7, 6, 5
    lengths = [1.0, 1.2, 0.8]
    q = inputs.octant(nx, ny, nz, seed=2).stack()  # (5, nz, ny, nx)
    c = cfg3(nx, ny, nz, limiter="sweby", beta=1.5, lx=lengths[0], ly=lengths[1], lz=lengths[2])
    dts = [1.5e-3] * 5
    r = O.run(c, O.prim_to_cons(c, q), 5, dts=dts).U
    n = [nx, ny, nz]
    nn = [n[perm[d]] for d in range(3)]
    ll = [lengths[perm[d]] for d in range(3)]
    cp = cfg3(nn[0], nn[1], nn[2], limiter="sweby", beta=1.5, lx=ll[0], ly=ll[1], lz=ll[2])
    rp = O.run(cp, O.prim_to_cons(cp, permute_axes(q, perm)), 5, dts=dts).U
    np.testing.assert_allclose(rp, permute_axes(r, perm), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_free_stream_preserved_exactly(bc):
    n = 6
    one = np.ones((n, n, n))
    q = np.stack([1.3 * one, 0.4 * one, -0.2 * one, 0.7 * one, 0.9 * one])
    c = cfg3(n, n, n, bc=bc)
    U0 = O.prim_to_cons(c, q)
    r = O.run(c, U0, 6)
    assert np.array_equal(r.U, U0)


def test_periodic_conservation_with_species():
    n = 10
    base = inputs.octant(n, n, n, seed=5)
    y = np.random.default_rng(1).uniform(0, 1, size=(2, n, n, n))
    q = inputs.with_species(base, y).stack()
    c = cfg3(n, n, n, bc="periodic", nspecies=2, time_order=3)
    U0 = O.prim_to_cons(c, q)
    r = O.run(c, U0, 10)
    for l in range(7):
        assert abs(math.fsum(r.U[l].ravel()) - math.fsum(U0[l].ravel())) < 1e-12
    # a constant fraction stays constant in 3D as well
    q[5] = 0.3
    r = O.run(c, O.prim_to_cons(c, q), 6)
    assert np.abs(r.U[5] - 0.3 * r.U[0]).max() < 1e-14


def test_smooth_wave_converges_at_second_order():
    errs = []
    for n in (16, 32):
        c = cfg3(n, n, n, bc="periodic", limiter="vanleer", cfl=0.4)
        r = O.run(c, O.prim_to_cons(c, inputs.smooth_wave_3d(n).stack()), 10**5, t_end=0.1)
        rho = r.U[0]
        errs.append(np.abs(rho - inputs.smooth_wave_3d(n, t=0.1).rho).mean())
        # the contact keeps the velocity and pressure uniform
        q = O.cons_to_prim(c, r.U)
        assert np.abs(q[1:4] - 1.0 / 3.0).max() < 1e-13 and np.abs(q[4] - 1.0).max() < 1e-13
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_cfl_dt_by_hand():
    # rho 1.4, p 1 -> c 1; (u, v, w) = (0.5, -0.25, 0.1) on 10 x 8 x 5 cells of the unit cube
    shape = (5, 8, 10)
    one = np.ones(shape)
    q = np.stack([1.4 * one, 0.5 * one, -0.25 * one, 0.1 * one, one])
    c = cfg3(10, 8, 5, cfl=0.45)
    expect = 0.45 / ((0.5 + 1) * 10 + (0.25 + 1) * 8 + (0.1 + 1) * 5)
    assert math.isclose(O.cfl_dt(c, O.prim_to_cons(c, q)), expect, rel_tol=1e-13)


def test_octant_problem_stays_physical():
    n = 16
    c = cfg3(n, n, n, limiter="vanleer", cfl=0.45)
    r = O.run(c, O.prim_to_cons(c, inputs.octant(n, seed=3).stack()), 30)
    q = O.cons_to_prim(c, r.U)
    assert np.all(np.isfinite(r.U)) and q[0].min() > 0 and q[4].min() > 0


def test_3d_config_validated():
    with pytest.raises(O.OracleError):
        O.run(O.OracleConfig(nx=4, ny=4, nz=3, dim=2), np.ones((4, 4, 4)), 1)
