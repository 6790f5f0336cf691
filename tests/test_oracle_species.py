"""Pins of the oracle's species transport (Sec. 5: the conservative form
d(rho y_k)/dt + div(rho y_k u) = 0 carried by the Lagrange flux).

None of these checks retypes the oracle's formulas: they use facts the
scheme must satisfy whatever its implementation -- a constant mass fraction
stays constant (the species flux is y times the mass flux), complementary
fractions keep summing to one, passive species leave the gas dynamics
untouched bit for bit, the pure-advection special case converges at second
order to the exact translated profile and obeys the maximum principle, and
the transposed problem gives the transposed answer.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs


def cons(cfg, prim):
    return O.prim_to_cons(cfg, prim.stack())


@pytest.mark.parametrize("time_order", [2, 3])
@pytest.mark.parametrize("bc,kind", [("transmissive", "quadrant"), ("periodic", "kh")])
def test_constant_fraction_stays_constant(bc, kind, time_order):
    nx, ny = 24, 19
    base = inputs.quadrant(nx, ny, seed=5) if kind == "quadrant" else inputs.kelvin_helmholtz(nx, ny, seed=2)
    prim = inputs.with_species(base, np.full((ny, nx), 0.37))
    cfg = O.OracleConfig(nx=nx, ny=ny, bc=bc, limiter="sweby", beta=1.5, nspecies=1, time_order=time_order)
    r = O.run(cfg, cons(cfg, prim), 12)
    rho, rhoy = r.U[0], r.U[4]
    assert np.abs(rhoy - 0.37 * rho).max() <= 4e-15 * np.abs(rho).max()


def test_complementary_fractions_sum_to_one():
    """y_2 = 1 - y_1: the limiter is odd, so the face fractions stay
    complementary and rho y_1 + rho y_2 = rho up to rounding."""
    prim = inputs.three_region(56, 24, seed=3)
    cfg = O.OracleConfig(nx=56, ny=24, lx=7.0, ly=3.0, limiter="vanleer", nspecies=2)
    r = O.run(cfg, cons(cfg, prim), 30)
    assert np.abs(r.U[4] + r.U[5] - r.U[0]).max() <= 1e-14 * np.abs(r.U[0]).max()
    # the fractions stay in [0, 1] up to rounding on this resting start
    y = r.U[4:] / r.U[0]
    assert y.min() >= -1e-12 and y.max() <= 1 + 1e-12


@pytest.mark.parametrize("dim", [1, 2])
def test_species_leave_gas_dynamics_unchanged(dim):
    if dim == 2:
        base = inputs.quadrant(20, 17, seed=8)
        cfg0 = O.OracleConfig(nx=20, ny=17, limiter="minmod")
    else:
        base = inputs.named_shock_tube("sod", 64)
        cfg0 = O.OracleConfig(nx=64, dim=1, limiter="minmod")
    rng = np.random.default_rng(1)
    y = rng.uniform(0.0, 1.0, size=(3,) + base.shape)
    cfg3 = O.OracleConfig(**{**cfg0.__dict__, "nspecies": 3})
    r0 = O.run(cfg0, cons(cfg0, base), 15)
    r3 = O.run(cfg3, cons(cfg3, inputs.with_species(base, y)), 15)
    assert np.array_equal(r0.U, r3.U[:4])
    assert np.array_equal(r0.dts, r3.dts)


def test_species_flux_is_mass_flux_times_upwind_fraction():
    """Phi_y = (rho y)_A u* with the same upwind side A as the mass flux."""
    rng = np.random.default_rng(4)
    n = 200
    qL = np.stack([rng.uniform(0.2, 2, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0.1, 2, n),
                   rng.uniform(0, 1, n), rng.uniform(0, 1, n)], 1)
    qR = np.stack([rng.uniform(0.2, 2, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0.1, 2, n),
                   rng.uniform(0, 1, n), rng.uniform(0, 1, n)], 1)
    c2 = O.OracleConfig(nx=4, ny=4, nspecies=2)
    c0 = O.OracleConfig(nx=4, ny=4)
    for d in (0, 1):
        F = O.face_flux(c2, d, qL, qR)
        F0 = O.face_flux(c0, d, qL[:, :4], qR[:, :4])
        assert np.array_equal(F[:, :4], F0)
        # the side whose density gives the mass flux: F_rho = rho_A u*, and
        # u* has the sign of F_rho
        ustar_pos = F[:, 0] > 0
        yA = np.where(ustar_pos[:, None], qL[:, 4:], qR[:, 4:])
        np.testing.assert_allclose(F[:, 4:], F[:, :1] * yA, rtol=1e-14, atol=1e-16)
        # equal states: the physical flux rho y u_n
        Fe = O.face_flux(c2, d, qL, qL)
        np.testing.assert_allclose(Fe[:, 4:], qL[:, :1] * qL[:, 4:] * qL[:, 1 + d:2 + d], rtol=1e-14, atol=1e-16)


def _scalar_error_1d(n, limiter, t_end=0.25):
    cfg = O.OracleConfig(nx=n, dim=1, bc="periodic", limiter=limiter, nspecies=1, cfl=0.4)
    r = O.run(cfg, cons(cfg, inputs.advected_scalar_1d(n)), 10**6, t_end=t_end)
    assert math.isclose(r.t, t_end, rel_tol=1e-12)
    y = r.U[4, 0] / r.U[0, 0]
    return np.abs(y - inputs.advected_scalar_1d(n, t=t_end).y[0, 0]).mean()


@pytest.mark.parametrize("limiter", ["vanleer", "sweby"])
def test_scalar_advection_converges_at_second_order(limiter):
    """Uniform rho, u, p: the species equation reduces to MUSCL advection of y,
    whose error against the exact translation falls by ~4 per refinement."""
    e = [_scalar_error_1d(n, limiter) for n in (64, 128, 256)]
    orders = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert min(orders) > 1.75, (e, orders)


def test_scalar_advection_2d_diagonal():
    errs = []
    for n in (32, 64):
        cfg = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter="vanleer", nspecies=1, cfl=0.4)
        r = O.run(cfg, cons(cfg, inputs.advected_scalar(n)), 10**6, t_end=0.2)
        y = r.U[4] / r.U[0]
        errs.append(np.abs(y - inputs.advected_scalar(n, t=0.2).y[0]).mean())
    assert errs[0] < 1e-2 and math.log2(errs[0] / errs[1]) > 1.75, errs


@pytest.mark.parametrize("limiter", ["minmod", "vanleer", "sweby"])
def test_indicator_obeys_maximum_principle(limiter):
    """The unsplit update is a convex combination of 1D MUSCL updates whose
    Courant number is below 1/2 under the CFL condition, and each of those is
    TVD for limiters with phi <= 2 min(1, r): the indicator stays in [0, 1]."""
    cfg = O.OracleConfig(nx=40, ny=40, bc="periodic", limiter=limiter, beta=2.0, nspecies=1, cfl=0.45)
    r = O.run(cfg, cons(cfg, inputs.advected_indicator(40)), 60)
    y = r.U[4] / r.U[0]
    assert y.min() >= -1e-13 and y.max() <= 1 + 1e-13
    # mass of the indicator conserved on the periodic mesh
    assert abs(math.fsum(r.U[4].ravel()) - math.fsum(cons(cfg, inputs.advected_indicator(40))[4].ravel())) < 1e-11


def test_species_transpose_symmetry():
    nx, ny = 14, 9
    prim = inputs.with_species(inputs.quadrant(nx, ny, seed=6),
                               np.random.default_rng(2).uniform(0, 1, size=(2, ny, nx)))
    c, ct = O.OracleConfig(nx=nx, ny=ny, nspecies=2), O.OracleConfig(nx=ny, ny=nx, nspecies=2)
    U = cons(c, prim)
    perm = [0, 2, 1, 3, 4, 5]
    dts = [1.5e-3] * 6
    a = O.run(c, U, 6, dts=dts).U
    b = O.run(ct, np.ascontiguousarray(U[perm].transpose(0, 2, 1)), 6, dts=dts).U
    np.testing.assert_allclose(b[perm].transpose(0, 2, 1), a, rtol=1e-12, atol=1e-14)


def test_species_conserved_periodic():
    prim = inputs.shear_layer_tracers(32, 24, seed=1, nspecies=3)
    cfg = O.OracleConfig(nx=32, ny=24, bc="periodic", nspecies=3, time_order=3)
    U0 = cons(cfg, prim)
    r = O.run(cfg, U0, 20)
    for l in range(7):
        assert abs(math.fsum(r.U[l].ravel()) - math.fsum(U0[l].ravel())) < 1e-11


def test_species_count_validated():
    with pytest.raises(O.OracleError):
        O.run(O.OracleConfig(nx=8, ny=8, nspecies=9), np.ones((13, 8, 8)), 1)
