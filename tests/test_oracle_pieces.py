"""Pins of the oracle's face-level building blocks.

* Limiter, eq. (sweby): beta = 1 is minmod and beta = 2 is superbee (textbook
  definitions written out here independently), hand-computed values, symmetry
  and oddness, and the van Leer harmonic-mean form.
* Interface solver, eqs. (13)-(14): uniform states, mirror symmetry, the two
  characteristic (acoustic) relations the solution must satisfy, and
  agreement with the exact Riemann solver in the weak-wave limit.
* Face flux, eq. (12): consistency with the physical Euler flux, rotation
  between the x and y directions, and the upwind choice.
"""
import math

import numpy as np
import pytest

from oracle import exact_riemann as X
from oracle import oracle as O

G = 1.4


def cfg(limiter="sweby", beta=1.5, riemann="maxc"):
    return O.OracleConfig(nx=4, ny=4, limiter=limiter, beta=beta, riemann=riemann)


def _rand_pairs(n=4000, seed=1):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=n) * np.exp(rng.normal(size=n))
    b = rng.normal(size=n) * np.exp(rng.normal(size=n))
    # include exact zeros and ties
    a[:50] = 0.0
    b[50:100] = 0.0
    b[100:150] = a[100:150]
    b[150:200] = 2.0 * a[150:200]
    b[200:250] = -a[200:250]
    return a, b


def test_sweby_beta1_is_minmod():
    a, b = _rand_pairs()
    got = O.limiter(cfg("minmod"), a, b)
    same = a * b > 0
    minmod = np.where(same, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)
    np.testing.assert_array_equal(got, minmod)
    np.testing.assert_array_equal(O.limiter(cfg("sweby", 1.0), a, b), minmod)


def test_sweby_beta2_is_superbee():
    a, b = _rand_pairs(seed=2)
    got = O.limiter(cfg("sweby", 2.0), a, b)
    # superbee in ratio form: slope = b * max(0, min(2r, 1), min(r, 2)), r = a/b
    with np.errstate(divide="ignore", invalid="ignore"):
        r = a / b
        sb = b * np.maximum(0.0, np.maximum(np.minimum(2 * r, 1.0), np.minimum(r, 2.0)))
    sb = np.where(a * b > 0, sb, 0.0)
    np.testing.assert_allclose(got, sb, rtol=1e-15, atol=0)


def test_sweby_hand_values():
    c = cfg("sweby", 1.5)
    # phi(1, 3) = max(min(1, 4.5), min(1.5, 3)) = 1.5
    # phi(-2, -1) = -max(min(2, 1.5), min(3, 1)) = -1.5
    # phi(1, 1.2) = max(min(1, 1.8), min(1.5, 1.2)) = 1.2
    # phi(1, -1) = 0
    got = O.limiter(c, [1.0, -2.0, 1.0, 1.0, 0.0], [3.0, -1.0, 1.2, -1.0, 5.0])
    np.testing.assert_array_equal(got, [1.5, -1.5, 1.2, 0.0, 0.0])


@pytest.mark.parametrize("lim,beta", [("minmod", 1.0), ("sweby", 1.5), ("sweby", 2.0), ("vanleer", 1.0)])
def test_limiter_symmetric_odd_and_bounded(lim, beta):
    a, b = _rand_pairs(seed=3)
    c = cfg(lim, beta)
    f = O.limiter(c, a, b)
    np.testing.assert_array_equal(f, O.limiter(c, b, a))
    np.testing.assert_array_equal(-f, O.limiter(c, -a, -b))
    same = a * b > 0
    assert np.all(f[~same] == 0.0)
    lo = np.minimum(np.abs(a), np.abs(b))
    hi = np.maximum(np.abs(a), np.abs(b))
    # second-order TVD region: min(|a|,|b|) <= |phi| <= min(2 min, max)
    assert np.all(np.abs(f[same]) >= lo[same] * (1 - 1e-15))
    assert np.all(np.abs(f[same]) <= np.minimum(2 * lo[same], hi[same]) * (1 + 1e-15))
    assert np.all(np.sign(f[same]) == np.sign(a[same]))


def test_vanleer_hand_values_and_ratio_form():
    c = cfg("vanleer")
    # 2ab/(a+b): (1,3) -> 1.5, (2,2) -> 2, (-1,-4) -> -1.6
    np.testing.assert_allclose(O.limiter(c, [1.0, 2.0, -1.0], [3.0, 2.0, -4.0]), [1.5, 2.0, -1.6], rtol=1e-15)
    a, b = _rand_pairs(seed=4)
    same = a * b > 0
    r = a[same] / b[same]
    # van Leer's ratio form phi(r) = (r + |r|)/(1 + |r|) times the downwind slope b
    np.testing.assert_allclose(O.limiter(c, a, b)[same], b[same] * (r + np.abs(r)) / (1 + np.abs(r)), rtol=1e-13)


def _rand_faces(n=500, seed=5):
    rng = np.random.default_rng(seed)
    L = np.stack([rng.uniform(0.1, 3, n), rng.uniform(-2, 2, n), rng.uniform(0.05, 5, n)], axis=1)
    R = np.stack([rng.uniform(0.1, 3, n), rng.uniform(-2, 2, n), rng.uniform(0.05, 5, n)], axis=1)
    return L, R


@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
def test_interface_uniform_state(riemann):
    L, _ = _rand_faces()
    ps, us = O.interface_solve(cfg(riemann=riemann), L, L)
    np.testing.assert_allclose(ps, L[:, 2], rtol=1e-14)
    np.testing.assert_allclose(us, L[:, 1], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
def test_interface_mirror_symmetry(riemann):
    L, R = _rand_faces(seed=6)
    c = cfg(riemann=riemann)
    ps, us = O.interface_solve(c, L, R)
    Lm, Rm = R.copy(), L.copy()
    Lm[:, 1] *= -1
    Rm[:, 1] *= -1
    ps2, us2 = O.interface_solve(c, Lm, Rm)
    np.testing.assert_allclose(ps2, ps, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(us2, -us, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
def test_interface_characteristic_relations(riemann):
    # The acoustic solver's star state lies on the left characteristic
    # p* - p_L + Z_L (u* - u_L) = 0 and the right one p* - p_R - Z_R (u* - u_R) = 0,
    # with Z_k = rho_k max(c_L, c_R) (eqs. 13-14) or rho_k c_k (per side).
    L, R = _rand_faces(seed=7)
    ps, us = O.interface_solve(cfg(riemann=riemann), L, R)
    cL = np.sqrt(G * L[:, 2] / L[:, 0])
    cR = np.sqrt(G * R[:, 2] / R[:, 0])
    if riemann == "maxc":
        ZL, ZR = L[:, 0] * np.maximum(cL, cR), R[:, 0] * np.maximum(cL, cR)
    else:
        ZL, ZR = L[:, 0] * cL, R[:, 0] * cR
    scale = np.abs(L[:, 2]) + np.abs(R[:, 2]) + (ZL + ZR) * (np.abs(L[:, 1]) + np.abs(R[:, 1]) + 1)
    assert np.all(np.abs(ps - L[:, 2] + ZL * (us - L[:, 1])) <= 1e-13 * scale)
    assert np.all(np.abs(ps - R[:, 2] - ZR * (us - R[:, 1])) <= 1e-13 * scale)


def test_interface_weak_wave_limit_matches_exact_riemann():
    # Equal sound speeds, small jumps: eqs. (13)-(14) agree with the exact
    # Riemann star state up to O(eps^2).
    c = cfg()
    errs = []
    for eps in (4e-3, 2e-3, 1e-3):
        L = X.State(1.0, 0.2, 1.0)
        R = X.State(1.0 + eps, 0.2 - 0.5 * eps, 1.0 + eps)  # same c: p/rho constant
        st = X.star_region(L, R, G)
        ps, us = O.interface_solve(c, [[L.rho, L.u, L.p]], [[R.rho, R.u, R.p]])
        errs.append(abs(ps[0] - st.p) + abs(us[0] - st.u))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.15)
    assert errs[2] < 1e-5


def _euler_flux_x(q):
    rho, u, v, p = q.T
    E = p / (G - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho * u, rho * u * u + p, rho * u * v, (E + p) * u], axis=1)


def _rand_prims(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.1, 3, n), rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(0.05, 5, n)], axis=1)


@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
def test_flux_consistency(riemann):
    q = _rand_prims(400, 8)
    c = cfg(riemann=riemann)
    np.testing.assert_allclose(O.face_flux(c, 0, q, q), _euler_flux_x(q), rtol=1e-13, atol=1e-13)
    # y-direction flux of (rho,u,v,p) is the x flux of (rho,v,u,p) with momenta swapped
    qs = q[:, [0, 2, 1, 3]]
    Fy = O.face_flux(c, 1, q, q)
    np.testing.assert_allclose(Fy[:, [0, 2, 1, 3]], _euler_flux_x(qs), rtol=1e-13, atol=1e-13)


def test_flux_rotation_and_upwinding():
    c = cfg()
    qL, qR = _rand_prims(400, 9), _rand_prims(400, 10)
    Fx = O.face_flux(c, 0, qL, qR)
    Fy = O.face_flux(c, 1, qL[:, [0, 2, 1, 3]], qR[:, [0, 2, 1, 3]])
    np.testing.assert_allclose(Fy[:, [0, 2, 1, 3]], Fx, rtol=1e-14, atol=1e-14)
    # mass flux is rho_upwind * u*, with the upwind side picked by the sign of u*
    ps, us = O.interface_solve(c, qL[:, [0, 1, 3]], qR[:, [0, 1, 3]])
    rho_up = np.where(us > 0, qL[:, 0], qR[:, 0])
    np.testing.assert_allclose(Fx[:, 0], rho_up * us, rtol=1e-14, atol=1e-15)
    # momentum flux carries p*, energy flux carries p* u*
    u_up = np.where(us > 0, qL[:, 1], qR[:, 1])
    np.testing.assert_allclose(Fx[:, 1], rho_up * u_up * us + ps, rtol=1e-13, atol=1e-13)


def test_flux_reversal_is_conservative():
    # Flipping the face normal (swap sides, negate normal velocities) negates the flux.
    c = cfg()
    qL, qR = _rand_prims(400, 11), _rand_prims(400, 12)
    F = O.face_flux(c, 0, qL, qR)
    mL, mR = qR.copy(), qL.copy()
    mL[:, 1] *= -1
    mR[:, 1] *= -1
    Fm = O.face_flux(c, 0, mL, mR)
    # components: mass and energy flip sign, x-momentum (p* and rho u u*) stays, y-momentum flips
    np.testing.assert_allclose(Fm[:, [0, 2, 3]], -F[:, [0, 2, 3]], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Fm[:, 1], F[:, 1], rtol=1e-12, atol=1e-12)


def test_prim_cons_roundtrip_and_eos():
    c = O.OracleConfig(nx=3, ny=2)
    q = np.stack([np.full((2, 3), 1.3), np.full((2, 3), 0.4), np.full((2, 3), -0.2), np.full((2, 3), 0.9)])
    U = O.prim_to_cons(c, q)
    # rho E = p/(gamma-1) + rho |u|^2 / 2 = 0.9/0.4 + 0.65 * 0.2
    assert U[3, 0, 0] == pytest.approx(0.9 / 0.4 + 0.5 * 1.3 * 0.2, rel=1e-15)
    np.testing.assert_allclose(O.cons_to_prim(c, U), q, rtol=1e-14)


def test_cfl_dt_hand_value():
    # rho = 1.4, p = 1 -> c = 1; u = 0.5, v = -0.25 on a 10 x 10 unit square:
    # dt = 0.45 / ((0.5 + 1)/0.1 + (0.25 + 1)/0.1) = 0.45 / 27.5
    c = O.OracleConfig(nx=10, ny=10, cfl=0.45)
    q = np.stack([np.full((10, 10), 1.4), np.full((10, 10), 0.5), np.full((10, 10), -0.25), np.ones((10, 10))])
    assert O.cfl_dt(c, O.prim_to_cons(c, q)) == pytest.approx(0.45 / 27.5, rel=1e-14)
    c1 = O.OracleConfig(nx=10, dim=1, cfl=0.5)
    q1 = q[:, :1, :]
    assert O.cfl_dt(c1, O.prim_to_cons(c1, q1)) == pytest.approx(0.5 * 0.1 / 1.5, rel=1e-14)
    assert math.isfinite(O.cfl_dt(c1, O.prim_to_cons(c1, q1)))
