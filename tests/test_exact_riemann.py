"""Pins of the exact Riemann solver (the 'analytic solution' of Sec. 4.2).

The solver is checked against what the mathematics fixes, not against itself:
Rankine-Hugoniot conditions across every shock, constant entropy and Riemann
invariant through every rarefaction fan, continuity of p and u across the
contact, the symmetric problem, the small-amplitude acoustic limit, and the
star values tabulated in the textbook the paper cites.
"""
import math
import os

import numpy as np
import pytest

from oracle import exact_riemann as X

G = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TUBES = {
    "sod": (X.State(1.0, 0.0, 1.0), X.State(0.125, 0.0, 0.1)),
    "two_rarefaction": (X.State(1.0, -2.0, 0.4), X.State(1.0, 2.0, 0.4)),
    "sonic_rarefaction": (X.State(5.0, 0.0, 5.0), X.State(0.125, 0.0, 0.1)),
    "shock_shock": (X.State(1.0, 5.0, 1.0), X.State(1.0, -5.0, 0.01)),
    "strong_left": (X.State(1.0, 0.0, 1000.0), X.State(1.0, 0.0, 0.01)),
}


def _rh_residuals(pre: X.State, post_rho, post_u, post_p, S):
    """Mass, momentum and energy flux jumps in the frame of a shock of speed S."""
    w1, w2 = pre.u - S, post_u - S
    mass = pre.rho * w1 - post_rho * w2
    mom = pre.rho * w1 * w1 + pre.p - (post_rho * w2 * w2 + post_p)
    en = w1 * (0.5 * pre.rho * w1 * w1 + G / (G - 1) * pre.p) - w2 * (0.5 * post_rho * w2 * w2 + G / (G - 1) * post_p)
    return mass, mom, en


@pytest.mark.parametrize("name", sorted(TUBES))
def test_rankine_hugoniot_and_isentropes(name):
    L, R = TUBES[name]
    st = X.star_region(L, R, G)
    ws = X.wave_speeds(L, R, G)
    scale = max(L.p, R.p, L.rho, R.rho)
    if "left_shock" in ws:
        for r in _rh_residuals(L, st.rho_L, st.u, st.p, ws["left_shock"]):
            assert abs(r) < 1e-10 * scale * max(1.0, abs(ws["left_shock"])) ** 3
    else:
        # entropy p / rho^gamma and the invariant u + 2c/(gamma-1) through the left fan
        xi = np.linspace(ws["left_head"], ws["left_tail"], 17)
        rho, u, p = X.sample(L, R, xi, G)
        np.testing.assert_allclose(p / rho**G, L.p / L.rho**G, rtol=1e-10)
        c = np.sqrt(G * p / rho)
        np.testing.assert_allclose(u + 2 * c / (G - 1), L.u + 2 * L.c(G) / (G - 1), rtol=1e-10, atol=1e-12)
        # the fan is a centred simple wave: u - c = xi inside it
        np.testing.assert_allclose(u - c, xi, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(st.p / st.rho_L**G, L.p / L.rho**G, rtol=1e-10)
    if "right_shock" in ws:
        for r in _rh_residuals(R, st.rho_R, st.u, st.p, ws["right_shock"]):
            assert abs(r) < 1e-10 * scale * max(1.0, abs(ws["right_shock"])) ** 3
    else:
        xi = np.linspace(ws["right_tail"], ws["right_head"], 17)
        rho, u, p = X.sample(L, R, xi, G)
        np.testing.assert_allclose(p / rho**G, R.p / R.rho**G, rtol=1e-10)
        c = np.sqrt(G * p / rho)
        np.testing.assert_allclose(u - 2 * c / (G - 1), R.u - 2 * R.c(G) / (G - 1), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(u + c, xi, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("name", sorted(TUBES))
def test_contact_continuity(name):
    L, R = TUBES[name]
    st = X.star_region(L, R, G)
    eps = 1e-9
    rl, ul, pl = X.sample(L, R, np.array([st.u - eps]), G)
    rr, ur, pr = X.sample(L, R, np.array([st.u + eps]), G)
    assert pl[0] == pytest.approx(pr[0], rel=1e-12)
    assert ul[0] == pytest.approx(ur[0], rel=1e-12, abs=1e-12)
    assert rl[0] == pytest.approx(st.rho_L, rel=1e-12)
    assert rr[0] == pytest.approx(st.rho_R, rel=1e-12)


def test_symmetric_problem_has_zero_contact_velocity():
    L, R = TUBES["two_rarefaction"]
    st = X.star_region(L, R, G)
    assert abs(st.u) < 1e-14
    assert st.rho_L == pytest.approx(st.rho_R, rel=1e-14)


def test_uniform_state_is_its_own_star_state():
    s = X.State(0.7, 0.3, 0.9)
    st = X.star_region(s, s, G)
    assert st.p == pytest.approx(0.9, rel=1e-13)
    assert st.u == pytest.approx(0.3, rel=1e-13)


def test_acoustic_limit():
    # For a weak jump the exact star state agrees with the linear acoustic
    # solution with Z = rho c to second order in the amplitude.
    base = X.State(1.0, 0.1, 1.0)
    Z = base.rho * base.c(G)
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        R = X.State(1.0, 0.1 + 0.3 * eps, 1.0 + eps)
        st = X.star_region(base, R, G)
        p_lin = 0.5 * (base.p + R.p) - 0.5 * Z * (R.u - base.u)
        u_lin = 0.5 * (base.u + R.u) - 0.5 * (R.p - base.p) / Z
        errs.append(abs(st.p - p_lin) + abs(st.u - u_lin))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_textbook_star_values():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "toro_star_values.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        vals = [float(v) for v in row[1:]]
        st = X.star_region(X.State(*vals[0:3]), X.State(*vals[3:6]), G)
        assert round(st.p, 5) == pytest.approx(vals[6], abs=1.5e-5)
        assert round(st.u, 5) == pytest.approx(vals[7], abs=1.5e-5)


def test_solution_on_cells_is_piecewise_and_monotone_for_sod():
    L, R = TUBES["sod"]
    rho, u, p = X.solution_on_cells(L, R, 400, 0.2)
    assert rho[0] == 1.0 and rho[-1] == 0.125
    # Sod's density decreases monotonically from left to right
    assert np.all(np.diff(rho) <= 1e-14)
    assert math.isclose(p.max(), 1.0) and math.isclose(p.min(), 0.1)
