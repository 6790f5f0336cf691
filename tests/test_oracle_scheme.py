"""Pins of the oracle's whole Heun/RK2 Lagrange-flux step (Sec. 4).

What fixes the scheme independently of this code:
  * a uniform state is preserved exactly (all slopes and flux differences vanish);
  * a contact (uniform u, v, p) keeps u, v, p constant (follows from eqs. 12-14);
  * periodic meshes conserve mass, momentum and energy (telescoping fluxes);
  * the scheme commutes with the x<->y transpose and with mirror reflections;
  * a 2D run of data constant in y equals the 1D run row by row;
  * the shock tubes of Sec. 4.2 approach the exact Riemann solution, stay
    positive, and their L1 error falls as the mesh is refined;
  * second-order L1 convergence on the translated smooth wave;
  * the dual-number tangent equals central finite differences at smooth states.
"""
import math
import os

import numpy as np
import pytest

from oracle import exact_riemann as X
from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fsum_planes(U):
    return np.array([math.fsum(U[l].ravel()) for l in range(4)])


@pytest.mark.parametrize("dim,bc", [(1, "transmissive"), (1, "periodic"), (2, "transmissive"), (2, "periodic")])
def test_free_stream_is_preserved_exactly(dim, bc):
    n = 12
    c = O.OracleConfig(nx=n, ny=n if dim == 2 else 1, dim=dim, bc=bc)
    ny = n if dim == 2 else 1
    q = np.stack([np.full((ny, n), 0.8), np.full((ny, n), 0.3), np.full((ny, n), -0.6), np.full((ny, n), 0.7)])
    U0 = O.prim_to_cons(c, q)
    r = O.run(c, U0, 5)
    np.testing.assert_array_equal(r.U, U0)


def test_contact_keeps_velocity_and_pressure():
    n = 32
    c = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter="vanleer")
    U0 = O.prim_to_cons(c, inputs.smooth_wave(n).stack())
    r = O.run(c, U0, 40)
    q = O.cons_to_prim(c, r.U)
    assert np.abs(q[1] - 0.5).max() < 1e-13
    assert np.abs(q[2] - 0.5).max() < 1e-13
    assert np.abs(q[3] - 1.0).max() < 1e-13


@pytest.mark.parametrize("lim", ["minmod", "sweby", "vanleer"])
def test_periodic_conservation(lim):
    n = 32
    c = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter=lim)
    U0 = O.prim_to_cons(c, inputs.kelvin_helmholtz(n, seed=3).stack())
    r = O.run(c, U0, 25)
    s0, s1 = fsum_planes(U0), fsum_planes(r.U)
    scale = np.array([math.fsum(np.abs(U0[l]).ravel()) for l in range(4)])
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)


def _transpose_state(U):
    # swap the axes and the two momentum components
    return np.ascontiguousarray(U[[0, 2, 1, 3]].transpose(0, 2, 1))


@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_transpose_symmetry(bc):
    nx, ny = 20, 14
    c = O.OracleConfig(nx=nx, ny=ny, bc=bc)
    ct = O.OracleConfig(nx=ny, ny=nx, bc=bc)
    U0 = O.prim_to_cons(c, inputs.quadrant(nx, ny, seed=7).stack())
    dts = O.run(c, U0, 12).dts
    a = O.run(c, U0, 12, dts=dts).U
    b = O.run(ct, _transpose_state(U0), 12, dts=dts).U
    np.testing.assert_allclose(_transpose_state(b), a, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_mirror_symmetry(axis):
    n = 18
    c = O.OracleConfig(nx=n, ny=n, bc="transmissive")
    U0 = O.prim_to_cons(c, inputs.quadrant(n, seed=11).stack())

    def mirror(U):
        if axis == "x":
            M = U[:, :, ::-1].copy()
            M[1] *= -1
        else:
            M = U[:, ::-1, :].copy()
            M[2] *= -1
        return np.ascontiguousarray(M)

    dts = O.run(c, U0, 10).dts
    a = O.run(c, U0, 10, dts=dts).U
    b = O.run(c, mirror(U0), 10, dts=dts).U
    np.testing.assert_allclose(mirror(b), a, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_2d_with_y_constant_data_equals_1d(bc):
    nx, ny = 40, 6
    q1 = inputs.named_shock_tube("sod", nx).stack()
    c1 = O.OracleConfig(nx=nx, dim=1, bc=bc, limiter="sweby", beta=1.5, cfl=0.4)
    U1 = O.prim_to_cons(c1, q1)
    r1 = O.run(c1, U1, 15)
    c2 = O.OracleConfig(nx=nx, ny=ny, dim=2, bc=bc, limiter="sweby", beta=1.5)
    q2 = np.ascontiguousarray(np.repeat(q1, ny, axis=1))
    r2 = O.run(c2, O.prim_to_cons(c2, q2), 15, dts=r1.dts)
    for j in range(ny):
        np.testing.assert_allclose(r2.U[:, j, :], r1.U[:, 0, :], rtol=1e-13, atol=1e-14)


def _paper_tubes():
    rows = []
    for ln in open(os.path.join(GOLDEN, "paper_shock_tubes.txt")):
        if ln.strip() and not ln.startswith("#"):
            f = ln.split()
            rows.append(dict(name=f[0], L=tuple(map(float, f[1:4])), R=tuple(map(float, f[4:7])), T=float(f[7]),
                             cells=[int(v) for v in f[8].split(",")], cfl=float(f[9]), beta=float(f[10])))
    return rows


PAPER_TUBES = _paper_tubes()


def _run_tube(L, R, T, n, cfl, beta):
    c = O.OracleConfig(nx=n, dim=1, limiter="sweby", beta=beta, cfl=cfl)
    U0 = O.prim_to_cons(c, inputs.shock_tube(n, L, R).stack())
    r = O.run(c, U0, 10**6, t_end=T)
    assert r.t == pytest.approx(T, abs=1e-15)
    q = O.cons_to_prim(c, r.U)[:, 0, :]
    ex = X.solution_on_cells(X.State(*L), X.State(*R), n, T)
    return q, ex


@pytest.mark.parametrize("tube", PAPER_TUBES, ids=[f"{t['name']}-T{t['T']}" for t in PAPER_TUBES])
def test_paper_shock_tubes_against_exact_solution(tube):
    errs = []
    for n in tube["cells"] + [2 * tube["cells"][-1]]:
        q, (rho_e, u_e, p_e) = _run_tube(tube["L"], tube["R"], tube["T"], n, tube["cfl"], tube["beta"])
        # positivity of density, pressure and internal energy (claimed in Sec. 4.2)
        assert np.all(q[0] > 0) and np.all(q[3] > 0)
        errs.append(np.abs(q[0] - rho_e).mean() / np.abs(rho_e).mean())
        # velocity and pressure: at most a few percent relative L1 away from exact
        assert np.abs(q[3] - p_e).mean() / np.abs(p_e).mean() < 0.06
    assert errs[-1] < 0.03
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:]))


def test_shock_shock_has_no_contact_oscillation():
    # Sec. 4.2, last tube: no pressure or velocity oscillation at the contact.
    L, R = (1.0, 5.0, 1.0), (1.0, -5.0, 0.01)
    q, (rho_e, u_e, p_e) = _run_tube(L, R, 0.16, 400, 0.25, 1.0)
    st = X.star_region(X.State(*L), X.State(*R))
    ws = X.wave_speeds(X.State(*L), X.State(*R))
    x = inputs.cell_centres(400)
    inner = (x - 0.5 > ws["left_shock"] * 0.16 + 0.03) & (x - 0.5 < ws["right_shock"] * 0.16 - 0.03)
    assert inner.sum() > 20
    assert np.abs(q[3][inner] / st.p - 1).max() < 0.02
    assert np.abs(q[1][inner] - st.u).max() < 0.02 * abs(L[1])


def test_baseline_sod_case():
    # Sod on 1000 cells, minmod, CFL 0.5, t = 0.2 against the exact solution.
    n = 1000
    c = O.OracleConfig(nx=n, dim=1, limiter="minmod", cfl=0.5)
    U0 = O.prim_to_cons(c, inputs.named_shock_tube("sod", n).stack())
    r = O.run(c, U0, 10**6, t_end=0.2)
    q = O.cons_to_prim(c, r.U)[:, 0, :]
    rho_e, u_e, p_e = X.solution_on_cells(X.State(1, 0, 1), X.State(0.125, 0, 0.1), n, 0.2)
    assert np.abs(q[0] - rho_e).mean() < 2e-3
    assert np.abs(q[1] - u_e).mean() < 3e-3
    assert np.abs(q[3] - p_e).mean() < 2e-3
    # star-region plateau between the contact and the shock
    st = X.star_region(X.State(1, 0, 1), X.State(0.125, 0, 0.1))
    x = inputs.cell_centres(n)
    ws = X.wave_speeds(X.State(1, 0, 1), X.State(0.125, 0, 0.1))
    plateau = (x > 0.5 + st.u * 0.2 + 0.02) & (x < 0.5 + ws["right_shock"] * 0.2 - 0.02)
    assert np.abs(q[3][plateau] / st.p - 1).max() < 1e-3
    assert np.abs(q[0][plateau] / st.rho_R - 1).max() < 1e-2


@pytest.mark.parametrize("lim,min_order", [("vanleer", 1.9), ("minmod", 1.75)])
def test_second_order_convergence_smooth_wave(lim, min_order):
    T = 0.25
    errs = []
    for n in (32, 64, 128):
        c = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter=lim, cfl=0.45)
        r = O.run(c, O.prim_to_cons(c, inputs.smooth_wave(n).stack()), 10**6, t_end=T)
        q = O.cons_to_prim(c, r.U)
        errs.append(np.abs(q[0] - inputs.smooth_wave(n, t=T).rho).mean())
    order = math.log2(errs[1] / errs[2])
    assert order >= min_order
    assert errs[2] < 5e-4


def test_1d_second_order_convergence():
    T = 0.25
    errs = []
    for n in (64, 128, 256):
        c = O.OracleConfig(nx=n, dim=1, bc="periodic", limiter="vanleer", cfl=0.45)
        r = O.run(c, O.prim_to_cons(c, inputs.smooth_wave_1d(n).stack()), 10**6, t_end=T)
        errs.append(np.abs(O.cons_to_prim(c, r.U)[0] - inputs.smooth_wave_1d(n, t=T).rho).mean())
    assert math.log2(errs[1] / errs[2]) >= 1.9


def test_t_end_is_hit_exactly_and_dts_follow_cfl():
    n = 50
    c = O.OracleConfig(nx=n, dim=1, limiter="minmod", cfl=0.5)
    U0 = O.prim_to_cons(c, inputs.named_shock_tube("sod", n).stack())
    r = O.run(c, U0, 10**6, t_end=0.05)
    assert r.t == 0.05
    assert r.dts[0] == pytest.approx(O.cfl_dt(c, U0), rel=1e-15)
    assert r.dts[-1] <= r.dts[-2]


def test_nonphysical_state_is_reported():
    n = 8
    c = O.OracleConfig(nx=n, dim=1)
    q = inputs.named_shock_tube("sod", n).stack()
    q[3, 0, 3] = -0.5
    r = O.run(c, O.prim_to_cons(c, q), 1, dts=[1e-3], allow_nonphysical=True)
    assert r.status == O.NONPHYSICAL


@pytest.mark.parametrize("state", ["smooth", "kh_perturbed"])
def test_tangent_matches_central_differences(state):
    n = 16
    c = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter="vanleer", cfl=0.4)
    # A uniform field sits on the limiter's kink phi(0, 0), where J is only
    # directionally differentiable, so every field gets a smooth background.
    if state == "smooth":
        q0 = inputs.smooth_wave(n).stack()
        amp = 0.05
    else:
        q0 = inputs.kelvin_helmholtz(n, seed=2).stack()
        amp = 1e-3
    for l in range(4):
        q0[l] += amp * inputs.smooth_perturbation(n, seed=5 + l)
    U0 = O.prim_to_cons(c, q0)
    dts = O.run(c, U0, 6).dts
    rng = np.random.default_rng(4)
    d = np.zeros_like(q0)
    d[0] = rng.normal(size=(n, n))
    d[3] = rng.normal(size=(n, n))
    UT, dUT = O.run_tangent(c, q0, d, dts)
    np.testing.assert_allclose(UT, O.run(c, U0, 6, dts=dts).U, rtol=1e-14, atol=1e-14)
    # A white-noise direction moves some limiter arguments across zero for
    # large h (branch flips); scan h and take the plateau.
    errs = []
    for h in (1e-5, 1e-6, 1e-7, 1e-8):
        Up = O.run(c, O.prim_to_cons(c, q0 + h * d), 6, dts=dts).U
        Um = O.run(c, O.prim_to_cons(c, q0 - h * d), 6, dts=dts).U
        fd = (Up - Um) / (2 * h)
        errs.append(np.abs(fd - dUT).max() / np.abs(dUT).max())
    assert min(errs) < 1e-6


@pytest.mark.parametrize("order", [2, 3])
def test_time_steps_equal_butcher_form(order):
    # The oracle's Heun (flux average) and SSP-RK3 (Shu-Osher convex
    # combinations) steps against the same methods in Butcher form, built here
    # from the oracle's residual L(U): Heun k1 = L(U), k2 = L(U + dt k1),
    # U + dt (k1 + k2)/2; SSP-RK3 k3 = L(U + dt (k1 + k2)/4),
    # U + dt (k1/6 + k2/6 + 2 k3/3).
    n = 20
    c = O.OracleConfig(nx=n, ny=n + 3, bc="periodic", limiter="vanleer", time_order=order)
    U0 = O.prim_to_cons(c, inputs.kelvin_helmholtz(n, n + 3, seed=8).stack())
    dt = 0.5 * O.cfl_dt(c, U0)
    k1 = O.residual(c, U0)
    k2 = O.residual(c, U0 + dt * k1)
    if order == 2:
        ref = U0 + dt * (k1 + k2) / 2
    else:
        k3 = O.residual(c, U0 + dt * (k1 + k2) / 4)
        ref = U0 + dt * (k1 / 6 + k2 / 6 + 2 * k3 / 3)
    got = O.run(c, U0, 1, dts=[dt]).U
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)


def test_ssprk3_keeps_invariants():
    n = 24
    c = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter="vanleer", time_order=3)
    U0 = O.prim_to_cons(c, inputs.kelvin_helmholtz(n, n, seed=2).stack())
    r = O.run(c, U0, 20)
    s0, s1 = fsum_planes(U0), fsum_planes(r.U)
    scale = np.array([math.fsum(np.abs(U0[l]).ravel()) for l in range(4)])
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)
    cw = O.OracleConfig(nx=n, ny=n, bc="periodic", limiter="vanleer", time_order=3)
    q = O.cons_to_prim(cw, O.run(cw, O.prim_to_cons(cw, inputs.smooth_wave(n).stack()), 20).U)
    assert np.abs(q[1] - 0.5).max() < 1e-13 and np.abs(q[3] - 1.0).max() < 1e-13
