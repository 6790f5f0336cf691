"""Planted mistakes in the oracle must be caught by its pins.

Each case edits one plausible slip into a private copy of the oracle source
(a dropped term, a flipped sign, a wrong index or branch), compiles it on the
CPU and runs a battery of the independent checks used to pin the oracle.
At least one check must fail for every mutant, and all checks must pass for
the unmodified source -- so the pins are shown to bite.
"""
import math
import os
import tempfile
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import exact_riemann as X
from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

MUTANTS = {
    "muscl_half_dropped": ("qL[l] = q_at(l, iL, j) + 0.5 * sL;", "qL[l] = q_at(l, iL, j) + sL;"),
    "pstar_jump_sign": ("- (rL * rR / rs) * a * (uR - uL);", "+ (rL * rR / rs) * a * (uR - uL);"),
    "ustar_pressure_sign": ("- (pR - pL) / (rs * a);", "- (pL - pR) / (rs * a);"),
    "upwind_flipped": ("(val(ustar) > 0.0) ? qL : qR;", "(val(ustar) > 0.0) ? qR : qL;"),
    "y_slope_wrong_axis": ("S sL = limiter(c, q_at(l, i, jL) - q_at(l, i, jL - 1),",
                           "S sL = limiter(c, q_at(l, i, jL) - q_at(l, i - 1, jL),"),
    "energy_flux_no_pu": ("F[3] = F[3] + pstar * ustar;", "F[3] = F[3];"),
    "heun_corrector_only": ("U[l][k] = U[l][k] - dt * ((bn + bs) / 2.0);", "U[l][k] = U[l][k] - dt * bs;"),
    "eos_half_dropped": ("q[3] = (c.gamma - 1.0) * rho * (E - 0.5 * (u * u + v * v));",
                         "q[3] = (c.gamma - 1.0) * rho * (E - (u * u + v * v));"),
    "sweby_beta_both": ("min_first(S(beta * aa), bb)", "min_first(S(beta * aa), S(beta * bb))"),
    "limiter_sign_lost": ("return val(a) > 0.0 ? m : S(-m);", "return m;"),
    "y_balance_sign": ("Ay * north - Ay * south", "Ay * south - Ay * north"),
    "max_c_is_min": ("S a = max_first(cL, cR);", "S a = min_first(cL, cR);"),
    "dt_without_y": ("if (c.dim == 2) s += (std::fabs(q[2]) + a) / c.dy;", ""),
    "momentum_pressure_wrong_axis": ("F[1 + dir] = F[1 + dir] + pstar;", "F[1] = F[1] + pstar;"),
    "rk3_stage2_weight": ("U2[l][k] = 0.75 * U[l][k] + 0.25 *", "U2[l][k] = 0.70 * U[l][k] + 0.30 *"),
    "species_fraction_not_divided": ("q[4 + k] = U[4 + k] / rho;", "q[4 + k] = U[4 + k];"),
    "species_cons_without_rho": ("U[4 + k] = rho * q[4 + k];", "U[4 + k] = q[4 + k];"),
    "species_fraction_of_wrong_species": ("q[4 + k] = U[4 + k] / rho;", "q[4 + k] = U[4 + c.nspecies - 1 - k] / rho;"),
    "species_update_skips_last": ("for (int l = 0; l < nf; ++l) Us[l][k] = U[l][k] - dt",
                                  "for (int l = 0; l < nf - (nf > 4); ++l) Us[l][k] = U[l][k] - dt"),
}


def battery():
    """Independent checks (closed forms, invariants, exact solutions); returns failures."""
    fails = []

    def check(name, cond):
        if not cond:
            fails.append(name)

    c = O.OracleConfig(nx=4, ny=4, limiter="sweby", beta=2.0)
    # superbee at beta = 2; minmod; van Leer; oddness
    got = O.limiter(c, [1.0, 1.0, -2.0], [3.0, 0.6, -1.0])
    check("superbee_values", np.allclose(got, [2.0, 1.0, -2.0]))
    got = O.limiter(O.OracleConfig(nx=4, ny=4, limiter="sweby", beta=1.5), [1.0, -2.0], [3.0, -1.0])
    check("sweby_values", np.allclose(got, [1.5, -1.5]))
    # acoustic characteristic relations of eqs. (13)-(14)
    rng = np.random.default_rng(0)
    L = np.stack([rng.uniform(0.2, 2, 50), rng.uniform(-1, 1, 50), rng.uniform(0.1, 2, 50)], 1)
    R = np.stack([rng.uniform(0.2, 2, 50), rng.uniform(-1, 1, 50), rng.uniform(0.1, 2, 50)], 1)
    ps, us = O.interface_solve(c, L, R)
    a = np.maximum(np.sqrt(1.4 * L[:, 2] / L[:, 0]), np.sqrt(1.4 * R[:, 2] / R[:, 0]))
    check("char_left", np.allclose(ps - L[:, 2] + L[:, 0] * a * (us - L[:, 1]), 0, atol=1e-12))
    check("char_right", np.allclose(ps - R[:, 2] - R[:, 0] * a * (us - R[:, 1]), 0, atol=1e-12))
    # flux consistency with the physical flux in both directions
    q = np.stack([rng.uniform(0.2, 2, 20), rng.uniform(-1, 1, 20), rng.uniform(-1, 1, 20), rng.uniform(0.1, 2, 20)], 1)
    E = q[:, 3] / 0.4 + 0.5 * q[:, 0] * (q[:, 1] ** 2 + q[:, 2] ** 2)
    Fx = np.stack([q[:, 0] * q[:, 1], q[:, 0] * q[:, 1] ** 2 + q[:, 3], q[:, 0] * q[:, 1] * q[:, 2], (E + q[:, 3]) * q[:, 1]], 1)
    Fy = np.stack([q[:, 0] * q[:, 2], q[:, 0] * q[:, 1] * q[:, 2], q[:, 0] * q[:, 2] ** 2 + q[:, 3], (E + q[:, 3]) * q[:, 2]], 1)
    check("flux_x", np.allclose(O.face_flux(c, 0, q, q), Fx, atol=1e-12))
    check("flux_y", np.allclose(O.face_flux(c, 1, q, q), Fy, atol=1e-12))
    # hand-computed CFL dt (rho 1.4, p 1 -> c 1; u .5, v -.25 on 10x10)
    cd = O.OracleConfig(nx=10, ny=10, cfl=0.45)
    qd = np.stack([np.full((10, 10), 1.4), np.full((10, 10), 0.5), np.full((10, 10), -0.25), np.ones((10, 10))])
    check("dt_hand", math.isclose(O.cfl_dt(cd, O.prim_to_cons(cd, qd)), 0.45 / 27.5, rel_tol=1e-12))
    # conservation on a periodic mesh
    cp = O.OracleConfig(nx=16, ny=16, bc="periodic")
    U0 = O.prim_to_cons(cp, inputs.kelvin_helmholtz(16, 16, seed=1).stack())
    try:
        r = O.run(cp, U0, 8, allow_nonphysical=True)
        drift = [abs(math.fsum(r.U[l].ravel()) - math.fsum(U0[l].ravel())) for l in range(4)]
        check("conservation", max(drift) < 1e-11 and np.all(np.isfinite(r.U)))
    except O.OracleError:
        check("conservation", False)
    # transpose symmetry on a non-square quadrant problem
    ct, ctt = O.OracleConfig(nx=12, ny=9), O.OracleConfig(nx=9, ny=12)
    Uq = O.prim_to_cons(ct, inputs.quadrant(12, 9, seed=3).stack())
    dts = [2e-3] * 5
    a1 = O.run(ct, Uq, 5, dts=dts, allow_nonphysical=True).U
    b1 = O.run(ctt, np.ascontiguousarray(Uq[[0, 2, 1, 3]].transpose(0, 2, 1)), 5, dts=dts, allow_nonphysical=True).U
    check("transpose", np.allclose(b1[[0, 2, 1, 3]].transpose(0, 2, 1), a1, rtol=1e-11, atol=1e-12))
    # Sod against the exact solution
    n = 200
    c1 = O.OracleConfig(nx=n, dim=1, limiter="minmod", cfl=0.5)
    try:
        rs = O.run(c1, O.prim_to_cons(c1, inputs.named_shock_tube("sod", n).stack()), 10**5, t_end=0.2,
                   allow_nonphysical=True)
        qs = O.cons_to_prim(c1, rs.U)[:, 0, :]
        rho_e, _, p_e = X.solution_on_cells(X.State(1, 0, 1), X.State(0.125, 0, 0.1), n, 0.2)
        check("sod_exact", np.abs(qs[0] - rho_e).mean() < 6e-3 and np.abs(qs[3] - p_e).mean() < 5e-3)
    except O.OracleError:
        check("sod_exact", False)
    # second-order convergence on the 1D smooth wave
    errs = []
    for m in (64, 128):
        cw = O.OracleConfig(nx=m, dim=1, bc="periodic", limiter="vanleer")
        try:
            rw = O.run(cw, O.prim_to_cons(cw, inputs.smooth_wave_1d(m).stack()), 10**5, t_end=0.2,
                       allow_nonphysical=True)
            errs.append(np.abs(O.cons_to_prim(cw, rw.U)[0] - inputs.smooth_wave_1d(m, t=0.2).rho).mean())
        except O.OracleError:
            errs.append(np.inf)
    check("order2", np.all(np.isfinite(errs)) and errs[1] > 0 and math.log2(errs[0] / errs[1]) > 1.8)
    # SSP-RK3 step against its Butcher form built from the residual
    c3 = O.OracleConfig(nx=10, ny=12, bc="periodic", time_order=3)
    U3 = O.prim_to_cons(c3, inputs.kelvin_helmholtz(10, 12, seed=4).stack())
    dt = 0.5 * O.cfl_dt(c3, U3)
    k1 = O.residual(c3, U3)
    k2 = O.residual(c3, U3 + dt * k1)
    k3 = O.residual(c3, U3 + dt * (k1 + k2) / 4)
    ref = U3 + dt * (k1 / 6 + k2 / 6 + 2 * k3 / 3)
    got = O.run(c3, U3, 1, dts=[dt], allow_nonphysical=True).U
    check("rk3_butcher", np.allclose(got, ref, rtol=1e-12, atol=1e-13))
    # species: a constant fraction stays constant; y_2 = 1 - y_1 keeps summing
    # to one; uniform-flow advection of y converges at second order
    cs = O.OracleConfig(nx=12, ny=9, nspecies=2)
    ps = inputs.quadrant(12, 9, seed=2)
    ys = np.stack([np.full((9, 12), 0.3), np.random.default_rng(1).uniform(0, 1, (9, 12))])
    ys[1] = np.where(ys[1] > 0.5, 1.0, 0.0)
    try:
        Us = O.run(cs, O.prim_to_cons(cs, np.concatenate([ps.stack(), ys])), 6, allow_nonphysical=True).U
        check("species_constant", np.abs(Us[4] - 0.3 * Us[0]).max() < 1e-13)
    except O.OracleError:
        check("species_constant", False)
    c2 = O.OracleConfig(nx=40, ny=20, lx=7.0, ly=3.0, nspecies=2)
    try:
        U2s = O.run(c2, O.prim_to_cons(c2, inputs.three_region(40, 20, seed=1).stack()), 8, allow_nonphysical=True).U
        check("species_sum", np.abs(U2s[4] + U2s[5] - U2s[0]).max() < 1e-13)
    except O.OracleError:
        check("species_sum", False)
    es = []
    for m in (64, 128):
        ca = O.OracleConfig(nx=m, dim=1, bc="periodic", nspecies=1, cfl=0.4)
        try:
            ra = O.run(ca, O.prim_to_cons(ca, inputs.advected_scalar_1d(m).stack()), 10**5, t_end=0.25,
                       allow_nonphysical=True)
            es.append(np.abs(ra.U[4, 0] / ra.U[0, 0] - inputs.advected_scalar_1d(m, t=0.25).y[0, 0]).mean())
        except O.OracleError:
            es.append(np.inf)
    check("species_order2", np.all(np.isfinite(es)) and es[1] > 0 and math.log2(es[0] / es[1]) > 1.75)
    return fails


@pytest.fixture(scope="module")
def mutant_libs():
    src = O.source_text()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")

    def make(item):
        name, (old, new) = item
        assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
        return name, O.compile_variant(src.replace(old, new), os.path.join(tmp, f"{name}.so"))

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(make, MUTANTS.items()))


def test_unmodified_oracle_passes_battery():
    assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(mutant_libs, name):
    with O.use_library(mutant_libs[name]):
        fails = battery()
    assert fails, f"planted mistake {name} went undetected"
