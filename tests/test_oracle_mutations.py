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
    "muscl_half_dropped": ("qL[l] = q_at(l, d, -1, i, j, k) + 0.5 * sL;", "qL[l] = q_at(l, d, -1, i, j, k) + sL;"),
    "pstar_jump_sign": ("- (rL * rR / rs) * a * (uR - uL);", "+ (rL * rR / rs) * a * (uR - uL);"),
    "ustar_pressure_sign": ("- (pR - pL) / (rs * a);", "- (pL - pR) / (rs * a);"),
    "upwind_flipped": ("(val(ustar) > 0.0) ? qL : qR;", "(val(ustar) > 0.0) ? qR : qL;"),
    "slope_on_wrong_axis": ("S sL = limiter(c, q_at(l, d, -1, i, j, k) - q_at(l, d, -2, i, j, k),",
                            "S sL = limiter(c, q_at(l, d, -1, i, j, k) - q_at(l, 0, -2, i, j, k),"),
    "energy_flux_no_pu": ("F[e] = F[e] + pstar * ustar;", "F[e] = F[e];"),
    "heun_corrector_only": ("U[l][x] = U[l][x] - dt * ((bn + bs) / 2.0);", "U[l][x] = U[l][x] - dt * bs;"),
    "eos_half_dropped": ("q[e] = (c.gamma - 1.0) * rho * (E - 0.5 * kin);", "q[e] = (c.gamma - 1.0) * rho * (E - kin);"),
    "sweby_beta_both": ("min_first(S(beta * aa), bb)", "min_first(S(beta * aa), S(beta * bb))"),
    "limiter_sign_lost": ("return val(a) > 0.0 ? m : S(-m);", "return m;"),
    "balance_sign": ("acc = acc + A * ahead - A * behind;", "acc = acc + A * behind - A * ahead;"),
    "max_c_is_min": ("S a = max_first(cL, cR);", "S a = min_first(cL, cR);"),
    "dt_speed_of_one_axis": ("s = s + (abs_s(q[1 + d]) + a) / h[d];", "s = s + (abs_s(q[1]) + a) / h[d];"),
    "momentum_pressure_wrong_axis": ("F[1 + dir] = F[1 + dir] + pstar;", "F[1] = F[1] + pstar;"),
    "rk3_stage2_weight": ("U2[l][x] = 0.75 * U[l][x] + 0.25 *", "U2[l][x] = 0.70 * U[l][x] + 0.30 *"),
    "species_fraction_not_divided": ("q[e + 1 + k] = U[e + 1 + k] / rho;", "q[e + 1 + k] = U[e + 1 + k];"),
    "species_cons_without_rho": ("U[e + 1 + k] = rho * q[e + 1 + k];", "U[e + 1 + k] = q[e + 1 + k];"),
    "species_fraction_of_wrong_species": ("q[e + 1 + k] = U[e + 1 + k] / rho;",
                                          "q[e + 1 + k] = U[e + c.nspecies - k] / rho;"),
    "species_update_skips_last": ("for (int l = 0; l < nf; ++l) Us[l][x] = U[l][x] - dt",
                                  "for (int l = 0; l < nf - (c.nspecies > 0); ++l) Us[l][x] = U[l][x] - dt"),
    "w_missing_from_eos": ("kin = kin + q[1 + d] * q[1 + d];", "kin = kin + (d < 2 ? q[1 + d] * q[1 + d] : S(0.0));"),
    "face_area_one_factor": ("const double A = m.h[(d + 1) % 3] * m.h[(d + 2) % 3];",
                             "const double A = m.h[(d + 1) % 3];"),
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
    # 3D: a z-only tube equals the 1D scheme; an axis permutation commutes
    # with the step; the 3D CFL dt by hand
    n = 24
    tube = inputs.named_shock_tube("sod", n).stack()[:, 0, :]
    c1 = O.OracleConfig(nx=n, dim=1, limiter="minmod")
    dts3 = [3e-3] * 6
    try:
        r1 = O.run(c1, O.prim_to_cons(c1, tube[:, None, :]), 6, dts=dts3, allow_nonphysical=True).U[:, 0, :]
        q3 = np.zeros((5, n, 1, 1))
        q3[0, :, 0, 0], q3[3, :, 0, 0], q3[4, :, 0, 0] = tube[0], tube[1], tube[3]
        cz = O.OracleConfig(nx=1, ny=1, nz=n, dim=3, limiter="minmod")
        rz = O.run(cz, O.prim_to_cons(cz, q3), 6, dts=dts3, allow_nonphysical=True).U.reshape(5, n)
        check("z_tube_is_1d", np.allclose(rz[[0, 3, 4]], r1[[0, 1, 3]], rtol=1e-13, atol=1e-14))
    except O.OracleError:
        check("z_tube_is_1d", False)
    qo = inputs.octant(5, 4, 3, seed=1).stack()
    co = O.OracleConfig(nx=5, ny=4, nz=3, dim=3, lx=1.0, ly=1.3, lz=0.7)
    cp = O.OracleConfig(nx=3, ny=5, nz=4, dim=3, lx=0.7, ly=1.0, lz=1.3)
    perm = [2, 0, 1]  # new axis d = old axis perm[d]

    def relabel(U):
        order = [0] + [1 + (2 - perm[2 - p]) for p in range(3)]
        out = np.transpose(U, order).copy()
        for d in range(3):
            out[1 + d] = np.transpose(U[1 + perm[d]], [2 - perm[2 - p] for p in range(3)])
        return np.ascontiguousarray(out)
    try:
        ro = O.run(co, O.prim_to_cons(co, qo), 3, dts=[2e-3] * 3, allow_nonphysical=True).U
        rp = O.run(cp, O.prim_to_cons(cp, relabel(qo)), 3, dts=[2e-3] * 3, allow_nonphysical=True).U
        check("permute_3d", np.allclose(rp, relabel(ro), rtol=1e-12, atol=1e-13))
    except O.OracleError:
        check("permute_3d", False)
    one = np.ones((5, 8, 10))
    qd = np.stack([1.4 * one, 0.5 * one, -0.25 * one, 0.1 * one, one])
    cd3 = O.OracleConfig(nx=10, ny=8, nz=5, dim=3, cfl=0.45)
    check("dt_hand_3d", math.isclose(O.cfl_dt(cd3, O.prim_to_cons(cd3, qd)), 0.45 / (15 + 10 + 5.5), rel_tol=1e-12))
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
