"""Discrete adjoint (lf_adjoint_*) against forward-mode dual numbers of the CPU
oracle and against central finite differences.

States: the seeded Kelvin-Helmholtz shear layer (or a four-quadrant problem)
plus a seeded smooth background of amplitude 1e-3 on every field.  The plain
piecewise-constant states sit exactly on the limiter's kink phi(0, 0) and on
ties of max(c_L, c_R), where the objective is only directionally
differentiable; the background moves the state off those points.  The dt
sequence of the forward run is frozen for every derivative.
"""
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux, LagrangeFluxError, run_differentiable  # noqa: E402


def perturbed_state(nx, ny, kind="kh", seed=0, amp=1e-3):
    q = (inputs.kelvin_helmholtz(nx, ny, seed=seed) if kind == "kh" else inputs.quadrant(nx, ny, seed=seed)).stack()
    for l in range(4):
        q[l] += amp * inputs.smooth_perturbation(nx, ny, seed=10 * seed + l)
    return q


def gpu_adjoint(q0, nsteps, lam_T_fn, precision="fp64", passes="auto", **kw):
    """Forward nsteps, then backward with lambda_T = lam_T_fn(U_T); returns (U_T, dts, grad_q0).
    `passes`: how the reverse sweep forms the forward quantities ('tables',
    'direct' or the precision's default)."""
    ny, nx = q0.shape[1:]
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(Config(nx=nx, ny=ny, precision=precision, **kw))
    s.set_adjoint_passes(passes)
    q = torch.from_numpy(q0).to("cuda", tdt)
    s.set_primitive(q[0], q[1], q[2], q[3])
    dts = s.adjoint_forward(nsteps)
    UT = torch.empty((4, ny, nx), dtype=tdt, device="cuda")
    s.get_state(UT)
    lam = lam_T_fn(UT).to(tdt).contiguous()
    gq = torch.empty_like(UT)
    s.adjoint_backward(lam, grad_q0=gq)
    s.close()
    return UT.double().cpu().numpy(), dts, gq.double().cpu().numpy()


@pytest.mark.parametrize("passes", ["tables", "direct"])
@pytest.mark.parametrize("limiter,bc,kind", [("vanleer", "periodic", "kh"), ("minmod", "periodic", "kh"),
                                             ("sweby", "periodic", "kh"),
                                             ("sweby", "transmissive", "quadrant"),
                                             ("minmod", "transmissive", "quadrant"),
                                             ("vanleer", "transmissive", "quadrant")])
def test_dot_product_against_oracle_tangent(limiter, bc, kind, passes):
    """<lambda_T, dU(T)> of the oracle's dual-number tangent equals
    <grad_q0, dq0> of the GPU adjoint, FP64, for both forms of the reverse
    sweep (prep tables, direct recomputation: the FP32 default)."""
    nx, ny, nsteps = 24, 19, 23  # ragged, and 23 steps -> checkpoint segments 5,5,5,5,3
    kw = dict(limiter=limiter, bc=bc, cfl=0.4, beta=1.5)
    q0 = perturbed_state(nx, ny, kind, seed=3)
    rng = np.random.default_rng(7)
    lamT = rng.normal(size=(4, ny, nx))
    UT, dts, gq = gpu_adjoint(q0, nsteps, lambda U: torch.from_numpy(lamT).cuda(), passes=passes, **kw)
    oc = O.OracleConfig(nx=nx, ny=ny, limiter=limiter, bc=bc, cfl=0.4, beta=1.5)
    for trial in range(3):
        dq = rng.normal(size=(4, ny, nx))
        U_or, dU = O.run_tangent(oc, q0, dq, dts)
        np.testing.assert_allclose(UT, U_or, rtol=1e-11, atol=1e-12)
        lhs = float((lamT * dU).sum())
        rhs = float((gq * dq).sum())
        assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs)), (trial, lhs, rhs)


def _oracle_grad_component(args):
    oc_kw, q0, k, dts, wT = args
    oc = O.OracleConfig(**oc_kw)
    ny, nx = q0.shape[1:]
    field, cell = divmod(k, nx * ny)
    dq = np.zeros_like(q0)
    dq[(0, 3)[field]].flat[cell] = 1.0
    _, dU = O.run_tangent(oc, q0, dq, dts)
    return k, float((wT * dU[0]).sum())


def test_full_gradient_against_dual_numbers_32():
    """dJ/drho0 and dJ/dp0 of J = sum (rho(T) - rho_target)^2 on 32 x 32, every
    component by a forward-mode dual-number run of the oracle."""
    n, nsteps = 32, 64
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.4)
    q0 = perturbed_state(n, n, "kh", seed=1)
    qt = q0.copy()
    qt[0] += 1e-2 * inputs.smooth_perturbation(n, n, seed=99)
    oc_kw = dict(nx=n, ny=n, **kw)
    oc = O.OracleConfig(**oc_kw)
    rho_target = O.run(oc, O.prim_to_cons(oc, qt), nsteps).U[0]
    rt = torch.from_numpy(rho_target).cuda()

    def lam(U):
        out = torch.zeros_like(U)
        out[0] = 2.0 * (U[0] - rt)
        return out

    UT, dts, gq = gpu_adjoint(q0, nsteps, lam, **kw)
    wT = 2.0 * (UT[0] - rho_target)
    jobs = [(oc_kw, q0, k, dts, wT) for k in range(2 * n * n)]
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        res = dict(ex.map(_oracle_grad_component, jobs, chunksize=32))
    dual = np.array([res[k] for k in range(2 * n * n)]).reshape(2, n, n)
    adj = np.stack([gq[0], gq[3]])
    err = np.abs(adj - dual).max() / np.abs(dual).max()
    print("adjoint vs dual-number gradient, max relative error:", err)
    assert err <= 1e-9


def _J(solver, q, dts, rho_target):
    solver.set_primitive(q[0], q[1], q[2], q[3])
    for dt in dts:
        solver.step_fixed(dt)
    U = torch.empty((4,) + q.shape[1:], dtype=q.dtype, device="cuda")
    solver.get_state(U)
    return float(((U[0] - rho_target) ** 2).sum())


def test_finite_differences_512():
    """512 x 512 periodic shear layer, 256 steps at CFL 0.4: <grad, d> against
    central differences on 64 seeded smooth directions in (rho0, p0) (sums of
    low Fourier modes), with the dt sequence frozen; h scanned and the best h
    taken.  Grid-scale (white-noise) directions move limiter arguments across
    zero, where J is only piecewise smooth; they agree to ~3e-6 at h = 1e-9
    and are not used for the 1e-6 bar."""
    n, nsteps = 512, 256
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.4)
    q0 = perturbed_state(n, n, "kh", seed=2)
    qt = q0.copy()
    qt[0] += 1e-2 * inputs.smooth_perturbation(n, n, seed=98)
    s = LagrangeFlux(Config(nx=n, ny=n, precision="fp64", **kw))
    qtt = torch.from_numpy(qt).cuda()
    s.set_primitive(qtt[0], qtt[1], qtt[2], qtt[3])
    s.run(max_steps=nsteps)
    rho_target = torch.empty((4, n, n), dtype=torch.float64, device="cuda")
    s.get_state(rho_target)
    rho_target = rho_target[0].clone()

    def lam(U):
        out = torch.zeros_like(U)
        out[0] = 2.0 * (U[0] - rho_target)
        return out

    UT, dts, gq = gpu_adjoint(q0, nsteps, lam, **kw)
    gq = torch.from_numpy(gq).cuda()
    qd = torch.from_numpy(q0).cuda()
    worst = 0.0
    for k in range(64):
        d = torch.zeros_like(qd)
        d[0] = torch.from_numpy(inputs.smooth_perturbation(n, n, seed=1000 + 2 * k)).cuda()
        d[3] = torch.from_numpy(inputs.smooth_perturbation(n, n, seed=1001 + 2 * k)).cuda()
        ad = float((gq * d).sum())
        best = np.inf
        for h in (1e-7, 1e-8, 1e-6):
            fd = (_J(s, qd + h * d, dts, rho_target) - _J(s, qd - h * d, dts, rho_target)) / (2 * h)
            best = min(best, abs(fd - ad) / abs(ad))
            if best <= 1e-7:
                break
        worst = max(worst, best)
        assert best <= 1e-6, (k, best)
    print("finite differences vs adjoint, worst relative error over 64 directions:", worst)
    s.close()


def test_fp32_adjoint_against_fp64_on_the_shear_layer():
    """Reported, with a sanity bound only (the FP32 bound is held on a resolved
    state by test_fp32_adjoint_on_a_resolved_state).  The linearisation depends on the
    limiter's partial derivatives, functions of the ratio of neighbouring
    differences; with a 1e-3 background those differences are ~3e-5 on values
    of 1-2, which FP32 resolves to ~0.5%, so the FP32 adjoint differs from the
    FP64 one by percents (measured 2-11% at 512^2 after 4-256 steps)."""
    n, nsteps = 512, 256
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.4)
    q0 = perturbed_state(n, n, "kh", seed=4)
    rng = np.random.default_rng(3)
    lamT = torch.from_numpy(rng.normal(size=(4, n, n))).cuda()
    _, _, g64 = gpu_adjoint(q0, nsteps, lambda U: lamT, "fp64", **kw)
    _, _, g32 = gpu_adjoint(q0, nsteps, lambda U: lamT, "fp32", **kw)
    rel = [float(np.linalg.norm(g32[l] - g64[l]) / np.linalg.norm(g64[l])) for l in range(4)]
    print("FP32 vs FP64 adjoint, relative L2 per (rho, u, v, p):", rel)
    assert max(rel) <= 0.25


def smooth_state(n, seed=0, amp=0.2):
    """Smooth density wave (rho = 1 + 0.2 sin(2 pi (x + y)), u = v = 0.5,
    p = 1) with a seeded smooth background of amplitude `amp` on every
    field, so that neighbouring differences (~4e-2 at n = 32) are far above
    FP32 rounding and the limiter derivatives are well resolved."""
    q = inputs.smooth_wave(n, n).stack()
    for l in range(4):
        q[l] += amp * inputs.smooth_perturbation(n, n, seed=20 * seed + l)
    return q


@pytest.mark.parametrize("passes", ["direct", "tables"])
@pytest.mark.parametrize("limiter", ["vanleer", "minmod"])
def test_fp32_adjoint_on_a_resolved_state(limiter, passes):
    """FP32 adjoint against the FP64 adjoint on a state FP32 resolves: relative
    L2 <= 1e-4 per gradient field (measured 7e-6 van Leer, 4e-5 minmod), for
    the FP32 default (direct passes) and the table passes.  Both runs share
    the frozen dt and the derivative conventions; only rounding differs.
    The bound needs a state where no limiter argument sits within FP32
    rounding of a branch point (ab = 0, or |a| = |b| for minmod): there
    FP32 and FP64 take different branches and the local derivative changes
    by O(1).  On a 64^2 state with a 5% background over 40 steps a handful
    of such cells gives 1-2e-3, and on the shear layer (differences of
    3e-5) percents (test_fp32_adjoint_against_fp64_on_the_shear_layer)."""
    n, nsteps = 32, 20
    kw = dict(limiter=limiter, bc="periodic", cfl=0.4)
    q0 = smooth_state(n, seed=1)
    rng = np.random.default_rng(5)
    lamT = torch.from_numpy(rng.normal(size=(4, n, n))).cuda()
    _, _, g64 = gpu_adjoint(q0, nsteps, lambda U: lamT, "fp64", **kw)
    _, _, g32 = gpu_adjoint(q0, nsteps, lambda U: lamT, "fp32", passes=passes, **kw)
    rel = [float(np.linalg.norm(g32[l] - g64[l]) / np.linalg.norm(g64[l])) for l in range(4)]
    print(f"FP32 ({passes}) vs FP64 adjoint, {limiter}, relative L2 per (rho, u, v, p):", rel)
    assert max(rel) <= 1e-4, rel


def test_adjoint_one_call_and_host_buffers():
    """lf_adjoint (forward and backward in one call) and host buffers give the
    same gradient as the split device-buffer calls, bit for bit."""
    n, nsteps = 40, 12
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.4)
    q0 = perturbed_state(n, n, "kh", seed=8)
    rng = np.random.default_rng(9)
    lam_np = rng.normal(size=(4, n, n))
    _, dts_ref, gq_ref = gpu_adjoint(q0, nsteps, lambda U: torch.from_numpy(lam_np).cuda(), **kw)
    s = LagrangeFlux(Config(nx=n, ny=n, precision="fp64", **kw))
    q = torch.from_numpy(q0).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    gU_h = np.empty((4, n, n))
    gq_h = np.empty((4, n, n))
    dts = s.adjoint(nsteps, lam_np, grad_U0=gU_h, grad_q0=gq_h)
    np.testing.assert_array_equal(dts, dts_ref)
    np.testing.assert_array_equal(gq_h, gq_ref)
    gU_d = torch.empty((4, n, n), dtype=torch.float64, device="cuda")
    s.adjoint_backward(torch.from_numpy(lam_np).cuda(), grad_U0=gU_d)
    np.testing.assert_array_equal(gU_d.cpu().numpy(), gU_h)
    with pytest.raises(ValueError):
        s.adjoint_backward(lam_np, grad_q0=gU_d)  # mixed host and device buffers
    s.close()


def test_autograd_matches_direct_adjoint():
    n, nsteps = 48, 10
    q0 = perturbed_state(n, n, "kh", seed=6)
    s = LagrangeFlux(Config(nx=n, ny=n, precision="fp64", limiter="vanleer", bc="periodic", cfl=0.4))
    q = [torch.from_numpy(q0[l]).cuda().requires_grad_(True) for l in range(4)]
    U = run_differentiable(s, q[0], q[1], q[2], q[3], nsteps)
    loss = (U[0] ** 2).sum() + U[3].sum()
    loss.backward()
    s.close()

    def lam(UT):
        out = torch.zeros_like(UT)
        out[0] = 2.0 * UT[0]
        out[3] = 1.0
        return out

    _, _, gq = gpu_adjoint(q0, nsteps, lam, limiter="vanleer", bc="periodic", cfl=0.4)
    for l in range(4):
        np.testing.assert_allclose(q[l].grad.cpu().numpy(), gq[l], rtol=1e-13, atol=1e-13)


def test_adjoint_argument_errors():
    s = LagrangeFlux(Config(nx=16, ny=16))
    lam = torch.zeros((4, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(LagrangeFluxError) as ei:
        s.adjoint_backward(lam)
    assert ei.value.status == 6  # no forward run recorded
    s.close()
    s = LagrangeFlux(Config(nx=16, ny=16, riemann="per_side"))
    q = torch.from_numpy(inputs.quadrant(16, 16).stack()).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    with pytest.raises(LagrangeFluxError) as ei:
        s.adjoint_forward(4)
    assert ei.value.status == 1
    s.close()
