"""Transported mass fractions (Sec. 5) on the GPU, through the C ABI, against
the FP64 CPU oracle.

Bars as for the gas dynamics: FP64 relative L1 <= 1e-12 per conservative
field (rho, rho u, rho v, rho E, rho y_k) after up to 100 steps; FP32 <= 2e-5
against the FP64 oracle.  Plus invariants that hold at any size: the gas
fields do not depend on the species bit for bit, a constant fraction stays
constant, complementary fractions keep summing to one, and the species
masses are conserved on a periodic mesh.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import (Config, LagrangeFlux, LagrangeFluxBatch,  # noqa: E402
                                            LagrangeFluxError, lf_set_mass_fractions, lf_step_noalloc)

FP64_TOL = 1e-12
FP32_TOL = 2e-5


def rel_l1(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / (den if den > 0 else max(a.size, 1))


def gpu_species_run(prim, precision="fp64", steps=100, dts=None, host=False, lx=1.0, ly=1.0, **kw):
    """prim: (4 + ns, ny, nx) primitive planes with mass fractions.  Returns
    the conservative state (4 + ns planes) after the run, and (t, steps)."""
    nf, ny, nx = prim.shape
    ns = nf - 4
    dim = kw.pop("dim", 2 if ny > 1 else 1)
    cfg = Config(nx=nx, ny=ny, dim=dim, precision=precision, nspecies=ns, xmax=lx, ymax=ly, **kw)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(cfg)
    if host:
        q = np.ascontiguousarray(prim.astype(cfg.np_dtype))
        s.set_primitive(q[0], q[1], q[2], q[3])
        if ns:
            s.set_mass_fractions(np.ascontiguousarray(q[4:]))
    else:
        q = torch.from_numpy(prim).to("cuda", tdt)
        s.set_primitive(q[0], q[1], q[2], q[3])
        if ns:
            s.set_mass_fractions(q[4:].contiguous())
    if dts is not None:
        for dt in dts:
            s.step_fixed(dt)
    else:
        s.run(max_steps=steps)
    if host:
        U = np.concatenate([s.get_state()] + ([s.get_partial_densities()] if ns else [])).astype(np.float64)
    else:
        U = torch.empty((nf, ny, nx), dtype=tdt, device="cuda")
        s.get_state(U[:4])
        if ns:
            s.get_partial_densities(U[4:])
        U = U.double().cpu().numpy()
    t, n = s.time()
    s.close()
    return U, t, n


def oracle_run(prim, steps=100, lx=1.0, ly=1.0, **kw):
    nf, ny, nx = prim.shape
    dim = kw.pop("dim", 2 if ny > 1 else 1)
    oc = O.OracleConfig(nx=nx, ny=ny, dim=dim, nspecies=nf - 4, lx=lx, ly=ly, **kw)
    return O.run(oc, O.prim_to_cons(oc, prim), steps)


def assert_close(U, ref, tol):
    for l in range(U.shape[0]):
        if l in (1, 2) and tol > 1e-10:  # FP32: momentum components against the momentum magnitude
            den = np.abs(ref[1]).sum() + np.abs(ref[2]).sum()
            e = np.abs(U[l] - ref[l]).sum() / den
        else:
            e = rel_l1(U[l], ref[l])
        assert e <= tol, f"field {l}: relative L1 {e:.3e} > {tol:.1e}"


@pytest.mark.parametrize("time_order", [2, 3])
@pytest.mark.parametrize("case", ["quadrant", "three_region", "shear"])
def test_species_fp64_against_oracle(case, time_order):
    lx = ly = 1.0
    if case == "quadrant":  # ragged: 203 columns (8 FP64 strips), 97 rows (2 tiles)
        base = inputs.quadrant(203, 97, seed=11)
        y = np.random.default_rng(5).uniform(0.0, 1.0, size=(2, 97, 203))
        prim = inputs.with_species(base, y).stack()
        kw = dict(limiter="vanleer", bc="transmissive", cfl=0.45)
    elif case == "three_region":
        prim = inputs.three_region(140, 60, seed=2).stack()
        lx, ly = inputs.TRIPLE_DOMAIN
        kw = dict(limiter="sweby", beta=1.5, bc="transmissive", cfl=0.4)
    else:
        prim = inputs.shear_layer_tracers(96, 70, seed=4, nspecies=1).stack()
        kw = dict(limiter="minmod", bc="periodic", cfl=0.45)
    ref = oracle_run(prim, 100, lx=lx, ly=ly, time_order=time_order, **kw)
    U, t, n = gpu_species_run(prim, "fp64", 100, lx=lx, ly=ly, time_order=time_order, **kw)
    assert n == 100 and t == pytest.approx(ref.t, rel=1e-13)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("nx,ns", [(1000, 1), (61, 2), (29, 2)])
def test_species_1d_fp64(nx, ns):
    base = inputs.named_shock_tube("sod", nx)
    x = inputs.cell_centres(nx)[None, :]
    ys = [np.where(x < 0.5, 1.0, 0.0), 0.5 + 0.3 * np.sin(6 * math.pi * x)][:ns]
    prim = inputs.with_species(base, np.stack(ys)).stack()
    kw = dict(limiter="minmod", cfl=0.5)
    ref = oracle_run(prim, 100, **kw)
    U, _, _ = gpu_species_run(prim, "fp64", 100, **kw)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("kind", ["advected", "shear"])
def test_species_fp32_against_fp64_oracle(kind):
    if kind == "advected":
        prim = inputs.advected_scalar(130, 70).stack()
        kw = dict(limiter="vanleer", bc="periodic", cfl=0.45)
    else:
        prim = inputs.shear_layer_tracers(128, 96, seed=7, nspecies=2).stack()
        kw = dict(limiter="vanleer", bc="periodic", cfl=0.45)
    ref = oracle_run(prim, 40, **kw)
    U, _, _ = gpu_species_run(prim, "fp32", steps=None, dts=ref.dts, **kw)
    assert_close(U, ref.U, FP32_TOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("time_order", [2, 3])
def test_gas_dynamics_bitwise_independent_of_species(precision, time_order):
    base = inputs.kelvin_helmholtz(150, 90, seed=3)
    kw = dict(limiter="sweby", beta=1.5, bc="periodic", cfl=0.45, time_order=time_order)
    U0, t0, _ = gpu_species_run(base.stack(), precision, 37, **kw)
    y = np.random.default_rng(3).uniform(0, 1, size=(2,) + base.shape)
    U2, t2, _ = gpu_species_run(inputs.with_species(base, y).stack(), precision, 37, **kw)
    assert t0 == t2
    assert np.array_equal(U0, U2[:4])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 1e-5)])
def test_constant_fraction_stays_constant_gpu(precision, tol):
    base = inputs.quadrant(120, 90, seed=8)
    prim = inputs.with_species(base, np.full((1,) + base.shape, 0.37)).stack()
    U, _, _ = gpu_species_run(prim, precision, 60, limiter="vanleer", cfl=0.45)
    assert np.abs(U[4] - 0.37 * U[0]).max() <= tol * np.abs(U[0]).max()


def test_complementary_fractions_and_species_mass_on_gpu():
    prim = inputs.shear_layer_tracers(160, 128, seed=5, nspecies=2).stack()
    cfg = Config(nx=160, ny=128, precision="fp64", nspecies=2, bc="periodic", limiter="vanleer")
    s = LagrangeFlux(cfg)
    q = torch.from_numpy(prim).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    s.set_mass_fractions(q[4:].contiguous())
    S0 = s.conservation_sums()
    assert S0.shape == (6,)
    s.run(max_steps=80)
    S1 = s.conservation_sums()
    for l in (0, 4, 5):
        assert abs(S1[l] - S0[l]) <= 1e-12 * abs(S0[l])
    rho_y = s.get_partial_densities()
    rho = s.get_state()[0]
    assert np.abs(rho_y[0] + rho_y[1] - rho).max() <= 1e-13 * np.abs(rho).max()
    y = s.get_mass_fractions()
    np.testing.assert_allclose(y, rho_y / rho[None], rtol=1e-15, atol=0)
    s.close()


def test_host_partial_densities_round_trip():
    prim = inputs.three_region(70, 30, seed=1).stack()
    oc = O.OracleConfig(nx=70, ny=30, nspecies=2, lx=7.0, ly=3.0, limiter="minmod")
    U0 = O.prim_to_cons(oc, prim)
    s = LagrangeFlux(Config(nx=70, ny=30, nspecies=2, xmax=7.0, ymax=3.0, limiter="minmod"))
    s.set_state(*[np.ascontiguousarray(U0[l]) for l in range(4)])
    s.set_partial_densities(np.ascontiguousarray(U0[4:]))
    assert np.array_equal(s.get_partial_densities(), U0[4:])
    ref = O.run(oc, U0, 50)
    s.run(max_steps=50)
    U = np.concatenate([s.get_state(), s.get_partial_densities()])
    assert_close(U, ref.U, FP64_TOL)
    s.close()


def test_full_size_8192_species_fp32():
    """8192^2 periodic shear layer with two tracers, the benchmark's species
    launch configuration: one step checked at sampled cells against the
    oracle on a patch, then 20 more steps against the invariants."""
    n = 8192
    prim = inputs.shear_layer_tracers(n, n, seed=0, nspecies=2).stack()
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.45)
    s = LagrangeFlux(Config(nx=n, ny=n, precision="fp32", nspecies=2, **kw))
    q = torch.from_numpy(prim).to("cuda", torch.float32)
    del prim
    s.set_primitive(q[0], q[1], q[2], q[3])
    s.set_mass_fractions(q[4:].contiguous())
    del q
    U0 = torch.empty((6, n, n), dtype=torch.float32, device="cuda")
    s.get_state(U0[:4])
    s.get_partial_densities(U0[4:])
    U0h = U0.cpu().numpy()
    dt = s.step(return_dt=True)
    s.get_state(U0[:4])
    s.get_partial_densities(U0[4:])
    rng = np.random.default_rng(1)
    samples = [(0, 0), (n - 1, n - 1), (n // 2, n // 4), (4095, 2048)] + [tuple(v) for v in rng.integers(0, n, (16, 2))]
    r = 6
    for ci, cj in samples:
        ii, jj = np.arange(ci - r, ci + r + 1) % n, np.arange(cj - r, cj + r + 1) % n
        patch = np.ascontiguousarray(U0h[:, jj][:, :, ii].astype(np.float64))
        oc = O.OracleConfig(nx=2 * r + 1, ny=2 * r + 1, lx=(2 * r + 1) / n, ly=(2 * r + 1) / n, nspecies=2,
                            limiter="vanleer")
        ref = O.run(oc, patch, 1, dts=[dt]).U[:, r, r]
        got = U0[:, cj, ci].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), (ci, cj, got, ref)
    del U0h
    s.run(max_steps=20)
    s.get_state(U0[:4])
    s.get_partial_densities(U0[4:])
    rho = U0[0].double()
    err = (U0[4].double() + U0[5].double() - rho).abs().max().item()
    assert err <= 2e-6 * rho.abs().max().item()
    s.close()


def test_species_argument_errors():
    s = LagrangeFlux(Config(nx=16, ny=16))
    y = torch.zeros((1, 16, 16), dtype=torch.float64, device="cuda")
    assert lf_set_mass_fractions(s._h, y.data_ptr(), 1) == 1  # the C call on a context without species
    with pytest.raises(ValueError):  # the binding checks the buffer size first
        s.set_mass_fractions(y)
    s.close()
    s = LagrangeFlux(Config(nx=16, ny=16, nspecies=1))
    q = torch.from_numpy(inputs.quadrant(16, 16).stack()).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    with pytest.raises(LagrangeFluxError) as ei:
        s.adjoint_forward(4)
    assert ei.value.status == 1
    s.close()
    with pytest.raises(LagrangeFluxError):
        LagrangeFluxBatch([Config(nx=16, ny=16, nspecies=1)])
    c = Config(nx=16, ny=16, nspecies=1).to_c()
    U = torch.zeros((5, 16, 16), dtype=torch.float64, device="cuda")
    st = lf_step_noalloc(c, U.data_ptr(), U.data_ptr(), 1e-3, None, None)
    assert st == 1
