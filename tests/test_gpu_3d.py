"""The three-dimensional step on the GPU, through the C ABI, against the FP64
CPU oracle (itself pinned by tests/test_oracle_3d.py).

Bars: FP64 relative L1 <= 1e-12 per conservative field after tens of steps;
FP32 <= 2e-5 against the FP64 oracle on the same dt sequence.  Meshes are
ragged against every tiling of the kernel: FP32 strips of 60 output columns,
FP64 strips of 28, four output rows per CTA, 64 planes per z-tile.
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

from paper_1607_08710_gb300.lagflux import (Config, LagrangeFlux, LagrangeFluxError,  # noqa: E402
                                            lf_get_primitive, lf_set_state)

FP64_TOL = 1e-12
FP32_TOL = 2e-5


def rel_l1(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / (den if den > 0 else max(a.size, 1))


def gpu3(q, precision="fp64", steps=None, dts=None, host=False, lengths=(1.0, 1.0, 1.0), **kw):
    nz, ny, nx = q.shape[1:]
    cfg = Config(nx=nx, ny=ny, nz=nz, dim=3, precision=precision, xmax=lengths[0], ymax=lengths[1],
                 zmax=lengths[2], **kw)
    s = LagrangeFlux(cfg)
    if host:
        s.set_primitives(np.ascontiguousarray(q.astype(cfg.np_dtype)))
    else:
        s.set_primitives(torch.from_numpy(q).to("cuda", torch.float64 if precision == "fp64" else torch.float32))
    if dts is not None:
        for dt in dts:
            s.step_fixed(dt)
    else:
        s.run(max_steps=steps)
    U = s.get_conservative().astype(np.float64)
    t, n = s.time()
    s.close()
    return U, t, n


def oracle3(q, steps, dts=None, lengths=(1.0, 1.0, 1.0), **kw):
    nz, ny, nx = q.shape[1:]
    oc = O.OracleConfig(nx=nx, ny=ny, nz=nz, dim=3, lx=lengths[0], ly=lengths[1], lz=lengths[2], **kw)
    return O.run(oc, O.prim_to_cons(oc, q), steps, dts=dts)


def assert_close(U, ref, tol, fp32=False):
    for l in range(U.shape[0]):
        if fp32 and l in (1, 2, 3):  # momentum components against the momentum magnitude
            den = sum(np.abs(ref[m]).sum() for m in (1, 2, 3))
            e = np.abs(U[l] - ref[l]).sum() / den
        else:
            e = rel_l1(U[l], ref[l])
        assert e <= tol, f"field {l}: relative L1 {e:.3e} > {tol:.1e}"


@pytest.mark.parametrize("shape,bc,limiter", [((23, 29, 37), "transmissive", "vanleer"),
                                              ((70, 13, 20), "periodic", "minmod"),
                                              ((9, 8, 61), "transmissive", "sweby"),
                                              ((1, 7, 5), "periodic", "vanleer")])
def test_octant_fp64_against_oracle(shape, bc, limiter):
    nz, ny, nx = shape
    q = inputs.octant(nx, ny, nz, seed=nx + ny + nz).stack()
    kw = dict(bc=bc, limiter=limiter, beta=1.5, cfl=0.45)
    ref = oracle3(q, 30, lengths=(1.0, 1.3, 0.7), **kw)
    U, t, n = gpu3(q, "fp64", steps=30, lengths=(1.0, 1.3, 0.7), **kw)
    assert n == 30 and t == pytest.approx(ref.t, rel=1e-13)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
def test_ssprk3_and_per_side_fp64(riemann):
    q = inputs.octant(20, 15, 34, seed=9).stack()
    kw = dict(bc="periodic", limiter="vanleer", riemann=riemann, time_order=3, cfl=0.4)
    ref = oracle3(q, 20, **kw)
    U, _, _ = gpu3(q, "fp64", steps=20, **kw)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("kind", ["wave", "shear"])
def test_fp32_against_fp64_oracle(kind):
    if kind == "wave":
        q = inputs.smooth_wave_3d(64, 20, 36).stack()
    else:
        q = inputs.shear_layer_3d(64, 40, 33, seed=2).stack()
    kw = dict(bc="periodic", limiter="vanleer", cfl=0.45)
    ref = oracle3(q, 25, **kw)
    U, _, _ = gpu3(q, "fp32", dts=ref.dts, **kw)
    assert_close(U, ref.U, FP32_TOL, fp32=True)


def test_host_buffers_and_conservation():
    q = inputs.octant(33, 21, 40, seed=4).stack()
    kw = dict(bc="periodic", limiter="vanleer", cfl=0.45)
    s = LagrangeFlux(Config(nx=33, ny=21, nz=40, dim=3, **kw))
    s.set_primitives(np.ascontiguousarray(q))
    S0 = s.conservation_sums()
    assert S0.shape == (5,)
    s.run(max_steps=40)
    S1 = s.conservation_sums()
    U = s.get_conservative()
    for l in range(5):
        assert abs(S1[l] - S0[l]) <= 1e-13 * max(1.0, abs(S0[l]))
        assert S1[l] == pytest.approx(math.fsum(U[l].ravel()), rel=1e-15, abs=1e-15)
    qb = s.get_primitives()
    oc = O.OracleConfig(nx=33, ny=21, nz=40, dim=3)
    np.testing.assert_allclose(qb, O.cons_to_prim(oc, U), rtol=1e-14, atol=1e-15)
    s.close()


def test_run_graph_equals_direct_steps():
    q = inputs.shear_layer_3d(60, 24, 40, seed=1).stack()
    outs = []
    for mode in ("run", "step"):
        s = LagrangeFlux(Config(nx=60, ny=24, nz=40, dim=3, precision="fp32", bc="periodic"))
        s.set_primitives(torch.from_numpy(q).cuda().float())
        if mode == "run":
            assert s.run(max_steps=70)[0] == 70
        else:
            for _ in range(70):
                s.step()
        outs.append(s.get_conservative())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_full_size_sampled_cells_fp32():
    """384^3 periodic 3D shear layer, the benchmark's 3D launch configuration:
    one step checked at sampled cells against the oracle on a patch."""
    n = 384
    q = inputs.shear_layer_3d(n, seed=0).stack()
    kw = dict(bc="periodic", limiter="vanleer", cfl=0.45)
    s = LagrangeFlux(Config(nx=n, ny=n, nz=n, dim=3, precision="fp32", **kw))
    s.set_primitives(torch.from_numpy(q).cuda().float())
    del q
    U0 = s.get_conservative()
    dt = s.step(return_dt=True)
    U1 = torch.empty((5, n, n, n), dtype=torch.float32, device="cuda")
    s.get_conservative(U1)
    rng = np.random.default_rng(0)
    samples = [(0, 0, 0), (n - 1, n - 1, n - 1), (59, 60, 63), (60, 5, 64)]
    samples += [tuple(v) for v in rng.integers(0, n, (12, 3))]
    r = 5
    for ci, cj, ck in samples:
        ii, jj, kk = (np.arange(c - r, c + r + 1) % n for c in (ci, cj, ck))
        patch = np.ascontiguousarray(U0[:, kk][:, :, jj][:, :, :, ii].astype(np.float64))
        m = 2 * r + 1
        oc = O.OracleConfig(nx=m, ny=m, nz=m, dim=3, lx=m / n, ly=m / n, lz=m / n, limiter="vanleer")
        ref = O.run(oc, patch, 1, dts=[dt]).U[:, r, r, r]
        got = U1[:, ck, cj, ci].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), (ci, cj, ck, got, ref)
    s.close()


def test_3d_argument_errors():
    s = LagrangeFlux(Config(nx=8, ny=8, nz=8, dim=3))
    a = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    p = a.data_ptr()
    assert lf_set_state(s._h, p, p, p, p, 1) == 1  # four-plane calls describe 1D/2D states only
    assert lf_get_primitive(s._h, p, p, p, p, 1) == 1
    with pytest.raises(LagrangeFluxError) as ei:
        s.adjoint_forward(2)
    assert ei.value.status == 1
    s.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (40, 1, 1), (1, 1, 33), (1, 17, 1), (3, 2, 2), (65, 5, 3)])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_degenerate_and_thin_meshes_fp64(shape, bc):
    """Meshes of one cell along some axes (the step must reduce to the lower-
    dimensional scheme there) and tiny meshes smaller than one strip, one
    row block or one z-tile."""
    nz, ny, nx = shape
    q = inputs.octant(nx, ny, nz, seed=7).stack()
    kw = dict(bc=bc, limiter="vanleer", cfl=0.4)
    ref = oracle3(q, 12, **kw)
    U, _, _ = gpu3(q, "fp64", steps=12, **kw)
    assert_close(U, ref.U, FP64_TOL)


def test_nonphysical_state_is_flagged_3d():
    q = inputs.octant(16, 12, 10, seed=1).stack()
    q[4, 5, 6, 7] = -0.5  # negative pressure in one cell
    s = LagrangeFlux(Config(nx=16, ny=12, nz=10, dim=3))
    s.set_primitives(np.ascontiguousarray(q))
    with pytest.raises(LagrangeFluxError) as ei:
        s.run(max_steps=3)
    assert ei.value.status == 4  # LF_ERR_NONPHYSICAL
    s.close()


def octant_with_species(nx, ny, nz, ns, seed):
    base = inputs.octant(nx, ny, nz, seed=seed)
    rng = np.random.default_rng(seed)
    y = rng.uniform(0.0, 1.0, size=(ns, nz, ny, nx))
    return inputs.with_species(base, y).stack()


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("time_order", [2, 3])
def test_species_3d_fp64_against_oracle(ns, time_order):
    q = octant_with_species(37, 14, 23, ns, seed=ns + 10 * time_order)
    kw = dict(bc="periodic", limiter="vanleer", cfl=0.4, time_order=time_order, nspecies=ns)
    ref = oracle3(q, 20, **kw)
    U, _, _ = gpu3(q, "fp64", steps=20, **kw)
    assert U.shape[0] == 5 + ns
    assert_close(U, ref.U, FP64_TOL)


def test_species_3d_fp32_and_invariants():
    n = 40
    base = inputs.shear_layer_3d(n, 24, 20, seed=3)
    inside = np.abs(inputs.cell_centres(24)[None, :, None] - 0.5) < 0.25
    y1 = np.broadcast_to(inside, base.shape).astype(np.float64)
    q = inputs.with_species(base, np.stack([y1, 1.0 - y1])).stack()
    kw = dict(bc="periodic", limiter="vanleer", cfl=0.45, nspecies=2)
    ref = oracle3(q, 20, **kw)
    U, _, _ = gpu3(q, "fp32", dts=ref.dts, **kw)
    assert_close(U, ref.U, FP32_TOL, fp32=True)
    # complementary fractions keep summing to one; species mass is conserved
    s = LagrangeFlux(Config(nx=n, ny=24, nz=20, dim=3, **kw))
    s.set_primitives(np.ascontiguousarray(q))
    S0 = s.conservation_sums()
    assert S0.shape == (7,)
    s.run(max_steps=30)
    S1 = s.conservation_sums()
    for l in (0, 5, 6):
        assert abs(S1[l] - S0[l]) <= 1e-12 * abs(S0[l])
    rho_y = s.get_partial_densities()
    assert rho_y.shape == (2, 20, 24, n)
    U = s.get_conservative()
    assert np.abs(rho_y[0] + rho_y[1] - U[0]).max() <= 1e-13 * np.abs(U[0]).max()
    np.testing.assert_allclose(s.get_mass_fractions(), rho_y / U[0][None], rtol=1e-15, atol=0)
    qb = s.get_primitives()
    np.testing.assert_allclose(qb[5:], rho_y / U[0][None], rtol=1e-15, atol=0)
    s.close()
