"""GPU (CUDA, through the C ABI) against the FP64 CPU oracle.

Bars:
  * FP64: relative L1 <= 1e-12 per conservative field after up to 100 steps
    (the two sides differ only in rounding order and FMA contraction).
  * FP32: relative L1 <= 2e-5 per field against the FP64 oracle on the same
    input after tens of steps (single-precision rounding, ~6e-8 per
    operation, grown through the run; the bound for the smooth-flow precision
    study is 1e-5, checked in test_gpu_precision.py).
Sizes span several warp strips (60 output columns in FP32, 28 in FP64) and 64-row tiles with
ragged tails.
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

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux, LagrangeFluxError  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 2e-5


def rel_l1(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.abs(b).sum()
    if den == 0.0:
        return np.abs(a - b).sum() / max(a.size, 1)
    return np.abs(a - b).sum() / den


def gpu_run(prim, precision="fp64", steps=None, t_end=0.0, dts=None, host=False, **kw):
    ny, nx = prim.shape[1], prim.shape[2]
    dim = kw.pop("dim", 2 if ny > 1 else 1)
    cfg = Config(nx=nx, ny=ny, dim=dim, precision=precision, **kw)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(cfg)
    if host:
        q = np.ascontiguousarray(prim.astype(cfg.np_dtype))
        s.set_primitive(q[0], q[1], q[2], q[3])
    else:
        q = torch.from_numpy(prim).to("cuda", tdt)
        s.set_primitive(q[0], q[1], q[2], q[3])
    if dts is not None:
        for dt in dts:
            s.step_fixed(dt)
        n, t = len(dts), None
    else:
        n, t = s.run(t_end=t_end, max_steps=steps if steps is not None else 2**31 - 1)
    if host:
        U = s.get_state().astype(np.float64)
    else:
        out = torch.empty((4, ny, nx), dtype=tdt, device="cuda")
        s.get_state(out)
        U = out.double().cpu().numpy()
    tt, nsteps = s.time()
    s.close()
    return U, nsteps, tt


def oracle_cfg(prim, **kw):
    ny, nx = prim.shape[1], prim.shape[2]
    dim = kw.pop("dim", 2 if ny > 1 else 1)
    return O.OracleConfig(nx=nx, ny=ny, dim=dim, **kw)


def assert_close(U, ref, tol):
    for l in range(4):
        e = rel_l1(U[l], ref[l])
        assert e <= tol, f"field {l}: relative L1 {e:.3e} > {tol:.1e}"


def assert_close_fp32(U, ref, tol=FP32_TOL):
    """FP32 against the FP64 oracle: a momentum component is measured against
    the momentum vector's magnitude, since a small component (e.g. the 1%
    shear-layer perturbation) is computed from terms as large as the other
    one and carries their single-precision rounding."""
    for l in range(4):
        den = np.abs(ref[l]).sum() if l in (0, 3) else np.abs(ref[1]).sum() + np.abs(ref[2]).sum()
        e = np.abs(np.asarray(U[l], np.float64) - ref[l]).sum() / (den if den > 0 else 1.0)
        assert e <= tol, f"field {l}: relative L1 {e:.3e} > {tol:.1e}"


def test_sod_1000_cells_fp64():
    prim = inputs.named_shock_tube("sod", 1000).stack()
    kw = dict(limiter="minmod", cfl=0.5)
    ref = O.run(oracle_cfg(prim, **kw), O.prim_to_cons(oracle_cfg(prim, **kw), prim), 10**6, t_end=0.2)
    U, n, t = gpu_run(prim, t_end=0.2, **kw)
    assert n == ref.steps
    assert t == 0.2
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("nx,ny,bc", [(256, 256, "transmissive"), (100, 77, "transmissive"), (128, 96, "periodic"),
                                      (57, 130, "periodic")])
def test_quadrant_fp64_100_steps(nx, ny, bc):
    prim = inputs.quadrant(nx, ny, seed=nx + ny).stack()
    kw = dict(limiter="vanleer", cfl=0.45, bc=bc)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 100)
    U, n, t = gpu_run(prim, steps=100, **kw)
    assert n == 100
    assert t == pytest.approx(ref.t, rel=1e-13)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("limiter,beta", [("minmod", 1.0), ("sweby", 1.5), ("sweby", 2.0), ("vanleer", 1.0)])
@pytest.mark.parametrize("riemann", ["maxc", "per_side"])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_variants_fp64(limiter, beta, riemann, bc):
    prim = inputs.kelvin_helmholtz(61, 45, seed=1).stack() if bc == "periodic" else inputs.quadrant(61, 45, seed=2).stack()
    kw = dict(limiter=limiter, beta=beta, riemann=riemann, bc=bc, cfl=0.4)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 30)
    U, n, _ = gpu_run(prim, steps=30, **kw)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("name", ["sod", "two_rarefaction", "sonic_rarefaction", "shock_shock"])
def test_paper_tubes_fp64(name):
    prim = inputs.named_shock_tube(name, 400).stack()
    kw = dict(limiter="sweby", beta=1.5 if name != "shock_shock" else 1.0, cfl=0.25)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 10**6, t_end=0.16)
    U, n, t = gpu_run(prim, t_end=0.16, **kw)
    assert n == ref.steps and t == 0.16
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("shape", [(1, 1), (1, 3), (2, 2), (3, 29), (29, 3), (1, 28), (65, 1), (5, 57)])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_tiny_and_ragged_2d(shape, bc):
    ny, nx = shape
    prim = inputs.quadrant(nx, ny, seed=3).stack()
    kw = dict(limiter="vanleer", bc=bc, cfl=0.4)
    oc = oracle_cfg(prim, dim=2, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 10)
    U, n, _ = gpu_run(prim, steps=10, dim=2, **kw)
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("nx", [1, 2, 27, 28, 29, 113, 4096])
def test_1d_sizes(nx):
    prim = inputs.named_shock_tube("sod", nx).stack()
    kw = dict(limiter="minmod", cfl=0.5, dim=1)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 20)
    U, n, _ = gpu_run(prim, steps=20, **kw)
    assert_close(U, ref.U, FP64_TOL)


def test_host_buffers_and_fixed_dt_replay():
    prim = inputs.quadrant(90, 70, seed=5).stack()
    kw = dict(limiter="vanleer", cfl=0.45)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 25)
    U, n, _ = gpu_run(prim, dts=ref.dts, host=True, **kw)
    assert n == 25
    assert_close(U, ref.U, FP64_TOL)


@pytest.mark.parametrize("kind", ["quadrant", "kh", "wave"])
def test_fp32_against_fp64_oracle(kind):
    n = 96
    if kind == "quadrant":
        prim, bc = inputs.quadrant(n, n, seed=9).stack(), "transmissive"
    elif kind == "kh":
        prim, bc = inputs.kelvin_helmholtz(n, n, seed=9).stack(), "periodic"
    else:
        prim, bc = inputs.smooth_wave(n).stack(), "periodic"
    kw = dict(limiter="vanleer", bc=bc, cfl=0.45)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 40)
    U, nsteps, _ = gpu_run(prim, precision="fp32", dts=ref.dts, **kw)
    assert_close_fp32(U, ref.U)


def test_fp64_conservation_periodic():
    n = 200
    prim = inputs.kelvin_helmholtz(n, n, seed=4).stack()
    cfg = Config(nx=n, ny=n, bc="periodic", limiter="vanleer", cfl=0.45)
    s = LagrangeFlux(cfg)
    q = torch.from_numpy(prim).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    s0 = s.conservation_sums()
    s.run(max_steps=100)
    s1 = s.conservation_sums()
    U = s.get_state()
    exact = np.array([math.fsum(U[l].ravel()) for l in range(4)])
    np.testing.assert_allclose(s1, exact, rtol=1e-15, atol=1e-15)
    scale = np.array([np.abs(U[l]).sum() for l in range(4)])
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale)
    s.close()


def test_nonphysical_state_is_flagged_and_time_stops():
    prim = inputs.quadrant(64, 64, seed=1).stack()
    prim[3, 10, 10] = -1.0  # negative pressure
    s = LagrangeFlux(Config(nx=64, ny=64))
    q = torch.from_numpy(prim).cuda()
    s.set_primitive(q[0], q[1], q[2], q[3])
    with pytest.raises(LagrangeFluxError) as ei:
        s.run(max_steps=5)
    assert ei.value.status == 4
    t, steps = s.time()
    assert steps == 0 and t == 0.0
    s.close()


def test_nan_state_is_flagged():
    prim = inputs.quadrant(40, 40, seed=1).stack()
    prim[0, 3, 3] = np.nan
    s = LagrangeFlux(Config(nx=40, ny=40, precision="fp32"))
    q = torch.from_numpy(prim).cuda().float()
    s.set_primitive(q[0], q[1], q[2], q[3])
    with pytest.raises(LagrangeFluxError):
        s.run(max_steps=3)
    s.close()


def test_step_before_state_is_an_error():
    s = LagrangeFlux(Config(nx=8, ny=8))
    with pytest.raises(LagrangeFluxError) as ei:
        s.step()
    assert ei.value.status == 6
    s.close()


def _patch_oracle_step(U_full, ci, cj, dt, precision, radius=6, **kw):
    """One oracle step on a periodic patch around (ci, cj); returns the centre cell."""
    ny, nx = U_full.shape[1:]
    ii = (np.arange(ci - radius, ci + radius + 1)) % nx
    jj = (np.arange(cj - radius, cj + radius + 1)) % ny
    patch = np.ascontiguousarray(U_full[:, jj][:, :, ii].astype(np.float64))
    oc = O.OracleConfig(nx=2 * radius + 1, ny=2 * radius + 1, lx=(2 * radius + 1) / nx, ly=(2 * radius + 1) / ny,
                        bc="transmissive", **kw)
    return O.run(oc, patch, 1, dts=[dt]).U[:, radius, radius]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_8192_sampled_cells(precision):
    """8192^2 periodic Kelvin-Helmholtz, the benchmark's launch configuration:
    one GPU step checked at sampled cells against the oracle on a patch (a cell
    after one step depends only on cells within 4 of it), and the GPU dt
    against the oracle's CFL dt of the whole mesh."""
    n = 8192
    prim = inputs.kelvin_helmholtz(n, n, seed=0).stack()
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.45)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(Config(nx=n, ny=n, precision=precision, **kw))
    q = torch.from_numpy(prim).to("cuda", tdt)
    s.set_primitive(q[0], q[1], q[2], q[3])
    del q
    U0 = torch.empty((4, n, n), dtype=tdt, device="cuda")
    s.get_state(U0)
    U0h = U0.cpu().numpy()
    del U0
    dt = s.step(return_dt=True)
    oc = O.OracleConfig(nx=n, ny=n, **kw)
    dt_ref = O.cfl_dt(oc, U0h.astype(np.float64))
    assert dt == pytest.approx(dt_ref, rel=1e-14 if precision == "fp64" else 1e-6)
    U1 = torch.empty((4, n, n), dtype=tdt, device="cuda")
    s.get_state(U1)
    rng = np.random.default_rng(0)
    samples = [(0, 0), (n - 1, n - 1), (0, n - 1), (n // 2, n // 4), (4095, 2048)]
    samples += [tuple(v) for v in rng.integers(0, n, size=(27, 2))]
    tol = 1e-13 if precision == "fp64" else 2e-6
    for ci, cj in samples:
        ref = _patch_oracle_step(U0h, ci, cj, dt, precision, **{k: v for k, v in kw.items() if k != "bc"})
        got = U1[:, cj, ci].double().cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol * scale, (ci, cj, got, ref)
    s.close()


def test_maximum_fp32_mesh_sampled_cells():
    """The largest FP32 mesh lf_init accepts: 46336 x 46340 cells, whose field
    plane (rows padded to 128 bytes) is just under 2^31 elements, where the
    kernels' 32-bit in-plane offsets peak (69 GB for the two states).  The
    periodic Kelvin-Helmholtz layer is built on the device from its 1D
    profiles; one CFL step is checked at sampled cells, the last rows and
    columns among them, against the oracle on patches, and the GPU dt against
    the oracle's CFL dt: the layer is a product of a y-profile (rho, u) and
    an x-profile (v), so a two-row mesh with the same dx and dy holding one
    row of each kind has the dt of the whole mesh."""
    nx, ny = 46336, 46340
    free, _ = torch.cuda.mem_get_info()
    if free < 115e9:
        pytest.skip("needs about 105 GB of free device memory")
    rho_y, u_y, v_x, p = inputs.kelvin_helmholtz_profiles(nx, ny, seed=0)
    kw = dict(limiter="vanleer", bc="periodic", cfl=0.45)
    s = LagrangeFlux(Config(nx=nx, ny=ny, precision="fp32", **kw))
    f32 = dict(device="cuda", dtype=torch.float32)
    planes = [torch.as_tensor(rho_y, **f32)[:, None].expand(ny, nx).contiguous(),
              torch.as_tensor(u_y, **f32)[:, None].expand(ny, nx).contiguous(),
              torch.as_tensor(v_x, **f32)[None, :].expand(ny, nx).contiguous(),
              torch.full((ny, nx), p, **f32)]
    s.set_primitive(*planes)
    del planes
    torch.cuda.empty_cache()
    U = torch.empty((4, ny, nx), **f32)
    s.get_state(U)
    rng = np.random.default_rng(1)
    samples = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx - 3, ny - 2), (nx // 2, ny // 4 + 1)]
    samples += [tuple(v) for v in zip(rng.integers(0, nx, 14), rng.integers(0, ny, 14))]
    r = 6
    patches = {}
    for ci, cj in samples:
        ii = torch.as_tensor(np.arange(ci - r, ci + r + 1) % nx, device="cuda")
        jj = torch.as_tensor(np.arange(cj - r, cj + r + 1) % ny, device="cuda")
        patches[(ci, cj)] = U[:, jj][:, :, ii].double().cpu().numpy()
    rows = U[:, [0, ny // 2]].double().cpu().numpy()  # one row outside the layer, one inside
    dt = s.step(return_dt=True)
    oc = O.OracleConfig(nx=nx, ny=2, ly=2.0 / ny, **kw)
    assert dt == pytest.approx(O.cfl_dt(oc, rows), rel=1e-6)
    s.get_state(U)
    okw = {k: v for k, v in kw.items() if k != "bc"}
    for ci, cj in samples:
        pc = O.OracleConfig(nx=2 * r + 1, ny=2 * r + 1, lx=(2 * r + 1) / nx, ly=(2 * r + 1) / ny,
                            bc="transmissive", **okw)
        ref = O.run(pc, patches[(ci, cj)], 1, dts=[dt]).U[:, r, r]
        got = U[:, cj, ci].double().cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), (ci, cj, got, ref)
    s.close()
    del U
    torch.cuda.empty_cache()


def test_run_graph_replay_equals_direct_steps():
    # lf_run issues steps as replays of a recorded 32-step CUDA graph plus a
    # direct remainder; lf_step launches directly.  Same kernels, same order:
    # the results must be identical bit for bit.
    prim = inputs.kelvin_helmholtz(96, 80, seed=3).stack()
    cfg = Config(nx=96, ny=80, bc="periodic", limiter="vanleer", cfl=0.45, precision="fp32")
    outs = []
    for mode in ("run", "step"):
        s = LagrangeFlux(cfg)
        q = torch.from_numpy(prim).cuda().float()
        s.set_primitive(q[0], q[1], q[2], q[3])
        if mode == "run":
            n, _ = s.run(max_steps=70)
            assert n == 70
        else:
            for _ in range(70):
                s.step()
        outs.append((s.get_state(), s.time()))
        s.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("dim,bc", [(2, "transmissive"), (2, "periodic"), (1, "transmissive")])
@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_ssprk3_matches_oracle(dim, bc, precision, tol):
    if dim == 2:
        prim = (inputs.quadrant(77, 61, seed=4) if bc == "transmissive" else inputs.kelvin_helmholtz(77, 61, seed=4)).stack()
    else:
        prim = inputs.named_shock_tube("sod", 333).stack()
    kw = dict(limiter="vanleer", bc=bc, cfl=0.45, time_order=3, dim=dim)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 40)
    U, n, t = gpu_run(prim, precision=precision, dts=ref.dts if precision == "fp32" else None,
                      steps=None if precision == "fp32" else 40, **kw)
    assert n == 40
    if precision == "fp64":
        assert_close(U, ref.U, tol)
    else:
        assert_close_fp32(U, ref.U, tol)


def _paper_tubes():
    import os
    rows = []
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", "paper_shock_tubes.txt")):
        if ln.strip() and not ln.startswith("#"):
            f = ln.split()
            for n in f[8].split(","):
                rows.append((f[0], tuple(map(float, f[1:4])), tuple(map(float, f[4:7])), float(f[7]), int(n),
                             float(f[9]), float(f[10])))
    return rows


@pytest.mark.parametrize("name,L,R,T,n,cfl,beta", _paper_tubes())
def test_paper_tubes_at_paper_settings_fp64(name, L, R, T, n, cfl, beta):
    """Sec. 4.2's shock tubes with the paper's cells, final times, CFL and
    Sweby beta (tests/golden/paper_shock_tubes.txt), GPU against the oracle."""
    prim = inputs.shock_tube(n, L, R).stack()
    kw = dict(limiter="sweby", beta=beta, cfl=cfl)
    oc = oracle_cfg(prim, **kw)
    ref = O.run(oc, O.prim_to_cons(oc, prim), 10**6, t_end=T)
    U, steps, t = gpu_run(prim, t_end=T, **kw)
    assert steps == ref.steps and t == T
    assert_close(U, ref.U, FP64_TOL)
