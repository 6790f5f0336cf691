"""Batched mode (lf_batch_*) against the FP64 oracle, problem by problem.

Each problem of a batch must evolve exactly as it would alone: same per-cell
arithmetic, its own CFL dt (Sec. 4, Heun step 1) and time.  FP64 bar:
relative L1 <= 1e-12 per field; FP32: <= 2e-5 against the FP64 oracle.
The tile height, the CUDA graph and the autotuner change only the schedule,
so results must be bitwise identical across them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux, LagrangeFluxBatch, LagrangeFluxError  # noqa: E402

SIZES = [(37, 61), (64, 64), (100, 33), (1, 5), (130, 70), (17, 200), (61, 61), (3, 2)]


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / (den if den > 0 else 1.0)


def field_errors(U, ref):
    """Relative L1 per field; a momentum component is measured against the
    momentum vector's magnitude (sum of both components), since in FP32 a
    small component (e.g. the 1% shear-layer perturbation) is computed from
    terms as large as the other component and carries their rounding."""
    out = []
    for l in range(4):
        den = np.abs(ref[l]).sum()
        if l in (1, 2):
            den = np.abs(ref[1]).sum() + np.abs(ref[2]).sum()
        out.append(np.abs(U[l] - ref[l]).sum() / (den if den > 0 else 1.0))
    return out


def make_batch(sizes, precision, bc="transmissive", kind="quadrant", rows=None):
    cfgs = [Config(nx=nx, ny=ny, precision=precision, limiter="vanleer", bc=bc, cfl=0.45) for nx, ny in sizes]
    b = LagrangeFluxBatch(cfgs)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    prims = []
    for p, (nx, ny) in enumerate(sizes):
        prim = (inputs.quadrant(nx, ny, seed=100 + p) if kind == "quadrant"
                else inputs.kelvin_helmholtz(nx, ny, seed=100 + p)).stack()
        prims.append(prim)
        q = torch.from_numpy(prim).to("cuda", tdt)
        b.set_primitive(p, q[0], q[1], q[2], q[3])
    if rows:
        b.set_rows(rows)
    return b, prims


def states(b, sizes):
    return [b.get_state(p).astype(np.float64) for p in range(len(sizes))]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("bc,kind", [("transmissive", "quadrant"), ("periodic", "kh")])
def test_batch_matches_oracle(precision, tol, bc, kind):
    steps = 30
    b, prims = make_batch(SIZES, precision, bc=bc, kind=kind)
    b.run(steps)
    got = states(b, SIZES)
    t, nsteps = b.times()
    b.close()
    for p, (nx, ny) in enumerate(SIZES):
        oc = O.OracleConfig(nx=nx, ny=ny, limiter="vanleer", bc=bc, cfl=0.45)
        ref = O.run(oc, O.prim_to_cons(oc, prims[p]), steps)
        assert nsteps[p] == steps
        assert t[p] == pytest.approx(ref.t, rel=1e-13 if precision == "fp64" else 1e-6)
        errs = [rel_l1(got[p][l], ref.U[l]) for l in range(4)] if precision == "fp64" else field_errors(got[p], ref.U)
        assert max(errs) <= tol, (p, errs)


def test_graph_rows_and_autotune_do_not_change_results():
    steps = 12
    runs = []
    for rows, graph, tune in [(64, True, False), (64, False, False), (16, True, False), (128, True, False),
                              (None, True, True)]:
        b, _ = make_batch(SIZES, "fp32", rows=rows)
        if tune:
            chosen = b.autotune(2)
            assert chosen in (16, 24, 32, 48, 64, 96, 128)
            t, s = b.times()
            assert np.all(s == 0) and np.all(t == 0.0)  # the trials left no trace
        b.run(steps, use_graph=graph)
        runs.append(states(b, SIZES))
        b.close()
    for other in runs[1:]:
        for p in range(len(SIZES)):
            np.testing.assert_array_equal(other[p], runs[0][p])


def test_graph_replays_accumulate():
    b, _ = make_batch(SIZES[:4], "fp64")
    b.run(5)
    b.run(5)  # replays the recorded 5-step graph
    first = states(b, SIZES[:4])
    t1, s1 = b.times()
    b.close()
    c, _ = make_batch(SIZES[:4], "fp64")
    c.run(10, use_graph=False)
    second = states(c, SIZES[:4])
    t2, s2 = c.times()
    c.close()
    assert np.all(s1 == 10) and np.all(s2 == 10)
    np.testing.assert_array_equal(t1, t2)
    for p in range(4):
        np.testing.assert_array_equal(first[p], second[p])


def test_bad_problem_is_isolated_and_reported():
    sizes = SIZES[:3]
    cfgs = [Config(nx=nx, ny=ny, precision="fp64") for nx, ny in sizes]
    b = LagrangeFluxBatch(cfgs)
    for p, (nx, ny) in enumerate(sizes):
        prim = inputs.quadrant(nx, ny, seed=p).stack()
        if p == 1:
            prim[3, 2, 2] = -1.0
        q = torch.from_numpy(prim).cuda()
        b.set_primitive(p, q[0], q[1], q[2], q[3])
    b.run(4)
    with pytest.raises(LagrangeFluxError) as ei:
        b.times()
    assert ei.value.status == 4
    b.close()


def test_batch_rejects_mixed_schemes_and_1d():
    with pytest.raises(LagrangeFluxError):
        LagrangeFluxBatch([Config(nx=8, ny=8), Config(nx=8, ny=8, limiter="minmod")])
    with pytest.raises(LagrangeFluxError):
        LagrangeFluxBatch([Config(nx=8, dim=1)])


def test_full_size_512_problems_sampled():
    """The benchmark's batched configuration: 512 seeded uneven meshes (sides
    log-uniform in [64, 1024]), FP32, autotuned, graph of the step loop.
    Sampled problems are checked against the FP64 oracle after 3 steps."""
    sizes = [tuple(int(v) for v in s) for s in inputs.batched_sizes(512, seed=0)]
    b, prims = make_batch(sizes, "fp32")
    b.autotune(2)
    b.run(3)
    t, s = b.times()
    assert np.all(s == 3)
    order = np.argsort([nx * ny for nx, ny in sizes])
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1]), 0, 511]
    for p in sample:
        nx, ny = sizes[p]
        got = b.get_state(p).astype(np.float64)
        oc = O.OracleConfig(nx=nx, ny=ny, limiter="vanleer", bc="transmissive", cfl=0.45)
        ref = O.run(oc, O.prim_to_cons(oc, prims[p]), 3)
        assert max(field_errors(got, ref.U)) <= 2e-5, (p, field_errors(got, ref.U))
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("bc,kind", [("transmissive", "quadrant"), ("periodic", "kh")])
def test_batch_equals_single_meshes_bitwise(precision, bc, kind):
    """A problem of a batch runs the same march (inner-strip or mapped, the
    same arithmetic) with its own CFL dt as the same mesh in its own context,
    so after the same steps the states agree bit for bit -- whatever the
    order in which the persistent kernel's warps took the units."""
    sizes = SIZES + [(300, 131)]
    steps = 17
    b, prims = make_batch(sizes, precision, bc=bc, kind=kind)
    b.run(steps)
    got = states(b, sizes)
    b.close()
    tdt = torch.float64 if precision == "fp64" else torch.float32
    for p, (nx, ny) in enumerate(sizes):
        s = LagrangeFlux(Config(nx=nx, ny=ny, precision=precision, limiter="vanleer", bc=bc, cfl=0.45))
        q = torch.from_numpy(prims[p]).to("cuda", tdt)
        s.set_primitive(q[0], q[1], q[2], q[3])
        s.run(max_steps=steps)
        single = s.get_state().astype(np.float64)
        s.close()
        assert np.array_equal(got[p], single), f"problem {p} ({nx}x{ny})"
