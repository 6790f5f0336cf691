"""Translation invariance of the GPU step on periodic meshes, bit for bit.

With periodic boundaries the scheme (Sec. 4: eqs. 12-14 on every face, the
CFL dt from a maximum over all cells) commutes with a shift of the mesh: every
cell's update depends only on the values around it, and the maximum does not
depend on the order of its terms.  The kernels compute each cell with the same
operations in the same order wherever it sits, so a shifted initial state must
give exactly the shifted result.  The shifts move cells between the strips
whose columns lie inside the row (the vector-copy march) and the edge strips
(the boundary-mapped march), between row tiles and tile prologues, and, in
3D, between CTA row blocks and plane tiles; any difference in the arithmetic
of those paths shows up as a changed bit.
"""
import numpy as np
import pytest

from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux  # noqa: E402


def run_periodic(q, steps, **kw):
    shape = q.shape[1:]
    if len(shape) == 3:
        nz, ny, nx = shape
        cfg = Config(nx=nx, ny=ny, nz=nz, dim=3, bc="periodic", **kw)
    else:
        ny, nx = shape
        cfg = Config(nx=nx, ny=ny, bc="periodic", **kw)
    s = LagrangeFlux(cfg)
    s.set_primitives(np.ascontiguousarray(q.astype(cfg.np_dtype)))
    n, t = s.run(max_steps=steps)
    assert n == steps
    U = s.get_conservative()
    s.close()
    return U, t


def assert_shift_invariant(q, shifts, steps, **kw):
    axes = tuple(range(1, q.ndim))
    U0, t0 = run_periodic(q, steps, **kw)
    assert np.all(np.isfinite(U0))
    for sh in shifts:
        Us, ts = run_periodic(np.roll(q, sh, axis=axes), steps, **kw)
        assert ts == t0  # the same dt sequence
        ref = np.roll(U0, sh, axis=axes)
        bad = np.argwhere(Us != ref)
        assert bad.size == 0, f"shift {sh}: {len(bad)} cells differ, first at {bad[0]}"


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("nspecies", [0, 2])
def test_periodic_translation_is_bitwise_2d(precision, nspecies):
    # 250 columns: five FP32 strips of 60 output columns (three inner), nine
    # FP64 strips of 28; 150 rows: three 64-row tiles, the last one ragged
    nx, ny = 250, 150
    base = inputs.kelvin_helmholtz(nx, ny, seed=4)
    if nspecies:
        rng = np.random.default_rng(11)
        base = inputs.with_species(base, rng.uniform(0.0, 1.0, size=(nspecies, ny, nx)))
    q = base.stack()
    assert_shift_invariant(q, [(13, 7), (64, 61), (1, 123), (0, 2)], steps=12, precision=precision,
                           limiter="vanleer", cfl=0.45, nspecies=nspecies)


@pytest.mark.parametrize("limiter", ["minmod", "sweby"])
def test_periodic_translation_is_bitwise_2d_limiters(limiter):
    nx, ny = 190, 70
    q = inputs.quadrant(nx, ny, seed=3).stack()
    assert_shift_invariant(q, [(5, 29), (35, 60)], steps=10, precision="fp32", limiter=limiter, beta=1.5,
                           cfl=0.4)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_periodic_translation_is_bitwise_3d(precision):
    # 190 columns: strips 1 and 2 of four lie inside the rows (FP32); 9 rows:
    # three 4-row blocks, the last ragged; 70 planes: two z-tiles
    nx, ny, nz = 190, 9, 70
    q = inputs.octant(nx, ny, nz, seed=5).stack()
    assert_shift_invariant(q, [(5, 3, 17), (64, 4, 60), (1, 0, 1)], steps=6, precision=precision,
                           limiter="vanleer", cfl=0.4)


def run_with_tile(q, steps, tile_rows, **kw):
    shape = q.shape[1:]
    if len(shape) == 3:
        nz, ny, nx = shape
        cfg = Config(nx=nx, ny=ny, nz=nz, dim=3, tile_rows=tile_rows, **kw)
    else:
        ny, nx = shape
        cfg = Config(nx=nx, ny=ny, tile_rows=tile_rows, **kw)
    s = LagrangeFlux(cfg)
    s.set_primitives(np.ascontiguousarray(q.astype(cfg.np_dtype)))
    if tile_rows:
        assert s.tile_rows == tile_rows
    s.run(max_steps=steps)
    U = s.get_conservative()
    s.close()
    return U


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("time_order,nspecies,bc", [(2, 0, "transmissive"), (3, 0, "periodic"), (2, 2, "periodic")])
def test_tile_height_does_not_change_results_2d(precision, time_order, nspecies, bc):
    """The tile height is a launch shape only: every row is computed with the
    same operations whether it opens a tile (prologue) or not."""
    nx, ny = 200, 131
    base = inputs.quadrant(nx, ny, seed=8)
    if nspecies:
        rng = np.random.default_rng(2)
        base = inputs.with_species(base, rng.uniform(0.0, 1.0, size=(nspecies, ny, nx)))
    q = base.stack()
    kw = dict(precision=precision, bc=bc, limiter="vanleer", cfl=0.45, time_order=time_order, nspecies=nspecies)
    ref = run_with_tile(q, 10, 0, **kw)
    for rows in (1, 3, 4, 16, 64, 128, 4096):
        U = run_with_tile(q, 10, rows, **kw)
        assert np.array_equal(U, ref), f"tile_rows={rows}"


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tile_height_does_not_change_results_3d(precision):
    nx, ny, nz = 70, 9, 45
    q = inputs.octant(nx, ny, nz, seed=6).stack()
    kw = dict(precision=precision, bc="transmissive", limiter="vanleer", cfl=0.4)
    ref = run_with_tile(q, 6, 0, **kw)
    for planes in (1, 5, 8, 64):
        U = run_with_tile(q, 6, planes, **kw)
        assert np.array_equal(U, ref), f"planes per tile {planes}"


@pytest.mark.parametrize("dim", [2, 3])
def test_autotune_leaves_no_trace(dim):
    if dim == 2:
        q = inputs.kelvin_helmholtz(300, 257, seed=1).stack()
        cfg = Config(nx=300, ny=257, precision="fp32", bc="periodic", cfl=0.45)
        cand = (4, 8, 16, 32, 64, 128)
    else:
        q = inputs.octant(64, 20, 40, seed=2).stack()
        cfg = Config(nx=64, ny=20, nz=40, dim=3, precision="fp32", bc="periodic", cfl=0.4)
        cand = (8, 16, 32, 64)
    s = LagrangeFlux(cfg)
    s.set_primitives(np.ascontiguousarray(q.astype(np.float32)))
    s.run(max_steps=3)
    U0, t0 = s.get_conservative(), s.time()
    rows = s.autotune(2)
    assert rows in cand and s.tile_rows == rows
    assert np.array_equal(s.get_conservative(), U0)
    assert s.time() == t0
    s.run(max_steps=4)
    U1 = s.get_conservative()
    s.close()
    # the same seven steps without the autotuning
    s = LagrangeFlux(cfg)
    s.set_primitives(np.ascontiguousarray(q.astype(np.float32)))
    s.run(max_steps=7)
    assert np.array_equal(s.get_conservative(), U1)
    s.close()


def test_tile_rows_arguments():
    s = LagrangeFlux(Config(nx=32, ny=1, dim=1))
    assert s.tile_rows == 0
    with pytest.raises(Exception):
        s.tile_rows = 8  # 1D meshes have no tiles
    s.close()
    s = LagrangeFlux(Config(nx=32, ny=32))
    with pytest.raises(Exception):
        s.tile_rows = 0
    with pytest.raises(Exception):
        s.autotune(1)  # no state yet
    s.tile_rows = 7
    assert s.tile_rows == 7
    s.close()
