"""The benchmark's full workloads -- the 8192^2 periodic Kelvin-Helmholtz layer
(ten CFL steps), the 384^3 periodic 3D shear layer (five) and the 512 batched
four-quadrant problems (ten) -- and the 2048^2 four-quadrant problem of the
FP64/FP32 configuration (its 400 steps) on the GPU, against the FP64 oracle run on the
whole meshes on the host's cores (the OpenMP build for the single meshes, the
same bits as the plain build, test_oracle_openmp.py; the plain build in a
pool of processes, one problem each, for the batch): every cell of every field
is compared, not samples.

Bars: FP64 relative L1 <= 1e-12 per conservative field and the oracle's own
CFL dt sequence to 1e-14; FP32 (state in FP32, dt from an FP64 reduction)
relative L1 <= 2e-5 per field against its own norm, on the GPU's dt sequence.
One exception, in both precisions: the 3D layer's rho w.  w starts at zero
and the initial flow is divergence-free, so after five steps rho w holds
only what the scheme generates at the density contacts, orders of magnitude
below the other momentum components; rounding-level differences are large
against its own norm (FP64 1.4e-8 measured), so it is measured against the
momentum magnitude |rho u| + |rho v| + |rho w| (its own-norm error is
printed beside it).
"""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from oracle import oracle as O
from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300.lagflux import Config, LagrangeFlux, LagrangeFluxBatch  # noqa: E402

N, STEPS = 8192, 10
KW = dict(limiter="vanleer", bc="periodic", cfl=0.45)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


@pytest.fixture(scope="module")
def prim():
    return inputs.kelvin_helmholtz(N, N, seed=0).stack()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_whole_8192_mesh_ten_steps_against_openmp_oracle(prim, precision):
    tdt = torch.float64 if precision == "fp64" else torch.float32
    s = LagrangeFlux(Config(nx=N, ny=N, precision=precision, **KW))
    q = torch.from_numpy(prim).to("cuda", tdt)
    s.set_primitive(q[0], q[1], q[2], q[3])
    del q
    U = torch.empty((4, N, N), dtype=tdt, device="cuda")
    s.get_state(U)
    U0 = U.double().cpu().numpy()  # the oracle starts from the GPU's conservative state
    dts = [s.step(return_dt=True) for _ in range(STEPS)]
    s.get_state(U)
    got = U.double().cpu().numpy()
    del U
    s.close()

    oc = O.OracleConfig(nx=N, ny=N, **KW)
    with O.use_library(O.build_omp()):
        O.threads(host_cores())
        ref = O.run(oc, U0, STEPS) if precision == "fp64" else O.run(oc, U0, STEPS, dts=dts)
    assert ref.steps == STEPS
    if precision == "fp64":
        np.testing.assert_allclose(dts, ref.dts, rtol=1e-14, atol=0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for field in range(4):
        err = np.abs(got[field] - ref.U[field]).sum() / np.abs(ref.U[field]).sum()
        print(f"8192^2 {precision} field {field}: relative L1 {err:.3e}")
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"


N3, STEPS3 = 384, 5


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_whole_384_cube_five_steps_against_openmp_oracle(precision):
    tdt = torch.float64 if precision == "fp64" else torch.float32
    q = inputs.shear_layer_3d(N3, seed=0).stack()
    s = LagrangeFlux(Config(nx=N3, ny=N3, nz=N3, dim=3, precision=precision, **KW))
    s.set_primitives(torch.from_numpy(q).to("cuda", tdt))
    del q
    U0 = s.get_conservative().astype(np.float64)
    dts = [s.step(return_dt=True) for _ in range(STEPS3)]
    got = s.get_conservative().astype(np.float64)
    s.close()

    oc = O.OracleConfig(nx=N3, ny=N3, nz=N3, dim=3, **KW)
    with O.use_library(O.build_omp()):
        O.threads(host_cores())
        ref = O.run(oc, U0, STEPS3) if precision == "fp64" else O.run(oc, U0, STEPS3, dts=dts)
    assert ref.steps == STEPS3
    if precision == "fp64":
        np.testing.assert_allclose(dts, ref.dts, rtol=1e-14, atol=0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    momentum = sum(np.abs(ref.U[m]).sum() for m in (1, 2, 3))
    for field in range(5):
        diff = np.abs(got[field] - ref.U[field]).sum()
        own = diff / np.abs(ref.U[field]).sum()
        err = diff / momentum if field == 3 else own
        print(f"384^3 {precision} field {field}: relative L1 {err:.3e} (against its own norm {own:.3e})")
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"


NPROB, STEPS_B = 512, 10
KW_B = dict(limiter="vanleer", bc="transmissive", cfl=0.45)


def _oracle_problem(args):
    """One batched problem of the benchmark run by the plain oracle (worker of a
    spawned process pool)."""
    p, nx, ny, steps = args
    oc = O.OracleConfig(nx=nx, ny=ny, **KW_B)
    r = O.run(oc, O.prim_to_cons(oc, inputs.quadrant(nx, ny, seed=p).stack()), steps)
    return p, r.U, r.t


@pytest.fixture(scope="module")
def batch_reference():
    sizes = [(int(a), int(b)) for a, b in inputs.batched_sizes(NPROB, seed=0)]
    ref = [None] * NPROB
    with ProcessPoolExecutor(max_workers=max(1, min(16, host_cores())), mp_context=mp.get_context("spawn")) as ex:
        for p, U, t in ex.map(_oracle_problem, [(p, a, b, STEPS_B) for p, (a, b) in enumerate(sizes)], chunksize=8):
            ref[p] = (U, t)
    return sizes, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_whole_512_problem_batch_ten_steps_against_oracle(batch_reference, precision):
    """The batched benchmark's problems (sides log-uniform in [64, 1024], seeded
    quadrant states, one persistent launch per stage, the step loop as a CUDA
    graph): every problem after ten CFL steps against the oracle run alone with
    its own CFL dt; FP32 takes its dt sequence from FP32 wave speeds, so its
    times differ from the oracle's at FP32 rounding."""
    sizes, ref = batch_reference
    tdt = torch.float64 if precision == "fp64" else torch.float32
    b = LagrangeFluxBatch([Config(nx=a, ny=c, precision=precision, **KW_B) for a, c in sizes])
    for p, (a, c) in enumerate(sizes):
        q = torch.from_numpy(inputs.quadrant(a, c, seed=p).stack()).to("cuda", tdt)
        b.set_primitive(p, q[0], q[1], q[2], q[3])
    b.run(STEPS_B)
    t, steps = b.times()
    got = [b.get_state(p).astype(np.float64) for p in range(len(sizes))]
    b.close()
    assert (steps == STEPS_B).all()
    tol = 1e-12 if precision == "fp64" else 2e-5
    ttol = 1e-13 if precision == "fp64" else 1e-5
    worst = 0.0
    for p, (U_ref, t_ref) in enumerate(ref):
        assert abs(t[p] - t_ref) <= ttol * t_ref, (p, t[p], t_ref)
        for field in range(4):
            err = np.abs(got[p][field] - U_ref[field]).sum() / np.abs(U_ref[field]).sum()
            worst = max(worst, err)
            assert err <= tol, f"{precision} problem {p} {sizes[p]} field {field}: relative L1 {err:.3e} > {tol}"
    print(f"512 batched problems {precision}: worst relative L1 over problems and fields {worst:.3e}")


N1, STEPS1 = 2048, 400
KW_1 = dict(limiter="vanleer", bc="transmissive", cfl=0.45)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2048_quadrant_400_steps_against_openmp_oracle(precision):
    """2048^2 cells on [0,1]^2, seeded four-quadrant Riemann problem, van Leer,
    CFL 0.45, transmissive boundaries, 400 steps: FP64 with the oracle's own CFL
    dt sequence, FP32 on the GPU's."""
    tdt = torch.float64 if precision == "fp64" else torch.float32
    prim = inputs.quadrant(N1, N1, seed=0).stack()
    s = LagrangeFlux(Config(nx=N1, ny=N1, precision=precision, **KW_1))
    q = torch.from_numpy(prim).to("cuda", tdt)
    s.set_primitive(q[0], q[1], q[2], q[3])
    U = torch.empty((4, N1, N1), dtype=tdt, device="cuda")
    s.get_state(U)
    U0 = U.double().cpu().numpy()
    dts = [s.step(return_dt=True) for _ in range(STEPS1)]
    s.get_state(U)
    got = U.double().cpu().numpy()
    s.close()
    oc = O.OracleConfig(nx=N1, ny=N1, **KW_1)
    with O.use_library(O.build_omp()):
        O.threads(host_cores())
        ref = O.run(oc, U0, STEPS1) if precision == "fp64" else O.run(oc, U0, STEPS1, dts=dts)
    assert ref.steps == STEPS1
    if precision == "fp64":
        np.testing.assert_allclose(dts, ref.dts, rtol=1e-13, atol=0)
    tol = 1e-12 if precision == "fp64" else 2e-5
    for field in range(4):
        err = np.abs(got[field] - ref.U[field]).sum() / np.abs(ref.U[field]).sum()
        print(f"2048^2 quadrant {precision} field {field}: relative L1 {err:.3e}")
        assert err <= tol, f"{precision} field {field}: relative L1 {err:.3e} > {tol}"
