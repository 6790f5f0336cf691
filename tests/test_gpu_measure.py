"""The library's measurement calls on the GPU: the FMA-throughput peaks that
the ALU rooflines divide by (lf_measure_peak) and the per-stage tracing of
batches (lf_batch_profile)."""
import pytest

from paper_1607_08710_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1607_08710_gb300 import lagflux as L  # noqa: E402


def test_measured_fma_peaks_are_plausible():
    """GB300: 152 SMs x 2 FP64 FMA per clock (1.26 TFLOP/s at 2.07 GHz) and
    128 FP32 FMA lanes per SM (80.5 TFLOP/s); the measured rates must lie
    within a factor of the nominal ones at any clock the GPU may run, and the
    paired FP32 form is at least as fast as the scalar one."""
    f64 = L.measure_peak("fp64", 0, 20.0)
    f32 = L.measure_peak("fp32", 0, 20.0)
    f32p = L.measure_peak("fp32_paired", 0, 20.0)
    print("measured peaks (TFLOP/s): fp64", f64, "fp32", f32, "fp32 paired", f32p)
    assert 0.3 < f64 < 2.0
    assert 20.0 < f32 < 120.0
    assert f32p >= 0.9 * f32
    assert f32 > 20 * f64


def test_measure_peak_rejects_bad_arguments():
    with pytest.raises(KeyError):
        L.measure_peak("int8")
    r = L.ctypes.c_double()
    assert L.lf_measure_peak(0, 7, 10.0, L.ctypes.byref(r)) == L.LF_ERR_ARG
    assert L.lf_measure_peak(0, 0, 0.0, L.ctypes.byref(r)) == L.LF_ERR_ARG
    assert L.lf_measure_peak(0, 0, 10.0, None) == L.LF_ERR_ARG


def test_batch_profile_advances_like_batch_run():
    """lf_batch_profile runs the same steps as lf_batch_run (direct launches):
    the states end bit for bit equal, the step counts advance, and both stage
    times are positive."""
    sizes = [(70, 45), (130, 64), (64, 200)]
    cfgs = [L.Config(nx=nx, ny=ny, precision="fp32", limiter="vanleer", bc="transmissive", cfl=0.45)
            for nx, ny in sizes]
    outs = []
    for mode in ("profile", "run"):
        b = L.LagrangeFluxBatch(cfgs)
        for p, (nx, ny) in enumerate(sizes):
            q = torch.from_numpy(inputs.quadrant(nx, ny, seed=p).stack()).cuda().float()
            b.set_primitive(p, q[0], q[1], q[2], q[3])
        if mode == "profile":
            ms = b.profile(5)
            assert ms[0] > 0 and ms[1] > 0
        else:
            b.run(5, use_graph=False)
        _, steps = b.times()
        assert list(steps) == [5, 5, 5]
        outs.append([b.get_state(p) for p in range(len(sizes))])
        b.close()
    for a, c in zip(outs[0], outs[1]):
        assert (a == c).all()
