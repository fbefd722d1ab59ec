"""The arithmetic throughput probe (dgsrhd_arith_probe) behind the FP64 roofline's denominator:
every operation runs, leaves finite chain sums, and reports 4 x threads x iters operations; the
FP64 primitives the library uses in place of CUDA's division, square root and reciprocal cube
root issue fewer FP64 instructions than those (the reason they exist), measured as throughput."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rate(kind, iters, sink, stream):
    from paper_2205_00095_gb300.solver import arith_probe
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        arith_probe(kind, 8, sink, stream)
        ev0.record(stream)
        ops = arith_probe(kind, iters, sink, stream)
        ev1.record(stream)
    torch.cuda.synchronize()
    return ops / (ev0.elapsed_time(ev1) * 1e-3), ops


def test_probe_runs_every_operation(gpu_lib):
    from paper_2205_00095_gb300 import _lib
    stream = torch.cuda.Stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.full((sms * 8 * 256,), float("nan"), dtype=torch.float64, device="cuda")
    for kind in _lib.PROBE:
        rate, ops = _rate(kind, 64, sink, stream)
        assert ops == 4 * sink.numel() * 64
        assert rate > 0.0
        assert torch.isfinite(sink).all(), kind


def test_probe_rejects_bad_arguments(gpu_lib):
    import ctypes
    from paper_2205_00095_gb300 import _lib
    lib = gpu_lib
    sink = torch.zeros(256, dtype=torch.float64, device="cuda")
    ops = ctypes.c_int64()
    for kind, iters, threads in ((len(_lib.PROBE), 1, 256), (-1, 1, 256), (0, 0, 256), (0, 1, 255),
                                 (0, 1, 0)):
        assert lib.dgsrhd_arith_probe(kind, iters, sink.data_ptr(), threads, None,
                                      ctypes.byref(ops)) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_arith_probe(0, 1, None, 256, None, ctypes.byref(ops)) == _lib.DGSRHD_EINVAL


def test_library_primitives_beat_cuda_division_and_sqrt(gpu_lib):
    stream = torch.cuda.Stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    r = {k: _rate(k, 2000, sink, stream)[0]
         for k in ("dfma", "ddiv", "recip", "dsqrt", "sqrt", "drsqrt", "rsqrt", "drcbrt", "rcbrt")}
    cost = {k: r["dfma"] / v for k, v in r.items()}
    print("\nDFMA-equivalents:", {k: round(v, 2) for k, v in cost.items()},
          f"DFMA {2 * r['dfma'] / 1e12:.3f} TFLOP/s")
    assert cost["recip"] < cost["ddiv"]
    assert cost["sqrt"] < cost["dsqrt"]
    assert cost["rcbrt"] < cost["drcbrt"]
    assert cost["rsqrt"] < cost["drsqrt"]
    assert np.isfinite(list(cost.values())).all()
