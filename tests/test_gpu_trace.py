"""Kernel timeline tracing (fa_trace_start / fa_trace_stop) on the GPU: every
block of every traced launch leaves one record, launches group cleanly in a
graph-replayed solve, results do not change, and a full ring drops records
instead of overrunning."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import to_dev, to_host

pytestmark = pytest.mark.gpu


def workload_ctx(stream):
    w = inputs.make_workload("wilson_4x4x4x8")
    ctx = fa.Context(w["dims"], stream)
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 0.05)
    ctx.set_poles(*fa.neuberger_poles(w["ns"]))
    return w, ctx


def test_trace_of_a_graph_replayed_solve():
    import torch
    stream = torch.cuda.Stream()
    w, ctx = workload_ctx(stream)
    with torch.cuda.stream(stream):
        b = to_dev(w["b"])
    stream.synchronize()
    kw = dict(ell=2, tol=1e-8, mode="pseudo", precision="f32", graph=True)
    ref = ctx.apply_f(b, **kw)
    stream.synchronize()
    y_ref = to_host(ref.y)
    fa.trace_start(1 << 18)
    r = ctx.apply_f(b, **kw)
    rec, dropped = fa.trace_stop(1 << 18)
    assert dropped == 0 and len(rec) > 0
    assert np.array_equal(to_host(r.y), y_ref)            # tracing changes no result
    assert np.all(rec["t_end_ns"] >= rec["t_start_ns"])
    launches = fa.trace_launches(rec)
    for L in launches:
        assert L["blocks"] == L["grid"], L                 # one record per block, no launch merged
    names = [L["name"] for L in launches]
    plain, dot, gram = names.count("k_hop1<f32>"), names.count("k_hop1<f32, dot>"), names.count("k_hop_gram<f32>")
    # an FP32 outer iteration at l = 2: four plain sweeps, three with <rt, out>, one Gram sweep
    assert gram > 0 and plain == 4 * gram and dot == 3 * gram, (plain, dot, gram)
    assert gram >= r.stats["outer_iters"]
    # the launches are in stream order
    starts = [L["start_ns"] for L in launches]
    assert starts == sorted(starts)
    assert all(a["end_ns"] < b2["start_ns"] for a, b2 in zip(launches, launches[1:]))


def test_trace_full_ring_drops_and_errors():
    import torch
    stream = torch.cuda.Stream()
    w, ctx = workload_ctx(stream)
    with torch.cuda.stream(stream):
        b = to_dev(w["b"])
    stream.synchronize()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fa.trace_start(nsm)                                       # one record per SM
    ctx.apply_f(b, ell=2, tol=1e-6, mode="double", precision="f32")
    rec, dropped = fa.trace_stop(4 * nsm)
    assert len(rec) <= nsm and dropped > 0
    with pytest.raises(fa.FAError) as e:
        fa.trace_stop()
    assert e.value.status == fa.FA_ESTATE
    with pytest.raises(fa.FAError) as e:
        fa.trace_start(0)
    assert e.value.status == fa.FA_EINVAL


def test_fp32_issue_rate_probe():
    """The FP32 issue-rate probe (denominator of the double-float sweep's
    roofline): positive, below the SMs x 128 lanes x 2.2 GHz ceiling, and the
    argument checks."""
    import ctypes
    import torch
    rate, ms = fa.fp32_issue_rate(3)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert ms > 0 and 0.2 * nsm * 128 * 1.0e9 < rate < nsm * 128 * 2.2e9, (rate, ms)
    lib = fa.load_library()
    r, m = ctypes.c_double(), ctypes.c_double()
    assert lib.fa_fp32_issue_rate(0, ctypes.byref(r), ctypes.byref(m)) == fa.FA_EINVAL
    assert lib.fa_fp32_issue_rate(1, None, ctypes.byref(m)) == fa.FA_EINVAL
