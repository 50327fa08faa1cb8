"""FP32 sweep launch shapes and the autotuner (GPU): the shape changes the
launch configuration only, so every shape gives the same result bit for bit;
the autotuner sets the faster shape and its cache skips the timing."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import make_context, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(16, 16, 16, 32), (6, 4, 6, 10)])
def test_shapes_give_identical_results(dims):
    U = inputs.su3_exp_gauge(dims, 0.5, 11)
    psi = to_dev(inputs.gaussian_spinor(dims, 12))
    ctx = make_context(dims, U, -1.8, 0.1, 0.037)
    outs = []
    for shape in ("wide", "narrow", "auto"):
        ctx.set_hop_shape(shape)
        assert ctx.hop_shape() == fa._SHAPE[shape]
        outs.append((to_host(ctx.apply_dw(psi, precision="f32")), to_host(ctx.apply_A(psi, precision="f32"))))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_autotune_picks_the_faster_shape_and_caches(tmp_path):
    dims = (16, 16, 16, 32)
    w = inputs.make_workload("wilson_16x16x16x32", dims)
    ctx = make_context(dims, w["U"], w["mass"], w["mu"], 0.03)
    import torch
    r = ctx.autotune(reps=10)
    t = r["times_ms"]
    assert not r["cached"] and all(x > 0 for x in t)
    # the automatic shape is kept unless the other is faster by more than 3 %
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    deflt = fa.SHAPE_NARROW if (np.prod(dims) + 127) // 128 <= 7 * sms else fa.SHAPE_WIDE
    other = 3 - deflt
    expect = other if t[other - 1] < 0.97 * t[deflt - 1] else deflt
    assert r["shape"] == expect and ctx.hop_shape() == expect
    cache = str(tmp_path / "tune.json")
    r1 = ctx.autotune(reps=5, cache=cache)
    ctx.set_hop_shape("auto")
    r2 = ctx.autotune(reps=5, cache=cache)
    assert not r1["cached"] and r2["cached"] and r2["shape"] == r1["shape"] == ctx.hop_shape()
    # a solve after tuning matches the untuned one bit for bit
    b = to_dev(w["b"])
    om, sg = fa.neuberger_poles(4)
    ctx.set_poles(om, sg)
    kw = dict(ell=2, tol=1e-6, mode="pseudo", precision="f32")
    y1 = to_host(ctx.apply_f(b, **kw).y)
    ctx.set_hop_shape("wide" if ctx.hop_shape() == fa.SHAPE_NARROW else "narrow")
    y2 = to_host(ctx.apply_f(b, **kw).y)
    assert np.array_equal(y1, y2)


def test_bad_shape_and_order_errors():
    dims = (4, 4, 4, 8)
    ctx = fa.Context(dims)
    with pytest.raises(fa.FAError) as e:
        fa._check(ctx.lib.fa_set_hop_shape(ctx.h, 7), "fa_set_hop_shape")
    assert e.value.status == fa.FA_EINVAL
    with pytest.raises(fa.FAError) as e:
        ctx.autotune(reps=2)
    assert e.value.status == fa.FA_ESTATE


def test_autotune_on_a_capturable_stream():
    """On a side stream the chains are replayed from a CUDA graph (as the solver
    replays its outer iterations); the stream is usable afterwards and the
    results do not change."""
    import torch
    dims = (16, 16, 16, 32)
    w = inputs.make_workload("wilson_16x16x16x32", dims)
    stream = torch.cuda.Stream()
    ctx = fa.Context(dims, stream)
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 0.03)
    with torch.cuda.stream(stream):
        psi = to_dev(w["b"])
    stream.synchronize()
    out = ctx.apply_dw(psi, precision="f32")
    stream.synchronize()
    before = to_host(out)
    r = ctx.autotune(reps=10)
    assert not r["cached"] and all(0 < x < 1.0 for x in r["times_ms"])
    assert r["shape"] in (fa.SHAPE_WIDE, fa.SHAPE_NARROW)
    out = ctx.apply_dw(psi, precision="f32")
    stream.synchronize()
    assert np.array_equal(before, to_host(out))
    ctx.set_poles(*fa.neuberger_poles(4))
    res = ctx.apply_f(psi, ell=2, tol=1e-6, mode="pseudo", precision="f32", graph=True)
    stream.synchronize()
    assert res.stats["status"] == 0
