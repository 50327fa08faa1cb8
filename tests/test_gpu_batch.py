"""Batched multi-shift solves (fa_apply_f_batched) and CUDA-graph replay.

Systems of one lattice shape share every kernel launch; each keeps its own
gauge field (or shares one), mu, scale, poles, scalars and convergence.  The
batched result of every system must equal the one-at-a-time solve of the same
system (same kernels, same per-system reductions), and match the oracle."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import oracle_double, rel, to_dev, to_host, workload_case
from oracle import dirac, scale

pytestmark = pytest.mark.gpu


def lattice_systems(dims, gauge_seed, mu, sources, stream=None, poles=10):
    """One owner context with the gauge field and one context per source sharing it."""
    U = inputs.su3_exp_gauge(dims, 0.5, gauge_seed)
    c = scale.power_scale(dirac.Operator(U, -1.8, mu).A, inputs.gaussian_spinor(dims, gauge_seed + 3), 100)
    om, sg = fa.neuberger_poles(poles)
    owner = fa.Context(dims, stream)
    owner.set_gauge(to_dev(U))
    ctxs = []
    for k in range(len(sources)):
        ctx = owner if k == 0 else fa.Context(dims, stream)
        if k > 0:
            ctx.share_gauge(owner)
        ctx.set_params(-1.8, mu, -1, c)
        ctx.set_poles(om, sg)
        ctxs.append(ctx)
    return ctxs, [to_dev(s) for s in sources], (U, c, om, sg)


def _batch_systems():
    d1, d2 = (4, 4, 4, 8), (3, 3, 3, 6)
    return [(301, d1, 0.05, inputs.point_source(d1, 0, 0)), (302, d2, 0.12, inputs.gaussian_spinor(d2, 11)),
            (301, d1, 0.05, inputs.point_source(d1, 2, 1)), (303, d1, 0.18, inputs.gaussian_spinor(d1, 12)),
            (302, d2, 0.12, inputs.point_source(d2, 3, 2)), (301, d1, 0.05, inputs.gaussian_spinor(d1, 9))]


SYSTEMS = _batch_systems()   # (gauge seed, dims, mu, source) of build_batch's systems, in its order


def build_batch(stream=None):
    d1, d2 = (4, 4, 4, 8), (3, 3, 3, 6)
    srcs1 = [inputs.point_source(d1, 0, 0), inputs.point_source(d1, 2, 1), inputs.gaussian_spinor(d1, 9)]
    srcs2 = [inputs.gaussian_spinor(d2, 11), inputs.point_source(d2, 3, 2)]
    srcs3 = [inputs.gaussian_spinor(d1, 12)]
    a, ba, ia = lattice_systems(d1, 301, 0.05, srcs1, stream)
    b, bb, ib = lattice_systems(d2, 302, 0.12, srcs2, stream)
    c, bc, ic = lattice_systems(d1, 303, 0.18, srcs3, stream)
    # interleave shapes on purpose: the batch groups them itself
    ctxs = [a[0], b[0], a[1], c[0], b[1], a[2]]
    srcs = [ba[0], bb[0], ba[1], bc[0], bb[1], ba[2]]
    return ctxs, srcs, (a, b, c)


@pytest.mark.parametrize("mode,precision", [("double", "f64"), ("pseudo", "f64"), ("single", "f64"),
                                            ("double", "f32"), ("pseudo", "f32")])
def test_batched_equals_one_at_a_time(mode, precision):
    """Systems of two lattice shapes in one batched solve (one launch per kernel
    for all of them; the FP32 sweep over lattice groups, several right-hand
    sides per block) against each system solved alone with the same sweep shape
    (128-thread FP32 sweeps, the Gram matrix in a kernel of its own): equal bit
    for bit."""
    ctxs, srcs, _ = build_batch()
    kw = dict(ell=2, tol=1e-10, mode=mode, precision=precision)
    ys, stats = fa.apply_f_batched(ctxs, srcs, **kw)
    for i, (ctx, b) in enumerate(zip(ctxs, srcs)):
        ctx.set_hop_shape("narrow")
        r = ctx.apply_f(b, gram_epilogue=False, **kw)
        ctx.set_hop_shape("auto")
        assert np.array_equal(to_host(ys[i]), to_host(r.y)), i
        assert stats[i]["outer_iters"] == r.stats["outer_iters"]
        assert stats[i]["iters_per_shift"] == r.stats["iters_per_shift"]


def test_batched_against_oracle():
    ctxs, srcs, (a, _, _) = build_batch()
    # both solves at tol 1e-12, so that the comparison at 1e-10 is not limited by
    # where each stops
    ys, _ = fa.apply_f_batched(ctxs, srcs, ell=2, tol=1e-12, mode="pseudo", precision="f64")
    d1 = (4, 4, 4, 8)
    U = inputs.su3_exp_gauge(d1, 0.5, 301)
    c = scale.power_scale(dirac.Operator(U, -1.8, 0.05).A, inputs.gaussian_spinor(d1, 304), 100)
    om, sg = fa.neuberger_poles(10)
    from oracle import msbicgstab as ms
    op = dirac.Operator(U, -1.8, 0.05, c)
    y_o = ms.multishift_double(op.A, inputs.gaussian_spinor(d1, 9), sg, om, 2, 1e-12)
    assert rel(to_host(ys[5]), y_o) < 1e-10


@pytest.mark.parametrize("mode,precision", [("double", "f64"), ("pseudo", "mixed"), ("double", "f32"),
                                            ("pseudo", "mixed_df")])
def test_graph_replay_equals_direct_launches(mode, precision):
    import torch
    w = workload_case("wilson_4x4x4x8")
    stream = torch.cuda.Stream()
    ctx = fa.Context(w["dims"], stream)
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], w["c"])
    ctx.set_poles(w["omega"], w["sigma"])
    with torch.cuda.stream(stream):
        b = to_dev(w["b"])
    stream.synchronize()
    kw = dict(ell=2, tol=1e-10, mode=mode, precision=precision)
    r0 = ctx.apply_f(b, **kw)
    r1 = ctx.apply_f(b, graph=True, **kw)
    r2 = ctx.apply_f(b, graph=True, **kw)
    stream.synchronize()
    assert np.array_equal(to_host(r0.y), to_host(r1.y))
    assert np.array_equal(to_host(r1.y), to_host(r2.y))
    assert r1.stats["outer_iters"] == r0.stats["outer_iters"]
    y_o, _ = oracle_double("wilson_4x4x4x8", None, 2, 1e-12)
    tol = {"f64": 1e-9, "mixed": 1e-8, "f32": 1e-6, "mixed_df": 1e-8}[precision]
    assert rel(to_host(r1.y), y_o) < tol


def test_batched_graph_mode():
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctxs, srcs, _ = build_batch(stream)
    stream.synchronize()
    ys0, _ = fa.apply_f_batched(ctxs, srcs, ell=2, tol=1e-10, mode="pseudo", precision="f32")
    ys1, _ = fa.apply_f_batched(ctxs, srcs, ell=2, tol=1e-10, mode="pseudo", precision="f32", graph=True)
    stream.synchronize()
    for a, b in zip(ys0, ys1):
        assert np.array_equal(to_host(a), to_host(b))


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_batched_precise_head_against_oracle(precision):
    """FA_MIXED / FA_MIXED_DF for a batch: the head runs until every system asks
    for the switch; every system then meets the 1e-8 bound against the oracle."""
    from oracle import msbicgstab as ms
    ctxs, srcs, (a, bgrp, cgrp) = build_batch()
    ys, st = fa.apply_f_batched(ctxs, srcs, ell=2, tol=1e-10, mode="pseudo", precision=precision)
    assert len({x["switch_outer"] for x in st}) == 1 and st[0]["switch_outer"] > 0
    for i, (gauge_seed, dims, mu, src) in enumerate(SYSTEMS):
        U = inputs.su3_exp_gauge(dims, 0.5, gauge_seed)
        c = scale.power_scale(dirac.Operator(U, -1.8, mu).A, inputs.gaussian_spinor(dims, gauge_seed + 3), 100)
        om, sg = fa.neuberger_poles(10)
        y_o = ms.multishift_double(dirac.Operator(U, -1.8, mu, c).A, src, sg, om, 2, 1e-12)
        assert rel(to_host(ys[i]), y_o) < 1e-8, i


@pytest.mark.parametrize("precision", ["f64", "f32", "mixed_df"])
def test_graph_cache_follows_context_changes(precision):
    """A graph-replayed solve after a change of mu / mass / scale (fa_set_params),
    of the gauge field, of the FP32 sweep shape or of l (which can reallocate the
    seed vectors) equals a solve with direct launches under the new settings: no
    cached outer iteration replays stale kernel arguments."""
    import torch
    w = workload_case("wilson_4x4x4x8")
    stream = torch.cuda.Stream()
    ctx = fa.Context(w["dims"], stream)
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], w["c"])
    ctx.set_poles(w["omega"], w["sigma"])
    with torch.cuda.stream(stream):
        b = to_dev(w["b"])
    stream.synchronize()
    kw = dict(ell=2, tol=1e-10, mode="pseudo", precision=precision)

    def same(**over):
        k = dict(kw, **over)
        g = to_host(ctx.apply_f(b, graph=True, **k).y)
        d = to_host(ctx.apply_f(b, graph=False, **k).y)
        stream.synchronize()
        assert np.array_equal(g, d), over
        return g

    y0 = same()
    ctx.set_params(w["mass"], 0.15, w["t_bc"], w["c"])           # new mu
    y1 = same()
    assert rel(y1, y0) > 1e-3
    ctx.set_params(-1.7, 0.15, w["t_bc"], 0.9 * w["c"])           # new mass and scale
    y2 = same()
    assert rel(y2, y1) > 1e-3
    U2 = inputs.su3_exp_gauge(w["dims"], 0.5, 777)
    ctx.set_gauge(to_dev(U2))                                     # new gauge field
    y3 = same()
    assert rel(y3, y2) > 1e-3
    ctx.set_hop_shape("wide")                                     # FP32 sweep shape
    same()
    ctx.set_hop_shape("auto")
    same(ell=4)                                                   # larger l reallocates
    same()
    # back to the first settings: the graphs follow again
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], w["c"])
    assert np.array_equal(same(), y0)


def test_point_source_batch_every_system_against_oracle():
    """The batched configuration's structure on stand-in lattices: 12 spin-colour
    point sources on each of three lattices of different shapes (mu drawn per
    lattice), 36 systems in one batched FP32 solve (l 2) and one with a
    double-float head (l 4); every system against the oracle at the bounds of
    the one-system solves (FP32 bulk 1e-6, precise head 1e-8)."""
    from oracle import msbicgstab as ms
    import torch
    rng = np.random.default_rng(404)
    shapes = [(4, 4, 4, 4), (3, 3, 3, 6), (4, 4, 4, 8)]
    stream = torch.cuda.Stream()
    ctxs, srcs, want = [], [], {2: [], 4: []}
    om, sg = fa.neuberger_poles(12)
    with torch.cuda.stream(stream):
        for k, dims in enumerate(shapes):
            mu = float(rng.uniform(0.0, 0.2))
            sources = [inputs.point_source(dims, sp, co) for sp in range(4) for co in range(3)]
            group, bs, (U, c, _, _) = lattice_systems(dims, 500 + k, mu, sources, stream, poles=12)
            ctxs += group
            srcs += bs
            op = dirac.Operator(U, -1.8, mu, c)
            for src in sources:
                for ell in (2, 4):
                    want[ell].append(ms.multishift_double(op.A, src, sg, om, ell, 1e-12))
    stream.synchronize()
    assert len(ctxs) == 36
    for ell, precision, bound in ((2, "f32", 1e-6), (4, "mixed_df", 1e-8)):
        ys, st = fa.apply_f_batched(ctxs, srcs, ell=ell, tol=1e-10, mode="pseudo", precision=precision, graph=True)
        stream.synchronize()
        assert all(x["status"] == 0 for x in st)
        worst = max(rel(to_host(y), w) for y, w in zip(ys, want[ell]))
        assert worst < bound, (ell, precision, worst)


def test_batched_autotuner_keeps_results():
    """fa_autotune_batched times the multi-RHS sweep's shapes and keeps the
    fastest; the batched solve with the chosen shape equals the default's bit
    for bit (the shape decides only which block runs which right-hand side)."""
    ctxs, srcs, _ = build_batch()
    kw = dict(ell=2, tol=1e-10, mode="pseudo", precision="f32")
    y0, _ = fa.apply_f_batched(ctxs, srcs, **kw)
    tune = fa.autotune_batched(ctxs, reps=5)
    assert tune["rhs_per_block"] in (1, 2, 3, 4, 6, 12, 16) and tune["min_blocks"] in (4, 7)
    assert all(t > 0 for t in tune["times_ms"].values())
    y1, _ = fa.apply_f_batched(ctxs, srcs, **kw)
    for a, b in zip(y0, y1):
        assert np.array_equal(to_host(a), to_host(b))
