"""fa_apply_A_noalloc, the entry point for callers that cannot let the library
allocate device memory (graph capture in global mode, framework-owned memory
budgets): it must give the same A v as fa_apply_A on two calls in a row, each
with fresh inputs, and reject lattices beyond its static scratch limit.

Collected last on purpose: it shares one static device array across calls,
so it runs after every other test of a session as well as alone."""
import ctypes

import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import make_context, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_noalloc_apply_A_matches_apply_A_twice():
    import torch
    dims = (8, 8, 8, 16)                       # 8192 sites: the static limit
    ctx = make_context(dims, inputs.su3_exp_gauge(dims, 0.5, 601), -1.8, 0.05, 0.031)
    lib = fa.load_library()
    for call, seed in enumerate((602, 603)):
        x = to_dev(inputs.gaussian_spinor(dims, seed))
        for dagger in (0, 1):
            want = to_host(ctx.apply_A(x, dagger=bool(dagger)))
            out = torch.empty_like(x)
            rc = lib.fa_apply_A_noalloc(ctx.h, ctx_ptr(x), ctx_ptr(out), dagger)
            assert rc == fa.FA_OK, (call, lib.fa_last_error())
            ctx.sync()
            assert rel(to_host(out), want) < 1e-13, (call, dagger)


def test_noalloc_rejects_lattices_beyond_the_limit():
    import torch
    dims = (8, 8, 8, 18)                       # 9216 sites
    ctx = make_context(dims, inputs.su3_exp_gauge(dims, 0.5, 604), -1.8, 0.05, 0.031)
    x = to_dev(inputs.gaussian_spinor(dims, 605))
    out = torch.zeros_like(x)
    lib = fa.load_library()
    assert lib.fa_apply_A_noalloc(ctx.h, ctx_ptr(x), ctx_ptr(out), 0) == fa.FA_EINVAL
    assert b"static scratch limit" in lib.fa_last_error()
    assert not bool(torch.any(out != 0))


def ctx_ptr(t):
    return ctypes.c_void_p(t.data_ptr())
