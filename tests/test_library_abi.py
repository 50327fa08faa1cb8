"""The C-ABI library loads and exports every entry point of include/fapath.h
(no GPU needed), and its host-side pole table matches the oracle's."""
import os
import re

import numpy as np
import pytest

import paper_1010_2592_gb300 as fa
from oracle import poles

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    """Compile libfapath.so first if this checkout has not built it yet."""
    if not os.path.exists(fa.LIB_PATH):
        from paper_1010_2592_gb300 import build
        build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fapath.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fa_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert set(declared_functions()) == set(fa.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = fa.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version():
    lib = fa.load_library()
    assert lib.fa_status_string(0) == b"ok"
    for s in range(-8, 0):
        assert lib.fa_status_string(s) != b"unknown status"
    assert b"sm_103a" in lib.fa_version()


@pytest.mark.parametrize("ns", [1, 10, 20, 32, 64])
def test_library_neuberger_poles_match_oracle(ns):
    om, sg = fa.neuberger_poles(ns)
    om_o, sg_o = poles.neuberger_poles(ns)
    assert np.allclose(om, om_o, rtol=1e-15, atol=0)
    assert np.allclose(sg, sg_o, rtol=1e-15, atol=1e-300)


@pytest.mark.parametrize("ns,eps", [(1, 0.5), (4, 0.05), (10, 0.01), (20, 0.003), (32, 1e-3)])
def test_library_zolotarev_poles_match_oracle(ns, eps):
    """Host code: the library's own elliptic functions (AGM scale) against the
    oracle's library routines (scipy.special)."""
    om, sg, d = fa.zolotarev_poles(ns, eps)
    om_o, sg_o, d_o = poles.zolotarev_poles(ns, eps)
    assert np.allclose(om, om_o, rtol=1e-10, atol=0)
    assert np.allclose(sg, sg_o, rtol=1e-10, atol=0)
    assert abs(d - d_o) <= 1e-6 * d_o + 1e-13   # the library reports the largest error over all alternation points


@pytest.mark.parametrize("ns,eps", [(40, 1e-8), (64, 1e-6), (24, 1e-12)])
def test_library_zolotarev_poles_against_high_precision(ns, eps):
    """Small eps and many poles, where cn of modulus sqrt(1 - eps^2) is tiny in
    the middle of the range: the library against the same construction in
    40-digit arithmetic (mpmath's elliptic functions)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    e = mp.mpf(eps)
    m = 1 - e * e
    K = mp.ellipk(m)
    c = [e * e * (mp.ellipfun("sn", l * K / (2 * ns), m=m) / mp.ellipfun("cn", l * K / (2 * ns), m=m)) ** 2
         for l in range(1, 2 * ns)]
    sig, zer = c[0::2], c[1::2]
    res = []
    for s in range(ns):
        r = mp.mpf(1)
        for z in zer:
            r *= z - sig[s]
        for t in range(ns):
            if t != s:
                r /= sig[t] - sig[s]
        res.append(r)
    xs = [e / mp.ellipfun("dn", j * K / (2 * ns), m=m) for j in range(2)]
    P = [x * sum(r / (x * x + sg) for r, sg in zip(res, sig)) for x in xs]
    D = 2 / (P[0] + P[1])
    om, sg, d = fa.zolotarev_poles(ns, eps)
    assert np.allclose(sg, [float(x) for x in sig], rtol=1e-12, atol=0)
    assert np.allclose(om, [float(D * r) for r in res], rtol=1e-10, atol=0)
    assert abs(d - float(abs(D * P[0] - 1))) <= 1e-6 * d + 1e-13


def test_library_zolotarev_poles_equioscillate_at_small_eps():
    """Where scipy's elliptic functions lose digits (modulus near 1), the
    library's poles still give the alternation of the best approximation."""
    from closed_forms import alternation
    ns, eps = 5, 1e-4
    om, sg, d = fa.zolotarev_poles(ns, eps)
    dd, signs = alternation(om, sg, eps, npts=2000001)
    assert len(signs) == 2 * ns + 1 and np.all(signs[1:] != signs[:-1])
    assert abs(dd - d) <= 1e-5 * d


def test_invalid_arguments_rejected_before_any_device_call():
    import ctypes
    lib = fa.load_library()
    h = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 8)
    assert lib.fa_create(ctypes.byref(h), bad, None) == fa.FA_EINVAL
    assert lib.fa_neuberger_poles(0, None, None) == fa.FA_EINVAL
    assert lib.fa_neuberger_poles(65, None, None) == fa.FA_EINVAL
    assert lib.fa_destroy(None) == fa.FA_OK
    assert lib.fa_set_params(None, -1.8, 0.1, -1, 1.0) == fa.FA_EINVAL
    om = np.empty(4)
    for bad_eps in (0.0, 1.0, -0.1, float("nan")):
        assert lib.fa_zolotarev_poles(4, bad_eps, om.ctypes.data, om.ctypes.data, None) == fa.FA_EINVAL
    assert lib.fa_zolotarev_poles(65, 0.1, om.ctypes.data, om.ctypes.data, None) == fa.FA_EINVAL

    ms, n = ctypes.c_double(), ctypes.c_longlong()
    assert lib.fa_hop_timing_split(None, fa.F32, 0, ctypes.byref(ms), ctypes.byref(n)) == fa.FA_EINVAL


def _struct_fields(name):
    """Field names, in order, of the typedef struct `name` in include/fapath.h."""
    src = open(os.path.join(ROOT, "include", "fapath.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[[^\]]*\]", "", decl).strip()     # drop array sizes
        if decl:
            # "type a, b, c": the first piece ends with the first name
            fields += [piece.split()[-1].lstrip("*") for piece in decl.split(",")]
    return fields


def test_binding_structs_follow_the_header():
    """The ctypes mirrors of fa_solver_params and fa_solver_stats list the
    header's fields in the header's order (a field added on one side only would
    shift every later one)."""
    assert [f for f, _ in fa.SolverParams._fields_] == _struct_fields("fa_solver_params")
    assert [f for f, _ in fa.SolverStats._fields_] == _struct_fields("fa_solver_stats")


def test_status_codes_follow_the_header():
    """Every fa_status code of the header has the same value in the binding."""
    src = open(os.path.join(ROOT, "include", "fapath.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(FA_E[A-Z]+|FA_OK)\s*=\s*(-?\d+)", src))
    assert len(codes) == 9
    for k, v in codes.items():
        assert getattr(fa, k) == v, k
