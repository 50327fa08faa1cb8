"""Write the stored expected values of the full-size parity test.

Runs the FP64 oracle only (never the CUDA path) on the 16^3 x 32 workload:
the power-iteration scale c, then the double-pass multi-shift BiCGstab(2)
with Neuberger's 20 poles at tol 1e-12, and stores c, the outer-iteration
counts and y* = f(A) b at 512 seeded sample positions, plus |y*|.

    python tests/golden/make_golden.py [workload] [tol]     (about 15 min of numpy)
    python tests/golden/make_golden.py --sites [workload]   (tol 1e-12, site samples)

With a tolerance other than 1e-12 the file is named <workload>_tol<tol>.json; the
benchmark reads the outer-iteration count of the tol-1e-9 run to scale its oracle
(CPU) baseline to a whole solve at the headline's tolerance.

--sites writes <workload>_sites.json: y* at all 12 spin-colour components of
48 seeded sites in every time slice (t = 0 and T-1, where the antiperiodic
sign acts, included), 18,432 entries for the 16^3 x 32 workload, so that the
relative 2-norm of the difference on the sample estimates the full-vector
error of a solve.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle import dirac, msbicgstab as ms, poles, scale  # noqa: E402


def oracle_solution(name, tol):
    """y* = f(A) b by the FP64 oracle's double-pass solve, with c and its stats."""
    w = inputs.make_workload(name)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], 1.0, w["t_bc"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c, w["t_bc"])
    om, sg = poles.neuberger_poles(w["ns"])
    st = ms.Stats()
    y = ms.multishift_double(op.A, w["b"], sg, om, w["ell"], tol, stats=st)
    return w, c, st, y


def main_sites(name="wilson_16x16x16x32", tol=1e-12, per_slice=48):
    t0 = time.time()
    w, c, st, y = oracle_solution(name, tol)
    X, Y, Z, T = w["dims"]
    rng = np.random.default_rng(4243)
    sites = []
    for t in range(T):
        flat = rng.choice(X * Y * Z, size=per_slice, replace=False)
        for f in sorted(flat.tolist()):
            x, r = f % X, f // X
            sites.append([t, r // Y, r % Y, x])       # canonical index order (t, z, y, x)
    idx = np.asarray(sites)
    vals = y[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].reshape(len(sites), 12)
    out = dict(
        workload=name, dims=list(w["dims"]), ell=w["ell"], ns=w["ns"], tol=tol, scale_c=c,
        outer_iters=st.n_outer, y_norm=float(np.linalg.norm(y)), sites_per_slice=per_slice,
        site_index_tzyx=idx.tolist(), y_re=np.round(vals.real, 17).tolist(), y_im=np.round(vals.imag, 17).tolist(),
        oracle_seconds=time.time() - t0,
        source="oracle.msbicgstab.multishift_double (FP64 numpy), written by tests/golden/make_golden.py --sites",
    )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_sites.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, st.n_outer, time.time() - t0)


def main(name="wilson_16x16x16x32", tol=1e-12, n_samples=512):
    t0 = time.time()
    w = inputs.make_workload(name)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], 1.0, w["t_bc"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c, w["t_bc"])
    om, sg = poles.neuberger_poles(w["ns"])
    st = ms.Stats()
    y = ms.multishift_double(op.A, w["b"], sg, om, w["ell"], tol, stats=st)
    rng = np.random.default_rng(4242)
    shape = y.shape
    idx = np.stack([rng.integers(0, n, n_samples) for n in shape], axis=1)
    vals = y[tuple(idx.T)]
    out = dict(
        workload=name, dims=list(w["dims"]), ell=w["ell"], ns=w["ns"], tol=tol, scale_c=c,
        outer_iters=st.n_outer, iters_per_shift=[int(v) for v in st.iters_per_shift],
        n_mv=st.n_mv, y_norm=float(np.linalg.norm(y)), sample_index=idx.tolist(),
        sample_re=vals.real.tolist(), sample_im=vals.imag.tolist(),
        oracle_seconds=time.time() - t0,
        source="oracle.msbicgstab.multishift_double (FP64 numpy), written by tests/golden/make_golden.py",
    )
    suffix = "" if tol == 1e-12 else f"_tol{tol:g}"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}{suffix}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, st.n_outer, time.time() - t0)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "--sites":
        main_sites(*(args[1:2] or ["wilson_16x16x16x32"]))
        sys.exit(0)
    main(args[0] if args else "wilson_16x16x16x32", float(args[1]) if len(args) > 1 else 1e-12)
