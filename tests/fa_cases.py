"""Shared set-up of the GPU parity tests: seeded inputs, oracle references."""
from __future__ import annotations

import functools

import numpy as np

import inputs
from oracle import dirac, msbicgstab as ms, poles, scale


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def to_host(t):
    return t.detach().cpu().numpy()


def make_context(dims, U, mass, mu, c, t_bc=-1, omega=None, sigma=None):
    import paper_1010_2592_gb300 as fa
    ctx = fa.Context(dims)
    ctx.set_gauge(to_dev(U))
    ctx.set_params(mass, mu, t_bc, c)
    if omega is not None:
        ctx.set_poles(omega, sigma)
    return ctx


@functools.lru_cache(maxsize=8)
def workload_case(name, dims=None):
    """Inputs, oracle scale c and poles of a workload (optionally resized)."""
    w = inputs.make_workload(name, dims)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], 1.0, w["t_bc"])
    c = scale.power_scale(op.A, w["v0"], 100)
    om, sg = poles.neuberger_poles(w["ns"])
    w.update(c=c, omega=om, sigma=sg)
    return w


@functools.lru_cache(maxsize=64)
def oracle_double(name, dims, ell, tol):
    w = workload_case(name, dims)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], w["c"], w["t_bc"])
    st = ms.Stats()
    y = ms.multishift_double(op.A, w["b"], w["sigma"], w["omega"], ell, tol, stats=st)
    return y, st


@functools.lru_cache(maxsize=64)
def oracle_single(name, dims, ell, tol):
    w = workload_case(name, dims)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], w["c"], w["t_bc"])
    st = ms.Stats()
    xs = ms.multishift_single(op.A, w["b"], w["sigma"], ell, tol, stats=st)
    return xs, st
