"""Test helper: build a library Sampler from a seeded workloads.Problem."""
import numpy as np

import paper_2507_14652_gb300 as hmc
import workloads as W


def sampler_from(prob, prec, chains=None, n_splits=1, rows_per_pass=0):
    C = prob.chains if chains is None else chains
    if prob.kind == W.KIND_MLP:
        return hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, C,
                               prior_sigma=prob.prior_sigma, noise_sigma=prob.noise_sigma, prec=prec,
                               act=prob.net.act, bias=prob.net.bias, n_splits=n_splits,
                               rows_per_pass=rows_per_pass)
    return hmc.Sampler.deeponet(prob.branch.widths, prob.trunk.widths, prob.u, prob.yq, prob.t, prob.mask,
                                prob.frozen, C, prior_sigma=prob.prior_sigma, noise_sigma=prob.noise_sigma,
                                prec=prec, out_bias=prob.out_bias, branch_act=prob.branch.act,
                                trunk_act=prob.trunk.act, branch_bias=prob.branch.bias,
                                trunk_bias=prob.trunk.bias, n_splits=n_splits, rows_per_pass=rows_per_pass)


def rel_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grad_ok(g, gref, tol):
    """North-star gradient tolerance: relative 2-norm error and a per-component bound."""
    g, gref = np.asarray(g, dtype=np.float64), np.asarray(gref, dtype=np.float64)
    rms = np.sqrt(np.mean(gref ** 2))
    comp = np.abs(g - gref) <= tol * (np.abs(gref) + rms)
    return rel_err(g, gref) <= tol and bool(comp.all()), rel_err(g, gref), float(
        np.max(np.abs(g - gref) / (np.abs(gref) + rms)))


def grad_ok_bf16(g, gref, tol=2e-2):
    """BF16 gradient tolerance, per gradient evaluation: relative 2-norm error and
    relative infinity-norm error both within tol."""
    g, gref = np.asarray(g, dtype=np.float64), np.asarray(gref, dtype=np.float64)
    r2 = rel_err(g, gref)
    rinf = float(np.max(np.abs(g - gref)) / max(np.max(np.abs(gref)), 1e-300))
    return r2 <= tol and rinf <= tol, r2, rinf
