"""Learned prolongator: training data from the plain method, GPU training, inference and the
accept/reject rule.

Every numeric step runs in librmg.so (features, operator-dependent weights, measured
convergence factors, the MLP's forward/backward/Adam kernels); this module only moves arrays
between those calls.

* Labels. For each training operator the plain method measures the two-grid A-norm error
  reduction (rmg_hier_convergence_factor) with linear interpolation and with the
  operator-dependent (series-resistance) weights; the label of every fine node is the
  per-axis weight vector of the better candidate.
* Training. rmg_mlp_train (Adam, batches drawn on the device).
* Inference. rmg_hier_mlp_weights predicts per-node, per-axis weights from the composite
  operator; co-located copies get identical weights.
* Acceptance. The learned weights are kept only if the measured V-cycle convergence factor is
  no worse than with linear interpolation (the plain prolongator is the fallback).
"""
from __future__ import annotations

import numpy as np

from . import rmg, upload

NFEAT = 32
ACTIVE = [8, 17, 26]          # active-axis flags in the feature vector
REMFRAC = [7, 16, 25]         # rem/3 in the feature vector (the linear weights)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform initial parameters (drawn on the host and passed to the library)."""
    rng = np.random.default_rng(seed)

    def layer(n_out, n_in):
        lim = np.sqrt(6.0 / n_in)
        return rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)

    W1, b1 = layer(64, NFEAT)
    W2, b2 = layer(64, 64)
    W3, b3 = layer(3, 64)
    W3 *= 0.1
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float32)


def _options(levels, smoother="chebyshev"):
    o = rmg.default_options(levels=levels)
    if smoother == "chebyshev":
        o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
    else:
        o.smoother, o.nu1, o.nu2, o.omega = rmg.JACOBI, 2, 2, 0.67
    return o


def label_operator(ctx, problem, levels=2, iters=6, seed=7, device="cuda:0"):
    """Features, labels and loss mask of one operator (device tensors) and the two measured
    two-grid factors (linear, operator-dependent)."""
    import torch
    dp = upload(problem, device)
    lay = rmg.Layout(ctx, problem.dim, problem.region_dims, dp.gids, problem.n_nodes,
                     dp.dirichlet)
    lay.operator_from_csr(problem.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, _options(levels))
    n_r = lay.sizes()["n_regional"]
    feats = torch.empty((n_r, NFEAT), dtype=torch.float32, device=device)
    h.mlp_features(0, feats)
    f_lin = h.convergence_factor(iters, seed)
    wr = torch.empty(3 * n_r, dtype=torch.float32, device=device)
    h.opdep_weights(0, wr)
    h.set_transfer_weights(0, wr)
    h.setup_numeric()
    f_op = h.convergence_factor(iters, seed)
    if f_op < f_lin:
        labels = wr.view(3, n_r).t().contiguous()
    else:
        labels = feats[:, REMFRAC].contiguous()
    interior = (dp.dirichlet[dp.gids] == 0).to(torch.float32)
    mask = (feats[:, ACTIVE] * interior[:, None]).contiguous()
    h.close()
    lay.close()
    return feats, labels, mask, (f_lin, f_op)


def training_set(ctx, seeds, make_problem, levels=2, iters=6, device="cuda:0"):
    """Concatenated features/labels/masks of the operators make_problem(seed)."""
    import torch
    F, Y, M, factors = [], [], [], []
    for s in seeds:
        f, y, m, fac = label_operator(ctx, make_problem(s), levels, iters, device=device)
        F.append(f); Y.append(y); M.append(m); factors.append(fac)
    return torch.cat(F), torch.cat(Y), torch.cat(M), np.asarray(factors)


def train(ctx, feats, labels, mask, steps=1500, batch=16384, lr=2e-3, seed=0, init_seed=0):
    net = rmg.MLP(ctx, init_params(init_seed))
    hist = net.train(feats, labels, mask, steps=steps, batch=batch, lr=lr, seed=seed)
    return net, hist


def apply_learned(h, net, n_regional, levels=(0,), iters=6, seed=7, device="cuda:0"):
    """Predict weights for the given levels, accept them if the measured convergence factor
    is no worse than with linear interpolation, otherwise restore linear interpolation."""
    import torch
    f_plain = h.convergence_factor(iters, seed)
    for l in levels:
        n_l = h.level_sizes(l)[0]
        wr = torch.empty(3 * n_l, dtype=torch.float32, device=device)
        h.mlp_weights(l, net, wr)
        h.set_transfer_weights(l, wr)
    h.setup_numeric()
    f_learned = h.convergence_factor(iters, seed)
    accepted = f_learned <= f_plain
    if not accepted:
        for l in levels:
            h.set_transfer_weights(l, None)
        h.setup_numeric()
    return dict(accepted=bool(accepted), factor_plain=f_plain, factor_learned=f_learned)
