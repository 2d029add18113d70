"""Learned prolongator: training data from the plain method, GPU training, inference and the
accept/reject rule.

Every numeric step runs in librmg.so (features, operator-dependent weights, measured
convergence factors and region energies, the MLP's forward/backward/Adam kernels, the blend of
learned and linear weights); this module only moves arrays between those calls.

* Labels. Training operators are labelled in batches: a batch of independent operators is laid
  side by side as one system with disconnected components (workloads.batch), so one two-grid
  hierarchy treats all of them. For every operator the plain method measures the two-grid
  A-norm error reduction (rmg_hier_region_energies summed over the operator's regions) with
  linear interpolation and with the operator-dependent (series-resistance) weights; the label
  of every fine node is the per-axis weight vector of the better candidate for its operator.
* Training. rmg_mlp_train (Adam, batches drawn on the device).
* Inference. rmg_hier_mlp_weights predicts per-node, per-axis weights from the composite
  operator; co-located copies get identical weights.
* Acceptance, per region. With linear and with learned weights the V-cycle runs as a
  stationary solver from the same random error; region k keeps the learned weights when its
  energy reduction (e_k^T A^(k) e_k after / before) is no worse than with linear interpolation.
  Nodes shared with a rejecting region keep linear weights (rmg_hier_blend_weights), so copies
  stay identical. The plain prolongator is the fallback and the yardstick: if the blended weights
  give a worse global factor than linear interpolation, linear interpolation is restored.
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


def factors_from_energies(e0, eK, iters, groups=None):
    """Energy reduction factors (eK / e0)^(1 / (2 iters)) of every region, or of every group of
    regions (groups: the group id of every region) with the energies summed over the group."""
    if groups is not None:
        k = int(np.max(groups)) + 1
        e0 = np.bincount(groups, weights=e0, minlength=k)
        eK = np.bincount(groups, weights=eK, minlength=k)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(e0 > 0, np.maximum(eK, 0.0) / np.where(e0 > 0, e0, 1.0), 0.0)
    return f ** (0.5 / iters)


def label_batch(ctx, problems, levels=2, iters=6, seed=7, device="cuda:0"):
    """Features, labels and loss mask (device tensors, rows = regional nodes of the batch) of
    independent operators labelled together, and their (linear, operator-dependent) two-grid
    factors, one row per operator."""
    import torch
    import workloads as W
    B = W.batch(problems)
    dp = upload(B, device, with_rhs=False)
    lay = rmg.Layout(ctx, B.dim, B.region_dims, dp.gids, B.n_nodes, dp.dirichlet)
    lay.operator_from_csr(B.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, _options(levels))
    n_r = lay.sizes()["n_regional"]
    feats = torch.empty((n_r, NFEAT), dtype=torch.float32, device=device)
    h.mlp_features(0, feats)
    e0, eK = h.region_energies(iters, seed)
    f_lin = factors_from_energies(e0, eK, iters, B.region_component)
    wr = torch.empty(3 * n_r, dtype=torch.float32, device=device)
    h.opdep_weights(0, wr)
    h.set_transfer_weights(0, wr)
    h.setup_numeric()
    e0, eK = h.region_energies(iters, seed)
    f_op = factors_from_energies(e0, eK, iters, B.region_component)
    # labels: the teacher's weights in the regions of operators where it wins, linear ones
    # elsewhere (the blend kernel, with "accept" = the teacher wins for the region's operator)
    better = (f_op < f_lin)[B.region_component].astype(np.uint8)
    lab = torch.empty(3 * n_r, dtype=torch.float32, device=device)
    h.blend_weights(0, better, wr, lab)
    labels = lab.view(3, n_r).t().contiguous()
    interior = (dp.dirichlet[dp.gids] == 0).to(torch.float32)
    mask = (feats[:, ACTIVE] * interior[:, None]).contiguous()
    h.close()
    lay.close()
    return feats, labels, mask, np.stack([f_lin, f_op], axis=1)


def label_operator(ctx, problem, levels=2, iters=6, seed=7, device="cuda:0"):
    """label_batch of a single operator (its factors as a tuple)."""
    f, y, m, fac = label_batch(ctx, [problem], levels, iters, seed, device)
    return f, y, m, (float(fac[0, 0]), float(fac[0, 1]))


def _coarse_unknowns(problem, levels):
    """Unknowns of the coarsest level of a box-tiled problem with Dirichlet faces (an estimate
    from the global node counts, (N - 1) / 3^(levels - 1) + 1 per axis, boundary removed)."""
    n = 1
    for N in problem.global_dims:
        if N == 1:
            continue
        c = (N - 1) // 3 ** (levels - 1) + 1
        n *= max(c - 2, 0)
    return n


def training_set(ctx, seeds, make_problem, levels=2, iters=6, device="cuda:0", batch=50,
                 max_coarse=12000):
    """Concatenated features/labels/masks of the operators make_problem(seed), labelled in
    batches of at most `batch` independent operators whose coarsest levels together stay
    within max_coarse unknowns (the dense coarse solver takes 16384); factors has one row per
    operator."""
    import torch
    F, Y, M, factors = [], [], [], []
    pending, coarse = [], 0

    def flush():
        f, y, m, fac = label_batch(ctx, pending, levels, iters, device=device)
        F.append(f); Y.append(y); M.append(m); factors.append(fac)

    for s in seeds:
        p = make_problem(s)
        nc = _coarse_unknowns(p, levels)
        if pending and (len(pending) >= batch or coarse + nc > max_coarse):
            flush()
            pending, coarse = [], 0
        pending.append(p)
        coarse += nc
    if pending:
        flush()
    return torch.cat(F), torch.cat(Y), torch.cat(M), np.concatenate(factors)


def train(ctx, feats, labels, mask, steps=1500, batch=16384, lr=2e-3, seed=0, init_seed=0):
    net = rmg.MLP(ctx, init_params(init_seed))
    hist = net.train(feats, labels, mask, steps=steps, batch=batch, lr=lr, seed=seed)
    return net, hist


def accept_per_region(h, candidate, n_regional, iters=6, seed=7, device="cuda:0"):
    """Keep the candidate level-0 weights (device float[3 * n_r], identical on co-located
    copies) in the regions where they help, linear interpolation elsewhere.

    A region's effect is measured with its neighbours on linear interpolation: for every colour
    class of the region graph (rmg_hier_region_colours; regions of one class never touch) the
    candidate is switched on in that class alone (rmg_hier_blend_weights), the V-cycle runs as
    a stationary solver from a fixed random error, and every region of the class is accepted
    when its energy reduction (e_k^T A^(k) e_k after / before, rmg_hier_region_energies) is no
    worse than with linear interpolation everywhere. The accepted regions are then switched on
    together; if that is globally worse than linear interpolation the plain prolongator is
    restored. Leaves the hierarchy set up with the chosen transfer. The host only compares the
    per-region scalars the library returns."""
    import torch
    h.set_transfer_weights(0, None)
    h.setup_numeric()
    p0, pK = h.region_energies(iters, seed)
    f_plain_r = factors_from_energies(p0, pK, iters)
    f_plain = float(factors_from_energies(np.array([p0.sum()]), np.array([pK.sum()]), iters)[0])
    h.set_transfer_weights(0, candidate)
    h.setup_numeric()
    c0, cK = h.region_energies(iters, seed)
    f_cand = float(factors_from_energies(np.array([c0.sum()]), np.array([cK.sum()]), iters)[0])
    colours, ncol = h.region_colours()
    mixed = torch.empty(3 * n_regional, dtype=torch.float32, device=device)
    accept = np.zeros(colours.size, dtype=np.uint8)
    for c in range(ncol):
        trial = (colours == c).astype(np.uint8)
        h.blend_weights(0, trial, candidate, mixed)
        h.set_transfer_weights(0, mixed)
        h.setup_numeric()
        t0, tK = h.region_energies(iters, seed)
        f_trial = factors_from_energies(t0, tK, iters)
        accept |= (trial.astype(bool) & (f_trial <= f_plain_r)).astype(np.uint8)
    h.blend_weights(0, accept, candidate, mixed)
    h.set_transfer_weights(0, mixed)
    h.setup_numeric()
    m0, mK = h.region_energies(iters, seed)
    f_mixed = float(factors_from_energies(np.array([m0.sum()]), np.array([mK.sum()]), iters)[0])
    kept = bool(accept.any()) and f_mixed <= f_plain
    if not kept:
        h.set_transfer_weights(0, None)
        h.setup_numeric()
    return dict(accepted=kept, regions=int(accept.size),
                regions_accepted=int(accept.sum()) if kept else 0, colours=int(ncol),
                factor_plain=f_plain, factor_candidate=f_cand, factor_blended=f_mixed,
                factor=f_mixed if kept else f_plain, weights=mixed if kept else None,
                accept=accept if kept else np.zeros_like(accept))


def apply_learned(h, net, n_regional, iters=6, seed=7, device="cuda:0"):
    """Predict level-0 weights with the network and accept them region by region
    (accept_per_region)."""
    import torch
    wr = torch.empty(3 * n_regional, dtype=torch.float32, device=device)
    h.mlp_weights(0, net, wr)
    res = accept_per_region(h, wr, n_regional, iters, seed, device)
    res["factor_learned"] = res["factor_candidate"]
    return res
