"""Operator-dependent interpolation weights and the small MLP of the learned prolongator.

The paper keeps linear interpolation and notes that matrix-dependent transfers (black box
multigrid) must produce identical stencils at co-located nodes (Sec. 3.2). The learned
prolongator predicts per-node, per-axis interpolation weights; its teacher is the
operator-dependent candidate below, computed from the composite matrix:

  along axis a, a fine node at remainder rem between coarse nodes X0 and X0 + 3 lies on a
  line of three edges with conductances k_e = -A(p_e, p_e+1); as resistors in series the
  weight of the right coarse node is sum_{e < rem} (1/k_e) / sum_e (1/k_e) (the 1D
  A-harmonic extension); rem/3 (linear) when a conductance is not positive.

The MLP functions are a plain FP64 restatement of the network (27 features padded to 32 ->
64 -> 64 -> 3, ReLU, ReLU, sigmoid) with the BF16 roundings of the GPU forward pass applied
at the same points, used to check the GPU gradients.

The network input (``features``) is, per fine node and axis, the line of three edges between
its two coarse neighbours read from the composite matrix: log10 of the three conductances
-A(p_e, p_e+1) and of the four diagonals A(p_i, p_i), each divided by the node's own
diagonal, then rem/3 and an active flag (zero along axes where the node sits on a coarse
index). Its output (``weights_from_outputs``) is the right-neighbour weight per active axis.
The paper has no learned transfer: the network, its features and its outputs are readings
of the scope, pinned by closed forms (a hand-set network, the constant-coefficient
Laplacian's features) rather than by the paper.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NFEAT = 32
H = 64
NOUT = 3


def opdep_weights(A: sp.csr_matrix, global_dims) -> np.ndarray:
    """(3, n) operator-dependent right weights per composite node and axis."""
    Nx, Ny, Nz = global_dims
    n = Nx * Ny * Nz
    A = sp.csr_matrix(A)
    g = np.arange(n)
    coord = [g % Nx, (g // Nx) % Ny, g // (Nx * Ny)]
    stride = [1, Nx, Nx * Ny]
    dims = [Nx, Ny, Nz]
    wr = np.zeros((3, n))
    for a in range(3):
        if dims[a] == 1:
            continue
        rem = coord[a] % 3
        act = np.flatnonzero(rem != 0)
        r = rem[act]
        p0 = act - r * stride[a]
        ks = []
        for e in range(3):
            i = p0 + e * stride[a]
            j = i + stride[a]
            ks.append(-np.asarray(A[i, j]).ravel())
        k = np.stack(ks)                       # (3, m)
        good = np.all(k > 0, axis=0)
        res = np.where(good, 1.0 / np.where(good, k, 1.0), 0.0)
        tot = res.sum(axis=0)
        num = np.where(r == 1, res[0], res[0] + res[1])
        w = np.where(good, num / np.where(good, tot, 1.0), r / 3.0)
        wr[a, act] = w
    return wr


# ------------------------------------------------------------------------------ MLP
def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * NFEAT].reshape(H, NFEAT); o += H * NFEAT
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + NOUT * H].reshape(NOUT, H); o += NOUT * H
    b3 = p[o:o + NOUT]; o += NOUT
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


NPARAMS = H * NFEAT + H + H * H + H + NOUT * H + NOUT


def forward(params, X, rounding=True):
    """Forward pass with the GPU's BF16 operand roundings (inputs, weights, hidden
    activations; ``rounding=False`` gives the exact FP64 network), FP64 accumulation.
    Returns the outputs and the cached activations."""
    rnd = bf16_round if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(params)
    Xb = rnd(X)
    Z1 = Xb @ rnd(W1).T + b1
    H1 = np.maximum(Z1, 0.0)
    H1b = rnd(H1)
    Z2 = H1b @ rnd(W2).T + b2
    H2 = np.maximum(Z2, 0.0)
    H2b = rnd(H2)
    Z3 = H2b @ rnd(W3).T + b3
    O = 1.0 / (1.0 + np.exp(-Z3))
    return O, (Xb, H1b, H2b, O)


def loss_and_grad(params, X, Y, M, rounding=True):
    """Masked mean squared error L = sum M (O - Y)^2 / (3 B) and its gradient by the chain
    rule (ReLU derivative taken where the activation is positive). The backward pass uses
    FP32 weights for the data gradients, as the GPU does."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    B = X.shape[0]
    O, (Xb, H1b, H2b, _) = forward(params, X, rounding)
    L = float(np.sum(M * (O - Y) ** 2) / (NOUT * B))
    dO = 2.0 * M * (O - Y) / (NOUT * B)
    dZ3 = dO * O * (1.0 - O)
    dW3 = dZ3.T @ H2b
    db3 = dZ3.sum(axis=0)
    dH2 = dZ3 @ W3
    dZ2 = dH2 * (H2b > 0)
    dW2 = dZ2.T @ H1b
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (H1b > 0)
    dW1 = dZ1.T @ Xb
    db1 = dZ1.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, grad


# ------------------------------------------------------------------------------ features
def features(A: sp.csr_matrix, global_dims) -> np.ndarray:
    """(n, 32) network inputs of every composite node (columns 27..31 are zero padding).

    Per axis a (9 columns from 9a): a node at remainder rem = c_a mod 3 != 0 lies between the
    coarse nodes p_0 = g - rem s_a and p_3 = p_0 + 3 s_a. With d_g = A(g, g) (1 when not
    positive): log10(max(k_e / d_g, 1e-12)) capped at 2 for the conductances
    k_e = -A(p_e, p_e + s_a), e = 0, 1, 2; log10(max(A(p_i, p_i) / d_g, 1e-12)) capped at 12
    for i = 0..3; rem / 3; 1. An axis with rem = 0, or one the grid does not have (2D: z), is
    all zero."""
    Nx, Ny, Nz = global_dims
    n = Nx * Ny * Nz
    A = sp.csr_matrix(A)
    diag = A.diagonal()
    g = np.arange(n)
    coord = [g % Nx, (g // Nx) % Ny, g // (Nx * Ny)]
    stride = [1, Nx, Nx * Ny]
    dims = [Nx, Ny, Nz]
    dref = np.where(diag > 0, diag, 1.0)
    F = np.zeros((n, NFEAT))
    for a in range(3):
        if dims[a] == 1:
            continue
        rem = coord[a] % 3
        act = np.flatnonzero(rem != 0)
        r = rem[act]
        p0 = act - r * stride[a]
        for e in range(3):
            i = p0 + e * stride[a]
            k = -np.asarray(A[i, i + stride[a]]).ravel()
            F[act, 9 * a + e] = np.minimum(np.log10(np.maximum(k / dref[act], 1e-12)), 2.0)
        for e in range(4):
            d = diag[p0 + e * stride[a]]
            F[act, 9 * a + 3 + e] = np.minimum(np.log10(np.maximum(d / dref[act], 1e-12)), 12.0)
        F[act, 9 * a + 7] = r / 3.0
        F[act, 9 * a + 8] = 1.0
    return F


def weights_from_outputs(feats, out) -> np.ndarray:
    """(3, n) right-neighbour weights: the network output along active axes, 0 elsewhere."""
    F = np.asarray(feats)
    O = np.asarray(out)
    return np.stack([np.where(F[:, 9 * a + 8] > 0.5, O[:, a], 0.0) for a in range(3)])


def blend_weights(region_dims, region_gids, accept, learned, dim) -> np.ndarray:
    """(3, n_r) regional weights: `learned` (3, n_r) at regional nodes whose composite node lies
    only in accepting regions, linear interpolation rem/3 (as FP32) elsewhere, 0 along axes
    where the node sits on a coarse index (local coordinate divisible by 3)."""
    dims = np.asarray(region_dims).reshape(-1, 3)
    sizes = dims.prod(axis=1)
    reg = np.repeat(np.arange(dims.shape[0]), sizes)
    gids = np.asarray(region_gids)
    ok_comp = np.ones(int(gids.max()) + 1, dtype=bool)
    np.logical_and.at(ok_comp, gids, np.asarray(accept, dtype=bool)[reg])
    ok = ok_comp[gids]
    local = np.concatenate([np.arange(s) for s in sizes])
    nx, ny = dims[reg, 0], dims[reg, 1]
    coord = [local % nx, (local // nx) % ny, local // (nx * ny)]
    out = np.zeros((3, gids.size))
    for a in range(3):
        rem = coord[a] % 3 if a < dim else np.zeros_like(local)
        lin = np.where(rem == 1, np.float32(1.0 / 3.0), np.float32(2.0 / 3.0)).astype(np.float64)
        out[a] = np.where(rem == 0, 0.0, np.where(ok, np.asarray(learned)[a], lin))
    return out
