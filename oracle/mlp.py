"""Learned warm start of the cell solves — FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module. The CUDA library never
imports, links or calls it, and this module shares no code with it.

The paper warm-starts every cell solve from the duals of the cell's previous
solve (Algorithm 2, input u_{C,J}; §6.1). This project adds a second
candidate, predicted by a small network from the cell's data, and keeps
whichever gives the smaller X-marginal error after one Y-iteration. This
module defines, for cells of 8×8 pixels (2×2 basic cells of 4×4):

* features (1089 numbers):
    [0, 64)      64·μ(x)/‖μ_J‖ on the cell's pixels, row-major;
    [64, 1088)   1024·ν_cell(y)/‖ν_cell‖ on the 32×32 pixel window whose
                 centre pixel (row 16, column 16 of the window) is the
                 centroid of ν_cell rounded to a pixel; support points
                 outside the window are left out;
    1088         log(ε/Δ²), Δ the pixel spacing of the level;
* the target: the cell's converged dual α in the frame of the ν_cell
  centroid, scaled by 1/ε and shifted to mean zero. Translating ν_cell by t
  changes the optimal α by −2⟨x, t⟩ + const (c(x, y+t) = c(x,y) − 2⟨x−y, t⟩
  + |t|²), so the frame removes that linear term: with the anchor pixel
  a = round(centroid − ((H−1)/2, (W−1)/2)) and D = (r₀ − a_r, c₀ − a_c) for a
  cell whose top-left pixel is (r₀, c₀),
      target(i, j) = [α(r₀+i, c₀+j) − 2Δ²(D_r·i + D_c·j)]/ε − mean;
  a prediction p maps back to α(r₀+i, c₀+j) = ε·p(i,j) + 2Δ²(D_r·i + D_c·j)
  up to a constant;
* the network: 1089 → 256 → 256 → 64, ReLU after the two hidden layers,
  y = W3·relu(W2·relu(W1·x + b1) + b2) + b3, weights used in bfloat16
  (round to nearest even from FP32), biases and all sums in FP64 here;
* the loss: mean over the batch and the 64 outputs of (y − target)².

Rounding of the centroid is to the nearest integer, ties to even.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 1089, 256, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    """Flat parameter vector → dict of arrays (layout of SHAPES, row-major)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(w):
    """FP32 values rounded to bfloat16 (8 significant bits), returned as float64.

    bfloat16 keeps the upper 16 bits of an IEEE binary32; rounding to nearest,
    ties to even, adds 0x7FFF plus the lowest kept bit before truncating."""
    b = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X):
    """Network output for a batch X (N × 1089); returns y and the cache for backward."""
    p = unpack(params)
    W1, W2, W3 = bf16_round(p["W1"]), bf16_round(p["W2"]), bf16_round(p["W3"])
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + p["b3"]
    return y, (X, z1, h1, z2, h2, W1, W2, W3)


def loss(y, T):
    d = y - np.asarray(T, dtype=np.float64)
    return float((d * d).mean())


def backward(params, X, T):
    """Loss and its gradient with respect to the flat parameters.

    The rounding of the weights to bfloat16 is treated as the identity in the
    derivative (the gradient of the loss at the rounded weights)."""
    y, (X, z1, h1, z2, h2, W1, W2, W3) = forward(params, X)
    N = X.shape[0]
    dy = 2.0 * (y - T) / (N * N_OUT)
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(axis=0)
    return loss(y, T), pack(g)


# ----------------------------------------------------------------------------
# features and targets of a cell
# ----------------------------------------------------------------------------
def _cell_rect(prob, J):
    # the cell's pixels in row-major order of its rectangle
    X = np.sort(prob.cell_points(J))
    r, c = np.divmod(X, prob.n)
    return X, int(r.min()), int(c.min()), int(r.max() - r.min() + 1), int(c.max() - c.min() + 1)


def centroid(prob, cols, nu_cell):
    """Mass-weighted mean pixel (row, column) of ν_cell, in pixel indices."""
    r, c = np.divmod(np.asarray(cols), prob.n)
    m = nu_cell.sum()
    return float((nu_cell * r).sum() / m), float((nu_cell * c).sum() / m)


def anchor(prob, J, cols, nu_cell):
    _, r0, c0, H, W = _cell_rect(prob, J)
    cr, cc = centroid(prob, cols, nu_cell)
    return int(np.rint(cr - 0.5 * (H - 1))), int(np.rint(cc - 0.5 * (W - 1)))


def cell_features(prob, J, cols, nu_cell, eps):
    """The 1089 inputs of the network for cell J (8×8 pixels)."""
    X, r0, c0, H, W = _cell_rect(prob, J)
    assert H == 8 and W == 8
    f = np.zeros(N_IN)
    mu = prob.mu[X]
    f[:64] = 64.0 * mu / mu.sum()
    cr, cc = centroid(prob, cols, nu_cell)
    wr, wc = int(np.rint(cr)) - 16, int(np.rint(cc)) - 16
    yr, yc = np.divmod(np.asarray(cols), prob.n)
    hr, hc = yr - wr, yc - wc
    inside = (hr >= 0) & (hr < 32) & (hc >= 0) & (hc < 32)
    hist = np.zeros((32, 32))
    np.add.at(hist, (hr[inside], hc[inside]), nu_cell[inside])
    f[64:1088] = 1024.0 * hist.ravel() / nu_cell.sum()
    f[1088] = np.log(eps / prob.spacing ** 2)
    return f


def cell_target(prob, J, alpha, eps, anc):
    """Target of cell J from its converged α (over all pixels) and anchor."""
    X, r0, c0, H, W = _cell_rect(prob, J)
    i, j = np.divmod(np.arange(H * W), W)
    Dr, Dc = r0 - anc[0], c0 - anc[1]
    d2 = prob.spacing ** 2
    t = (alpha[X] - 2.0 * d2 * (Dr * i + Dc * j)) / eps
    return t - t.mean()


def alpha_from_prediction(prob, J, pred, eps, anc):
    """α on the cell's pixels from a prediction (inverse of cell_target up to a constant)."""
    X, r0, c0, H, W = _cell_rect(prob, J)
    i, j = np.divmod(np.arange(H * W), W)
    d2 = prob.spacing ** 2
    return eps * np.asarray(pred) + 2.0 * d2 * ((r0 - anc[0]) * i + (c0 - anc[1]) * j)


def training_pairs(prob, part, rows_before, alpha_after, eps, cells=None):
    """(features, targets, cell indices) of the 8×8 cells of one half-sweep:
    features from ν_cell gathered from the basic marginals before the solve,
    targets from the duals after it."""
    from . import dd as odd
    F, T, idx = [], [], []
    todo = range(len(prob.parts[part])) if cells is None else cells
    for jn in todo:
        J = prob.parts[part][jn]
        X, r0, c0, H, W = _cell_rect(prob, J)
        if H != 8 or W != 8:
            continue
        cols, nu_cell = odd.gather(rows_before, J)
        F.append(cell_features(prob, J, cols, nu_cell, eps))
        T.append(cell_target(prob, J, alpha_after, eps, anchor(prob, J, cols, nu_cell)))
        idx.append(jn)
    return np.array(F), np.array(T), np.array(idx, dtype=np.int64)
