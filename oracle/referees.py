"""Independent referees for the oracle (test infrastructure only).

These solve the full problem in one piece, with code paths unrelated to the
oracle's cell solver, so that agreement pins the oracle:

* sinkhorn_scaling: the Sinkhorn algorithm of Remark 2.4 in its scaling form
  (u, v, k = exp(−c/ε), reference measure μ⊗ν), FP64, no log-domain tricks;
  usable while exp(−‖c‖/ε) does not underflow.
* lp_optimum: the unregularised Kantorovich problem (eq. OTPrimal) solved as a
  linear programme by scipy's HiGHS solver.
"""
from __future__ import annotations

import numpy as np


def sinkhorn_scaling(mu, nu, C, eps, tol=1e-13, max_iter=200000):
    """Returns (π, u, v) with π = u ⊗ v · k · (μ ⊗ ν), iterated until the
    X-marginal L1 error after a Y-iteration is ≤ tol."""
    mu = np.asarray(mu, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    k = np.exp(-np.asarray(C, dtype=np.float64) / eps)
    u = np.ones(mu.size)
    for _ in range(max_iter):
        v = 1.0 / (k.T @ (u * mu))            # Y-iteration (dν̂/dν = 1)
        u_new = 1.0 / (k @ (v * nu))          # X-iteration
        pi = (u[:, None] * v[None, :]) * k * mu[:, None] * nu[None, :]
        if np.abs(pi.sum(axis=1) - mu).sum() <= tol:
            return pi, u, v
        u = u_new
    raise RuntimeError("sinkhorn_scaling did not converge")


def lp_optimum(mu, nu, C):
    """min ⟨c, π⟩ over π ≥ 0 with marginals μ, ν. Returns (cost, π)."""
    from scipy.optimize import linprog
    from scipy.sparse import kron, identity, vstack, csr_matrix

    mu = np.asarray(mu, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    nx, ny = mu.size, nu.size
    ones_y = csr_matrix(np.ones((1, ny)))
    ones_x = csr_matrix(np.ones((1, nx)))
    A = vstack([kron(identity(nx), ones_y), kron(ones_x, identity(ny))]).tocsr()
    b = np.concatenate([mu, nu])
    res = linprog(np.asarray(C, dtype=np.float64).ravel(), A_eq=A, b_eq=b,
                  bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun), res.x.reshape(nx, ny)


def odd_even_transposition_sort_steps(perm, n_steps):
    """Textbook odd-even transposition sort: returns the list of arrays after
    each phase. Phase 1 compares pairs (0,1), (2,3), …; phase 2 compares
    (1,2), (3,4), …, alternating."""
    a = list(perm)
    out = []
    for step in range(n_steps):
        start = 0 if step % 2 == 0 else 1
        for k in range(start, len(a) - 1, 2):
            if a[k] > a[k + 1]:
                a[k], a[k + 1] = a[k + 1], a[k]
        out.append(np.array(a))
    return out
