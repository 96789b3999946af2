"""FP64 CPU oracle of entropic domain decomposition for optimal transport.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module. The CUDA library never
imports, links or calls it, and this module shares no code with it.

It follows Bonafini & Schmitzer, "Domain decomposition for entropy regularized
optimal transport":

* the problem: minimise ε·KL(π|K) over couplings π of μ and ν, with
  K = exp(−c/ε)·(μ⊗ν) (§2.2, eq. EntropicOTPrimal; §3 eq. Problem);
* Algorithm 2 (practical domain decomposition, §6.1): for every composite cell J
  of the current partition, ν_cell = Σ_{i∈J} ν_i, a Sinkhorn solve on
  (μ_J, ν_cell) warm-started from u_{C,J}, extraction of the new basic
  Y-marginals ν_i = P_Y(π_cell restricted to X_i × Y), BalanceMeasures and
  Truncate;
* the Sinkhorn solver and its stopping rule (§6.2): start with a Y-iteration,
  stop once, right after a Y-iteration, Σ_x |P_X π − μ| is at most
  ‖μ_J‖·Err, so the last step is always a Y-iteration;
* the multi-scale scheme (§6.4): coarse images are push-forwards under the
  quad-tree parent map, fine basic marginals are initialised by eq.
  FineBasicMarginals, and ε·log u is kept fixed when ε changes;
* basic/composite partitions for images (§7.1): s×s basic cells, partition A
  of 2×2 blocks, partition B the same blocks shifted by one basic cell;
* objective values (Lemma 4.2, Prop. 2.5, §6.3): KL(π|K) − ‖K‖ of a
  partition's coupling summed cell by cell, and the primal-dual gaps of the
  cell problems.

Potentials are kept in the counting-measure form f = α + ε·log μ,
g = β + ε·log ν with π(x,y) = exp((f(x) + g(y) − c(x,y))/ε); α = ε·log u and
β = ε·log v are the paper's scalings in log form. With fixed marginals the
minimiser does not depend on this choice of reference measure.

Readings of points the paper leaves open (each is listed with its reason in
the design notes of the repository):

* BalanceMeasures (§6.2): surplus cells (‖ν_i‖ > ‖μ_i‖) give up the fraction
  d_i/‖ν_i‖ of every entry; the removed mass is shared among deficit cells in
  proportion to their deficits. This keeps non-negativity, the sum Σ_i ν_i and
  the support, as the paper requires.
* Truncate (§6.1 item (ii), §7.1): entries of ν_i not above the absolute
  threshold (1e-15) are dropped.
* Sinkhorn stopping test (§6.2) after truncation: the X-marginal is compared
  with μ_J rescaled to ‖ν_cell‖ (see sinkhorn_cell), because truncated mass
  makes ‖ν_cell‖ < ‖μ_J‖ and the unscaled error can then never reach
  ‖μ_J‖·Err for small Err.
* Dual refinement (§6.4 ends with "glue, then interpolate linearly in log
  space"): without gluing, each fine pixel takes the coarse α of its parent
  pixel plus a first-order correction from finite differences of α inside the
  parent's composite cell (central differences inside, one-sided at the cell
  edge). Both partitions at the new level start from this α (Algorithm 2,
  input u).
* Composite cells that consist of one basic cell (corners of partition B) are
  solved like the others; Example 3.3 shows it is redundant for the basic
  marginals, and solving keeps the duals of partition B complete.
* The local safeguard of §7.3 ("temporarily increasing ε"; off unless
  Params.safeguard): a cell whose solve stops at max_iter with an X-error
  above 10·Err·‖μ_J‖ is solved again at 4ε, then at ε (4ε once more if ε
  fails), else at 16ε … 4⁶ε, keeping the first solve that converges
  (safeguard_solve).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------
@dataclass
class Params:
    err: float = 1e-6          # Sinkhorn stopping threshold Err (§6.2)
    max_iter: int = 10000      # cap on Sinkhorn iterations per cell solve
    trunc: float = 1e-15       # Truncate threshold on ν_i entries (§7.1)
    balance: bool = True       # run BalanceMeasures (§6.2)
    safeguard: bool = False    # the local safeguard of §7.3 (see safeguard_solve)
    main_max_iter: int = 0     # > 0: cap of the first solve of each cell only (the
                               # safeguard's re-solves keep max_iter): a forced failure


# ----------------------------------------------------------------------------
# a generic discrete problem with a basic partition (§3, Def. 3.1)
# ----------------------------------------------------------------------------
class Problem:
    """μ on X, ν on Y, a cost function and a basic partition of X.

    basic: list of integer arrays, basic[i] = indices of the points of X_i.
    parts: dict name -> list of composite cells, each a list of basic indices.
    cost(X, Y): matrix c(x, y) for index arrays X (rows) and Y (columns).
    """

    def __init__(self, mu, nu, cost, basic, parts):
        self.mu = np.asarray(mu, dtype=np.float64).ravel()
        self.nu = np.asarray(nu, dtype=np.float64).ravel()
        self.cost = cost
        self.basic = [np.asarray(b, dtype=np.int64) for b in basic]
        self.parts = parts
        self.basic_mass = np.array([self.mu[b].sum() for b in self.basic])
        if np.any(self.basic_mass <= 0):
            raise ValueError("every basic cell needs positive mass (Def. 3.1)")

    def cell_points(self, J):
        return np.concatenate([self.basic[i] for i in J])


def matrix_problem(mu, nu, C, basic, parts):
    """Problem with an explicit cost matrix C[x, y]."""
    C = np.asarray(C, dtype=np.float64)
    return Problem(mu, nu, lambda X, Y: C[np.ix_(X, Y)], basic, parts)


# ----------------------------------------------------------------------------
# images: pixels, basic cells, partitions A and B (§7.1)
# ----------------------------------------------------------------------------
def grid_basic_cells(n, b):
    """b×b pixel blocks in row-major order of blocks; pixels row-major inside."""
    nb = n // b
    cells = []
    for r in range(nb):
        for s in range(nb):
            ii = np.arange(r * b, (r + 1) * b)
            jj = np.arange(s * b, (s + 1) * b)
            cells.append((ii[:, None] * n + jj[None, :]).ravel())
    return cells


def grid_partitions(nb):
    """Partition A: 2×2 blocks of basic cells. Partition B: the same blocks
    shifted by one basic cell, so it has single cells at the corners and 2×1
    blocks along the edges (§7.1 "Basic and composite partitions")."""
    A, B = [], []
    for a in range(nb // 2):
        for c in range(nb // 2):
            A.append([r * nb + s for r in (2 * a, 2 * a + 1) for s in (2 * c, 2 * c + 1)])
    for a in range(nb // 2 + 1):
        for c in range(nb // 2 + 1):
            rr = [r for r in (2 * a - 1, 2 * a) if 0 <= r < nb]
            cc = [s for s in (2 * c - 1, 2 * c) if 0 <= s < nb]
            B.append([r * nb + s for r in rr for s in cc])
    return {"A": A, "B": B}


class GridProblem(Problem):
    """Two n×n images on [0,1]² (pixel spacing `spacing`), cost |x−y|²."""

    def __init__(self, mu_img, nu_img, b, spacing):
        n = mu_img.shape[0]
        self.n, self.b, self.spacing = n, b, spacing
        self.nb = n // b
        if n % b or self.nb % 2:
            raise ValueError("n/b must be an even integer")
        d2 = spacing * spacing

        def cost(X, Y):
            xi, xj = np.divmod(X, n)
            yi, yj = np.divmod(Y, n)
            return d2 * ((xi[:, None] - yi[None, :]) ** 2 + (xj[:, None] - yj[None, :]) ** 2).astype(np.float64)

        super().__init__(mu_img, nu_img, cost, grid_basic_cells(n, b), grid_partitions(self.nb))


def pyramid(img, levels):
    """[coarsest, …, finest]: each coarse pixel holds the mass of its four
    children (push-forward under the quad-tree parent map, §6.4, §7.1)."""
    out = [np.asarray(img, dtype=np.float64)]
    for _ in range(levels - 1):
        a = out[0]
        m = a.shape[0] // 2
        out.insert(0, a.reshape(m, 2, m, 2).sum(axis=(1, 3)))
    return out


# ----------------------------------------------------------------------------
# the cell solver (§6.2) in log form
# ----------------------------------------------------------------------------
def logsumexp(a, axis):
    m = a.max(axis=axis, keepdims=True)
    return (m + np.log(np.exp(a - m).sum(axis=axis, keepdims=True))).squeeze(axis)


def sinkhorn_cell(C, mu_x, nu_y, f, eps, err, max_iter):
    """Sinkhorn on one composite cell, warm-started from f (Remark 2.4, §6.2).

    Y-iteration: g(y) = ε·log ν(y) − ε·log Σ_x exp((f(x) − c(x,y))/ε)
    X-iteration: f(x) = ε·log μ(x) − ε·log Σ_y exp((g(y) − c(x,y))/ε)
    After each Y-iteration the X-marginal error is compared with ‖μ_J‖·Err;
    the solver stops on a Y-iteration. Truncate removes a little mass from the
    basic marginals, so ‖ν_cell‖ can fall short of ‖μ_J‖ and no plan on the
    cell then matches μ_J exactly; the stopping test therefore measures the
    X-marginal against μ rescaled to the mass of ν_cell (the paper's rule
    whenever no mass was truncated):
        Σ_x |P_X π(x) − μ(x)·‖ν_cell‖/‖μ_J‖| ≤ ‖μ_J‖·Err.
    Returns f, g, the plan P (|X|×|Y|), the number of Y-iterations and the
    final X-marginal error Σ_x |P_X π(x) − μ(x)| (not rescaled).
    """
    logmu, lognu = np.log(mu_x), np.log(nu_y)
    tol = err * mu_x.sum()
    target = mu_x * (nu_y.sum() / mu_x.sum())
    it = 0
    while True:
        it += 1
        g = eps * lognu - eps * logsumexp((f[:, None] - C) / eps, axis=0)
        P = np.exp((f[:, None] + g[None, :] - C) / eps)
        px = P.sum(axis=1)
        if np.abs(px - target).sum() <= tol or it >= max_iter:
            return f, g, P, it, np.abs(px - mu_x).sum()
        f = eps * logmu - eps * logsumexp((g[None, :] - C) / eps, axis=1)


# ----------------------------------------------------------------------------
# Algorithm 2 building blocks
# ----------------------------------------------------------------------------
def gather(rows, J):
    """ν_cell = Σ_{i∈J} ν_i on the union of the supports (Algorithm 2)."""
    cols = np.unique(np.concatenate([rows[i][0] for i in J]))
    nu_cell = np.zeros(cols.size)
    for i in J:
        nu_cell[np.searchsorted(cols, rows[i][0])] += rows[i][1]
    return cols, nu_cell


def balance_measures(parts, targets):
    """BalanceMeasures (§6.2), proportional reading (see module docstring).

    parts: list of arrays ν_i on a common support; targets: ‖μ_i‖.
    Modifies parts in place; returns them.
    """
    m = np.array([p.sum() for p in parts])
    d = m - np.asarray(targets)
    sur = [k for k in range(len(parts)) if d[k] > 0]
    dfc = [k for k in range(len(parts)) if d[k] < 0]
    if not sur or not dfc:
        return parts
    delta = np.zeros_like(parts[0])
    for k in sur:
        take = parts[k] * (d[k] / m[k])
        parts[k] = parts[k] - take
        delta += take
    dtot = -d[dfc].sum()
    for k in dfc:
        parts[k] = parts[k] + delta * (-d[k] / dtot)
    return parts


@dataclass
class SweepInfo:
    cost: float = 0.0                  # Σ_J ⟨c, π_J⟩
    err_x: float = 0.0                 # Σ_J Σ_x |P_X π_J(x) − μ(x)|
    iters: list = field(default_factory=list)
    truncated_mass: float = 0.0
    converged: list = field(default_factory=list)   # per cell: the kept solve met its stopping test
    eps_used: list = field(default_factory=list)    # per cell: ε of the kept solve
    rescued: int = 0                   # cells the safeguard solved again
    escalated: int = 0                 # of these, cells kept at a larger ε


SAFEGUARD_FACTOR = 4.0   # ε factor of each safeguard attempt
SAFEGUARD_STEPS = 6      # attempts up to SAFEGUARD_FACTOR**6·ε


def solve_converged(P, mu_x, nu_y, err):
    """The stopping test of sinkhorn_cell for a plan P: Σ_x |P_X π − μ·‖ν‖/‖μ‖|
    ≤ ‖μ‖·Err."""
    target = mu_x * (nu_y.sum() / mu_x.sum())
    return bool(np.abs(P.sum(axis=1) - target).sum() <= err * mu_x.sum())


def safeguard_solve(C, mu_x, nu_y, alpha_x, eps, err, max_iter):
    """The local safeguard of §7.3 ("fixed locally, e.g. by temporarily
    increasing ε") for a cell whose solve at ε stopped at max_iter with an
    X-error above 10·Err·‖μ_J‖. The paper fixes neither the factor nor the
    order; read here as: solve at 4ε from the duals α the failed solve ended
    with; if that converges, solve at ε from its result, and if that fails,
    at 4ε once more; if 4ε fails, at 16ε, 64ε, … up to 4⁶ε (max_iter/4
    iterations each, at least 64), keeping the first solve that converges. ε·log u = α carries over from one ε to the next (as at a
    change of ε in §6.4). Returns f, g, P, total iterations, the unscaled
    X-error, the ε of the kept solve and whether it converged."""
    logmu = np.log(mu_x)
    short = max(max_iter // 4, 64)
    total = 0

    def attempt(alpha, e, cap):
        nonlocal total
        f, g, P, it, ex = sinkhorn_cell(C, mu_x, nu_y, alpha + e * logmu, e, err, cap)
        total += it
        return f, g, P, ex, f - e * logmu, solve_converged(P, mu_x, nu_y, err)

    e4 = SAFEGUARD_FACTOR * eps
    f, g, P, ex, a4, ok = attempt(alpha_x, e4, max_iter)
    if ok:
        f1, g1, P1, ex1, a1, ok1 = attempt(a4, eps, max_iter)
        if ok1:
            return f1, g1, P1, total, ex1, eps, True
        f, g, P, ex, _, ok = attempt(a1, e4, max_iter)
        return f, g, P, total, ex, e4, ok
    e, a = e4, a4
    for _ in range(2, SAFEGUARD_STEPS + 1):
        e *= SAFEGUARD_FACTOR
        f, g, P, ex, a, ok = attempt(a, e, short)
        if ok:
            break
    return f, g, P, total, ex, e, ok


def half_sweep(prob, part, rows, alpha, eps, params, plans=None, cells=None):
    """One iteration of Algorithm 2 over the composite partition `part`.

    rows: list over basic cells of (cols sorted int array, vals float array).
    alpha: array over X holding α = ε·log u_{C,J} for this partition; updated
    in place. Returns the new rows and a SweepInfo. If `plans` is a dict, the
    cell plans are stored there as plans[J index] = (X, cols, P). `cells`
    restricts the loop to the listed composite cells (the cells of one
    partition are independent, so a subset is solved exactly as in the full
    loop); rows of other basic cells are returned unchanged.
    """
    new_rows = list(rows)
    info = SweepInfo()
    todo = range(len(prob.parts[part])) if cells is None else cells
    for jn in todo:
        J = prob.parts[part][jn]
        cols, nu_cell = gather(rows, J)
        X = prob.cell_points(J)
        mu_x = prob.mu[X]
        # the cell problem lives on the support of μ_J (§2: couplings of μ and
        # ν); a pixel without mass carries no plan and keeps α = 0
        live = mu_x > 0
        C = prob.cost(X[live], cols)
        f0 = alpha[X[live]] + eps * np.log(mu_x[live])
        cap = params.main_max_iter if params.main_max_iter > 0 else params.max_iter
        f, g, P_live, it, err_x = sinkhorn_cell(C, mu_x[live], nu_cell, f0, eps, params.err, cap)
        ok = solve_converged(P_live, mu_x[live], nu_cell, params.err)
        e_used = eps
        if params.safeguard and not ok and err_x > 10.0 * params.err * mu_x[live].sum():
            a_fail = f - eps * np.log(mu_x[live])
            f, g, P_live, it2, err_x, e_used, ok = safeguard_solve(C, mu_x[live], nu_cell, a_fail, eps,
                                                                   params.err, params.max_iter)
            it += it2
            info.rescued += 1
            info.escalated += int(ok and e_used != eps)
        alpha[X[live]] = f - e_used * np.log(mu_x[live])
        alpha[X[~live]] = 0.0
        info.converged.append(ok)
        info.eps_used.append(e_used)
        P = np.zeros((X.size, cols.size))
        P[live] = P_live
        info.cost += float((C * P_live).sum())
        info.err_x += float(err_x)
        info.iters.append(it)
        if plans is not None:
            plans[jn] = (X, cols, P)
        # extraction of the new basic marginals
        parts, o = [], 0
        for i in J:
            k = prob.basic[i].size
            parts.append(P[o:o + k].sum(axis=0))
            o += k
        if params.balance:
            balance_measures(parts, [prob.basic_mass[i] for i in J])
        for i, v in zip(J, parts):
            keep = v > params.trunc
            info.truncated_mass += float(v[~keep].sum())
            new_rows[i] = (cols[keep], v[keep])
    return new_rows, info


def product_state(prob):
    """ν_i = ‖μ_i‖·ν on all of Y: the product coupling μ⊗ν (§6.4)."""
    cols = np.arange(prob.nu.size)
    return [(cols.copy(), m * prob.nu) for m in prob.basic_mass]


def rows_from_csr(row_ptr, col, val):
    return [(np.asarray(col[row_ptr[k]:row_ptr[k + 1]], dtype=np.int64),
             np.asarray(val[row_ptr[k]:row_ptr[k + 1]], dtype=np.float64))
            for k in range(len(row_ptr) - 1)]


def rows_to_dense(rows, ny):
    D = np.zeros((len(rows), ny))
    for k, (c, v) in enumerate(rows):
        D[k, c] = v
    return D


def y_marginal_error(prob, rows):
    """Σ_y |Σ_i ν_i(y) − ν(y)| (the Y-marginal error in L1)."""
    s = np.zeros(prob.nu.size)
    for c, v in rows:
        np.add.at(s, c, v)
    return float(np.abs(s - prob.nu).sum())


# ----------------------------------------------------------------------------
# the coupling behind a state, objective values (Lemma 4.2, Prop. 2.5)
# ----------------------------------------------------------------------------
def partition_plan(prob, part, rows, alpha, eps):
    """π = Σ_J π_J for the partition solved last: on each cell, f from
    α_{C,J} and one Y-iteration against ν_cell (so P_Y π = ν exactly).
    Returns a dense |X|×|Y| array (small problems only)."""
    P = np.zeros((prob.mu.size, prob.nu.size))
    for J in prob.parts[part]:
        cols, nu_cell = gather(rows, J)
        X = prob.cell_points(J)
        C = prob.cost(X, cols)
        f = alpha[X] + eps * np.log(prob.mu[X])
        g = eps * np.log(nu_cell) - eps * logsumexp((f[:, None] - C) / eps, axis=0)
        P[np.ix_(X, cols)] = np.exp((f[:, None] + g[None, :] - C) / eps)
    return P


def cell_objectives(prob, part, rows, alpha, eps):
    """Objective values of the coupling of partition_plan, cell by cell (§6.3:
    the primal score is summed over the composite cells of the last loop).

    On a cell J, f = α + ε·log μ on the pixels with mass and one Y-iteration
    against ν_cell give π_J = u_J ⊗ v_J · K on X_J × supp ν_cell with
    log u_J = α/ε and log v_J = β_J/ε, β_J = g − ε·log ν. Per cell:

    * primal_J = Σ π_J·(log π_J − log K − 1), the cell's share of
      KL(π|K) − ‖K‖ (the denominator of eq. RelPDGap);
    * gap_J = KL(π_J|K_J) − J_J(u_J, v_J), the primal-dual gap of the cell
      problem: marginals μ_J and ν_cell, kernel K_J = K restricted to
      X_J × supp ν_cell, J_J the dual objective of eq. EntropicOTDualObjective
      on that problem (Prop. 2.5). π_J meets ν_cell exactly and μ_J only up to
      the Sinkhorn tolerance, so gap_J has no fixed sign; it is zero at the
      cell's optimum.

    Returns (primal, gap): FP64 arrays in the order of prob.parts[part].
    """
    primal, gap = [], []
    for J in prob.parts[part]:
        cols, nu_cell = gather(rows, J)
        X = prob.cell_points(J)
        X = X[prob.mu[X] > 0]
        C = prob.cost(X, cols)
        mu_x, nu_y = prob.mu[X], prob.nu[cols]
        a = alpha[X]
        f = a + eps * np.log(mu_x)
        g = eps * np.log(nu_cell) - eps * logsumexp((f[:, None] - C) / eps, axis=0)
        P = np.exp((f[:, None] + g[None, :] - C) / eps)
        beta = g - eps * np.log(nu_y)
        pj = kl_minus_mass(P, C, mu_x, nu_y, eps)
        kl = pj + kernel_mass(C, mu_x, nu_y, eps)
        primal.append(pj)
        gap.append(kl - dual_objective(a, beta, mu_x, nu_cell, C, mu_x, nu_y, eps))
    return np.array(primal), np.array(gap)


def kl_minus_mass(P, C, mu, nu, eps):
    """KL(π|K) − ‖K‖ = Σ_{π>0} π·(log π − log K − 1), K = e^{−c/ε}·μ⊗ν
    (Definition 2.1 with φ(s) = s log s − s + 1; ‖K‖ is the constant that the
    paper subtracts in eq. RelPDGap)."""
    m = P > 0
    logK = -C / eps + np.log(mu)[:, None] + np.log(nu)[None, :]
    return float((P[m] * (np.log(P[m]) - logK[m] - 1.0)).sum())


def kernel_mass(C, mu, nu, eps):
    """‖K‖ = Σ_{x,y} e^{−c(x,y)/ε} μ(x) ν(y)."""
    return float((np.exp(-C / eps) * mu[:, None] * nu[None, :]).sum())


def kl_div(P, Q):
    """KL(P|Q) for non-negative arrays with supp P ⊂ supp Q (Definition 2.1)."""
    m = P > 0
    return float((P[m] * np.log(P[m] / Q[m])).sum() - P.sum() + Q.sum())


def dual_objective(alpha, beta, mu_hat, nu_hat, C, mu, nu, eps):
    """J(u,v) of eq. EntropicOTDualObjective with log u = α/ε, log v = β/ε:
    ⟨μ̂, log u⟩ + ⟨ν̂, log v⟩ − Σ u⊗v·K + ‖K‖."""
    K = np.exp(-C / eps) * mu[:, None] * nu[None, :]
    uv = np.exp((alpha[:, None] + beta[None, :]) / eps)
    return float(mu_hat @ (alpha / eps) + nu_hat @ (beta / eps) - (uv * K).sum() + K.sum())


# ----------------------------------------------------------------------------
# multi-scale: refinement of the basic marginals and of the duals (§6.4)
# ----------------------------------------------------------------------------
def refine_basic_marginals(coarse, fine, rows_c):
    """Eq. FineBasicMarginals: ν_i⁰(y) = ν(y)·ν̂_{Pa(i)}(pa(y))/ν̂(pa(y))·μ(X_i)/μ̂(X̂_{Pa(i)}).

    coarse, fine: GridProblem at two consecutive levels with the same b, so a
    coarse basic cell (r, s) is the parent of fine cells (2r+{0,1}, 2s+{0,1})
    and a coarse pixel (p, q) the parent of fine pixels (2p+{0,1}, 2q+{0,1}).
    """
    nc, nf = coarse.n, fine.n
    nbc, nbf = coarse.nb, fine.nb
    rows_f = [None] * (nbf * nbf)
    for R in range(nbf):
        for S in range(nbf):
            i = R * nbf + S
            j = (R // 2) * nbc + (S // 2)
            cc, vc = rows_c[j]
            pi, pj = np.divmod(cc, nc)
            ys, ws = [], []
            for di in (0, 1):
                for dj in (0, 1):
                    y = (2 * pi + di) * nf + (2 * pj + dj)
                    ys.append(y)
                    ws.append(fine.nu[y] * vc / coarse.nu[cc] * fine.basic_mass[i] / coarse.basic_mass[j])
            y = np.concatenate(ys)
            w = np.concatenate(ws)
            o = np.argsort(y, kind="stable")
            rows_f[i] = (y[o], w[o])
    return rows_f


def _fd(a, axis):
    """Finite differences along one axis: central inside, one-sided at the
    edges, zero when the extent is 1."""
    k = a.shape[axis]
    if k == 1:
        return np.zeros_like(a)
    d = np.empty_like(a)
    a_ = np.moveaxis(a, axis, 0)
    d_ = np.moveaxis(d, axis, 0)
    d_[0] = a_[1] - a_[0]
    d_[-1] = a_[-1] - a_[-2]
    if k > 2:
        d_[1:-1] = 0.5 * (a_[2:] - a_[:-2])
    return d


def refine_duals(coarse, fine, alpha_c, part):
    """Dual initialisation at the next level (reading of §6.4, see module
    docstring): per composite cell of `part` at the coarse level, the fine
    children of a coarse pixel p get α(p) ± ¼·∂α(p) along each axis."""
    nc, nf, b = coarse.n, fine.n, coarse.b
    alpha_f = np.empty(nf * nf)
    A2 = alpha_c.reshape(nc, nc)
    for J in coarse.parts[part]:
        rs = sorted({i // coarse.nb for i in J})
        ss = sorted({i % coarse.nb for i in J})
        r0, r1 = rs[0] * b, (rs[-1] + 1) * b
        s0, s1 = ss[0] * b, (ss[-1] + 1) * b
        blk = A2[r0:r1, s0:s1]
        dr, ds = _fd(blk, 0), _fd(blk, 1)
        for di, orr in ((0, -0.25), (1, 0.25)):
            for dj, oss in ((0, -0.25), (1, 0.25)):
                val = blk + orr * dr + oss * ds
                R = 2 * np.arange(r0, r1) + di
                S = 2 * np.arange(s0, s1) + dj
                alpha_f[(R[:, None] * nf + S[None, :]).ravel()] = val.ravel()
    return alpha_f


# ----------------------------------------------------------------------------
# dual gluing (§6.3, "Estimating the primal-dual gap") and eq. RelPDGap
# ----------------------------------------------------------------------------
def gluing_graph(prob):
    """Edges of the gluing graph of §6.3: the vertices are the cells of
    partition A; for every cell J_B of B and every ordered pair (J1, J2) of
    distinct A cells that both meet J_B there is one edge (J1, J2) labelled
    J_B (an edge per orientation, and several edges between two vertices when
    several B cells connect them). Returns [(j1, j2, jb, X1, X2)] with j1, j2
    indices into prob.parts["A"], jb into prob.parts["B"], X1 = the pixels of
    J1 ∩ J_B and X2 those of J2 ∩ J_B."""
    A, B = prob.parts["A"], prob.parts["B"]
    a_of = {i: j for j, J in enumerate(A) for i in J}
    edges = []
    for jb, JB in enumerate(B):
        meet = {}
        for i in JB:
            meet.setdefault(a_of[i], []).append(i)
        for j1 in sorted(meet):
            for j2 in sorted(meet):
                if j1 != j2:
                    X1 = np.concatenate([prob.basic[i] for i in meet[j1]])
                    X2 = np.concatenate([prob.basic[i] for i in meet[j2]])
                    edges.append((j1, j2, jb, X1, X2))
    return edges


def _log_mu_mean_exp(mu, t):
    """log of the μ-weighted mean of exp(t) (the ⨍ … dμ of §6.3), stably."""
    live = mu > 0
    return float(logsumexp(t[live] + np.log(mu[live]), axis=0) - np.log(mu[live].sum()))


def helmholtz_potential(n_nodes, j1, j2, logq):
    """The least-squares step of §6.3 (discrete Helmholtz decomposition of the
    edge values): V minimising Σ_e ((V(j1_e) − V(j2_e)) + logq_e)² with
    Σ V = 0 (sign reading: see glue_duals), as a dense least-squares problem
    with the gauge as one more row (the edge residuals do not see it)."""
    D = np.zeros((len(j1) + 1, n_nodes))
    rhs = np.zeros(len(j1) + 1)
    for e in range(len(j1)):
        D[e, j1[e]] += 1.0
        D[e, j2[e]] -= 1.0
        rhs[e] = -logq[e]
    D[-1, :] = 1.0
    return np.linalg.lstsq(D, rhs, rcond=None)[0]


def glue_duals(prob, alpha_A, alpha_B, eps):
    """Glued X-dual of §6.3 from the composite duals of both partitions.

    Edge weights, with u = exp(α/ε):
        q(J1,J2) = ⨍_{J1∩J_B} u_{A,J1}/u_{B,J_B} dμ · ⨍_{J2∩J_B} u_{B,J_B}/u_{A,J2} dμ.
    A potential V on the A cells solves the least-squares problem
        min Σ_edges ((V(J1) − V(J2)) + log q(J1,J2))²,   Σ_J V(J) = 0,
    and û_J = exp(V(J))·u_{A,J}. The sign in front of log q is the reading
    under which this agrees with the path-product construction of the same
    section (û_J = Π_k q(J_k, J_{k+1})·u_{A,J} along a path J_0 … J_n = J):
    for consistent duals u_{A,J} = λ_J u*, u_{B,J} = κ_J u*, log q(J1,J2) =
    log λ_{J1} − log λ_{J2} and both give û ∝ u*.
    Returns (alpha_hat, V) with alpha_hat = ε·log û on every pixel (α_A + ε·V
    on each A cell; 0 on pixels without mass, like α)."""
    A = prob.parts["A"]
    edges = gluing_graph(prob)
    mu = prob.mu
    j1 = np.array([e[0] for e in edges], dtype=np.int64)
    j2 = np.array([e[1] for e in edges], dtype=np.int64)
    logq = np.array([_log_mu_mean_exp(mu[X1], (alpha_A[X1] - alpha_B[X1]) / eps) +
                     _log_mu_mean_exp(mu[X2], (alpha_B[X2] - alpha_A[X2]) / eps)
                     for _, _, _, X1, X2 in edges])
    V = helmholtz_potential(len(A), j1, j2, logq)
    alpha_hat = np.asarray(alpha_A, dtype=np.float64).copy()
    for j, J in enumerate(A):
        X = prob.cell_points(J)
        alpha_hat[X] += eps * V[j]
    alpha_hat[mu == 0] = 0.0
    return alpha_hat, V


def best_y_dual(prob, alpha_hat, eps):
    """β̂ = ε·log v̂ for the Y-scaling that maximises J(û, ·) (one Y-iteration
    on the whole problem, Remark 2.4): v̂(y) = 1 / Σ_x û(x) e^{−c(x,y)/ε} μ(x).
    The paper glues the cells' v_J like û; this v̂ is at least as good a dual
    candidate for the given û. Dense (small problems)."""
    live = prob.mu > 0
    X = np.flatnonzero(live)
    C = prob.cost(X, np.arange(prob.nu.size))
    t = (alpha_hat[X][:, None] - C) / eps + np.log(prob.mu[X])[:, None]
    return -eps * logsumexp(t, axis=0)


def relative_pd_gap(prob, P, alpha_hat, beta_hat, eps):
    """eq. RelPDGap: (KL(π|K) − J(û,v̂)) / (KL(π|K) − ‖K‖) for a coupling P
    (dense |X|×|Y|) and duals log û = α̂/ε, log v̂ = β̂/ε (J of eq.
    EntropicOTDualObjective; ‖K‖ cancels in the numerator). Returns
    (relative gap, gap, primal score KL(π|K) − ‖K‖)."""
    live = prob.mu > 0
    X = np.flatnonzero(live)
    Y = np.arange(prob.nu.size)
    C = prob.cost(X, Y)
    primal = kl_minus_mass(P[X], C, prob.mu[X], prob.nu, eps)
    uvK = np.exp((alpha_hat[X][:, None] + beta_hat[None, :] - C) / eps) * prob.mu[X][:, None] * prob.nu[None, :]
    dual_minus_K = prob.mu[X] @ (alpha_hat[X] / eps) + prob.nu @ (beta_hat / eps) - uvK.sum()
    gap = primal - dual_minus_K
    return gap / primal, gap, primal


def fill_massless_affine(prob, alpha):
    """A copy of α in which every pixel without mass takes the value of the
    least-squares affine fit a + s_r·i + s_c·j of α over the pixels with mass
    of its A cell (i, j: pixel row and column). A pixel without mass has no
    dual (the problem lives on the support of μ, §2); §6.4 interpolates the
    glued dual between pixel centres, and this gives those pixels values that
    continue the cell's dual instead of an arbitrary constant. Each basic
    cell has positive mass (Def. 3.1), so an A cell has pixels with mass in
    all four of its basic cells, which no straight line meets, and the fit is
    unique."""
    out = np.asarray(alpha, dtype=np.float64).copy()
    for J in prob.parts["A"]:
        X = prob.cell_points(J)
        live = prob.mu[X] > 0
        if live.all():
            continue
        i, j = np.divmod(X, prob.n)
        D = np.stack([np.ones(X.size), i, j], axis=1).astype(np.float64)
        coef = np.linalg.lstsq(D[live], out[X[live]], rcond=None)[0]
        out[X[~live]] = D[~live] @ coef
    return out


def refine_duals_glued(coarse, fine, alpha_hat_c):
    """Dual initialisation at the next level as §6.4 describes it: the glued
    coarse X-dual, interpolated linearly in log space (on α̂ = ε·log û)
    onto the fine pixel centres. Coarse centres sit at coarse indices k;
    fine pixel I of a level twice as fine sits at t = I/2 − 1/4 in coarse
    index units, so every fine pixel lies between two coarse centres at
    fractions 1/4 and 3/4 per axis (bilinear weights); the outermost fine
    pixels lie a quarter step outside the outermost centres and take the
    linear extrapolation of the last two. Affine α̂ is reproduced exactly.
    The same α is used for both partitions."""
    nc, nf = coarse.n, fine.n
    A2 = np.asarray(alpha_hat_c, dtype=np.float64).reshape(nc, nc)

    def weights(I):
        t = I / 2.0 - 0.25
        k0 = np.clip(np.floor(t).astype(np.int64), 0, nc - 2)
        return k0, t - k0

    I = np.arange(nf)
    k0, w = weights(I)
    rows = A2[k0, :] * (1.0 - w)[:, None] + A2[k0 + 1, :] * w[:, None]        # nf × nc
    full = rows[:, k0] * (1.0 - w)[None, :] + rows[:, k0 + 1] * w[None, :]    # nf × nf
    return full.ravel()


# ----------------------------------------------------------------------------
# the full coarse-to-fine run
# ----------------------------------------------------------------------------
@dataclass
class RunResult:
    prob: GridProblem
    rows: list
    alpha: dict
    eps: float
    last_part: str
    history: list


def run_schedule(mu_img, nu_img, b, levels, schedule, params, *, on_half_sweep=None,
                 before_half_sweep=None, dual_refinement="cell"):
    """Algorithm 2 inside the multi-scale / ε-scaling driver (§6.4).

    schedule: list of (eps, sweeps, level); level 0 is the coarsest image,
    levels-1 the input resolution. One sweep = a half-sweep on A then on B.
    The run starts at level 0 from the product coupling with α = 0.
    before_half_sweep(prob, part, rows, alpha, eps) and on_half_sweep(prob,
    part, rows, alpha, eps, info) are called around every half-sweep (rows and
    α before, respectively after it).
    dual_refinement: "cell" refines the last partition's α cell by cell
    (refine_duals); "glued" glues α_A and α_B (glue_duals) and interpolates
    the glued dual (refine_duals_glued), as §6.4 describes; "hybrid" starts
    the A cells from the cell-wise refinement and the B cells from the glued
    one (both are feasible starts; only the iteration counts differ).
    """
    mus, nus = pyramid(mu_img, levels), pyramid(nu_img, levels)
    n = mu_img.shape[0]
    lev = 0

    def level_problem(l):
        return GridProblem(mus[l], nus[l], b, 2.0 ** (levels - 1 - l) / n)

    prob = level_problem(0)
    rows = product_state(prob)
    alpha = {"A": np.zeros(prob.mu.size), "B": np.zeros(prob.mu.size)}
    history, eps, last = [], None, "B"
    for eps_s, sweeps, L in schedule:
        while lev < L:
            fine = level_problem(lev + 1)
            rows = refine_basic_marginals(prob, fine, rows)
            if dual_refinement in ("glued", "hybrid") and eps is not None:
                a_hat, _ = glue_duals(prob, alpha["A"], alpha["B"], eps)
                a0 = refine_duals_glued(prob, fine, fill_massless_affine(prob, a_hat))
                a0[fine.mu == 0] = 0.0
                a_cell = refine_duals(prob, fine, alpha[last], last) if dual_refinement == "hybrid" else a0
                alpha = {"A": a_cell.copy(), "B": a0.copy()}
            else:
                a0 = refine_duals(prob, fine, alpha[last], last)
                alpha = {"A": a0.copy(), "B": a0.copy()}
            prob, lev = fine, lev + 1
        eps = eps_s
        for _ in range(sweeps):
            for part in ("A", "B"):
                if before_half_sweep is not None:
                    before_half_sweep(prob, part, rows, alpha[part], eps)
                rows, info = half_sweep(prob, part, rows, alpha[part], eps, params)
                last = part
                history.append((lev, eps, part, info))
                if on_half_sweep is not None:
                    on_half_sweep(prob, part, rows, alpha[part], eps, info)
    return RunResult(prob, rows, alpha, eps, last, history)
