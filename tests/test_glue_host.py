"""dd_glue_potential, the least-squares step of the dual gluing (§6.3), is
host code of the C ABI: it runs here without a GPU and is compared with the
oracle's dense least squares (oracle.dd.helmholtz_potential) and with closed
forms."""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def lib():
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def _gluing_edges(n, b):
    prob = odd.GridProblem(syn.gaussian_mixture(n, 2, 0), syn.gaussian_mixture(n, 2, 1), b, 1.0 / n)
    edges = odd.gluing_graph(prob)
    j1 = np.array([e[0] for e in edges], dtype=np.int32)
    j2 = np.array([e[1] for e in edges], dtype=np.int32)
    return len(prob.parts["A"]), j1, j2


def test_matches_the_oracle_on_the_gluing_graph(lib):
    nA, j1, j2 = _gluing_edges(64, 2)               # 16×16 A cells, 17×17 B cells
    rng = np.random.default_rng(11)
    logq = rng.normal(0.0, 1.0, j1.size)
    V, it, res = lib.dd_glue_potential(nA, j1, j2, logq)
    want = odd.helmholtz_potential(nA, j1, j2, logq)
    assert res <= 1e-12 and it > 0
    assert np.abs(V - want).max() <= 1e-9 * np.abs(want).max()


def test_exact_gradient_is_recovered(lib):
    # log q(j1, j2) = φ(j2) − φ(j1): the residuals vanish at V = φ − mean φ
    nA, j1, j2 = _gluing_edges(32, 2)
    phi = np.random.default_rng(12).normal(0.0, 3.0, nA)
    V, _, _ = lib.dd_glue_potential(nA, j1, j2, phi[j2] - phi[j1])
    assert np.abs(V - (phi - phi.mean())).max() < 1e-9


def test_components_loops_and_errors(lib):
    # two components (a path 0-1-2 and an edge 3-4) and a loop edge: each
    # component has mean zero, as the minimum-norm least-squares solution
    j1 = np.array([0, 1, 3, 2, 1], dtype=np.int32)
    j2 = np.array([1, 2, 4, 2, 0], dtype=np.int32)
    logq = np.array([0.5, -1.0, 2.0, 7.0, 0.25])
    V, _, _ = lib.dd_glue_potential(5, j1, j2, logq)
    want = odd.helmholtz_potential(5, j1, j2, logq)
    assert abs(V[:3].sum()) < 1e-12 and abs(V[3:].sum()) < 1e-12
    assert np.abs(V - want).max() < 1e-10
    with pytest.raises(lib.DDError) as e:
        lib.dd_glue_potential(5, np.array([0], np.int32), np.array([5], np.int32), np.array([1.0]))
    assert e.value.status == lib.DD_ERR_ARG
    with pytest.raises(lib.DDError) as e:
        lib.dd_glue_potential(5, np.array([0], np.int32), np.array([1], np.int32), np.array([np.nan]))
    assert e.value.status == lib.DD_ERR_ARG
    with pytest.raises(lib.DDError) as e:
        lib.dd_glue_potential(5, j1, j2, logq, max_iter=0)
    assert e.value.status == lib.DD_ERR_NOT_CONVERGED


def _duals(n, eps, seed):
    rng = np.random.default_rng(seed)
    k = np.arange(n)
    smooth = 0.002 * ((k[:, None] - n / 2.0) ** 2 + 0.5 * (k[None, :] - n / 3.0) ** 2)
    return (smooth + eps * rng.normal(0.0, 1.0, (n, n))).ravel()


def test_glued_duals_match_the_oracle(lib):
    n, b, eps = 32, 4, 0.01
    mu = syn.gaussian_mixture(n, 3, 30)
    mu[3, 5] = 0.0                    # a pixel without mass keeps α̂ = 0
    nu = syn.gaussian_mixture(n, 3, 31)
    aA, aB = _duals(n, eps, 1), _duals(n, eps, 2)
    prob = odd.GridProblem(mu, nu, b, 1.0 / n)
    want, Vw = odd.glue_duals(prob, aA, aB, eps)
    got, V = lib.dd_glue_duals_host(mu, aA, aB, b, eps)
    assert got[3, 5] == 0.0
    assert np.abs(got.ravel() - want).max() <= 1e-9 * np.abs(want).max()
    assert np.abs(V - Vw).max() <= 1e-9 * max(1.0, np.abs(Vw).max())


def test_glued_duals_of_consistent_rescalings(lib):
    # u_{A,J} = λ_J u*, u_{B,J} = κ_J u*: α̂ − α* is one constant
    n, b, eps = 32, 2, 0.02
    mu = syn.gaussian_mixture(n, 2, 32)
    a_star = _duals(n, eps, 3)
    rng = np.random.default_rng(4)
    nb = n // b
    lamA = rng.normal(0.0, 3.0, (nb // 2, nb // 2))
    lamB = rng.normal(0.0, 3.0, (nb // 2 + 1, nb // 2 + 1))
    r = np.arange(n) // b
    aA = a_star + eps * lamA[(r // 2)[:, None], (r // 2)[None, :]].ravel()
    aB = a_star + eps * lamB[((r + 1) // 2)[:, None], ((r + 1) // 2)[None, :]].ravel()
    got, _ = lib.dd_glue_duals_host(mu, aA, aB, b, eps)
    assert np.ptp(got.ravel() - a_star) / eps < 1e-9


def test_interpolation_matches_the_oracle(lib):
    coarse = odd.GridProblem(syn.gaussian_mixture(16, 2, 40), syn.gaussian_mixture(16, 2, 41), 2, 1.0 / 16)
    fine = odd.GridProblem(syn.gaussian_mixture(32, 2, 40), syn.gaussian_mixture(32, 2, 41), 2, 1.0 / 32)
    a = np.random.default_rng(13).normal(0.0, 1.0, (16, 16))
    got = lib.dd_interpolate_dual_host(a)
    want = odd.refine_duals_glued(coarse, fine, a.ravel()).reshape(32, 32)
    assert np.abs(got - want).max() < 1e-12
    k = np.arange(16.0)
    t = np.arange(32) / 2.0 - 0.25
    aff = 0.5 - 2.0 * k[:, None] + 0.25 * k[None, :]
    assert np.abs(lib.dd_interpolate_dual_host(aff) - (0.5 - 2.0 * t[:, None] + 0.25 * t[None, :])).max() < 1e-12
    with pytest.raises(lib.DDError):
        lib.dd_interpolate_dual_host(np.zeros((1, 1)))


def _csr(P):
    rp = np.zeros(P.shape[0] + 1, dtype=np.int64)
    cols, vals = [], []
    for x in range(P.shape[0]):
        nz = np.flatnonzero(P[x] > 0)
        cols.append(nz)
        vals.append(P[x, nz])
        rp[x + 1] = rp[x] + nz.size
    return rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals)


@pytest.mark.parametrize("sweeps,err,max_iter", [(2, 1e-6, 5), (40, 1e-13, 20000)])
def test_relative_pd_gap_matches_the_oracle(lib, sweeps, err, max_iter):
    # without truncation the coupling of the last partition reaches every
    # (x, y), so the restricted kernel is the whole kernel and the host gap
    # equals the oracle's dense eq. RelPDGap; at convergence it vanishes
    n, b, eps = 16, 4, 0.01
    mu = syn.gaussian_mixture(n, 3, 50)
    nu = syn.gaussian_mixture(n, 3, 51)
    prob = odd.GridProblem(mu, nu, b, 1.0 / n)
    rows = odd.product_state(prob)
    alpha = {"A": np.zeros(n * n), "B": np.zeros(n * n)}
    par = odd.Params(err=err, trunc=0.0, max_iter=max_iter)
    for l in range(2 * sweeps):
        part = "AB"[l % 2]
        rows, _ = odd.half_sweep(prob, part, rows, alpha[part], eps, par)
    a_hat, _ = odd.glue_duals(prob, alpha["A"], alpha["B"], eps)
    P = odd.partition_plan(prob, "B", rows, alpha["B"], eps)
    assert (P > 0).all()
    b_hat = odd.best_y_dual(prob, a_hat, eps)
    rel_w, gap_w, prim_w = odd.relative_pd_gap(prob, P, a_hat, b_hat, eps)
    rel, gap, prim = lib.dd_relative_pd_gap_host(mu, nu, eps, _csr(P), a_hat)
    assert prim == pytest.approx(prim_w, rel=1e-10)
    assert gap == pytest.approx(gap_w, rel=1e-7, abs=1e-12 * abs(prim_w))
    if sweeps == 40:
        assert abs(rel) < 1e-8
    else:
        assert rel > 1e-6


def _rows_csr(rows):
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    for i, (c, _) in enumerate(rows):
        rp[i + 1] = rp[i] + c.size
    return rp, np.concatenate([c for c, _ in rows]).astype(np.int32), np.concatenate([v for _, v in rows])


def test_coupling_image(lib, tmp_path):
    # §7.2: the product coupling paints every pixel with the μ-weighted mean
    # colour; the identity coupling (ν_i = μ on X_i) paints the checkerboard
    # of the basic cells itself; overlapping ν_i mix in proportion to mass
    n, b = 16, 4
    mu = syn.gaussian_mixture(n, 2, 60)
    prob = odd.GridProblem(mu, mu, b, 1.0 / n)
    colours = lib.checkerboard_colours(n // b)
    img = lib.dd_coupling_image_host(n, _rows_csr(odd.product_state(prob)), colours)
    mean = (prob.basic_mass[:, None] * colours).sum(axis=0) / prob.basic_mass.sum()
    assert np.abs(img - mean[None, None, :]).max() < 1e-6
    ident = [(np.sort(X), mu.ravel()[np.sort(X)]) for X in prob.basic]
    img = lib.dd_coupling_image_host(n, _rows_csr(ident), colours)
    cell = (np.arange(n)[:, None] // b) * (n // b) + np.arange(n)[None, :] // b
    assert np.abs(img - colours[cell]).max() < 1e-7
    rows = [(np.array([5]), np.array([1.0])), (np.array([5, 6]), np.array([3.0, 2.0]))]
    two = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    img = lib.dd_coupling_image_host(4, _rows_csr(rows), two)
    assert np.allclose(img[1, 1], [0.25, 0.0, 0.75]) and np.allclose(img[1, 2], [0.0, 0.0, 1.0])
    assert np.all(img[0, 0] == 0.0)                   # no mass: black
    path = tmp_path / "c.ppm"
    lib.write_ppm(path, img)
    data = path.read_bytes()
    assert data.startswith(b"P6\n4 4\n255\n") and len(data) == len(b"P6\n4 4\n255\n") + 48


@pytest.mark.parametrize("n,b", [(16, 4), (24, 4), (40, 4), (32, 8), (36, 2)])
def test_gluing_graph_is_the_nine_point_stencil(n, b):
    # The GPU gluing stores no edge list: on the grid of A cells (row-major,
    # A cell (R, C) = basic cells {2R, 2R+1} × {2C, 2C+1}) it applies the
    # Laplacian DᵀD of the oracle's gluing graph as a 9-point stencil with
    # weight 4 on the 4-neighbours and 2 on the diagonal ones, and builds
    # the right-hand side −Dᵀ log q (log q = s⁺_i + s⁻_{i'} for the ordered
    # pair (i, i') of basic cells of one B cell) per A cell from the B cells
    # at its four corners. Both against the oracle's edges, for grids whose
    # A-cell count is and is not a multiple of the 8 CTAs of the CG.
    prob = odd.GridProblem(syn.gaussian_mixture(n, 2, 0), syn.gaussian_mixture(n, 2, 1), b, 1.0 / n)
    nb = n // b
    na = nb // 2
    A = prob.parts["A"]
    assert len(A) == na * na
    for j, J in enumerate(A):   # row-major A cells, as on the device
        R, C = divmod(j, na)
        cells = sorted((i // nb, i % nb) for i in J)
        assert cells == [(2 * R + dr, 2 * C + dc) for dr in (0, 1) for dc in (0, 1)]
    edges = odd.gluing_graph(prob)
    L = np.zeros((na * na, na * na))
    for j1, j2, _, _, _ in edges:
        L[j1, j1] += 1
        L[j2, j2] += 1
        L[j1, j2] -= 1
        L[j2, j1] -= 1
    S = np.zeros_like(L)
    for R in range(na):
        for C in range(na):
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    R2, C2 = R + dr, C + dc
                    if (dr, dc) == (0, 0) or not (0 <= R2 < na and 0 <= C2 < na):
                        continue
                    w = 4.0 if dr == 0 or dc == 0 else 2.0
                    S[R * na + C, R2 * na + C2] -= w
                    S[R * na + C, R * na + C] += w
    assert np.array_equal(L, S)
    # right-hand side from random s± per basic cell
    rng = np.random.default_rng(5)
    sp = rng.normal(size=nb * nb)
    sm = rng.normal(size=nb * nb)

    def basic_of(X):
        r, c = divmod(int(X[0]), n)
        return (r // b) * nb + c // b

    rhs = np.zeros(na * na)
    for j1, j2, _, X1, X2 in edges:
        lq = sp[basic_of(X1)] + sm[basic_of(X2)]
        rhs[j1] -= lq
        rhs[j2] += lq
    corner = np.zeros(na * na)
    for R in range(na):
        for C in range(na):
            for dr in (0, 1):
                for dc in (0, 1):
                    Rb, Cb = R + dr, C + dc
                    own = (2 * R + dr) * nb + 2 * C + dc
                    for ei in (2 * Rb - 1, 2 * Rb):
                        for ej in (2 * Cb - 1, 2 * Cb):
                            o = ei * nb + ej
                            if 0 <= ei < nb and 0 <= ej < nb and o != own:
                                corner[R * na + C] += sp[o] + sm[own] - sp[own] - sm[o]
    assert np.allclose(corner, rhs, rtol=0, atol=1e-12)


def test_host_functions_reject_what_the_header_rejects(lib):
    # the error paths documented in dd.h for the host functions (no GPU)
    n, b = 16, 4
    mu = syn.gaussian_mixture(n, 2, 70)
    nu = syn.gaussian_mixture(n, 2, 71)
    a = np.zeros(n * n)

    def status(fn, *args):
        with pytest.raises(lib.DDError) as e:
            fn(*args)
        return e.value.status

    # gluing: n/b odd, a basic cell without mass, negative μ, non-finite α, ε ≤ 0
    assert status(lib.dd_glue_duals_host, np.ones((12, 12)), np.zeros(144), np.zeros(144), 4, 0.1) == lib.DD_ERR_ARG
    m0 = mu.copy()
    m0[:b, :b] = 0.0
    assert status(lib.dd_glue_duals_host, m0, a, a, b, 0.1) == lib.DD_ERR_ARG
    m1 = mu.copy()
    m1[3, 3] = -1e-9
    assert status(lib.dd_glue_duals_host, m1, a, a, b, 0.1) == lib.DD_ERR_ARG
    a1 = a.copy()
    a1[7] = np.inf
    assert status(lib.dd_glue_duals_host, mu, a1, a, b, 0.1) == lib.DD_ERR_ARG
    assert status(lib.dd_glue_duals_host, mu, a, a, b, 0.0) == lib.DD_ERR_ARG
    # the gap: an entry of π where ν has no mass, a pixel with ν > 0 that π
    # does not reach, a negative entry
    prob = odd.GridProblem(mu, nu, b, 1.0 / n)
    P = np.outer(prob.mu, prob.nu)
    rp, col, val = _csr(P)
    rel, _, _ = lib.dd_relative_pd_gap_host(mu, nu, 0.05, (rp, col, val), a)
    assert np.isfinite(rel)
    nu0 = nu.copy().ravel()
    nu0[int(col[0])] = 0.0
    assert status(lib.dd_relative_pd_gap_host, mu, nu0.reshape(n, n), 0.05, (rp, col, val), a) == lib.DD_ERR_ARG
    P2 = P.copy()
    P2[:, 5] = 0.0
    assert status(lib.dd_relative_pd_gap_host, mu, nu, 0.05, _csr(P2), a) == lib.DD_ERR_ARG
    v2 = val.copy()
    v2[3] = -v2[3]
    assert status(lib.dd_relative_pd_gap_host, mu, nu, 0.05, (rp, col, v2), a) == lib.DD_ERR_ARG
    # the image: a column outside the image
    rows = [(np.array([n * n]), np.array([1.0]))]
    assert status(lib.dd_coupling_image_host, n, _rows_csr(rows), np.zeros((1, 3), np.float32)) == lib.DD_ERR_ARG
