"""dd_solve_cell_noalloc: a cell solve for callers that cannot allocate device
memory when they need a solve (device memory owned by another runtime or
pool, latency-critical loops that must not stall on the allocator).

It must give the same basic marginals as the allocating path, dd_half_sweep,
on a problem whose partition A is a single cell, on two calls in a row (the
second warm-started from the first call's duals), and the FP64 oracle's
result on single cells of every supported size (b = 2, 4, 8), including a
support of the maximum size and supports far from the cell. Rejected inputs
leave the caller's buffers untouched. This file is collected last so that a
failure here does not hide the other tests.
"""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L1, the tolerance of the other parity tests


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    torch.cuda.set_device(0)
    return dd


def _dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=torch.device("cuda", 0))


def test_noalloc_cell_solve_matches_half_sweep(lib):
    import torch
    dd = lib
    n, b, eps = 8, 4, 0.02          # 2×2 basic cells: partition A is one cell
    mu = syn.gaussian_mixture(n, 2, 80)
    nu = syn.gaussian_mixture(n, 2, 81)
    stream = torch.cuda.current_stream()

    # allocating path: context + two A half-sweeps
    g = dd.DD(mu, nu, b, 1, [(eps, 1, 0)], err_tol=1e-6, stream=stream)

    # no-alloc path: caller-owned device buffers
    yy = np.arange(n * n)
    mu_t = _dev(mu.ravel(), torch.float64)
    yr, yc = _dev(yy // n, torch.int32), _dev(yy % n, torch.int32)
    nu_t = _dev(nu.ravel(), torch.float64)
    alpha_t = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    out_t = torch.zeros(4 * n * n, dtype=torch.float64, device="cuda")

    for call in range(2):
        g.half_sweep(0, eps)
        rp, col, val = g.basic_marginals()
        ref = np.zeros((4, n * n))
        for i in range(4):
            ref[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
        dd.dd_solve_cell_noalloc(mu_t.data_ptr(), b, 1.0 / n, n * n, yr.data_ptr(), yc.data_ptr(),
                                 nu_t.data_ptr(), eps, 1e-6, 2000, 1e-15, alpha_t.data_ptr(),
                                 out_t.data_ptr(), stream)
        got = out_t.cpu().numpy().reshape(4, n * n)
        rel = np.abs(got - ref).sum() / ref.sum()
        assert rel < TOL, (call, rel)
        assert abs(got.sum() - nu.sum()) < 1e-12          # Y-marginal reproduced
    g.close()


# ---- single cells against the FP64 oracle ----------------------------------
def _cell_problem(b, spacing, yr, yc, mu, nu):
    """The oracle's problem for one 2b×2b cell (4 basic cells, row-major in
    the 2×2 block) and a support given by offsets from the cell corner."""
    H = 2 * b
    basic = []
    for kr in range(2):
        for kc in range(2):
            ii = np.arange(kr * b, (kr + 1) * b)
            jj = np.arange(kc * b, (kc + 1) * b)
            basic.append((ii[:, None] * H + jj[None, :]).ravel())
    d2 = spacing * spacing

    def cost(X, Y):
        xr, xc = np.divmod(X, H)
        return d2 * ((xr[:, None] - yr[Y][None, :]) ** 2 + (xc[:, None] - yc[Y][None, :]) ** 2).astype(np.float64)

    return odd.Problem(mu, nu, cost, basic, {"A": [[0, 1, 2, 3]]})


def _case(b, offsets, seed):
    """μ on the cell and ν on the support grid offsets × offsets (row-major),
    both smooth, positive and of mass 1."""
    rng = np.random.default_rng(seed)
    H = 2 * b
    yr, yc = np.meshgrid(offsets, offsets, indexing="ij")
    yr, yc = yr.ravel().astype(np.int32), yc.ravel().astype(np.int32)
    span = float(offsets[-1] - offsets[0]) + 1.0
    nu = np.exp(-0.5 * (((yr - b) / (span / 4)) ** 2 + ((yc - b + 3) / (span / 5)) ** 2)) + 0.05 * rng.random(yr.size)
    nu /= nu.sum()
    xi = np.arange(H)
    mu = (np.exp(-0.5 * ((xi[:, None] - 2) / 3.0) ** 2 - 0.5 * ((xi[None, :] - H + 2) / 4.0) ** 2)
          + 0.1 + 0.05 * rng.random((H, H))).ravel()
    mu /= mu.sum()
    return yr, yc, mu, nu


CASES = [
    # b, support offsets per axis, eps, spacing
    (2, np.arange(-4, 8), 2e-3, 1 / 64),                  # 4×4 cell, 144 points
    (8, np.arange(-12, 28), 2e-3, 1 / 128),               # 16×16 cell, 1600 points
    (4, np.arange(-60, 68), 1e-3, 1 / 1024),              # 8×8 cell, 16384 points (the limit)
    (4, np.arange(-1890, 1891, 210), 2e-3, 1 / 4096),     # 19² points up to 1890 px away
]


@pytest.mark.parametrize("b,offsets,eps,spacing", CASES, ids=["b2", "b8", "b4_max_ny", "b4_far"])
def test_noalloc_matches_oracle(lib, b, offsets, eps, spacing):
    import torch
    dd = lib
    yr, yc, mu, nu = _case(b, offsets, seed=b)
    ny = yr.size
    prob = _cell_problem(b, spacing, yr, yc, mu, nu)
    rows = [(np.arange(ny), nu.copy())] + [(np.zeros(0, np.int64), np.zeros(0))] * 3
    alpha_ref = np.zeros(mu.size)
    stream = torch.cuda.current_stream()
    mu_t, nu_t = _dev(mu, torch.float64), _dev(nu, torch.float64)
    yr_t, yc_t = _dev(yr, torch.int32), _dev(yc, torch.int32)
    alpha_t = torch.zeros(mu.size, dtype=torch.float64, device="cuda")
    out_t = torch.zeros(4 * ny, dtype=torch.float64, device="cuda")
    for call in range(2):
        new_rows, info = odd.half_sweep(prob, "A", rows, alpha_ref, eps, odd.Params(err=1e-10, max_iter=20000))
        ref = np.zeros((4, ny))
        for i in range(4):
            ref[i, new_rows[i][0]] = new_rows[i][1]
        dd.dd_solve_cell_noalloc(mu_t.data_ptr(), b, spacing, ny, yr_t.data_ptr(), yc_t.data_ptr(),
                                 nu_t.data_ptr(), eps, 1e-7, 5000, 1e-15, alpha_t.data_ptr(),
                                 out_t.data_ptr(), stream)
        got = out_t.cpu().numpy().reshape(4, ny)
        rel = np.abs(got - ref).sum() / ref.sum()
        assert rel < TOL, (call, rel, info.iters)
        # BalanceMeasures: every basic cell carries its μ-mass
        for i in range(4):
            assert abs(got[i].sum() - mu[prob.basic[i]].sum()) < 1e-12
        # α agrees with the oracle's up to one constant (the gauge)
        d = alpha_t.cpu().numpy() - alpha_ref
        assert np.ptp(d) / eps < 1e-3, np.ptp(d) / eps


def test_noalloc_rejects_bad_input_and_keeps_outputs(lib):
    import torch
    dd = lib
    b, n = 4, 8
    yr, yc, mu, nu = _case(b, np.arange(-2, 10), seed=3)
    ny = yr.size
    mu_t, nu_t = _dev(mu, torch.float64), _dev(nu, torch.float64)
    yr_t, yc_t = _dev(yr, torch.int32), _dev(yc, torch.int32)
    alpha_t = torch.full((mu.size,), 7.0, dtype=torch.float64, device="cuda")
    out_t = torch.full((4 * ny,), 3.0, dtype=torch.float64, device="cuda")

    def call(**kw):
        a = dict(mu=mu_t, yr=yr_t, yc=yc_t, nu=nu_t, ny=ny, max_iter=2000)
        a.update(kw)
        dd.dd_solve_cell_noalloc(a["mu"].data_ptr(), b, 1 / 64, a["ny"], a["yr"].data_ptr(), a["yc"].data_ptr(),
                                 a["nu"].data_ptr(), 0.01, 1e-6, a["max_iter"], 1e-15, alpha_t.data_ptr(),
                                 out_t.data_ptr())

    # more support points than the fixed scratch holds: rejected before any work
    with pytest.raises(dd.DDError) as e:
        call(ny=16385)
    assert e.value.status == dd.DD_ERR_ARG and "16384" in str(e.value)
    # unsorted support
    bad = yc.copy()
    bad[0], bad[1] = bad[1], bad[0]
    with pytest.raises(dd.DDError) as e:
        call(yc=_dev(bad, torch.int32))
    assert e.value.status == dd.DD_ERR_ARG
    # ν of another mass than μ
    with pytest.raises(dd.DDError) as e:
        call(nu=_dev(nu * 1.01, torch.float64))
    assert e.value.status == dd.DD_ERR_ARG and "mass" in str(e.value)
    assert torch.all(alpha_t == 7.0) and torch.all(out_t == 3.0)
    # a solve cut off at max_iter: reported, with a feasible result
    with pytest.raises(dd.DDError) as e:
        call(max_iter=1)
    assert e.value.status == dd.DD_ERR_NOT_CONVERGED
    got = out_t.cpu().numpy().reshape(4, ny)
    assert np.abs(got.sum(axis=0) - nu).sum() < 1e-12
    # and the scratch is still usable
    call()
