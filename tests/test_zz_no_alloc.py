"""dd_solve_cell_noalloc: a cell solve for callers that cannot allocate device
memory (for example while a stream is being captured into a CUDA graph).

It must give the same basic marginals as the allocating path, dd_half_sweep,
on a problem whose partition A is a single cell, on two calls in a row (the
second warm-started from the first call's duals). This file is collected last
so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L1, the tolerance of the other parity tests


def test_noalloc_cell_solve_matches_half_sweep():
    import torch
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd

    torch.cuda.set_device(0)
    n, b, eps = 8, 4, 0.02          # 2×2 basic cells: partition A is one cell
    mu = syn.gaussian_mixture(n, 2, 80)
    nu = syn.gaussian_mixture(n, 2, 81)
    stream = torch.cuda.current_stream()

    # allocating path: context + two A half-sweeps
    g = dd.DD(mu, nu, b, 1, [(eps, 1, 0)], err_tol=1e-6, stream=stream)

    # no-alloc path: caller-owned device buffers
    dev = torch.device("cuda", 0)
    mu_t = torch.tensor(mu.ravel(), dtype=torch.float64, device=dev)
    yy = np.arange(n * n)
    yr = torch.tensor(yy // n, dtype=torch.int32, device=dev)
    yc = torch.tensor(yy % n, dtype=torch.int32, device=dev)
    nu_t = torch.tensor(nu.ravel(), dtype=torch.float64, device=dev)
    alpha_t = torch.zeros(n * n, dtype=torch.float64, device=dev)
    out_t = torch.zeros(4 * n * n, dtype=torch.float64, device=dev)

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


def test_noalloc_rejects_oversized_input():
    import torch
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd

    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    ibuf = torch.zeros(16, dtype=torch.int32, device=dev)
    with pytest.raises(dd.DDError) as e:
        dd.dd_solve_cell_noalloc(buf.data_ptr(), 4, 1 / 8, 16385, ibuf.data_ptr(), ibuf.data_ptr(),
                                 buf.data_ptr(), 0.02, 1e-6, 10, 1e-15, buf.data_ptr(), buf.data_ptr())
    assert e.value.status == dd.DD_ERR_ARG
    assert "16384" in str(e.value)
