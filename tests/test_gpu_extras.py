"""The §7.2 colour image computed on the GPU, and the peak-memory counters of
the sparse plan."""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def test_coupling_image_on_the_gpu(lib):
    # the device image equals the mean colour of the basic marginals computed
    # from their download, and the image of the oracle's state
    mu = syn.gaussian_mixture(32, 3, 60)
    nu = syn.gaussian_mixture(32, 3, 61)
    sched = [(0.02, 2, 0), (0.01, 2, 0)]
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-6)
    g.run_schedule()
    rng = np.random.default_rng(0)
    colours = rng.uniform(0, 1, size=(64, 3)).astype(np.float32)
    img = g.coupling_image(colours)
    rp, col, val = g.basic_marginals()
    g.close()
    rows = odd.rows_from_csr(rp, col, val)
    D = odd.rows_to_dense(rows, 32 * 32)            # basic cells × Y pixels
    mass = D.sum(axis=0)
    want = (colours.astype(np.float64).T @ D).T / np.where(mass > 0, mass, 1.0)[:, None]
    np.testing.assert_allclose(img.reshape(-1, 3), want, atol=2e-6)
    ref = odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))
    Dr = odd.rows_to_dense(ref.rows, 32 * 32)
    want_r = (colours.astype(np.float64).T @ Dr).T / Dr.sum(axis=0)[:, None]
    np.testing.assert_allclose(img.reshape(-1, 3), want_r, atol=1e-4)


def test_peak_plan_memory_is_reported(lib):
    mu = syn.gaussian_mixture(64, 3, 62)
    nu = syn.gaussian_mixture(64, 3, 63)
    g = lib.DD(mu, nu, 4, 3, syn.paper_schedule(64, 3, 2), err_tol=1e-6, mode=1)
    g.run_schedule()
    p = g.profile()
    _, _, _, _, nnz = g.info()
    g.close()
    assert p.peak_nnz >= nnz > 0
    assert p.peak_state_bytes >= 2 * 12 * nnz          # two CSR buffers of ≥ nnz entries
    assert p.peak_work_bytes >= 32 * nnz
