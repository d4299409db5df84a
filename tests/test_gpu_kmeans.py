"""Library k-means (kernel c) against the oracle's rule set: identical labels, centroids and inertia."""
import numpy as np
import pytest
import torch

from oracle import kmeans as km

pytestmark = pytest.mark.gpu


def blobs(n_per, k, d, sep, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((k, d)) * sep
    return np.concatenate([C[c] + rng.standard_normal((n_per, d)) for c in range(k)])


@pytest.mark.parametrize("n_per,k,d,n_init,seed", [(50, 4, 3, 1, 0), (300, 10, 10, 3, 1), (997, 7, 40, 2, 2),
                                                   (2000, 20, 20, 1, 3), (100, 50, 50, 1, 4)])
def test_kmeans_bitwise_parity(built_lib, n_per, k, d, n_init, seed):
    from paper_2210_16435_gb300.solver import kmeans

    X = blobs(n_per, k, d, 1.5, seed) * 1e-3
    lab, cen, inertia, iters = kmeans(torch.as_tensor(X, device="cuda"), k, seed=seed, n_init=n_init, max_iter=100)
    olab, omu, oin = km.kmeans(X, k, seed=seed, n_init=n_init, max_iter=100)
    assert np.array_equal(lab.cpu().numpy(), olab)
    assert np.array_equal(cen.cpu().numpy(), omu)
    assert inertia == oin


def test_kmeans_shuffled_rows_and_empty_clusters(built_lib):
    """Random row order (no label runs) and more clusters than distinct points (empty clusters)."""
    from paper_2210_16435_gb300.solver import kmeans

    rng = np.random.default_rng(7)
    X = rng.permutation(blobs(200, 5, 8, 3.0, 7))
    lab, cen, inertia, _ = kmeans(torch.as_tensor(X, device="cuda"), 5, seed=3, n_init=2)
    olab, omu, oin = km.kmeans(X, 5, seed=3, n_init=2, max_iter=100)
    assert np.array_equal(lab.cpu().numpy(), olab) and np.array_equal(cen.cpu().numpy(), omu) and inertia == oin
    Y = np.repeat(rng.standard_normal((3, 4)), [40, 30, 30], axis=0)
    lab, cen, inertia, _ = kmeans(torch.as_tensor(Y, device="cuda"), 6, seed=1)
    olab, omu, oin = km.kmeans(Y, 6, seed=1, n_init=1, max_iter=100)
    assert np.array_equal(lab.cpu().numpy(), olab) and np.array_equal(cen.cpu().numpy(), omu)


def test_kmeans_host_buffers(built_lib):
    from paper_2210_16435_gb300 import binding as B

    X = blobs(100, 3, 5, 2.0, 9)
    Xc = np.ascontiguousarray(X)
    lab = np.empty(len(X), dtype=np.int32)
    inertia, _ = B.sfairsc_kmeans(len(X), 5, Xc.ctypes.data, 3, 11, 1, 100, lab.ctypes.data)
    olab, _, oin = km.kmeans(X, 3, seed=11, n_init=1, max_iter=100)
    assert np.array_equal(lab, olab) and inertia == oin
