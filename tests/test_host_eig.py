"""The library's host FP64 symmetric eigensolver (projected matrix of the Krylov method) vs numpy."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "paper_2210_16435_gb300", "csrc", "eig_host.cpp")
DRIVER = r'''
#include "internal.h"
namespace sfairsc {
void check_cuda(cudaError_t, const char*) {}
void fail(int, const std::string&) { throw 1; }
}
extern "C" void eig(int m, double* A, double* w) { sfairsc::host_symmetric_eig(m, A, w); }
extern "C" int eig_limited(int m, double* A, double* w, int sweeps) { return sfairsc::host_symmetric_eig(m, A, w, sweeps) ? 1 : 0; }
extern "C" int eig_jacobi(int m, double* A, double* w) { return sfairsc::host_symmetric_eig_jacobi(m, A, w) ? 1 : 0; }
'''


@pytest.fixture(scope="module")
def eiglib():
    d = tempfile.mkdtemp()
    drv = os.path.join(d, "drv.cpp")
    open(drv, "w").write(DRIVER)
    so = os.path.join(d, "libeig.so")
    inc = ["-I" + os.path.join(ROOT, "paper_2210_16435_gb300", "csrc"), "-I/usr/local/cuda/include",
           "-I" + os.path.join(ROOT, "include")]
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", *inc, SRC, drv, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.eig.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.eig_limited.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.eig_jacobi.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (5, 2), (20, 3), (64, 4), (100, 6), (136, 5), (250, 7)])
def test_random_symmetric(eiglib, m, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m))
    A = A + A.T
    M = np.asfortranarray(A.copy())
    w = np.empty(m)
    eiglib.eig(m, M.ctypes.data, w.ctypes.data)
    ref = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(w, ref, atol=1e-12 * np.abs(ref).max())
    V = M
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-11 * np.abs(ref).max())


def test_arrowhead_and_clusters(eiglib):
    """The thick-restart shape: diagonal Ritz block, coupling row, tridiagonal tail, repeated values."""
    m, K = 40, 24
    rng = np.random.default_rng(9)
    A = np.zeros((m, m))
    A[np.arange(K), np.arange(K)] = np.sort(np.concatenate([np.zeros(4), np.full(4, 0.3), rng.random(K - 8)]))
    A[K, :K] = A[:K, K] = rng.standard_normal(K) * 1e-7
    for i in range(K, m):
        A[i, i] = rng.random() + 1
        if i + 1 < m:
            A[i, i + 1] = A[i + 1, i] = rng.random()
    M = np.asfortranarray(A.copy())
    w = np.empty(m)
    eiglib.eig(m, M.ctypes.data, w.ctypes.data)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-13)
    np.testing.assert_allclose(A @ M, M * w, atol=1e-12)


def test_sweep_limit_reports_failure_and_jacobi_recovers(eiglib):
    """A QR iteration cut off after 3 steps says so; the Jacobi fallback then gives the decomposition."""
    m = 30
    rng = np.random.default_rng(11)
    A = rng.standard_normal((m, m))
    A = A + A.T
    M = np.asfortranarray(A.copy())
    w = np.empty(m)
    assert eiglib.eig_limited(m, M.ctypes.data, w.ctypes.data, 3) == 0
    M = np.asfortranarray(A.copy())
    assert eiglib.eig_limited(m, M.ctypes.data, w.ctypes.data, -1) == 1
    M = np.asfortranarray(A.copy())
    assert eiglib.eig_jacobi(m, M.ctypes.data, w.ctypes.data) == 1
    ref = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(w, ref, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(M.T @ M, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(A @ M, M * w, atol=1e-11 * np.abs(ref).max())


def test_nonfinite_projected_matrix_is_flagged(eiglib):
    """A NaN never deflates: the QR iteration reports failure and Jacobi refuses the input."""
    m = 12
    A = np.diag(np.arange(m, dtype=float)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    A[5, 6] = A[6, 5] = np.nan
    w = np.empty(m)
    M = np.asfortranarray(A.copy())
    assert eiglib.eig_limited(m, M.ctypes.data, w.ctypes.data, -1) == 0
    M = np.asfortranarray(A.copy())
    assert eiglib.eig_jacobi(m, M.ctypes.data, w.ctypes.data) == 0


def test_random_sizes_threaded_and_limited(eiglib):
    """Sizes across the threaded range (from m = 48 the vectors are formed on several threads while
    the QR iteration runs), dense, clustered and banded inputs, and calls cut off by a sweep limit."""
    rng = np.random.default_rng(21)
    for it in range(40):
        m = int(rng.integers(40, 257))
        A = rng.standard_normal((m, m))
        A = (A + A.T) / 2
        if it % 3 == 1:  # clustered values, tiny couplings (a converged thick-restart block)
            A = np.diag(1e-3 * rng.integers(0, 5, m)) + 1e-9 * A
        elif it % 3 == 2:  # banded (a block-tridiagonal tail)
            A = np.triu(np.tril(A, 4), -4)
        M = np.asfortranarray(A.copy())
        w = np.empty(m)
        if it % 10 == 9:
            assert eiglib.eig_limited(m, M.ctypes.data, w.ctypes.data, 2) == 0
            continue
        assert eiglib.eig_limited(m, M.ctypes.data, w.ctypes.data, -1) == 1
        scale = np.abs(A).max()
        np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * scale)
        np.testing.assert_allclose(M.T @ M, np.eye(m), atol=1e-12)
        np.testing.assert_allclose(A @ M, M * w, atol=1e-12 * scale)
