"""Fused operator kernel (Sec. 3.4 (i)-(ii)) against the oracle's literal matvec."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from conftest import graph_tensors
from msbm import cell_sizes_equal, cell_sizes_from_proportions, graph_from_dense, sample_msbm
from oracle.sfairsc import SFairSCOperator, operator_from_graph

pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def msbm(n, k, h, deg, seed, unequal=False):
    cells = (cell_sizes_from_proportions(n, np.linspace(1, 3, k), 1.0 / np.arange(1, h + 1)) if unequal
             else cell_sizes_equal(n, k, h))
    from msbm import category_probabilities
    probs = category_probabilities(cells, min(deg, 0.4 * n), (0.5, 0.25, 0.15, 0.10))
    return sample_msbm(cells, probs, seed=seed)


def check_operator(g, prec, vdt, nvec, normalized=True, seed=0):
    from paper_2210_16435_gb300.solver import FairSC

    rp, ci, v, gr = graph_tensors(g, DT[vdt])
    s = FairSC(rp, ci, v, gr, k=2, h=g.h, normalized=normalized, prec=prec)
    # the oracle sees exactly the weights the library sees
    vals = v.to(torch.float64).cpu().numpy()
    W = sp.csr_matrix((vals, g.col_idx, g.row_ptr), shape=(g.n, g.n))
    op = SFairSCOperator(W, g.groups, g.h, normalized=normalized)
    assert s.sigma == pytest.approx(op.sigma, rel=1e-12)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((g.n, nvec))
    if prec == "mixed":
        w = w.astype(np.float32).astype(np.float64)
    got = s.apply_operator(torch.as_tensor(w, device="cuda")).double().cpu().numpy()
    ref = op.apply(w)
    scale = op.sigma * np.abs(w).max()
    err = np.abs(got - ref).max() / scale
    tol = 1e-13 if prec == "fp64" else 3e-6
    assert err < tol, (prec, vdt, nvec, err)
    s.close()
    return err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nvec", [1, 2, 3, 4])
def test_operator_msbm_shapes(built_lib, prec, nvec):
    g = msbm(3000, 5, 3, 40, seed=1)
    check_operator(g, prec, "f64", nvec)


@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_operator_value_dtypes(built_lib, vdt):
    g = msbm(2500, 4, 2, 30, seed=2)
    for prec in ["fp64", "mixed"]:
        check_operator(g, prec, vdt, 4)


@pytest.mark.parametrize("h", [1, 2, 5, 10, 32])
def test_operator_group_counts(built_lib, h):
    g = msbm(4000, 3, h, 48, seed=3 + h, unequal=True)
    check_operator(g, "fp64", "f64", 2)
    check_operator(g, "mixed", "f32", 1)


def test_operator_unnormalized_extension(built_lib):
    g = msbm(2000, 4, 3, 36, seed=9)
    check_operator(g, "fp64", "f64", 4, normalized=False)
    check_operator(g, "mixed", "f32", 2, normalized=False)


def test_operator_ragged_and_tiny(built_lib):
    # n not a multiple of 32, tiny graphs, a dense block and a path (degree 1-2 rows)
    rng = np.random.default_rng(4)
    for n in [37, 101, 1000 + 13]:
        A = np.triu((rng.random((n, n)) < 0.2) * rng.uniform(0.1, 2.0, (n, n)), 1)
        for i in range(n - 1):
            A[i, i + 1] = max(A[i, i + 1], 0.5)
        W = A + A.T
        groups = rng.integers(0, 3, n)
        groups[:3] = [0, 1, 2]
        g = graph_from_dense(W, groups)
        check_operator(g, "fp64", "f64", 3)
        check_operator(g, "mixed", "f32", 4)
    P = np.zeros((300, 300))
    for i in range(299):
        P[i, i + 1] = P[i + 1, i] = 1.0
    g = graph_from_dense(P, np.arange(300) % 2)
    check_operator(g, "fp64", "f64", 1)


def test_operator_high_degree_rows(built_lib):
    """Rows far longer than a warp (degree ~ 380, the n = 2,000 workload's density)."""
    from msbm import configs

    g = configs.msbm_n2000_k5_h2()["graph"]
    check_operator(g, "fp64", "f64", 4)
    check_operator(g, "mixed", "f64", 1)


def test_operator_many_ctas_large(built_lib):
    """A graph large enough to use every SM (n = 200,000, degree 32)."""
    g = msbm(200_000, 20, 5, 32, seed=11, unequal=True)
    check_operator(g, "fp64", "bf16", 4)
    check_operator(g, "mixed", "bf16", 4)


def test_operator_host_buffers(built_lib):
    """Host (CPU) tensors go through the same C call with copies in and out."""
    from paper_2210_16435_gb300.solver import FairSC
    from paper_2210_16435_gb300 import binding as B

    g = msbm(1500, 3, 2, 20, seed=12)
    rp, ci, v, gr = graph_tensors(g, torch.float64, device="cpu")
    s = FairSC(rp, ci, v, gr, k=2, h=2, prec="fp64")
    w = torch.randn(g.n, dtype=torch.float64)
    out = torch.empty_like(w)
    B.sfairsc_apply_operator(s.ctx, w.data_ptr(), out.data_ptr(), 1)
    ref = operator_from_graph(g).apply(w.numpy())
    assert np.abs(out.numpy() - ref).max() < 1e-12 * s.sigma * w.abs().max().item()
