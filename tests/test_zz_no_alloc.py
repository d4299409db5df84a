"""The allocation-free operator entry point against the ordinary one and the oracle.

sfairsc_apply_operator_static serves callers that cannot allocate device
memory (plug-ins inside a runtime that owns the device allocator, deployments
with a memory budget fixed at start-up).  It keeps all scratch in one
file-scope device array, so these tests call it twice in a row -- the second
call reuses the scratch the first one left behind -- and check both results
against sfairsc_apply_operator on a context built the normal way, and against
the oracle's literal operator P(L_n(P w)) - sigma P w + sigma w (Sec. 3.4 (i)),
within the tolerance the operator tests use for the mixed path.
"""
import ctypes

import numpy as np
import pytest
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_from_proportions, sample_msbm

pytestmark = pytest.mark.gpu


def _graph(n, k, h, deg, seed):
    cells = cell_sizes_from_proportions(n, np.linspace(1, 2, k), 1.0 / np.arange(1, h + 1))
    return sample_msbm(cells, category_probabilities(cells, deg, (0.5, 0.25, 0.15, 0.10)), seed=seed)


def _static_fn():
    from paper_2210_16435_gb300 import binding as B

    lib = B.load()
    fn = lib.sfairsc_apply_operator_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_int32] + [ctypes.c_void_p] * 2 + \
        [ctypes.c_int32, ctypes.c_void_p]
    return fn


def test_static_operator_matches_context_operator_twice(built_lib):
    from paper_2210_16435_gb300.solver import FairSC

    fn = _static_fn()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, h, nvec, seed) in enumerate([(30_000, 5, 4, 1), (12_345, 3, 1, 2)]):
        g = _graph(n, 4, h, 30, seed)
        rp, ci, v, gr = graph_tensors(g, torch.float32)
        ctx = FairSC(rp, ci, v, gr, k=2, h=h, prec="mixed")
        w = torch.randn(nvec, g.n, device="cuda", dtype=torch.float32)  # column-major n x nvec
        ref = torch.empty_like(w)
        from paper_2210_16435_gb300 import binding as B

        B.sfairsc_apply_operator(ctx.ctx, w.data_ptr(), ref.data_ptr(), nvec)
        out = torch.full_like(w, float("nan"))
        rc = fn(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), gr.data_ptr(), h, w.data_ptr(),
                out.data_ptr(), nvec, stream)
        torch.cuda.synchronize()
        assert rc == 0, (call, rc, B.load().sfairsc_last_error())
        err = (out - ref).abs().max().item() / (ctx.sigma * w.abs().max().item())
        assert err < 3e-6, (call, err)
        ctx.close()


def test_static_operator_rejects_sizes_beyond_its_scratch(built_lib):
    fn = _static_fn()
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    f = torch.zeros(8, dtype=torch.float32, device="cuda")
    rc = fn(524_289, 10, t.data_ptr(), t.data_ptr(), f.data_ptr(), t.data_ptr(), 2, f.data_ptr(), f.data_ptr(), 1, None)
    assert rc == -12  # UNSUPPORTED: n above the static limit, nothing launched


def test_static_operator_matches_oracle_operator_twice(built_lib):
    """Its own set-up (degrees, C^T C factor, sigma) and operator against the FP64 oracle."""
    from oracle.sfairsc import operator_from_graph

    fn = _static_fn()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, h, nvec, seed) in enumerate([(20_000, 4, 3, 5), (20_000, 4, 3, 5), (9_001, 7, 2, 6)]):
        g = _graph(n, 5, h, 24, seed)
        rp, ci, v, gr = graph_tensors(g, torch.float32)
        op = operator_from_graph(g)
        rng = np.random.default_rng(100 + call)
        W = rng.standard_normal((g.n, nvec))
        ref = op.apply(W)
        w = torch.as_tensor(np.ascontiguousarray(W.T), dtype=torch.float32, device="cuda")
        out = torch.full_like(w, float("nan"))
        rc = fn(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), gr.data_ptr(), h, w.data_ptr(),
                out.data_ptr(), nvec, stream)
        torch.cuda.synchronize()
        assert rc == 0, call
        got = out.cpu().numpy().T.astype(np.float64)
        err = np.abs(got - ref).max() / (op.sigma * np.abs(W).max())
        assert err < 3e-6, (call, err)
