"""Eigenvector-level backward (a loss on H and on the eigenvalues) against the oracle.

Small graphs: element by element against the oracle's closed form, which sums over every
eigenpair of Algorithm 2's pencil (dense), through the C ABI and through the autograd
function.  Homogeneity: for a loss linear in H, sum_e w_e g_e = -loss / 2 (H(cW) = H(W) / sqrt(c)).
At n = 20,000: a directional central difference of the loss with the oracle's own Lanczos
(tol 1e-13, sign rule applied) against the library's gradient.
"""
import numpy as np
import pytest
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_equal, sample_msbm
from oracle import gradient

pytestmark = pytest.mark.gpu


def graph(n, k, h, deg, seed):
    cells = cell_sizes_equal(n, k, h)
    return sample_msbm(cells, category_probabilities(cells, deg, (0.5, 0.25, 0.15, 0.10)), seed=seed)


@pytest.mark.parametrize("n,k,h,seed", [(240, 3, 2, 1), (400, 4, 3, 2), (300, 3, 1, 3)])
def test_vector_gradient_matches_oracle(built_lib, n, k, h, seed):
    from paper_2210_16435_gb300.solver import FairEmbedding, FairSC

    g = graph(n, k, h, 30, seed)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, k))
    gl = rng.standard_normal(k)
    gref, lref, Href = gradient.vector_gradient(g.row_ptr, g.col_idx, g.values, g.groups, h, k, G, gbar_lam=gl)
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=k, h=h, prec="fp64", tol=1e-12)
    lam, H, _, _ = s.solve(want_labels=False)
    assert np.abs(H.cpu().numpy() - Href).max() <= 1e-8 * np.abs(Href).max()  # same signs, same vectors
    got, _, it, rr = s.backward_vectors(torch.as_tensor(G), torch.as_tensor(gl))
    s.close()
    assert rr <= 1e-10 and it < 1000
    scale = np.abs(gref).max()
    assert np.abs(got.cpu().numpy() - gref).max() <= 1e-6 * scale
    # the same through autograd: loss = sum(G * H) + gl . lambda
    vals = v.clone().requires_grad_(True)
    lam_t, H_t = FairEmbedding.apply(vals, rp, ci, gr, k, h, None, {"prec": "fp64", "tol": 1e-12})
    loss = (H_t * torch.as_tensor(G, device="cuda")).sum() + (lam_t * torch.as_tensor(gl, device="cuda")).sum()
    loss.backward()
    assert np.abs(vals.grad.cpu().numpy() - gref).max() <= 1e-6 * scale


def test_vector_gradient_homogeneity(built_lib):
    from paper_2210_16435_gb300.solver import FairSC

    g = graph(3000, 5, 3, 40, 4)
    k = 5
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=k, h=3, prec="fp64", tol=1e-12)
    _, H, _, _ = s.solve(want_labels=False)
    G = torch.randn(g.n, k, dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    got, _, _, rr = s.backward_vectors(G)
    s.close()
    lhs = float(np.dot(g.values, got.cpu().numpy()))
    rhs = -0.5 * float((G * H.cpu()).sum())
    assert rr <= 1e-10
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs)


def test_vector_gradient_directional_fd_n20k(built_lib):
    from oracle.lanczos import thick_restart_lanczos
    from oracle.problem import adjacency
    from oracle.sfairsc import SFairSCOperator, embed, operator_from_graph
    from paper_2210_16435_gb300.solver import FairSC

    g = graph(20_000, 4, 2, 40, 5)
    k = 4
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=k, h=2, prec="fp64", tol=1e-12)
    lam, H, _, _ = s.solve(want_labels=False)
    rng = np.random.default_rng(6)
    G = rng.standard_normal((g.n, k))
    got, _, _, rr = s.backward_vectors(torch.as_tensor(G))
    s.close()
    got = got.cpu().numpy()
    op0 = operator_from_graph(g)
    # a random direction on the undirected weights (both CSR entries move together)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    key_lo = np.minimum(rows, g.col_idx) * g.n + np.maximum(rows, g.col_idx)
    _, inv = np.unique(key_lo, return_inverse=True)
    du = rng.standard_normal(inv.max() + 1)[inv]
    directional = float(np.dot(du, got))

    def loss(step):
        vals = g.values + step * du
        op = SFairSCOperator(adjacency(g.row_ptr, g.col_idx, vals), g.groups, 2, sigma=op0.sigma)
        lam2, X2, _ = thick_restart_lanczos(op.apply, g.n, k + 1, tol=1e-13, anorm=op.sigma, seed=0)
        return float(np.sum(G * embed(op, X2[:, :k])))

    eps = 1e-5
    fd = (loss(eps) - loss(-eps)) / (2 * eps)
    assert abs(fd - directional) <= 1e-4 * abs(directional), (fd, directional)


def test_vector_backward_status(built_lib):
    """A MIXED context is refused (its eigenvectors are too rough to deflate with); a conjugate
    gradient cut short reports NOT_CONVERGED."""
    from paper_2210_16435_gb300.binding import SFairSCError
    from paper_2210_16435_gb300.solver import FairSC

    g = graph(400, 4, 3, 30, 8)
    rp, ci, v, gr = graph_tensors(g)
    G = torch.randn(g.n, 4, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    s = FairSC(rp, ci, v, gr, k=4, h=3, prec="mixed")
    s.solve(want_labels=False)
    with pytest.raises(SFairSCError) as e:
        s.backward_vectors(G)
    assert e.value.status == -12  # UNSUPPORTED
    s.close()
    s = FairSC(rp, ci, v, gr, k=4, h=3, prec="fp64", tol=1e-12)
    s.solve(want_labels=False)
    with pytest.raises(SFairSCError) as e:
        s.backward_vectors(G, max_iter=1)
    assert e.value.status == -7  # NOT_CONVERGED
    _, _, it, rr = s.backward_vectors(G)
    s.close()
    assert rr <= 1e-10 and it < 1000
