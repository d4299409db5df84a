"""Pins of the oracle with a dense constraint matrix F (the random-Laplacian experiment, Exp. 4).

The fair SC problem min tr(H^T L H), H^T D H = I, F^T H = 0 (eq. normal-prob-fair)
is stated for any F of full column rank; the experiments' random Laplacian
uses a random dense F.  Checked: Algorithm 2 (explicit nullspace basis, dense)
and s-FairSC (eq. asigma, dense and matrix-free with the own Lanczos) give one
spectrum (Prop. 3.3); the invariants F^T H = 0 and H^T D H = I hold; only
range(F) matters (F and F R for an invertible R give the same problem), so the
group constraints passed as a dense F times R reproduce the label path; and a
graph without structure still has lambda_1 > 0 once a random F removes
D^{1/2} 1 from the feasible set (unlike the group constraints, Sec. 3.3).
"""
import numpy as np
import pytest

from msbm import configs, graph_from_dense
from oracle import fairsc, problem
from oracle.sfairsc import SFairSCOperator, smallest_eigenpairs


@pytest.mark.parametrize("n,h,seed", [(300, 5, 0), (500, 3, 1), (400, 2, 2)])
def test_dense_f_formulations_agree(n, h, seed):
    c = configs.random_laplacian(n, h, seed=seed)
    g, F = c["graph"], c["F"]
    W = g.to_scipy()
    k = 5
    l1, H1 = fairsc.fairsc_dense(W, None, h, k, F=F)
    l3, H3, _, _, _ = fairsc.sfairsc_dense(W, None, h, k, F=F)
    op = SFairSCOperator(W, None, h, F=F)
    l4, X4 = smallest_eigenpairs(op, k, tol=1e-13, method="lanczos")
    np.testing.assert_allclose(l3, l1, atol=1e-12)
    np.testing.assert_allclose(l4, l1, atol=1e-11)
    d = problem.degrees(W)
    for H in (H1, H3):
        np.testing.assert_allclose(F.T @ H, 0.0, atol=1e-11)
        np.testing.assert_allclose((H.T * d) @ H, np.eye(k), atol=1e-11)
    # lambda_1 > 0: D^{1/2} 1 is not in null(C^T) for a random F
    assert l1[0] > 1e-3


def test_only_range_of_f_matters_and_groups_as_dense_f():
    rng = np.random.default_rng(5)
    n, h, k = 240, 4, 4
    A = (rng.random((n, n)) < 0.1) * rng.uniform(0.5, 2.0, (n, n))
    Wd = np.triu(A, 1)
    Wd = Wd + Wd.T
    for i in range(n):
        j = (i + 1) % n
        Wd[i, j] = Wd[j, i] = max(Wd[i, j], 0.2)
    groups = rng.integers(0, h, n)
    groups[:h] = np.arange(h)
    g = graph_from_dense(Wd, groups)
    W = g.to_scipy()
    _, Fg, _ = problem.fairness_constraints(groups, h)
    R = rng.standard_normal((h - 1, h - 1)) + 3 * np.eye(h - 1)
    l_lab, _ = fairsc.fairsc_dense(W, groups, h, k)
    l_dense, _ = fairsc.fairsc_dense(W, None, h, k, F=Fg @ R)
    np.testing.assert_allclose(l_dense, l_lab, atol=1e-12)
    op = SFairSCOperator(W, None, h, F=Fg @ R)
    op_lab = SFairSCOperator(W, groups, h)
    w = rng.standard_normal((n, 3))
    np.testing.assert_allclose(op.apply(w), op_lab.apply(w), atol=1e-12)
