"""The experiments' m-SBM (Exp. 1, App. C): s-FairSC on the GPU against FairSC (Algorithm 2).

Graphs: k = 5 equal clusters, h in {2, 5, 10} equal groups, edge probabilities
(a, b, c, d) = (10, 7, 4, 1) (log n / n)^(2/3) with a same cluster & same group
> b other cluster & same group > c same cluster & other group > d, so that
edges follow the groups more than the clusters.  The paper reports that SC
fails to recover the fair ground truth while FairSC and s-FairSC do, with the
same error rate (eq. err).  Checked: the library's eigenvalues equal FairSC's
(dense Algorithm 2 in the oracle), its k-means labels give FairSC's error rate
and balance (eq. bal) to within two vertices, plain SC on the same graph
(h = 1) does clearly worse on both, and the oracle's k-means on the library's
H gives the library's labels.
"""
import numpy as np
import pytest
import torch

from conftest import graph_tensors
from msbm import configs
from oracle import fairsc
from oracle.kmeans import kmeans as oracle_kmeans
from oracle.metrics import average_balance, error_rate

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,h", [(1000, 2), (1000, 5), (1000, 10), (2000, 5)])
def test_paper_msbm_sfairsc_matches_fairsc(built_lib, n, h):
    from paper_2210_16435_gb300.solver import FairSC

    c = configs.paper_msbm(n, h)
    g, k = c["graph"], c["k"]
    lref, Href = fairsc.fairsc_dense(g.to_scipy(), g.groups, h, k)
    lab_ref, _, _ = oracle_kmeans(Href, k, seed=0, n_init=10, max_iter=300)
    err_ref = error_rate(lab_ref, g.clusters, k)
    rp, ci, v, gr = graph_tensors(g)
    for prec, tol in (("fp64", 1e-6), ("mixed", 1e-4)):
        s = FairSC(rp, ci, v, gr, k=k, h=h, prec=prec, kmeans_n_init=10, kmeans_max_iter=300)
        lam, H, lab, info = s.solve()
        s.close()
        lam, H, lab = lam.cpu().numpy(), H.cpu().numpy(), lab.cpu().numpy()
        big = np.abs(lref) >= 1e-3 * info["sigma"]
        rel = np.where(big, np.abs(lam - lref) / np.maximum(np.abs(lref), 1e-300), np.abs(lam - lref) / info["sigma"])
        assert rel.max() <= tol, (prec, rel.max())
        err = error_rate(lab, g.clusters, k)
        assert abs(err - err_ref) <= 4.0 / n, (prec, err, err_ref)
        assert abs(average_balance(lab, g.groups, k, h) - average_balance(lab_ref, g.groups, k, h)) <= 0.05
        if prec == "fp64":
            mine, _, _ = oracle_kmeans(H, k, seed=0, n_init=10, max_iter=300)
            assert np.array_equal(mine, lab)
    # plain SC (Algorithm 1, the same graph without the constraint) splits by group instead
    s = FairSC(rp, ci, v, gr * 0, k=k, h=1, prec="fp64", kmeans_n_init=10, kmeans_max_iter=300)
    _, _, lab_sc, _ = s.solve()
    s.close()
    lab_sc = lab_sc.cpu().numpy()
    assert error_rate(lab_sc, g.clusters, k) > err_ref + 0.3
    assert average_balance(lab_sc, g.groups, k, h) < average_balance(lab_ref, g.groups, k, h) - 0.2
    torch.cuda.synchronize()
