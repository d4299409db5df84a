"""Failure paths of the C ABI, made on the host (no GPU fault, trap or hang).

NOT_CONVERGED: a restart budget of one cycle at a tolerance the cycle cannot
reach; the outputs are still written.
SHIFT: a Hotelling shift below lambda_k (Prop. 3.3 needs sigma > lambda_k), so
the eigenvalue sigma of range(C) (Prop. 3.2) appears among the k smallest.
DEVICE_TIMEOUT: the fault-injection option makes the first operator launch wait
on a device flag that nothing sets; the wait gives up after the short limit, the
kernel returns, the call reports DEVICE_TIMEOUT, and the next solve on the same
context is correct.
"""
import numpy as np
import pytest
import torch

from conftest import graph_tensors
from msbm import category_probabilities, cell_sizes_equal, sample_msbm
from oracle import fairsc

pytestmark = pytest.mark.gpu


def _graph(n, k, h, deg, seed):
    cells = cell_sizes_equal(n, k, h)
    return sample_msbm(cells, category_probabilities(cells, deg, (0.5, 0.25, 0.15, 0.10)), seed=seed)


def test_not_converged_after_restart_budget(built_lib):
    from paper_2210_16435_gb300.solver import FairSC

    g = _graph(4000, 16, 4, 40, 21)
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=16, h=4, prec="fp64", tol=1e-13, max_restarts=1)
    lam, H, _, info = s.solve(want_labels=False, allow_not_converged=True)
    s.close()
    assert s.status == -7 and info["status"] == -7
    assert info["restarts"] == 1
    assert info["max_resid"] > 1e-13
    lam = lam.cpu().numpy()
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(H.cpu().numpy()))
    assert np.all(np.diff(lam) >= -1e-9)


def test_shift_below_lambda_k_is_reported(built_lib):
    from paper_2210_16435_gb300.solver import FairSC
    from paper_2210_16435_gb300.binding import SFairSCError

    g = _graph(2000, 10, 5, 60, 22)
    k = 10
    lref, *_ = fairsc.sfairsc_dense(g.to_scipy(), g.groups, 5, k)
    sigma = 0.5 * lref[k - 1]
    assert sigma > lref[0] + 1e-3
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=k, h=5, prec="fp64", block=4, sigma=sigma)
    with pytest.raises(SFairSCError) as e:
        s.solve(want_labels=False)
    assert e.value.status == -8
    s.close()


def test_device_wait_timeout_then_clean_solve(built_lib):
    from paper_2210_16435_gb300.solver import FairSC
    from paper_2210_16435_gb300.binding import SFairSCError

    g = _graph(600, 3, 2, 30, 23)
    k = 3
    rp, ci, v, gr = graph_tensors(g)
    s = FairSC(rp, ci, v, gr, k=k, h=2, prec="fp64", wait_limit_us=2000, fault_inject=1)
    with pytest.raises(SFairSCError) as e:
        s.solve(want_labels=False)
    assert e.value.status == -11
    # the hook is spent; the counters were reset: the same context solves correctly
    lam, _, _, info = s.solve(want_labels=False)
    s.close()
    assert info["status"] == 0
    lref, *_ = fairsc.sfairsc_dense(g.to_scipy(), g.groups, 2, k)
    assert np.abs(lam.cpu().numpy() - lref).max() <= 1e-8
    torch.cuda.synchronize()
