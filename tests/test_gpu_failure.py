"""Failure detection without a fault: every bounded device wait gives up, reports
EVD_ERR_TIMEOUT through the plan's status word, and lets its kernel return.

evd_wait_selftest runs one wait that never completes (a progress flag nothing
publishes, a grid barrier short of one CTA, an mbarrier nobody arrives at while the
CTA holds tensor memory) with a short limit.  The status comes back with the
location code, the call returns well within a second or two, and a solve on the
same plan afterwards is correct: the context and the plan's barrier state survive.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2511_16174_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def evd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_16174_gb300 import evd as m
    return m


@pytest.mark.parametrize("kind,where", [(0, 9901), (1, 9902), (2, 9903)])
def test_wait_that_runs_out_reports_timeout_and_returns(evd, kind, where):
    n = 300
    plan = evd.Plan(n, job="V", b=32, nb=64)
    ws = plan.workspace()
    assert plan.status() == (0, 0)
    t0 = time.perf_counter()
    plan.wait_selftest(kind)
    code, info = plan.status()  # synchronizes the plan's stream
    elapsed = time.perf_counter() - t0
    assert code == 7 and info == where, (code, info)  # EVD_ERR_TIMEOUT
    assert elapsed < 10.0
    assert plan.status() == (0, 0)  # cleared on read
    # the same plan solves correctly afterwards (SBR's cooperative panel kernel uses
    # the grid barrier whose counters the timed-out barrier left behind)
    A = inputs.goe(n, 9900 + kind)
    Ad = evd.empty_colmajor(n, n)
    Ad.copy_(torch.from_numpy(A))
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Q = evd.empty_colmajor(n, n)
    plan.syevd(Ad, w, Q, ws)
    plan.check("solve after a timed-out wait")
    w_ref, _ = oracle.eigh(A, want_vectors=False)
    m = oracle.metrics(A, w.cpu().numpy(), Q.cpu().numpy(), w_ref=w_ref)
    acc = oracle.acceptance(n, float(np.max(np.abs(w_ref))))
    assert m["dlam"] <= acc["dlam"] and m["orth_max"] <= acc["orth_max"] and m["resid"] <= acc["resid"], m
