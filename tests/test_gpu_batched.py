"""Batched solve and the (b, nb) autotuner, through the C ABI.

* Uneven batch (sizes from 1 to 1030, longest-first over lanes), run as one captured
  CUDA graph: every matrix's eigenvalues agree with the oracle within the acceptance
  bound, and every Q meets the orthogonality and residual bounds.  A second run with
  the same buffers replays the graph and gives the same results bit for bit.
* Autotuner: returns a candidate pair, writes it to the JSON cache, answers the
  second call from the cache, and a plan created with b = nb = 0 picks the cached
  pair when EVD_AUTOTUNE_CACHE names the file.
"""
import json
import os
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


def test_batched_uneven_sizes_match_oracle(evd):
    sizes = [3, 17, 64, 100, 257, 300, 513, 600, 1030, 40, 8, 1, 129, 700]
    mats = [inputs.goe(n, 8000 + i) for i, n in enumerate(sizes)]
    batch = evd.Batch(sizes, job="V")
    results = []
    for rep in range(2):
        for A, t in zip(mats, batch.A):
            t.copy_(torch.from_numpy(A))
        batch.run()
        torch.cuda.synchronize()
        assert evd.batched_last_graph()
        results.append(([w.cpu().numpy() for w in batch.w], [q.cpu().numpy() for q in batch.Q]))
    for i in range(len(sizes)):
        assert np.array_equal(results[0][0][i], results[1][0][i])
        assert np.array_equal(results[0][1][i], results[1][1][i])
    for A, w, Q in zip(mats, results[1][0], results[1][1]):
        n = A.shape[0]
        w_ref, _ = oracle.eigh(A, want_vectors=False) if n > 8 else oracle.jacobi(A)
        m = oracle.metrics(A, w, Q, w_ref=np.sort(w_ref))
        acc = oracle.acceptance(n, float(np.max(np.abs(w_ref))) if n else 0.0)
        assert m["dlam"] <= acc["dlam"], (n, m)
        assert m["orth_max"] <= acc["orth_max"], (n, m)
        assert m["resid"] <= acc["resid"], (n, m)


def test_autotune_cache_and_plan_lookup(evd, tmp_path):
    path = str(tmp_path / "tune.json")
    n = 600
    b, nb = evd.autotune(n, job="V", cache_path=path)
    assert (b, nb) in [(32, 32), (32, 64), (32, 128), (64, 64), (64, 128), (128, 128)]
    text = open(path).read()
    entries = json.loads(text)
    assert entries[-1]["n_bucket"] == 512 and entries[-1]["b"] == b and entries[-1]["nb"] == nb
    t0 = time.perf_counter()
    assert evd.autotune(n, job="V", cache_path=path) == (b, nb)  # from the cache
    assert time.perf_counter() - t0 < 0.5
    os.environ["EVD_AUTOTUNE_CACHE"] = path
    try:
        plan = evd.Plan(n, job="V")
        assert (plan.b, plan.nb) == (b, nb)
        plan.close()
    finally:
        del os.environ["EVD_AUTOTUNE_CACHE"]
