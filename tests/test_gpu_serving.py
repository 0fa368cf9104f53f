"""Continuous-batching server: results equal the oracle's for each request
alone, whatever the mix (tolerance 0)."""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_served_results_equal_each_request_alone(oracle):
    import torch
    assert torch.cuda.is_available()
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import serving as SV
    reqs = [r for r in I.serving_requests(40) if r.n <= 10][:8]
    prepared = {}
    for k, r in enumerate(reqs):
        w = r.workload()
        w.t_end = min(w.t_end, 2e-3)
        prepared[r.rid] = w
        r.arrival = 0.002 * k          # arrivals while earlier ones run
    srv = SV.Server(budget_bytes=2e9, max_slots=3, slice_periods=7, keep_counts=True)
    try:
        recs = srv.serve(reqs, prepared)
    finally:
        srv.close()
    assert sorted(r.rid for r in recs) == sorted(r.rid for r in reqs)
    for rec in recs:
        w = prepared[rec.rid]
        o, _, _ = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
        assert np.array_equal(rec.counts, o), rec.rid
        assert rec.latency >= 0
