"""The relax server on the GPU: requests that arrive while others run join
the batch, and every result is bitwise the same as the request relaxed by
itself (mmp_relax on its own context with the same shape)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests():
    from inputs import serve_requests
    from paper_2411_18194_gb300.serve import Request
    out = []
    for i, (t, w) in enumerate(serve_requests(40)):
        if max(w.problem.shape) <= 128:       # small grids keep the test short
            out.append(Request(i, w, 0.002 * len(out), torque_tol=5e-2, max_time=5e-12))
        if len(out) == 5:
            break
    return out


def test_served_results_equal_solo_results():
    from paper_2411_18194_gb300 import serve
    mixed = _requests()
    srv = serve.RelaxServer(budget_bytes=8e9, attempts_per_round=3, keep_results=True)
    done = srv.run(mixed)
    srv.close()
    assert len(done) == len(mixed) and srv.peak_members >= 2
    alone = serve.serve_one_at_a_time(_requests(), keep_results=True)
    by_id = {r.id: r for r in alone}
    for r in done:
        assert r.status == 0
        assert np.array_equal(r.result, by_id[r.id].result), r.workload.problem.shape
    st = serve.latency_stats(done)
    assert st["solves"] == len(mixed) and st["p99_s"] >= st["p50_s"] > 0
