"""Serving loop: each request's count is the oracle's and the same alone and in the
mix (GPU)."""
import time

import numpy as np
import pytest

import graphgen
import oracle
import paper_2009_12457_gb300 as bb
from paper_2009_12457_gb300 import serve
from paper_2009_12457_gb300.autotune import Autotuner

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def request_key(rid, scales=(8, 9, 10, 11, 12, 13), seeds=6):
    """Scale and graph seed of request rid, from the counter-based draw of its id."""
    d = graphgen.draw(5, 9, rid)
    return (scales[d % len(scales)], (d >> 32) % seeds)


_SOURCE_CACHE = {}


def source(key):
    if key not in _SOURCE_CACHE:
        scale, seed = key
        _SOURCE_CACHE[key] = graphgen.rmat(scale, 16, 1000 + seed)
    return _SOURCE_CACHE[key]


def test_served_counts_equal_counts_alone():
    arrivals = serve.poisson_trace(400.0, 1.5, seed=5)
    keys = [request_key(i) for i in range(len(arrivals))]
    alone, exact = {}, {}
    for k in set(keys):
        with bb.Graph(*source(k)) as g:
            alone[k] = g.count(p=2)
        n, rp, ci = source(k)
        pr = oracle.prepare(n, rp, ci)
        exact[k] = oracle.tc_intersect(n, pr["rowptr"], pr["colidx"])
    assert alone == exact
    # a budget of a few graphs forces evictions
    srv = serve.Server(source, device_budget_bytes=12 << 20, max_batch=32, workers=2, p=2)
    try:
        reqs = serve.run_open_loop(srv, keys, arrivals)
    finally:
        srv.close()
    assert len(reqs) == len(keys)
    assert all(r.status == 0 for r in reqs)
    wrong = [(r.rid, r.key, r.count, exact[r.key], r.batch_size) for r in reqs
             if r.count != exact[r.key]]
    assert not wrong, wrong[:10]
    assert srv.evictions > 0 and srv.hits > 0
    assert max(r.batch_size for r in reqs) > 1  # requests really shared launches
    summary = serve.latency_summary(reqs)
    assert summary["p99_ms"] >= summary["p50_ms"] > 0


def test_serial_baselines_match():
    keys = [request_key(i) for i in range(12)]
    counts, rate = serve.serial_baseline(source, keys, p=2)
    cached, rate_cached = serve.serial_cached_baseline(source, keys, p=2)
    assert counts == cached
    for k, c in zip(keys, counts):
        with bb.Graph(*source(k)) as g:
            assert c == g.count(p=3)
    assert rate > 0 and rate_cached > 0


def test_device_memory_report():
    mem = bb.bbtc_device_memory(torch.cuda.current_device())
    free, total = torch.cuda.mem_get_info()
    assert 0 < mem["total"] == total
    assert mem["pool_used"] <= mem["pool_reserved"]
    assert mem["available"] >= free - (1 << 30)


def test_autotuner_choice_gives_the_same_count(tmp_path):
    n, rp, ci = graphgen.rmat(14, 16, 3)
    tuner = Autotuner(cache_path=str(tmp_path / "tune.json"), repeats=1)
    with bb.Graph(n, rp, ci) as g:
        ref = g.count(p=1)
        choice = tuner.tune(g, p_choices=(1, 2, 4))
        assert choice["p"] in (1, 2, 4) and choice["count_ms"] > 0
        assert bb.bbtc_count(g.handle, Autotuner.opts(choice)) == ref
    again = Autotuner(cache_path=str(tmp_path / "tune.json"))
    with bb.Graph(n, rp, ci) as g:
        assert again.choice(g, tune_if_missing=False)["p"] == choice["p"]


def test_a_bad_graph_fails_only_its_own_requests():
    """A request whose graph cannot be prepared (an out-of-range column) fails with
    its own status; the requests that share its batch are still counted, and the
    server keeps serving."""
    bad_rp = np.array([0, 1, 2], dtype=np.int64)
    bad_ci = np.array([1, 5], dtype=np.int32)      # 5 is outside [0, 2)

    def mixed_source(key):
        return (2, bad_rp, bad_ci) if key == "bad" else source(key)

    good = [request_key(i) for i in range(40)]
    keys = good[:20] + ["bad"] + good[20:] + ["bad"]
    alone = {}
    for k in set(good):
        with bb.Graph(*source(k)) as g:
            alone[k] = g.count(p=2)
    srv = serve.Server(mixed_source, device_budget_bytes=1 << 30, max_batch=64, workers=1, p=2)
    try:
        reqs = [serve.Request(i, k, time.perf_counter()) for i, k in enumerate(keys)]
        with srv.cv:  # one burst; batches form as its graphs become ready
            for r in reqs:
                srv.submit(r)
        srv.drain(len(reqs))
        later = [serve.Request(len(keys) + i, k, time.perf_counter())
                 for i, k in enumerate(good[:5])]
        for r in later:                              # still serving
            srv.submit(r)
        srv.drain(len(reqs) + len(later))
    finally:
        srv.close()
    for r in reqs:
        if r.key == "bad":
            assert r.status != 0
        else:
            assert r.status == 0 and r.count == alone[r.key], (r.key, r.status, r.count)
    assert srv.errors
    assert all(r.status == 0 and r.count == alone[r.key] for r in later)
