"""Host-side logic of the serving loop and the autotuner (no GPU)."""
import json

import numpy as np

from paper_2009_12457_gb300 import autotune, serve


def test_poisson_trace_is_seeded_and_has_the_right_rate():
    a = serve.poisson_trace(1000.0, 5.0, seed=5)
    b = serve.poisson_trace(1000.0, 5.0, seed=5)
    assert np.array_equal(a, b)
    assert np.all(np.diff(a) > 0) and a[-1] < 5.0
    assert abs(len(a) - 5000) < 5 * np.sqrt(5000)  # within 5 sigma of the mean
    assert not np.array_equal(a, serve.poisson_trace(1000.0, 5.0, seed=6))


def test_latency_summary():
    reqs = []
    for i in range(100):
        r = serve.Request(i, ("g", i % 3), arrival=float(i))
        r.finish = float(i) + 0.001 * (i + 1)
        r.batch_size = 1 + i % 4
        reqs.append(r)
    s = serve.latency_summary(reqs)
    assert abs(s["p50_ms"] - 50.5) < 1.0
    assert abs(s["p99_ms"] - 99.0) < 1.5
    assert s["requests"] == 100 and s["mean_batch"] == 2.5
    assert abs(s["graphs_per_s"] - 100 / (99.1 - 0.0)) < 1e-6


def test_size_classes_group_similar_graphs():
    a = autotune.size_class({"n": 1 << 20, "m": 16 << 20})
    b = autotune.size_class({"n": (1 << 20) + 5, "m": (16 << 20) + 999})
    c = autotune.size_class({"n": 1 << 20, "m": 64 << 20})
    assert a == b and a != c


def test_autotuner_cache_round_trip(tmp_path):
    path = tmp_path / "t.json"
    t = autotune.Autotuner(cache_path=str(path))
    t.cache["m2^20_d2^5"] = {"p": 4, "kernel": "hashmap", "hash_threshold": 0, "chunk": 256,
                              "count_ms": 1.0}
    t._save()
    again = autotune.Autotuner(cache_path=str(path))
    assert again.cache == json.loads(path.read_text())
    opts = autotune.Autotuner.opts(again.cache["m2^20_d2^5"])
    assert opts.p == 4 and opts.kernel == 2 and opts.chunk == 256


def test_coverage_metric_by_hand():
    from paper_2009_12457_gb300 import workload
    # costs: task 3 is the heaviest, then 0, then 2, then 1
    cost = np.array([5.0, 1.0, 2.0, 9.0])
    perfect = np.array([5.0, 1.0, 2.0, 9.0])
    assert workload.coverage(perfect, cost, xs=(1, 2, 3, 4)) == {1: 0.25, 2: 0.5, 3: 0.75, 4: 1.0}
    # an estimate that ranks the heaviest task last needs the whole list for x = 1
    bad = np.array([4.0, 3.0, 2.0, 1.0])
    assert workload.coverage(bad, cost, xs=(1,))[1] == 1.0
    # ties keep Alg. 4 order: all-equal estimates scan tasks 0,1,2,3
    flat = np.zeros(4)
    assert workload.coverage(flat, cost, xs=(1, 2))[1] == 1.0
    assert workload.coverage(flat, cost, xs=(1, 2))[2] == 1.0


def test_spearman_by_hand():
    from paper_2009_12457_gb300 import workload
    assert workload.spearman(np.array([1, 2, 3, 4]), np.array([10, 20, 30, 40])) == 1.0
    assert workload.spearman(np.array([1, 2, 3, 4]), np.array([4, 3, 2, 1])) == -1.0
    # ties take average ranks: x = [1, 1, 2], y = [1, 2, 3] -> ranks (0.5, 0.5, 2) vs (0, 1, 2)
    r = workload.spearman(np.array([1, 1, 2]), np.array([1, 2, 3]))
    assert abs(r - 0.8660254037844386) < 1e-12


def test_estimates_from_a_plan():
    from paper_2009_12457_gb300 import workload
    plan = {"cuts": np.array([0, 2, 5]), "block_nnz": np.array([[3, 4], [0, 6]]),
            "tasks": np.array([[0, 0, 0], [0, 0, 1], [0, 1, 1], [1, 1, 1]]),
            "exec_time": np.array([4.5, 6.0, 8.0, 12.0])}
    e = workload.estimates(plan)
    assert np.allclose(e["nnz"], [9, 3 + 4 + 4, 4 + 6 + 4, 18])
    assert np.allclose(e["degree"], [4.5, 1.5 + 2 + 2, 2 + 2 + 2, 6])
    assert np.allclose(e["density"], [3 * 0.75, 0.75 + 4 / 6 + 4 / 6, 4 / 6 + 6 / 9 + 4 / 6, 3 * 6 / 9])
    assert np.allclose(e["bbtc"], [4.5, 6.0, 8.0, 12.0])


def test_opts_keep_output_arrays_alive():
    """bbtc_opts holds raw pointers; make_opts must keep the arrays behind them
    alive, so that a temporary output is not freed before the library writes it."""
    import gc
    import weakref
    import numpy as np
    import paper_2009_12457_gb300 as bb
    arr = np.zeros(4096, dtype=np.uint64)
    ref = weakref.ref(arr)
    opts = bb.make_opts(p=2, per_graph_out=arr)
    del arr
    gc.collect()
    assert ref() is not None and opts.per_graph_out == ref().ctypes.data
    del opts
    gc.collect()
    assert ref() is None
