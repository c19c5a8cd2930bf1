"""The benchmark workloads at full size against the oracle's stored values (GPU).

Every expected value here comes from tests/golden/, written by
tests/golden/make_golden.py from graphgen and the CPU oracle alone: the exact
triangle count of each workload (Sec. 2), the per-task counts of R-MAT scale 23
with every triangle placed in its task (Sec. 4.2, Alg. 4 order), the count of
each of the 4096 batched graphs, and the triangles at sampled vertices of the
Friendster-shaped graph. All comparisons are exact.
"""
import numpy as np
import pytest

import graphgen
import paper_2009_12457_gb300 as bb
from tests import goldens

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def rmat_s23():
    n, rp, ci = graphgen.rmat_s23()
    with bb.Graph(n, torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                  symmetric=True) as g:
        yield g


def test_rmat_s23_per_task_all_p_and_kernels(rmat_s23):
    want = goldens.config_counts()["rmat_s23_ef16_seed2"]
    per_task = goldens.rmat_s23_per_task()
    assert rmat_s23.info()["m"] == want["m"]
    for p in (4, 8, 16):
        total, tasks = per_task[p]
        assert total == want["triangles"]
        for kernel in ("auto", "hashmap", "intersect"):
            out = rmat_s23.count(p=p, kernel=kernel, per_task=True)
            assert out["total"] == want["triangles"], (p, kernel)
            assert np.array_equal(out["per_task"], tasks), (p, kernel)


def test_rmat_s23_resident_and_streamed(rmat_s23):
    want = goldens.config_counts()["rmat_s23_ef16_seed2"]["triangles"]
    for p in (1, 2):
        assert rmat_s23.count(p=p) == want
    # blocks streamed from pinned host memory through a 1 GB device pool
    assert rmat_s23.count(p=8, device_budget_bytes=1 << 30) == want
    assert rmat_s23.timings()["stream_rounds"] >= 2


def test_batch_4096_per_graph_counts():
    ref = goldens.batch4096()
    graphs = graphgen.batch_graphs(len(ref))
    assert [g[0] for g in graphs] == ref[:, 1].tolist()
    voff, rowptr, colidx = bb.batch_csr(graphs)
    want = ref[:, 3].astype(np.uint64)
    # one union handle, one counting launch for all 4096 graphs
    with bb.BatchGraph(vertex_offsets=voff, rowptr=torch.from_numpy(rowptr).cuda(),
                       colidx=torch.from_numpy(colidx).cuda(), symmetric=True) as u:
        for p in (1, 2):
            out = u.count(p=p, per_graph=True)
            assert out["total"] == int(want.sum())
            assert np.array_equal(out["per_graph"], want), p
    # separate handles counted together (each its own plan, one launch)
    sel = list(range(0, len(graphs), 16))
    hs = [bb.Graph(*graphs[g], symmetric=True) for g in sel]
    try:
        counts, stats = bb.bbtc_count_batch([h.handle for h in hs], bb.make_opts(p=0))
        assert not np.any(stats)
        assert np.array_equal(counts, want[sel])
        for h, g in zip(hs[:32], sel[:32]):
            assert h.info()["m"] == ref[g, 2]
    finally:
        for h in hs:
            h.close()


def test_friendster_shaped_total_vertices_and_streamed():
    want = goldens.config_counts().get("chunglu_friendster_seed3")
    if want is None:
        pytest.skip("no stored oracle count for the Friendster-shaped graph")
    n, rp, ci = graphgen.chunglu_friendster()
    d_rp, d_ci = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
    del rp, ci
    with bb.Graph(n, d_rp, d_ci, symmetric=True) as g:
        del d_rp, d_ci
        assert g.info()["m"] == want["m"]
        assert g.info()["wedges_in"] == want["wedges"]
        out = g.count(p=1, per_vertex=True)
        assert out["total"] == want["triangles"]
        pv = out["per_vertex"]
        assert int(pv.sum()) == 3 * want["triangles"]
        sample = goldens.chunglu_friendster_vertices()
        ids = np.array(sorted(sample), dtype=np.int64)
        assert np.array_equal(pv[ids], np.array([sample[x] for x in ids], dtype=np.uint64))
        del out, pv
        # blocks streamed from pinned host memory under a 24 GB device budget
        assert g.count(p=8, device_budget_bytes=24 << 30) == want["triangles"]
