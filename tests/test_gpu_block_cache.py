"""The library's cache of large device blocks (GPU).

Blocks of 64 MB and more freed by one handle are handed to the next request of
a similar size, on a stream that first waits for the block's last use. Counts
through reused blocks must equal the oracle's stored count of R-MAT scale 23
(Sec. 2: the exact triangle count), whichever stream the handles use, and the
memory report counts idle cached blocks as available.
"""
import pytest

import graphgen
import paper_2009_12457_gb300 as bb
from tests import goldens

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_reused_blocks_across_streams_and_memory_report():
    want = goldens.config_counts()["rmat_s23_ef16_seed2"]["triangles"]
    n, rp, ci = graphgen.rmat_s23()
    d_rp, d_ci = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
    torch.cuda.synchronize()  # the inputs are read on other streams
    dev = torch.cuda.current_device()
    streams = [torch.cuda.Stream(), torch.cuda.Stream(), None]
    before = bb.bbtc_device_memory(dev)["available"]
    for k in range(6):
        st = streams[k % len(streams)]
        h = bb.bbtc_graph_create_async(n, d_rp, d_ci, bb.INPUT_SYMMETRIC, st)
        try:
            p = 1 + (k % 3)  # plans of different sizes take blocks of different sizes
            assert bb.bbtc_count(h, bb.make_opts(p=p, stream=st)) == want, (k, p)
        finally:
            bb.bbtc_graph_destroy(h)
    torch.cuda.synchronize()
    mem = bb.bbtc_device_memory(dev)
    assert mem["pool_used"] <= mem["pool_reserved"]
    # the handles' blocks are idle in the cache now: they count as available
    assert mem["available"] >= before - (256 << 20)
