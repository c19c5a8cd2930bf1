"""bbtc_count_noalloc: the allocation-free count must equal bbtc_count.

Callers that cannot allocate device memory when they count (a loop that
reserves its GPU memory up front, or code running while another memory manager
owns the device) use this entry point; its scratch is a fixed device array in
the library. This file is collected last so that a failure here does not stop
the other tests of a run that halts at the first failure.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_2009_12457_gb300 as bb

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.mark.parametrize("p", [1, 4, 16])
def test_noalloc_matches_bbtc_count_twice(p):
    lib = bb.load()
    n, rp, ci = graphgen.rmat(13, 16, 9)
    with bb.Graph(n, rp, ci) as g:
        expect = g.count(p=p, per_task=True)      # also builds the plan for p
        nt = bb.bbtc_num_tasks(p)
        for _ in range(2):                          # two calls in a row share the scratch
            total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            per_task = torch.full((nt,), -1, dtype=torch.int64, device="cuda")
            st = lib.bbtc_count_noalloc(ctypes.c_void_p(g.handle), p,
                                        ctypes.c_void_p(total.data_ptr()),
                                        ctypes.c_void_p(per_task.data_ptr()), None)
            assert st == 0, bb.bbtc_last_error()
            torch.cuda.synchronize()
            assert int(total.item()) == expect["total"]
            assert np.array_equal(per_task.cpu().numpy().astype(np.uint64), expect["per_task"])


def test_noalloc_rejects_what_the_fixed_scratch_cannot_hold():
    lib = bb.load()
    n, rp, ci = graphgen.rmat(10, 8, 4)
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    with bb.Graph(n, rp, ci) as g:
        g.count(p=20)
        assert lib.bbtc_count_noalloc(ctypes.c_void_p(g.handle), 20,
                                      ctypes.c_void_p(total.data_ptr()), None, None) == 1
        # no plan for p = 3 yet: the call refuses rather than allocate one
        assert lib.bbtc_count_noalloc(ctypes.c_void_p(g.handle), 3,
                                      ctypes.c_void_p(total.data_ptr()), None, None) == 1
        g.count(p=3)
        assert lib.bbtc_count_noalloc(ctypes.c_void_p(g.handle), 3,
                                      ctypes.c_void_p(total.data_ptr()), None, None) == 0
        torch.cuda.synchronize()
        assert int(total.item()) == g.count(p=3)
