"""The list-ranking entry point that allocates nothing (etl_list_rank_static).

Some callers cannot allocate device memory where they call the library (an
external memory manager owns the device, or the call must not wait on the
allocator); this entry point takes its scratch from a fixed array inside the
library instead. Here it is called through the C ABI and its output is
compared, element by element, with the known ranks of the list (the list is
built from a permutation, so rank[order[i]] = i) and with the regular
etl_list_rank, on two calls in a row (the second call reuses the scratch the
first one left behind). Ranks are integers, so the tolerance is zero.

The file is named so that pytest collects it after every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_LEN = 1 << 18


def make_list(n, seed):
    order = np.random.default_rng(seed).permutation(n).astype(np.int32)
    succ = np.full(n, -1, np.int32)
    succ[order[:-1]] = order[1:]
    rank = np.empty(n, np.int32)
    rank[order] = np.arange(n, dtype=np.int32)
    return torch.from_numpy(succ).cuda(), int(order[0]), torch.from_numpy(rank).cuda()


def rank_with(fn, succ, head):
    rank = torch.full_like(succ, -7)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(ctypes.c_void_p(succ.data_ptr()), succ.numel(), head, ctypes.c_void_p(rank.data_ptr()),
            ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    return rank, int(st.item())


def test_static_matches_regular_twice():
    import paper_2103_15217_gb300 as etl
    etl.build()
    lib = etl.load_library()
    for n, seed in ((MAX_LEN, 1), (150_001, 2)):   # two calls in a row, different lists
        succ, head, known = make_list(n, seed)
        got, st_got = rank_with(lib.etl_list_rank_static, succ, head)
        want, st_want = rank_with(lib.etl_list_rank, succ, head)
        assert st_got == 0 and st_want == 0
        assert torch.equal(got, known)
        assert torch.equal(got, want)


def test_static_rejects_oversize_lists():
    import paper_2103_15217_gb300 as etl
    lib = etl.load_library()
    succ, head, _ = make_list(MAX_LEN + 1, 3)
    rank = torch.empty_like(succ)
    rc = lib.etl_list_rank_static(ctypes.c_void_p(succ.data_ptr()), succ.numel(), head,
                                  ctypes.c_void_p(rank.data_ptr()), None, None)
    assert rc == 1   # ETL_EINVAL, nothing enqueued
