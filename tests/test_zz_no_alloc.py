"""hyperim_coverage_noalloc through the C ABI against the existing coverage entry point.

The no-allocation variant serves callers that cannot allocate device memory (for example a
serving loop whose memory is reserved up front, or a host application whose own allocator owns
the GPU). Its per-stratum coverage must equal the one hyperim_select_seeds reports, call after
call: the second call checks that the shared scratch left by the first one does not leak into
the result. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01911_gb300 import build
    build.build()
    import paper_2406_01911_gb300 as H
    return H


def noalloc_coverage(H, n, pool, seeds):
    import torch
    v = pool.view()
    d_seeds = torch.as_tensor(np.asarray(seeds, dtype=np.int32)).cuda()
    lam = torch.full((16,), -1, dtype=torch.int64, device="cuda")  # garbage: the call zeroes it
    stream = torch.cuda.current_stream()
    st = H.lib().hyperim_coverage_noalloc(
        int(n), C.c_void_p(v["rr_off"]), C.c_void_p(v["rr_mem"]), C.c_void_p(v["rr_stratum"]),
        int(v["count"]), C.c_void_p(d_seeds.data_ptr()), len(seeds), C.c_void_p(lam.data_ptr()),
        C.c_void_p(stream.cuda_stream))
    assert st == 0, H.lib().hyperim_last_error()
    stream.synchronize()
    return lam.cpu().numpy().astype(np.uint64)


def test_noalloc_coverage_matches_select_seeds(H):
    n, hes = gc.random_graph(21, 3000, 2400, 7)
    off, mem = gc.csr(hes)
    g = H.Graph(n, off, mem, "wc", 0, seed=5)
    r1 = g.pool(tag=0, roots="stratified").sample(4000)
    r2 = g.pool(tag=1, roots="stratified").sample(3000)
    # first call: the seeds greedy picks on r1, counted on r2
    seeds_a, res_a = g.select_seeds(r1, r2, 25, mode="fixed")
    got_a = noalloc_coverage(H, n, r2, seeds_a)
    assert got_a.tolist() == res_a["lambda_r2"].tolist()
    # second call in a row, other seeds and pool: the flags of the first call must be gone
    seeds_b, res_b = g.select_seeds(r2, r1, 4, mode="fixed")
    got_b = noalloc_coverage(H, n, r1, seeds_b)
    assert got_b.tolist() == res_b["lambda_r2"].tolist()


def test_noalloc_rejects_too_many_vertices(H):
    import torch
    lam = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = H.lib().hyperim_coverage_noalloc(int(H.NOALLOC_MAX_N) + 1, None, None, None, 0, None, 0,
                                         C.c_void_p(lam.data_ptr()), None)
    assert st == -1
    assert b"too small" in H.lib().hyperim_last_error()
