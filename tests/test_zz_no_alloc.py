"""The allocation-free Jaccard entry point, sccg_jaccard_static, against sccg_jaccard.

Some callers of this library may not allocate device memory: plugins inside a host application
that owns all device memory through its own pool (their own cudaMalloc would bypass it or fail),
deployments that forbid allocation after start-up, and latency-critical loops in which
cudaMalloc/cudaFree would synchronise the device. They use sccg_jaccard_static, whose scratch is a
fixed array compiled into the library rather than context memory. This file checks it through the
C ABI, on two calls in a row, against the context-based sccg_jaccard (exact equality: the results
are integers and correctly rounded doubles). It is named to run last and builds everything it needs,
so it passes both alone and after the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("sum_inter", "sum_union", "n_nonzero", "n_pairs", "J", "Jprime")


@pytest.fixture(scope="module")
def lib_and_ctx():
    import paper_1208_0277_gb300 as P
    P.build()
    return P, P._native.load(), P.Context(0)


def static_jaccard(P, lib, inter, uni):
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    st = lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), inter.numel(), out.data_ptr(),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sccg_status_str(st)
    torch.cuda.synchronize()
    return P._native.JaccardC.from_buffer_copy(out.cpu().numpy().tobytes())


def synthetic_areas(seed, n):
    """inter <= union int64 arrays with about a third of the pairs not intersecting."""
    rng = np.random.default_rng(seed)
    uni = rng.integers(1, 5000, n).astype(np.int64)
    inter = (rng.random(n) * uni).astype(np.int64)
    inter[rng.random(n) < 0.3] = 0
    return torch.from_numpy(inter).cuda(), torch.from_numpy(uni).cuda()


def test_static_jaccard_matches_context_jaccard_on_two_calls_in_a_row(lib_and_ctx):
    P, lib, ctx = lib_and_ctx
    from paper_1208_0277_gb300 import workload as W
    # first call spans five slots of the fixed array, the second only one: the second must not see
    # the first call's partial sums
    cases = [synthetic_areas(1, 300_000)]
    w = W.single_tile(seed=0, n=400)
    A, B = ctx.upload(w.A), ctx.upload(w.B)
    pa, pb = ctx.candidate_pairs(A, B)
    cases.append(ctx.pair_areas(A, B, pa, pb))
    for inter, uni in cases:
        ref = ctx.jaccard(inter, uni)
        got = static_jaccard(P, lib, inter, uni)
        for k in FIELDS:
            assert getattr(got, k) == ref[k], k


def test_static_jaccard_rejects_what_it_cannot_hold(lib_and_ctx):
    P, lib, ctx = lib_and_ctx
    inter, uni = synthetic_areas(2, 16)
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more pairs than 4096 slots x 65,536 pairs: refused before anything is launched
    assert lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), 4096 * 65536 + 1, out.data_ptr(), s) == 2
    # the result must be device memory
    host = np.zeros(6, dtype=np.int64)
    assert lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), 16, host.ctypes.data, s) == 1
    # and the empty case still writes a result
    got = static_jaccard(P, lib, inter[:0], uni[:0])
    assert got.n_pairs == 0 and got.n_nonzero == 0 and got.J == 0.0 and got.Jprime == 0.0
