"""The allocation-free Jaccard entry point, sccg_jaccard_static, against sccg_jaccard and the oracle.

Some callers of this library may not allocate device memory: plugins inside a host application
that owns all device memory through its own pool (their own cudaMalloc would bypass it or fail),
deployments that forbid allocation after start-up, and latency-critical loops in which
cudaMalloc/cudaFree would synchronise the device. They use sccg_jaccard_static, whose scratch is a
fixed array compiled into the library rather than context memory. This file checks it through the
C ABI, on two calls in a row, against the context-based sccg_jaccard and the CPU oracle (exact
equality: the results are integers and correctly rounded doubles), at its pair limit against the
closed form J(A, A) = J'(A, A) = 1, and in a driver context the caller created itself. It is named
to run last and builds everything it needs, so it passes both alone and after the other tests."""
import ctypes

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("sum_inter", "sum_union", "n_nonzero", "n_pairs", "J", "Jprime")
STATIC_MAX_PAIRS = 4096 * 65536


@pytest.fixture(scope="module")
def lib_and_ctx():
    import paper_1208_0277_gb300 as P
    P.build()
    O.build()
    return P, P._native.load(), P.Context(0)


def static_jaccard(P, lib, inter, uni, n=None):
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    st = lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), inter.numel() if n is None else n,
                                 out.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
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


def test_static_jaccard_matches_context_jaccard_and_oracle_on_two_calls_in_a_row(lib_and_ctx):
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
        want = O.jaccard(inter.cpu().numpy(), uni.cpu().numpy())
        for k in FIELDS:
            assert getattr(got, k) == ref[k], k
            if k != "n_pairs":
                assert getattr(got, k) == want[k], k
        assert got.n_pairs == inter.numel()


def test_static_jaccard_at_its_pair_limit(lib_and_ctx):
    """2^28 pairs, each with inter == union (J(A, A) = J'(A, A) = 1 in closed form): every slot of the
    fixed array holds a partial sum, and the fixed-point sum of the ratios must not wrap."""
    P, lib, ctx = lib_and_ctx
    n = STATIC_MAX_PAIRS
    ones = torch.ones(n, dtype=torch.int64, device="cuda")
    got = static_jaccard(P, lib, ones, ones)
    assert (got.n_pairs, got.n_nonzero, got.sum_inter, got.sum_union) == (n, n, n, n)
    assert got.J == 1.0 and got.Jprime == 1.0
    ref = ctx.jaccard(ones, ones)
    for k in FIELDS:
        assert getattr(got, k) == ref[k], k
    del ones
    torch.cuda.empty_cache()


def test_static_jaccard_rejects_what_it_cannot_hold(lib_and_ctx):
    P, lib, ctx = lib_and_ctx
    inter, uni = synthetic_areas(2, 16)
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more pairs than 4096 slots x 65,536 pairs: refused before anything is launched
    assert lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), STATIC_MAX_PAIRS + 1, out.data_ptr(), s) == 2
    # the result must be device memory
    host = np.zeros(6, dtype=np.int64)
    assert lib.sccg_jaccard_static(inter.data_ptr(), uni.data_ptr(), 16, host.ctypes.data, s) == 1
    # the context Jaccard refuses counts whose exact J' sum could overflow 128 bits (checked before
    # any launch or pointer access)
    res = P._native.JaccardC()
    assert lib.sccg_jaccard(ctx.h, inter.data_ptr(), uni.data_ptr(), 1 << 43, ctypes.addressof(res), s) == 2
    # and the empty case still writes a result
    got = static_jaccard(P, lib, inter[:0], uni[:0])
    assert got.n_pairs == 0 and got.n_nonzero == 0 and got.J == 0.0 and got.Jprime == 0.0


def test_static_jaccard_in_a_context_the_caller_created(lib_and_ctx):
    """A host application may create its own driver context (cuCtxCreate) and make it current before
    calling the library; that context holds its own copy of the fixed array. Calls there and then back
    in the primary context must each use their own context's array."""
    P, lib, ctx = lib_and_ctx
    try:
        cu = ctypes.CDLL("libcuda.so.1")
        create = cu.cuCtxCreate_v2
    except (OSError, AttributeError):
        pytest.skip("driver API not reachable through ctypes")
    vp = ctypes.c_void_p
    u64 = ctypes.c_uint64
    inter, uni = synthetic_areas(3, 100_000)
    h_inter, h_uni = inter.cpu().numpy(), uni.cpu().numpy()
    want = O.jaccard(h_inter, h_uni)
    first = static_jaccard(P, lib, inter, uni)              # primary context (torch's)
    old = vp()
    assert cu.cuCtxGetCurrent(ctypes.byref(old)) == 0
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
    new = vp()
    assert create(ctypes.byref(new), 0, dev) == 0           # now current
    bufs = []
    try:
        nbytes = h_inter.nbytes
        d = {}
        for name, nb in (("inter", nbytes), ("uni", nbytes), ("out", 48)):
            p = u64()
            assert cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nb)) == 0
            bufs.append(p)
            d[name] = p
        assert cu.cuMemcpyHtoD_v2(d["inter"], h_inter.ctypes.data_as(vp), ctypes.c_size_t(nbytes)) == 0
        assert cu.cuMemcpyHtoD_v2(d["uni"], h_uni.ctypes.data_as(vp), ctypes.c_size_t(nbytes)) == 0
        for _ in range(2):
            st = lib.sccg_jaccard_static(d["inter"].value, d["uni"].value, len(h_inter), d["out"].value, None)
            assert st == 0, lib.sccg_status_str(st)
            assert cu.cuCtxSynchronize() == 0
            raw = (ctypes.c_uint8 * 48)()
            assert cu.cuMemcpyDtoH_v2(raw, d["out"], ctypes.c_size_t(48)) == 0
            got = P._native.JaccardC.from_buffer_copy(bytes(raw))
            for k in FIELDS:
                if k != "n_pairs":
                    assert getattr(got, k) == want[k], k
    finally:
        for p in bufs:
            cu.cuMemFree_v2(p)
        cu.cuCtxDestroy_v2(new)
        cu.cuCtxSetCurrent(old)
    again = static_jaccard(P, lib, inter, uni)               # back in the primary context
    for k in FIELDS:
        assert getattr(again, k) == getattr(first, k), k
