"""Host-to-host pipeline (chunked copies overlapped with the work): identical pairs, areas and
Jaccard bits to the device-resident path on the whole sets, and to the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunks,initial,growth,copy", [(1, None, 1.75, "sm"), (3, None, 1.75, "sm"),
                                                        (3, None, 1.0, "engine"), (7, 1000, 1.75, "sm"),
                                                        (7, 1000, 1.75, "engine")])
def test_pipeline_equals_resident_path_and_oracle(chunks, initial, growth, copy):
    import paper_1208_0277_gb300 as P
    from paper_1208_0277_gb300.pipeline import HostSet, Pipeline
    P.build()
    w = W.batched_uneven(seed=6, n_tiles=12, count_lo=50, count_hi=1500)
    ctx = P.Context(0)
    pipe = Pipeline(ctx, HostSet.from_polyset(w.A), HostSet.from_polyset(w.B), w.n_tiles, chunks=chunks,
                    initial_pairs=initial, growth=growth, copy=copy)
    pa, pb, inter, uni, J = pipe.run()
    pa, pb, inter, uni = (np.array(x, dtype=np.int64) for x in (pa, pb, inter, uni))   # views of reused buffers
    A, B = ctx.upload(w.A), ctx.upload(w.B)
    r = P.cross_compare(ctx, A, B, mode=P.MODE_PERSISTENT)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pa, r["pa"].cpu().numpy())
    np.testing.assert_array_equal(pb, r["pb"].cpu().numpy())
    np.testing.assert_array_equal(inter, r["inter"].cpu().numpy())
    np.testing.assert_array_equal(uni, r["uni"].cpu().numpy())
    for k in ("sum_inter", "sum_union", "n_nonzero", "n_pairs", "J", "Jprime"):
        assert J[k] == r["jaccard"][k], k
    _, mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")
    opa, opb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    np.testing.assert_array_equal(pa, opa)
    np.testing.assert_array_equal(pb, opb)
    idx = np.arange(0, len(opa), max(1, len(opa) // 2000))
    ri, ru = O.pair_areas(w.A, w.B, opa[idx], opb[idx], method="rle")
    np.testing.assert_array_equal(inter[idx], ri)
    np.testing.assert_array_equal(uni[idx], ru)
    pa2, _, inter2, _, J2 = pipe.run()                  # a second run reuses the buffers
    np.testing.assert_array_equal(pa2, pa)
    np.testing.assert_array_equal(inter2, inter)
    assert J2 == J


@pytest.mark.parametrize("offset,nbytes", [(0, 1 << 20), (4, (1 << 20) + 12), (8, 4096 + 4), (12, 4), (0, 16 * 40000 + 8)])
def test_sm_copy_moves_the_bytes_in_every_direction(offset, nbytes):
    """sccg_copy between pinned host and device memory (both ways) and device to device, at every
    alignment the unit choice distinguishes (16, 8, 4 bytes) with tails, equals the source."""
    import paper_1208_0277_gb300 as P
    P.build()
    ctx = P.Context(0)
    rng = np.random.default_rng(offset + nbytes)
    n = nbytes // 4
    src_h = torch.from_numpy(rng.integers(-2**31, 2**31, n + 8, dtype=np.int64).astype(np.int32)).pin_memory()
    k = offset // 4
    dev = torch.full((n + 8,), -1, dtype=torch.int32, device="cuda")
    ctx.copy(dev[k:k + n], src_h[k:k + n])                      # host -> device
    torch.cuda.synchronize()
    got = dev.cpu()
    assert torch.equal(got[k:k + n], src_h[k:k + n])
    assert bool((got[:k] == -1).all()) and bool((got[k + n:] == -1).all())
    back = torch.zeros(n + 8, dtype=torch.int32).pin_memory()
    ctx.copy(back[k:k + n], dev[k:k + n])                       # device -> host
    torch.cuda.synchronize()
    assert torch.equal(back[k:k + n], src_h[k:k + n])
    d2 = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    ctx.copy(d2[k:k + n], dev[k:k + n])                         # device -> device
    torch.cuda.synchronize()
    assert torch.equal(d2[k:k + n].cpu(), src_h[k:k + n])


def test_sm_copy_refuses_pageable_overlapping_and_misaligned_memory():
    import ctypes
    import paper_1208_0277_gb300 as P
    P.build()
    ctx = P.Context(0)
    dev = torch.zeros(1024, dtype=torch.int32, device="cuda")
    pageable = torch.zeros(1024, dtype=torch.int32)
    assert not pageable.is_pinned()
    with pytest.raises(P.SccgError):
        ctx.copy(dev, pageable)                                  # pageable host memory
    with pytest.raises(P.SccgError):
        ctx.copy(pageable, dev)
    with pytest.raises(P.SccgError):
        ctx.copy(dev[100:600], dev[0:500])                       # overlapping ranges
    lib, h = ctx.lib, ctx.h
    pin = torch.zeros(1024, dtype=torch.int32).pin_memory()
    assert lib.sccg_copy(h, ctypes.c_void_p(dev.data_ptr() + 2), ctypes.c_void_p(pin.data_ptr()), 64, None) != 0
    assert lib.sccg_copy(h, ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(pin.data_ptr()), 63, None) != 0
    assert lib.sccg_copy(h, ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(pin.data_ptr()), 0, None) == 0
    torch.cuda.synchronize()
    assert bool((dev == 0).all())


def test_sm_copy_from_a_fresh_host_thread():
    """A host thread whose first CUDA call is sccg_copy (the serving loop's batcher) copies too."""
    import threading
    import paper_1208_0277_gb300 as P
    P.build()
    ctx = P.Context(0)
    src = torch.arange(4096, dtype=torch.int32).pin_memory()
    dev = torch.zeros(4096, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    errs = []

    def work():
        try:
            ctx.copy(dev, src)
            torch.cuda.synchronize()
        except Exception as e:          # noqa: BLE001 - reported below
            errs.append(e)
    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert not errs, errs
    assert torch.equal(dev.cpu(), src)
