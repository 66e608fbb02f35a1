"""Host-to-host pipeline (chunked copies overlapped with the work): identical pairs, areas and
Jaccard bits to the device-resident path on the whole sets, and to the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunks,initial,growth", [(1, None, 1.75), (3, None, 1.75), (3, None, 1.0), (7, 1000, 1.75)])
def test_pipeline_equals_resident_path_and_oracle(chunks, initial, growth):
    import paper_1208_0277_gb300 as P
    from paper_1208_0277_gb300.pipeline import HostSet, Pipeline
    P.build()
    w = W.batched_uneven(seed=6, n_tiles=12, count_lo=50, count_hi=1500)
    ctx = P.Context(0)
    pipe = Pipeline(ctx, HostSet.from_polyset(w.A), HostSet.from_polyset(w.B), w.n_tiles, chunks=chunks,
                    initial_pairs=initial, growth=growth)
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
