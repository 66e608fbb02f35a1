"""Autotuner: the cache file round-trips on CPU; on the GPU the tuner times real launches, leaves the
context at the best parameters it found, and those parameters give the oracle's results."""
import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import tune
from paper_1208_0277_gb300 import workload as W


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tuned.json")
    assert tune.load(path, "k") is None
    tune.save(path, "k", {"params": {"T": 8192, "split_pixels": 4096, "warps_per_cta": 4}, "ms": 1.5,
                          "mode": "persistent", "table": []})
    tune.save(path, "k2", {"params": {"T": 2048, "split_pixels": 1024, "warps_per_cta": 8}, "ms": 2.0,
                           "mode": "plain", "table": []})
    assert tune.load(path, "k")["params"]["T"] == 8192
    assert tune.load(path, "k2")["mode"] == "plain"


@pytest.mark.gpu
@pytest.mark.parametrize("mode,raster", [(0, False), (1, False), (1, True)])
def test_tuner_picks_from_its_grid_and_keeps_results_exact(mode, raster):
    """Without rasters the tuner searches T, the item size, warps per CTA and threads per item; with
    rasters (persistent form) the threads per pair (raster_heavy: one warp or one CTA) and resident
    CTAs per SM."""
    torch = pytest.importorskip("torch")
    import paper_1208_0277_gb300 as P
    P.build()
    w = W.single_tile(seed=9, n=600)
    ctx = P.Context(0)
    A, B = ctx.upload(w.A, raster=raster), ctx.upload(w.B, raster=raster)
    pa, pb = ctx.candidate_pairs(A, B)
    res = tune.tune(ctx, A, B, pa, pb, mode=mode, reps=2, warm=1)
    p = ctx.params()
    if raster:
        assert res["params"]["raster_heavy"] in tune.HEAVY_GRID + (1024,)
        assert res["params"]["raster_lanes"] in tune.RASTER_LANES_GRID
        assert res["params"]["ctas_per_sm"] in tune.CTAS_GRID
        assert len(res["table"]) <= 1 + len(tune.HEAVY_GRID) + len(tune.CTAS_GRID) + len(tune.RASTER_LANES_GRID)
        assert len({tuple(sorted(t.items())) for t, _ in res["table"]}) == len(res["table"])   # none twice
    else:
        assert res["params"]["T"] in tune.T_GRID + tuple(T for _, T in tune.FORM_GRID) + (8192,)
        assert res["params"]["warps_per_cta"] in tune.WPC_GRID + (4,)
        assert len(res["table"]) >= 1 + len(tune.T_GRID) - 1
    for k, v in res["params"].items():
        assert p[k] == v
    inter, uni = ctx.pair_areas(A, B, pa, pb, mode=mode)
    torch.cuda.synchronize()
    ref = O.cross_compare(w.A, w.B)
    np.testing.assert_array_equal(inter.cpu().numpy(), ref["inter"])
    np.testing.assert_array_equal(uni.cpu().numpy(), ref["uni"])
