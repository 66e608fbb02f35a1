"""Other spatial operators (Sec. 3.4): ST_Contains from the pixel areas and ST_Touches by the stated
edge/vertex rule, through the C ABI, against the oracle (exact)."""
import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rect_sets(seed, n):
    rng = np.random.Generator(np.random.PCG64(seed))
    rects = []
    for _ in range(2 * n):
        x0, y0 = rng.integers(0, 12, 2) * 2
        w, h = rng.integers(1, 5, 2) * 2
        rects.append([[x0, y0], [x0 + w, y0], [x0 + w, y0 + h], [x0, y0 + h]])
    return W.from_rings(rects[:n]), W.from_rings(rects[n:])


@pytest.fixture(scope="module")
def sccg():
    import paper_1208_0277_gb300 as P
    P.build()
    return P


@pytest.mark.parametrize("kind", ["rects", "stars", "stairs"])
def test_touches_and_contains_match_oracle(sccg, kind):
    if kind == "rects":
        A, B = rect_sets(3, 80)
    elif kind == "stars":
        w = W.single_tile(seed=7, n=400)
        A, B = w.A, w.B
    else:
        rng = np.random.Generator(np.random.PCG64(9))
        ra, _ = W.staircase_rings(rng, 80, max_cols=10, max_h=10, origin_span=30)
        rb, _ = W.staircase_rings(rng, 80, max_cols=10, max_h=10, origin_span=30)
        A, B = W.from_rings(ra), W.from_rings(rb)
    ctx = sccg.Context(0)
    dA, dB = ctx.upload(A), ctx.upload(B)
    pa, pb = ctx.candidate_pairs(dA, dB)
    inter, uni = ctx.pair_areas(dA, dB, pa, pb)
    t = ctx.touches(dA, dB, pa, pb)
    c = ctx.contains(dA, dB, pa, pb, inter)
    torch.cuda.synchronize()
    ref = O.cross_compare(A, B)
    assert len(ref["pa"]) == pa.numel() and len(ref["pa"]) > 0
    np.testing.assert_array_equal(t.cpu().numpy(), O.touches_pairs(A, B, ref["pa"], ref["pb"]))
    np.testing.assert_array_equal(c.cpu().numpy(), O.contains_flags(ref["area_a"], ref["area_b"], ref["pa"],
                                                                     ref["pb"], ref["inter"]))
    if kind == "rects":
        assert t.sum().item() > 0 and (c.cpu().numpy() & 1).sum() > 0    # the cases really occur


def test_operators_flag_invalid_pairs(sccg):
    A, B = rect_sets(4, 10)
    ctx = sccg.Context(0)
    dA, dB = ctx.upload(A), ctx.upload(B)
    pa = torch.tensor([0, 99, 3], dtype=torch.int32, device="cuda")
    pb = torch.tensor([0, 1, -1], dtype=torch.int32, device="cuda")
    inter = torch.tensor([1, 1, 1], dtype=torch.int64, device="cuda")
    assert ctx.touches(dA, dB, pa, pb).cpu().tolist()[1:] == [255, 255]
    assert ctx.contains(dA, dB, pa, pb, inter).cpu().tolist()[1:] == [255, 255]
