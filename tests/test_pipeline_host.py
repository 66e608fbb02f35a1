"""Host logic of the pipelined front end: how the tiles are cut into chunks (no GPU needed)."""
import numpy as np
import pytest

from paper_1208_0277_gb300.pipeline import Pipeline


class _Set:
    def __init__(self, tiles, nv):
        self.tile_np = np.asarray(tiles, dtype=np.int32)
        self.off_np = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
        self.n = len(tiles)


def _sets(n_tiles, n, seed):
    rng = np.random.default_rng(seed)
    A = _Set(np.sort(rng.integers(0, n_tiles, n)), rng.integers(3, 60, n))
    B = _Set(np.sort(rng.integers(0, n_tiles, n)), rng.integers(3, 60, n))
    return A, B


@pytest.mark.parametrize("n_tiles,k,growth", [(625, 4, 1.75), (625, 4, 1.0), (625, 9, 1.5), (7, 4, 1.75),
                                              (3, 8, 1.75), (1, 4, 2.0), (50, 1, 1.75)])
def test_chunks_partition_the_tiles(n_tiles, k, growth):
    A, B = _sets(n_tiles, 20 * n_tiles, n_tiles + k)
    c = Pipeline._cut(A, B, n_tiles, min(k, n_tiles), growth)
    assert c[0][0] == 0 and c[-1][1] == n_tiles
    assert all(t0 < t1 for t0, t1 in c)
    assert all(c[i][1] == c[i + 1][0] for i in range(len(c) - 1))
    assert len(c) <= k


def test_chunk_sizes_grow_geometrically():
    A, B = _sets(2000, 200000, 1)
    c = Pipeline._cut(A, B, 2000, 4, 2.0)
    verts = np.zeros(2000)
    for S in (A, B):
        np.add.at(verts, S.tile_np, np.diff(S.off_np))
    sizes = np.array([verts[t0:t1].sum() for t0, t1 in c])
    np.testing.assert_allclose(sizes / sizes.sum(), np.array([1, 2, 4, 8]) / 15, atol=0.01)


def test_empty_tiles_and_sets():
    A = _Set([], [])
    B = _Set([0, 0, 5], [4, 4, 4])
    c = Pipeline._cut(A, B, 6, 3, 1.75)
    assert c[0][0] == 0 and c[-1][1] == 6
    assert all(t0 < t1 for t0, t1 in c)


def test_copy_mode_is_checked_before_any_device_work():
    with pytest.raises(ValueError):
        Pipeline(None, None, None, 1, copy="dma")
