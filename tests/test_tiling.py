"""Host logic of the fused kernel's tilings (CPU only): every candidate tiling covers
every node of every instance exactly once, with z-chunks of 2 to 241 planes, and the
automatic chunk looks at the whole batch."""
import numpy as np
import pytest

import paper_2607_06794_b300 as P


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2607_06794_b300 import build
    build.build()


MAX_PIECE = 241  # 240 planes per chunk, 241 when a 1-plane rest is merged


def batch(name):
    if name == "c2":
        return [P.Config(256, 128, 64)]
    if name == "tall":
        return [P.Config(16, 16, 300)]
    if name == "tiny":
        return [P.Config(5, 3, 2), P.Config(40, 9, 3)]
    if name == "ragged_batch":
        return [P.Config(64 + 43 * k, 64 + 11 * k, 48 - 5 * k) for k in range(6)]
    raise KeyError(name)


@pytest.mark.parametrize("name", ["c2", "tall", "tiny", "ragged_batch"])
def test_every_tiling_covers_every_node_once(name):
    cfgs = batch(name)
    assert P.tiling_count() >= 6
    for k in range(P.tiling_count()):
        tab = P.tiling_table(cfgs, k)
        cover = [np.zeros((c.nz, c.ny, c.nx), np.int32) for c in cfgs]
        for inst, x0, y0, z0, z1, w, h in tab.tolist():
            c = cfgs[inst]
            assert 2 <= z1 - z0 <= MAX_PIECE
            assert w == min(32, c.nx - x0) and 1 <= h <= 8 and h <= c.ny - y0
            cover[inst][z0:z1, y0:y0 + h, x0:x0 + w] += 1
        for cv in cover:
            assert cv.min() == 1 and cv.max() == 1, f"tiling {k}: nodes covered {cv.min()}..{cv.max()} times"


def test_tall_columns_are_cut_into_chunks_of_at_most_240_planes():
    for k in range(P.tiling_count()):
        tab = P.tiling_table(batch("tall"), k)
        assert (tab[:, 4] - tab[:, 3]).max() <= MAX_PIECE
        assert len(np.unique(tab[:, 3])) >= 2


def test_automatic_chunk_counts_the_columns_of_the_whole_batch():
    # 64 lattices of 64x64x48: 512 tile columns of 32x8 over the batch fill the GPU,
    # so the automatic chunk keeps whole columns; one lattice alone is split in z
    one = [P.Config(64, 64, 48)]
    many = one * 64
    auto = 0  # candidate 0 is the automatic chunk on 32x8 columns
    t1, tm = P.tiling_table(one, auto), P.tiling_table(many, auto)
    assert (t1[:, 4] - t1[:, 3]).max() < 48
    assert np.all(tm[:, 4] - tm[:, 3] == 48)


def test_bad_arguments_are_rejected():
    with pytest.raises(RuntimeError):
        P.tiling_table(batch("c2"), P.tiling_count())
    with pytest.raises(RuntimeError):
        P.tiling_table([P.Config(8, 8, 1)], 0)
