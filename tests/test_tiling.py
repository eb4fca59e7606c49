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


def test_mixed_tilings_take_whole_columns_in_full_waves_then_short_chunks():
    # 512x256x128: 1024 columns of 32x4 (592 resident blocks of 128 threads on 148 SMs)
    # or 512 of 32x8 (296 of 256 threads); the mixed candidates take one full wave of whole
    # columns first, then cut the other columns into equal chunks, level by level
    cfgs = [P.Config(512, 256, 128)]
    mixed = 0
    for k in range(P.tiling_count()):
        tab = P.tiling_table(cfgs, k)
        lens = tab[:, 4] - tab[:, 3]
        if len(np.unique(lens)) < 2:
            continue
        mixed += 1
        wave = 148 * (16 // int(tab[:, 6].max()))  # 16 warps of 128 registers per SM
        whole = int(np.sum(lens == 128))
        assert whole > 0 and whole % wave == 0, k
        assert np.all(lens[:whole] == 128), k  # the whole columns go out first
        tail = tab[whole:]
        assert len(np.unique(tail[:, 4] - tail[:, 3])) == 1, k
        assert np.all(np.diff(tail[:, 3]) >= 0), k  # chunk level by level
        assert len(tail) / wave > 0.8 * np.ceil(len(tail) / wave), k  # the last wave is nearly full
        cover = np.zeros((128, 256, 512), np.int8)
        for inst, x0, y0, z0, z1, w, h in tab.tolist():
            cover[z0:z1, y0:y0 + h, x0:x0 + w] += 1
        assert cover.min() == 1 and cover.max() == 1, k
    assert mixed >= 2


def test_bad_arguments_are_rejected():
    with pytest.raises(RuntimeError):
        P.tiling_table(batch("c2"), P.tiling_count())
    with pytest.raises(RuntimeError):
        P.tiling_table([P.Config(8, 8, 1)], 0)
