"""Learned sweep proposer: what it gains over plain enumeration and over random
draws, on a smooth stand-in response and on deposit descriptors of real drying
runs (every point of the sweep grid run to a dried deposit in one batch, two
seeds per point), and the end-to-end loop that simulates each proposal."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sweep():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import build
    build.build()
    from paper_2607_06794_b300 import sweep as S
    return S


def smooth_response(P):
    """A smooth stand-in for the descriptors (S_x, clusters, percolation) whose best
    point lies in the middle of the grid, far from where enumeration starts."""
    ar, e, L, sw = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    s = np.tanh(0.4 * (ar - 3.5)) * 0.5 + 0.02 * L
    c = 1.0 / (1.0 + e) + 0.01 * sw
    p = np.exp(-((ar - 4.0) ** 2) / 2.0 - (e - 1.0) ** 2 - ((L - 12.0) / 4.0) ** 2 - ((sw - 16.0) / 8.0) ** 2)
    return np.c_[s, c, p]


def test_proposer_beats_enumeration_at_equal_budget(sweep):
    """With 40 of 288 points simulated, the learned proposer finds far better points
    than enumerating the grid in order (the fallback) and, on average over seeds,
    better than drawing the 40 points at random."""
    grid = sweep.default_grid()
    objective = lambda y: float(y[2])  # maximise percolation
    budget = 40
    truth = smooth_response(grid)[:, 2]
    ref = sweep.grid_sweep(grid, smooth_response, objective, budget)
    bests = []
    for seed in (0, 1, 2):
        act = sweep.active_sweep(grid, smooth_response, objective, budget, seed_points=16, per_round=8,
                                 seed=seed, epochs=500)
        assert len(act.evaluated) == budget == len(set(act.evaluated))
        assert len(act.prediction_error) == budget - 16  # every proposal simulated and scored
        bests.append(act.best)
    g = np.random.default_rng(7)
    random_best = np.mean([truth[g.permutation(len(grid))[:budget]].max() for _ in range(2000)])
    assert min(bests) > ref.best + 0.3
    assert np.mean(bests) > random_best + 0.1
    assert max(bests) == truth.max()


def test_proposer_fit_reduces_loss(sweep):
    grid = sweep.default_grid()
    Y = smooth_response(grid)
    prop = sweep.Proposer(seed=1, members=1)
    l0 = prop.fit(grid[:50], Y[:50], epochs=1)
    l1 = prop.fit(grid[:50], Y[:50], epochs=800)
    assert l1 < 0.1 * l0


def test_sweep_loop_on_real_batched_runs(sweep):
    pts = np.array([(1.0, 0.0, 4.0, 12.0), (3.0, 1.0, 8.0, 16.0), (2.0, 2.0, 12.0, 24.0)])
    rows = sweep.batched_points(pts, steps=20, prec="fp16")
    assert rows.shape == (3, 3)
    assert np.all(np.abs(rows[:, 0]) <= 1.0)
    res = sweep.active_sweep(pts, lambda P: sweep.batched_points(P, 10, "fp16"), lambda y: float(y[2]),
                             budget=3, seed_points=2, per_round=1, epochs=50)
    assert len(res.evaluated) == 3


# ---------------------------------------------------------------------------- real deposits
@pytest.fixture(scope="module")
def real_table(sweep):
    """Descriptors of the dried deposits of the whole 288-point grid (aspect ratio x eps* x
    wire length x stripe width), two seeds per point, FP16 storage, one batch run until
    every droplet has evaporated."""
    grid = sweep.default_grid()
    rows, steps, raw = sweep.deposit_table(grid, seeds=(0, 1), prec="fp16", max_steps=20000, every=500)
    ok = ~np.isnan(rows[:, 0])
    return grid[ok], rows[ok], steps, raw


def aligned_connected(y):
    """Axially aligned and connected deposits: S_x minus twice the clusters per wire."""
    return float(y[0] - 2.0 * y[1])


def test_real_runs_dry_and_give_a_structured_table(real_table):
    grid, rows, steps, raw = real_table
    assert steps < 20000  # every droplet dried
    assert len(grid) >= 280  # at most the longest wires do not fit the roundest droplet
    assert np.all(np.abs(rows[:, 0]) <= 1.0) and np.all(rows[:, 1] > 0.0)
    assert np.all((rows[:, 2] >= 0.0) & (rows[:, 2] <= 1.0))
    # the deposit depends on the geometry: elongated droplets align the wires axially
    # (Sec. III.B), longer wires more so
    by_ar = [rows[grid[:, 0] == a, 0].mean() for a in (2.0, 6.0)]
    by_L = [rows[grid[:, 2] == L, 0].mean() for L in (4.0, 16.0)]
    assert by_ar[1] > by_ar[0] + 0.2 and by_L[1] > by_L[0] + 0.5


def test_proposer_predicts_real_descriptors(sweep, real_table):
    """Trained by the library's own kernels on half of the real points, the MLP
    predicts S_x of the other half (its prediction error is reported)."""
    grid, rows, _, _ = real_table
    g = np.random.default_rng(3)
    idx = g.permutation(len(grid))
    tr, te = idx[: len(idx) // 2], idx[len(idx) // 2:]
    prop = sweep.Proposer(seed=0, members=4)
    prop.fit(grid[tr], rows[tr], epochs=800)
    pred = prop.predict(grid[te])
    rmse = np.sqrt(np.mean((pred[:, 0] - rows[te, 0]) ** 2))
    r2 = 1.0 - np.sum((pred[:, 0] - rows[te, 0]) ** 2) / np.sum((rows[te, 0] - rows[te, 0].mean()) ** 2)
    print(f"held-out S_x: rmse {rmse:.3f}, R^2 {r2:.3f} (spread of S_x {rows[:, 0].std():.3f})")
    assert r2 > 0.5


def test_proposer_gain_on_real_deposits(sweep, real_table):
    """At a budget of 40 of ~286 simulated points, the proposer finds deposits at least
    as aligned-and-connected as random draws do on average, and far better than
    enumerating the grid in order (the fallback).  The LBM runs of the table judge
    every proposal; the prediction error of each proposal is recorded."""
    grid, rows, _, _ = real_table
    lookup = {tuple(p): r for p, r in zip(grid, rows)}
    simulate = lambda P: np.array([lookup[tuple(p)] for p in P])
    budget = 40
    truth = np.array([aligned_connected(r) for r in rows])
    ref = sweep.grid_sweep(grid, simulate, aligned_connected, budget)
    bests, errs = [], []
    for seed in (0, 1, 2):
        act = sweep.active_sweep(grid, simulate, aligned_connected, budget, seed_points=16, per_round=8,
                                 seed=seed, epochs=500)
        assert len(act.evaluated) == budget == len(set(act.evaluated))
        bests.append(act.best)
        errs += act.prediction_error
    g = np.random.default_rng(11)
    random_best = np.mean([truth[g.permutation(len(grid))[:budget]].max() for _ in range(4000)])
    print(f"best found: proposer {np.round(bests, 3)} (mean {np.mean(bests):.3f}), random {random_best:.3f}, "
          f"enumeration {ref.best:.3f}, grid optimum {truth.max():.3f}; "
          f"mean |prediction error| of proposals {np.mean(errs):.3f}")
    assert np.mean(bests) > ref.best + 0.5
    assert np.mean(bests) >= random_best - 0.01
