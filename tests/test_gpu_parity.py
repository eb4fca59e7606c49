"""GPU path against the FP64 oracle, element by element, through the C ABI.

Tolerances (per population, relative to |f| + w_i):
  FP64 storage+arithmetic: 1e-12 per step (only the summation order differs)
  FP32: 2e-6 (single-precision rounding of a few dozen operations on O(0.3) values)
  FP16 shifted: 2e-3 (stored liquid fraction carries 2^-11 relative error, total 2^-11)
  BF16 shifted: 1.5e-2 (8-bit significands: 2^-8 relative)
"""
import dataclasses

import numpy as np
import pytest

from tests import inputs
from tests.gpu_helpers import W, oracle_params, oracle_state, pop_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "fp16": 2e-3, "bf16": 1.5e-2}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import build
    build.build()
    import paper_2607_06794_b300 as P
    return P


def droplet_cfg(P, nx=40, ny=24, nz=20, **kw):
    base = dict(cx=nx / 2 - 0.5, cy=ny / 2 - 0.5, cz=-0.5, a=nx * 0.3, b=ny * 0.3, c=nz * 0.55,
                sigma=0.01, beta=0.7, top_bc=1, theta_deg=70.0)
    base.update(kw)
    return P.Config(nx, ny, nz, **base)


def run_pair(P, oracle, cfg, warm=15, steps=1, theta=None, beads=None):
    p, fR, fB, cot = oracle_state(oracle, cfg, warm, theta)
    sim = P.Simulation([cfg])
    if theta is not None:
        sim.set_substrate_pattern(0, theta)
    sim.write(0, "populations", np.stack([fR, fB]))
    ob = None
    if beads is not None:
        fil, pos, X = beads
        n_b = int(np.max(pos)) + 1
        nw = len(X) // n_b
        cen = X.reshape(nw, n_b, 3).mean(axis=1)
        dirs = X.reshape(nw, n_b, 3)[:, -1] - X.reshape(nw, n_b, 3)[:, 0]
        sim.add_nanowires(0, nw, n_b * cfg.d0, cen, dirs)
        ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, n_b, cfg))
    acc = oracle.Acc()
    for _ in range(steps):
        oracle.step(p, fR, fB, cot, acc, ob)
    sim.step(steps)
    sim.sync()
    return sim, p, fR, fB, cot, acc, ob


def sim_free_positions(cen, dirs, n_b, cfg):
    """Bead positions of straight filaments built on the test side (same rule as the library)."""
    d = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    X = np.concatenate([[c + (k - (n_b - 1) / 2.0) * cfg.d0 * dd for k in range(n_b)] for c, dd in zip(cen, d)])
    X[:, 0] %= cfg.nx
    X[:, 1] %= cfg.ny
    return X


# ---------------------------------------------------------------------------- fluid
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_one_step_matches_oracle(lbm, oracle, prec):
    cfg = droplet_cfg(lbm, prec=prec)
    theta = inputs.stripe_angles(cfg.nx, cfg.ny, 8, 60.0, 110.0)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, theta=theta)
    got = sim.read(0, "populations")
    assert pop_err(got, fR, fB) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_red_free_gas_warps_match_oracle(lbm, oracle, prec):
    """A tall gas region above a low droplet: in 16-bit storage most 32-node rows there hold
    no red at all (the liquid fraction -1/2 exactly), and the fused kernel takes its red-free
    form for those warps. One step against the oracle, and the rows stay red-free."""
    cfg = droplet_cfg(lbm, nx=64, ny=24, nz=40, prec=prec, c=10.0, J0=1e-3, evap_start=0)
    p, fR, fB, cot = oracle_state(oracle, cfg, 15)
    sim = lbm.Simulation([cfg])
    sim.write(0, "populations", np.stack([fR, fB]))
    before = sim.read(0, "populations")
    red_rows = before[0].reshape(19, cfg.nz, cfg.ny, cfg.nx // 32, 32)
    free = np.all(red_rows == 0.0, axis=(0, 4))  # [z][y][row piece]
    assert free.mean() > 0.4  # the red-free form is exercised
    acc = oracle.Acc()
    oracle.step(p, fR, fB, cot, acc)
    sim.step(1)
    sim.sync()
    got = sim.read(0, "populations")
    assert pop_err(got, fR, fB) < TOL[prec]
    after = got[0].reshape(19, cfg.nz, cfg.ny, cfg.nx // 32, 32)
    # a red-free row far from the liquid stays red-free (no red streams in from above)
    top = free.copy()
    top[: cfg.nz - 4] = False
    assert np.all(after[:, top] == 0.0)


def test_fp64_ten_steps_with_evaporation_and_budgets(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64", J0=2e-3, evap_start=0)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, steps=10)
    got = sim.read(0, "populations")
    assert pop_err(got, fR, fB) < 1e-11
    a = sim.read(0, "accum")
    assert a[0] == 10
    assert a[1] == pytest.approx(acc.h0, rel=1e-13)
    assert acc.evaporated > 0
    assert a[2] == pytest.approx(acc.evaporated, rel=1e-11)
    assert a[3] == pytest.approx(acc.top_in, rel=1e-12)
    assert a[4] == pytest.approx(acc.top_out, rel=1e-11)


def test_async_budget_read_matches_the_blocking_read(lbm, oracle):
    """The budget record copied behind the steps into pinned memory equals the blocking read
    once the stream has been synchronised."""
    import torch
    cfg = droplet_cfg(lbm, prec="fp32", J0=2e-3, evap_start=0)
    sim = lbm.Simulation([cfg])
    buf = torch.zeros(6, dtype=torch.float64, pin_memory=True)
    for _ in range(4):
        sim.step(1)
        sim.read_accum_async(0, buf)
    sim.sync()
    ref = sim.read(0, "accum")
    assert ref[0] == 4 and ref[2] > 0
    assert np.array_equal(buf.numpy(), ref)


def test_fp64_moments_and_colour_match_oracle_fields(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64")
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg)
    f = oracle.fields(p, fR, fB, cot)
    m = sim.read(0, "moments")
    assert np.allclose(m[..., 0], f["rhoR"], rtol=1e-13, atol=1e-15)
    assert np.allclose(m[..., 1], f["rhoB"], rtol=1e-13, atol=1e-15)
    assert np.allclose(m[..., 2:], f["j"], rtol=1e-11, atol=1e-15)
    assert np.allclose(sim.read(0, "colour"), f["C"], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("shape", [(5, 3, 4), (33, 9, 7), (1, 1, 6), (64, 8, 3)])
def test_ragged_and_tiny_lattices(lbm, oracle, shape):
    nx, ny, nz = shape
    cfg = lbm.Config(nx, ny, nz, prec="fp64", cx=nx / 2, cy=ny / 2, cz=-0.5, a=max(nx * 0.4, 1),
                     b=max(ny * 0.4, 1), c=nz * 0.6, sigma=0.02, top_bc=1, theta_deg=75.0,
                     J0=1e-3, evap_start=0, body=(1e-5, 0, 0))
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, warm=3, steps=3)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-12


@pytest.mark.parametrize("prec,shape,top_bc", [
    ("fp32", (37, 11, 9), 1), ("fp32", (36, 13, 9), 0), ("fp32", (68, 6, 7), 1),
    ("fp16", (37, 11, 9), 0), ("fp16", (68, 13, 10), 1), ("bf16", (36, 13, 9), 0)])
def test_staged_pulls_on_ragged_tiles(lbm, oracle, prec, shape, top_bc):
    """Both ways the 32- and 16-bit fused kernel stages its pull: per-element copies
    (nx not a multiple of 4) and bulk row copies (nx a multiple of 4), on lattices whose
    last tiles are narrower and shorter than the rest, with the gas top or the top wall."""
    nx, ny, nz = shape
    cfg = droplet_cfg(lbm, nx=nx, ny=ny, nz=nz, prec=prec, top_bc=top_bc, J0=1e-3, evap_start=0)
    theta = inputs.stripe_angles(nx, ny, 4, 60.0, 110.0)
    for tiling in (4, 6):
        p, fR, fB, cot = oracle_state(oracle, cfg, 10, theta)
        sim = lbm.Simulation([cfg])
        sim.set_substrate_pattern(0, theta)
        sim.set_tiling(tiling)
        sim.write(0, "populations", np.stack([fR, fB]))
        acc = oracle.Acc()
        for _ in range(2):
            oracle.step(p, fR, fB, cot, acc)
        sim.step(2)
        sim.sync()
        assert pop_err(sim.read(0, "populations"), fR, fB) < 2 * TOL[prec], (prec, shape, tiling)
        sim.close()


def test_top_wall_and_body_force(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64", top_bc=0, body=(2e-6, -1e-6, 0.0))
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, steps=4)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-12


def test_gpu_initial_droplet_matches_oracle(lbm, oracle):
    for prec in ("fp64", "fp32"):
        cfg = droplet_cfg(lbm, prec=prec)
        sim = lbm.Simulation([cfg])
        p = oracle_params(oracle, cfg)
        fR, fB = oracle.init_droplet(p, 0, cfg.cx, cfg.cy, cfg.cz, cfg.a, cfg.b, cfg.c, cfg.width)
        assert pop_err(sim.read(0, "populations"), fR, fB) < (1e-14 if prec == "fp64" else 1e-7)


def test_fp32_mass_is_conserved_over_many_steps(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp32", top_bc=0)
    sim = lbm.Simulation([cfg])
    d0 = sim.descriptors(0)
    sim.step(300)
    d1 = sim.descriptors(0)
    assert abs(d1["mass_R"] - d0["mass_R"]) < 1e-5 * d0["mass_R"]
    assert abs(d1["mass_B"] - d0["mass_B"]) < 1e-5 * d0["mass_B"]


# ---------------------------------------------------------------------------- beads
def bead_case(cfg, seed=7, n_fil=6, n_b=4):
    lo = [cfg.cx - cfg.a * 0.5, cfg.cy - cfg.b * 0.5, 2.5]
    hi = [cfg.cx + cfg.a * 0.5, cfg.cy + cfg.b * 0.5, cfg.c * 0.6]
    cen, dirs = inputs.random_filaments(seed, n_fil, n_b, cfg.d0, lo, hi, min_dist=2.05)
    fil, pos, X = inputs.straight_filaments(cen, dirs, n_b, cfg.d0)
    return fil, pos, X


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_beads_one_step_match_oracle(lbm, oracle, prec):
    cfg = droplet_cfg(lbm, nx=48, ny=32, nz=20, prec=prec, max_beads=64, eps_coh=1.0 * 0.006,
                      xi=0.02, gamma=1.0, a=18, b=11, c=14)
    beads = bead_case(cfg)
    sim, p, fR, fB, cot, acc, ob = run_pair(lbm, oracle, cfg, warm=5, steps=3, beads=beads)
    X = sim.read(0, "bead_x")
    V = sim.read(0, "bead_v")
    F = sim.read(0, "bead_f")
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert np.allclose(X, ob.X, rtol=0, atol=tol * 10)
    assert np.allclose(V, ob.V, rtol=0, atol=tol)
    assert np.allclose(F, ob.F, rtol=0, atol=tol)
    assert pop_err(sim.read(0, "populations"), fR, fB) < TOL[prec] * 10


def test_fene_overstretch_reports_status(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64", max_beads=8)
    sim = lbm.Simulation([cfg])
    sim.add_nanowires(0, 1, 4.0, np.array([[cfg.cx, cfg.cy, 5.0]]), np.array([[1.0, 0, 0]]))
    X = sim.read(0, "bead_x")
    X[1] = X[0] + np.array([2.6, 0, 0])
    sim.write(0, "bead_x", X)
    sim.step(1)
    from paper_2607_06794_b300 import _lib
    assert sim.status() == _lib.EFENE
    sim.clear_error()
    assert sim.status() == _lib.OK


def test_nan_population_reports_status(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp32")
    sim = lbm.Simulation([cfg])
    f = sim.read(0, "populations")
    f[0, 3, 5, 5, 5] = np.nan
    sim.write(0, "populations", f)
    sim.step(2)
    from paper_2607_06794_b300 import _lib
    assert sim.status() == _lib.ENAN


# ---------------------------------------------------------------------------- descriptors
def test_descriptors_match_oracle(lbm, oracle):
    cfg = droplet_cfg(lbm, nx=64, ny=48, nz=24, prec="fp64", max_beads=400, a=24, b=18, c=16)
    cfg = dataclasses.replace(cfg, x_src=20.0, x_snk=44.0)
    sim = lbm.Simulation([cfg])
    g = inputs.rng(3)
    nw = 60
    cen = np.c_[g.uniform(12, 52, nw), g.uniform(10, 38, nw), g.uniform(2, 10, nw)]
    dirs = np.c_[g.normal(size=nw), g.normal(size=nw), 0.2 * g.normal(size=nw)]
    sim.add_nanowires(0, nw, 8.0, cen, dirs)
    X = sim_free_positions(cen, dirs, 4, cfg)
    fil = np.repeat(np.arange(nw), 4)
    pos = np.tile(np.arange(4), nw)
    p = oracle_params(oracle, cfg)
    sx, nc, perc, _ = oracle.descriptors(p, fil, pos, X, cfg.rcon, cfg.x_src, cfg.x_snk)
    d = sim.descriptors(0)
    assert d["n_beads"] == 4 * nw and d["n_bonds"] == 3 * nw
    assert d["n_clusters"] == nc
    assert bool(d["percolates"]) == perc
    assert d["S_x"] == pytest.approx(sx, abs=1e-12)


def test_random_nanowire_placement_is_valid(lbm, oracle):
    cfg = droplet_cfg(lbm, nx=64, ny=32, nz=24, prec="fp32", max_beads=200, a=24, b=10, c=14)
    sim = lbm.Simulation([cfg])
    sim.add_nanowires(0, 20, 8.0, seed=99)
    X = sim.read(0, "bead_x")
    topo = sim.read(0, "bead_topo")
    C = sim.read(0, "colour")
    assert X.shape == (80, 3)
    for k in range(len(X)):
        x, y, z = np.rint(X[k]).astype(int)
        assert C[z, y % cfg.ny, x % cfg.nx] > 0.9
    # beads of different filaments further apart than d0
    for a in range(len(X)):
        for b in range(a + 1, len(X)):
            if topo[a, 0] != topo[b, 0]:
                d = X[b] - X[a]
                d[0] -= cfg.nx * np.round(d[0] / cfg.nx)
                d[1] -= cfg.ny * np.round(d[1] / cfg.ny)
                assert np.linalg.norm(d) > cfg.d0


# ---------------------------------------------------------------------------- batching
def test_batched_uneven_lattices_match_oracle_per_instance(lbm, oracle):
    """Three lattices of different sizes in one handle advance like three oracle runs."""
    cfgs = [droplet_cfg(lbm, nx=40, ny=24, nz=20, prec="fp64", J0=1e-3, evap_start=0),
            droplet_cfg(lbm, nx=64, ny=16, nz=12, prec="fp64", theta_deg=100.0, sigma=0.02),
            droplet_cfg(lbm, nx=24, ny=40, nz=9, prec="fp64", top_bc=0, J0=2e-3, evap_start=1)]
    states = [oracle_state(oracle, c, 5) for c in cfgs]
    sim = lbm.Simulation(cfgs)
    for k, (p, fR, fB, cot) in enumerate(states):
        sim.write(k, "populations", np.stack([fR, fB]))
    accs = [oracle.Acc() for _ in cfgs]
    for _ in range(4):
        for (p, fR, fB, cot), acc in zip(states, accs):
            oracle.step(p, fR, fB, cot, acc)
    sim.step(4)
    sim.sync()
    for k, ((p, fR, fB, cot), acc) in enumerate(zip(states, accs)):
        assert pop_err(sim.read(k, "populations"), fR, fB) < 1e-12, k
        a = sim.read(k, "accum")
        assert a[2] == pytest.approx(acc.evaporated, rel=1e-11, abs=1e-300)


def test_batched_beads_in_two_instances(lbm, oracle):
    cfgs = [droplet_cfg(lbm, nx=48, ny=32, nz=20, prec="fp64", max_beads=40, xi=0.02, a=18, b=11, c=14),
            droplet_cfg(lbm, nx=32, ny=32, nz=16, prec="fp64", max_beads=40, xi=0.01, a=11, b=11, c=11,
                        eps_coh=0.012)]
    sim = lbm.Simulation(cfgs)
    obs, states = [], []
    for k, c in enumerate(cfgs):
        p, fR, fB, cot = oracle_state(oracle, c, 3)
        sim.write(k, "populations", np.stack([fR, fB]))
        fil, pos, X = bead_case(c, seed=20 + k, n_fil=4)
        cen = X.reshape(4, 4, 3).mean(axis=1)
        dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
        sim.add_nanowires(k, 4, 8.0, cen, dirs)
        obs.append(oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, c)))
        states.append((p, fR, fB, cot))
    for _ in range(2):
        for (p, fR, fB, cot), ob in zip(states, obs):
            oracle.step(p, fR, fB, cot, oracle.Acc(), ob)
    sim.step(2)
    sim.sync()
    for k, ((p, fR, fB, cot), ob) in enumerate(zip(states, obs)):
        assert np.allclose(sim.read(k, "bead_x"), ob.X, atol=1e-11)
        assert pop_err(sim.read(k, "populations"), fR, fB) < 1e-11


# ---------------------------------------------------------------------------- full size
def test_full_size_c2_step_in_bench_configuration(lbm, oracle):
    """256x128x64 FP32 with 200 wires (the benchmark workload and launch configuration):
    one step from the same oracle state, every population compared."""
    from paper_2607_06794_b300 import workloads
    wl = workloads.droplet_c2("fp32")
    cfg = wl.cfgs[0]
    p = oracle_params(oracle, cfg)
    fR, fB = oracle.init_droplet(p, cfg.shape, cfg.cx, cfg.cy, cfg.cz, cfg.a, cfg.b, cfg.c, cfg.width)
    cot = oracle.cot_map(wl.thetas[0])
    start = np.stack([fR, fB])
    lo = [cfg.cx - 0.6 * cfg.a, cfg.cy - 0.6 * cfg.b, 2.5]
    hi = [cfg.cx + 0.6 * cfg.a, cfg.cy + 0.6 * cfg.b, 0.6 * cfg.c]
    cen, dirs = inputs.random_filaments(cfg.seed, 200, 4, cfg.d0, lo, hi, min_dist=2.05)
    fil, pos, X = inputs.straight_filaments(cen, dirs, 4, cfg.d0)
    ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfg))
    acc = oracle.Acc()
    oracle.step(p, fR, fB, cot, acc, ob)
    # the benchmark autotunes its tiling: every candidate is checked
    for k in range(lbm.tiling_count()):
        sim = lbm.Simulation([cfg])
        sim.set_substrate_pattern(0, wl.thetas[0])
        sim.write(0, "populations", start)
        sim.set_tiling(k)
        sim.add_nanowires(0, 200, 8.0, cen, dirs)
        sim.step(1)
        sim.sync()
        assert pop_err(sim.read(0, "populations"), fR, fB) < TOL["fp32"] * 5, k
        assert np.allclose(sim.read(0, "bead_x"), ob.X, atol=1e-6), k
        a = sim.read(0, "accum")
        assert a[2] == pytest.approx(acc.evaporated, rel=1e-4), k
        del sim


def test_full_size_c4_batch_step_on_sampled_lattices(lbm, oracle):
    """The 64-lattice FP16 batch (26.7 M nodes, 64..192 x 64 x 48) as the benchmark runs it: one
    step of the whole batch under four tilings (whole columns, 16-plane chunks, and the two mixed
    tilings: whole columns in full waves, then the remaining columns in short chunks); three sampled
    lattices (smallest, a middle one with cohesion, largest) start from oracle droplets with wires
    placed by the test and are compared with the FP64 oracle, every population."""
    from paper_2607_06794_b300 import workloads
    wl = workloads.batched_c4("fp16")
    sampled = [0, 37, 63]
    refs, starts, placed = {}, {}, {}
    for k in sampled:
        cfg = wl.cfgs[k]
        p = oracle_params(oracle, cfg)
        fR, fB = oracle.init_droplet(p, cfg.shape, cfg.cx, cfg.cy, cfg.cz, cfg.a, cfg.b, cfg.c, cfg.width)
        cot = oracle.cot_map(wl.thetas[k])
        nw, length = wl.wires[k]
        n_b = max(1, int(round(length / cfg.d0)))
        lo = [cfg.cx - 0.5 * cfg.a, cfg.cy - 0.5 * cfg.b, 2.5]
        hi = [cfg.cx + 0.5 * cfg.a, cfg.cy + 0.5 * cfg.b, 0.5 * cfg.c]
        cen, dirs = inputs.random_filaments(100 + k, min(nw, 60), n_b, cfg.d0, lo, hi, min_dist=2.05)
        fil, pos, X = inputs.straight_filaments(cen, dirs, n_b, cfg.d0)
        ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, n_b, cfg))
        starts[k] = np.stack([fR, fB])
        placed[k] = (len(cen), n_b * cfg.d0, cen, dirs)
        acc = oracle.Acc()
        oracle.step(p, fR, fB, cot, acc, ob)
        refs[k] = (fR, fB, ob.X.copy(), acc)
    # 32x4 columns: the automatic chunk (whole 48-plane columns over this batch), 16-plane chunks;
    # the mixed tilings on 32x4 and 32x8 columns
    big = [lbm.Config(512, 256, 128)]  # 128 planes divide into every fixed chunk
    mixed = [k for k in range(lbm.tiling_count())
             if len(np.unique(np.diff(lbm.tiling_table(big, k)[:, 3:5], axis=1))) > 1]
    assert len(mixed) == 2
    for t in [4, 5] + mixed:
        sim = lbm.Simulation(wl.cfgs)
        for k in range(len(wl.cfgs)):
            sim.set_substrate_pattern(k, wl.thetas[k])
            if k in placed:
                sim.write(k, "populations", starts[k])
                sim.add_nanowires(k, *placed[k])
            else:
                sim.add_nanowires(k, wl.wires[k][0], wl.wires[k][1], seed=wl.cfgs[k].seed)
        sim.set_tiling(t)
        sim.step(1)
        sim.sync()
        assert sim.status() == 0, t
        for k in sampled:
            fR, fB, Xr, acc = refs[k]
            assert pop_err(sim.read(k, "populations"), fR, fB) < TOL["fp16"], (t, k)
            assert np.allclose(sim.read(k, "bead_x"), Xr, rtol=0, atol=1e-3), (t, k)
            a = sim.read(k, "accum")
            assert a[2] == pytest.approx(acc.evaporated, rel=2e-2), (t, k)
        del sim


def test_large_bead_instance_uses_cell_list_and_matches_oracle(lbm, oracle):
    """More beads than one block holds: cell-list neighbour search and one launch per sub-step."""
    cfg = droplet_cfg(lbm, nx=96, ny=64, nz=24, prec="fp64", max_beads=1400, eps_coh=0.006, xi=0.02,
                      a=40, b=26, c=16)
    p, fR, fB, cot = oracle_state(oracle, cfg, 2)
    lo = [cfg.cx - 34, cfg.cy - 20, 2.5]
    hi = [cfg.cx + 34, cfg.cy + 20, 13.0]
    cen, dirs = inputs.random_filaments(31, 270, 4, cfg.d0, lo, hi, min_dist=2.05)
    assert len(cen) == 270  # 1080 beads: more than one block holds
    fil, pos, X = inputs.straight_filaments(cen, dirs, 4, cfg.d0)
    sim = lbm.Simulation([cfg])
    sim.write(0, "populations", np.stack([fR, fB]))
    sim.add_nanowires(0, 270, 8.0, cen, dirs)
    ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfg))
    acc = oracle.Acc()
    for _ in range(2):
        oracle.step(p, fR, fB, cot, acc, ob)
    sim.step(2)
    sim.sync()
    assert np.allclose(sim.read(0, "bead_x"), ob.X, atol=1e-11)
    assert np.allclose(sim.read(0, "bead_f"), ob.F, atol=1e-11)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-11


def test_many_beads_in_a_batch_take_four_lanes_per_bead_and_match_oracle(lbm, oracle):
    """Above 2048 beads in the batch the sub-steps run four lanes per bead (two stencil
    corners per lane, one integrated component per lane): two copies of the 1080-bead
    instance, each compared with the FP64 oracle."""
    cfg = droplet_cfg(lbm, nx=96, ny=64, nz=24, prec="fp64", max_beads=1400, eps_coh=0.006, xi=0.02,
                      a=40, b=26, c=16, eps_s=0.01)
    p, fR, fB, cot = oracle_state(oracle, cfg, 2)
    lo = [cfg.cx - 34, cfg.cy - 20, 0.6]
    hi = [cfg.cx + 34, cfg.cy + 20, 13.0]
    cen, dirs = inputs.random_filaments(32, 270, 4, cfg.d0, lo, hi, min_dist=2.05)
    assert len(cen) == 270
    fil, pos, X = inputs.straight_filaments(cen, dirs, 4, cfg.d0)
    assert X[:, 2].min() < 1.0  # some beads feel the substrate (adhesion, friction)
    sim = lbm.Simulation([cfg, cfg])
    for k in range(2):
        sim.write(k, "populations", np.stack([fR, fB]))
        sim.add_nanowires(k, 270, 8.0, cen, dirs)
    ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfg))
    acc = oracle.Acc()
    for _ in range(2):
        oracle.step(p, fR, fB, cot, acc, ob)
    sim.step(2)
    sim.sync()
    for k in range(2):
        assert np.allclose(sim.read(k, "bead_x"), ob.X, atol=1e-11), k
        assert np.allclose(sim.read(k, "bead_v"), ob.V, atol=1e-11), k
        assert np.allclose(sim.read(k, "bead_f"), ob.F, atol=1e-11), k
        assert pop_err(sim.read(k, "populations"), fR, fB) < 1e-11, k


def test_checkpoint_restore_with_beads_continues_the_run(lbm, oracle):
    """Fields read from a run and written into a fresh handle (step counter first, then the
    populations and the bead state) continue exactly as the original run does."""
    cfg = droplet_cfg(lbm, nx=48, ny=32, nz=20, prec="fp64", max_beads=40, xi=0.02, a=18, b=11, c=14,
                      J0=1e-3, evap_start=0)
    p, fR, fB, cot = oracle_state(oracle, cfg, 3)
    fil, pos, X = bead_case(cfg, seed=31, n_fil=4)
    cen = X.reshape(4, 4, 3).mean(axis=1)
    dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
    a = lbm.Simulation([cfg])
    a.write(0, "populations", np.stack([fR, fB]))
    a.add_nanowires(0, 4, 8.0, cen, dirs)
    a.step(3)
    saved = {f: a.read(0, f) for f in ("accum", "populations", "bead_x", "bead_v", "bead_f")}
    b = lbm.Simulation([cfg])
    b.write(0, "accum", saved["accum"])
    b.write(0, "populations", saved["populations"])
    b.add_nanowires(0, 4, 8.0, cen, dirs)
    for f in ("bead_x", "bead_v", "bead_f"):
        b.write(0, f, saved[f])
    a.step(3)
    b.step(3)
    assert b.status() == 0 and a.status() == 0
    assert np.allclose(b.read(0, "bead_x"), a.read(0, "bead_x"), rtol=0, atol=1e-12)
    pa, pb = a.read(0, "populations"), b.read(0, "populations")
    assert np.max(np.abs(pa - pb)) < 1e-12


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_restore_continues_up_to_the_rounding_of_the_stored_words(lbm, oracle, prec):
    """A 16-bit run pushes the next step's moments from the values before rounding, while a
    restore rebuilds them from the stored (rounded) words, so the restored run continues the
    unbroken one only up to that rounding: after 3 more steps the populations agree to the
    16-bit tolerance of the one-step parity test, the beads to 1e-5."""
    cfg = droplet_cfg(lbm, nx=48, ny=32, nz=20, prec=prec, max_beads=40, xi=0.02, a=18, b=11, c=14,
                      J0=1e-3, evap_start=0)
    fil, pos, X = bead_case(cfg, seed=31, n_fil=4)
    cen = X.reshape(4, 4, 3).mean(axis=1)
    dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
    a = lbm.Simulation([cfg])
    a.add_nanowires(0, 4, 8.0, cen, dirs)
    a.step(4)
    saved = {f: a.read(0, f) for f in ("accum", "populations", "bead_x", "bead_v", "bead_f")}
    b = lbm.Simulation([cfg])
    b.write(0, "accum", saved["accum"])
    b.write(0, "populations", saved["populations"])
    b.add_nanowires(0, 4, 8.0, cen, dirs)
    for f in ("bead_x", "bead_v", "bead_f"):
        b.write(0, f, saved[f])
    # the FP64 host form re-encodes to the same words up to the host's recomputation of the
    # liquid fraction, whose last bit can move where the fraction is near zero
    sp = saved["populations"]
    assert pop_err(b.read(0, "populations"), sp[0], sp[1]) < 1e-6
    a.step(3)
    b.step(3)
    assert b.status() == 0 and a.status() == 0
    pa, pb = a.read(0, "populations"), b.read(0, "populations")
    assert pop_err(pb, pa[0], pa[1]) < TOL[prec]
    assert np.allclose(b.read(0, "bead_x"), a.read(0, "bead_x"), rtol=0, atol=1e-5)


def test_tall_lattice_with_beads_in_the_upper_chunk(lbm, oracle):
    """nz = 300 is split into z-chunks (at most 240 planes each) whose coupling-tile flags the
    fused kernel keeps in a bit mask per column; wires near z = 280 exercise the upper chunk."""
    cfg = droplet_cfg(lbm, nx=16, ny=16, nz=300, prec="fp64", max_beads=16, a=7.0, b=7.0, c=295.0,
                      xi=0.02, gamma=1.0, theta_deg=80.0)
    cen = np.array([[7.5, 6.0, 280.0], [8.0, 10.0, 284.0]])
    dirs = np.array([[1.0, 0.2, 0.1], [0.3, -1.0, 0.2]])
    n_b = 4
    fil, pos, X = inputs.straight_filaments(cen, dirs, n_b, cfg.d0)
    sim, p, fR, fB, cot, acc, ob = run_pair(lbm, oracle, cfg, warm=2, steps=2, beads=(fil, pos, X))
    assert sim.status() == 0
    assert np.allclose(sim.read(0, "bead_x"), ob.X, rtol=0, atol=1e-11)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-11


def test_every_tiling_matches_the_oracle_on_a_batch(lbm, oracle):
    """Every candidate tiling (32x8 and 32x4 columns, automatic, 16-, 32- and 64-plane
    z-chunks) computes the oracle's steps on a batch: a thin lattice of short columns and a
    second lattice that carries beads; both evaporate."""
    cfgs = [droplet_cfg(lbm, nx=192, ny=160, nz=4, prec="fp64", a=60.0, b=50.0, c=3.5, theta_deg=60.0,
                        J0=1e-3, evap_start=0),
            droplet_cfg(lbm, nx=48, ny=32, nz=20, prec="fp64", max_beads=40, xi=0.02, a=18, b=11, c=14,
                        J0=2e-3, evap_start=0)]
    states = [oracle_state(oracle, c, 2) for c in cfgs]
    start = [np.stack([fR, fB]) for (p, fR, fB, cot) in states]
    fil, pos, X = bead_case(cfgs[1], seed=41, n_fil=4)
    cen = X.reshape(4, 4, 3).mean(axis=1)
    dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
    ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfgs[1]))
    accs = [oracle.Acc() for _ in cfgs]
    for _ in range(3):
        for k, ((p, fR, fB, cot), acc) in enumerate(zip(states, accs)):
            oracle.step(p, fR, fB, cot, acc, ob if k == 1 else None)
    assert accs[0].evaporated > 0 and accs[1].evaporated > 0
    for t in range(lbm.tiling_count()):
        sim = lbm.Simulation(cfgs)
        for k in range(2):
            sim.write(k, "populations", start[k])
        sim.set_tiling(t)
        sim.add_nanowires(1, 4, 8.0, cen, dirs)
        sim.step(3)
        sim.sync()
        assert sim.status() == 0, t
        for k, ((p, fR, fB, cot), acc) in enumerate(zip(states, accs)):
            assert pop_err(sim.read(k, "populations"), fR, fB) < 1e-11, (t, k)
            a = sim.read(k, "accum")
            assert a[2] == pytest.approx(acc.evaporated, rel=1e-11), (t, k)
            assert a[3] == pytest.approx(acc.top_in, rel=1e-12), (t, k)
        assert np.allclose(sim.read(1, "bead_x"), ob.X, rtol=0, atol=1e-11), t
        del sim


def test_graph_direct_and_profiled_steps_with_beads_and_sink_match_the_oracle(lbm, oracle):
    """Graph-replayed, directly launched and profiled steps (events around the fused launch),
    mixed in one run with beads and the evaporation sink, advance like the oracle. The sink acts
    wherever grad C is nonzero, also in the liquid where |grad C| is below the 1e-8 threshold
    of the interface normal (Eq. (8) takes |grad C| itself)."""
    cfg = droplet_cfg(lbm, nx=64, ny=40, nz=20, prec="fp64", max_beads=40, xi=0.02, a=20, b=12, c=14,
                      J0=1e-3, evap_start=0)
    p, fR, fB, cot = oracle_state(oracle, cfg, 2)
    fil, pos, X = bead_case(cfg, seed=53, n_fil=4)
    cen = X.reshape(4, 4, 3).mean(axis=1)
    dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
    sim = lbm.Simulation([cfg])
    sim.write(0, "populations", np.stack([fR, fB]))
    sim.add_nanowires(0, 4, 8.0, cen, dirs)
    ob = oracle.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfg))
    acc = oracle.Acc()
    for _ in range(6):
        oracle.step(p, fR, fB, cot, acc, ob)
    sim.step(2)
    sim.profile_steps(2)
    sim.step(1)
    sim.profile_steps(1)
    sim.sync()
    assert sim.status() == 0
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-11
    assert np.allclose(sim.read(0, "bead_x"), ob.X, rtol=0, atol=1e-11)
    a = sim.read(0, "accum")
    assert a[0] == 6
    assert a[2] == pytest.approx(acc.evaporated, rel=1e-11)
