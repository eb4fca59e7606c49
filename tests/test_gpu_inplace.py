"""Esoteric-pull in-place population storage (one buffer read and written in place,
plus ghost slots at the walls) against the FP64 oracle and against the two-buffer
storage: the same step, so the same numbers, in about half the population memory."""
import numpy as np
import pytest

from tests import inputs
from tests.gpu_helpers import oracle_state, pop_err
from tests.test_gpu_parity import TOL, bead_case, droplet_cfg, run_pair, sim_free_positions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import build
    build.build()
    import paper_2607_06794_b300 as P
    return P


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_inplace_one_step_matches_oracle(lbm, oracle, prec):
    cfg = droplet_cfg(lbm, prec=prec, inplace=1)
    theta = inputs.stripe_angles(cfg.nx, cfg.ny, 8, 60.0, 110.0)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, theta=theta)
    assert pop_err(sim.read(0, "populations"), fR, fB) < TOL[prec]


def test_inplace_fp64_steps_with_evaporation_and_gas_top_budgets(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64", J0=2e-3, evap_start=0, inplace=1)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, steps=11)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-11
    a = sim.read(0, "accum")
    assert a[0] == 11
    assert a[2] == pytest.approx(acc.evaporated, rel=1e-11)
    assert a[3] == pytest.approx(acc.top_in, rel=1e-12)
    assert a[4] == pytest.approx(acc.top_out, rel=1e-11)


def test_inplace_top_wall_and_body_force(lbm, oracle):
    cfg = droplet_cfg(lbm, prec="fp64", top_bc=0, body=(2e-6, -1e-6, 0.0), inplace=1)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, steps=5)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-12


@pytest.mark.parametrize("shape,prec,top_bc", [((5, 3, 4), "fp64", 1), ((33, 9, 7), "fp64", 0),
                                               ((1, 1, 6), "fp64", 1), ((64, 8, 3), "fp64", 0),
                                               ((37, 11, 2), "fp32", 0), ((36, 13, 9), "fp16", 1)])
def test_inplace_ragged_and_tiny_lattices(lbm, oracle, shape, prec, top_bc):
    nx, ny, nz = shape
    cfg = lbm.Config(nx, ny, nz, prec=prec, cx=nx / 2, cy=ny / 2, cz=-0.5, a=max(nx * 0.4, 1),
                     b=max(ny * 0.4, 1), c=nz * 0.6, sigma=0.02, top_bc=top_bc, theta_deg=75.0,
                     J0=1e-3, evap_start=0, body=(1e-5, 0, 0), inplace=1)
    sim, p, fR, fB, cot, acc, _ = run_pair(lbm, oracle, cfg, warm=3, steps=3)
    assert pop_err(sim.read(0, "populations"), fR, fB) < (1e-12 if prec == "fp64" else 2 * TOL[prec])


def test_inplace_beads_match_oracle(lbm, oracle):
    cfg = droplet_cfg(lbm, nx=48, ny=32, nz=20, prec="fp64", max_beads=64, eps_coh=1.0 * 0.006,
                      xi=0.02, gamma=1.0, a=18, b=11, c=14, inplace=1)
    beads = bead_case(cfg)
    sim, p, fR, fB, cot, acc, ob = run_pair(lbm, oracle, cfg, warm=5, steps=3, beads=beads)
    assert np.allclose(sim.read(0, "bead_x"), ob.X, rtol=0, atol=1e-10)
    assert np.allclose(sim.read(0, "bead_v"), ob.V, rtol=0, atol=1e-11)
    assert pop_err(sim.read(0, "populations"), fR, fB) < 1e-11


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_inplace_equals_two_buffer_storage(lbm, prec):
    """The same arithmetic in another memory layout: 25 steps of a droplet with a stripe
    pattern and evaporation give the same populations and budgets under both layouts, under
    two tilings, up to the rounding-order noise of the moment push (tile-edge shares are
    added with atomics, whose order varies from run to run under either layout)."""
    theta = inputs.stripe_angles(64, 40, 10, 60.0, 110.0)
    out = {}
    for inplace in (0, 1):
        for tiling in (2, 6):
            cfg = droplet_cfg(lbm, nx=64, ny=40, nz=24, prec=prec, J0=1e-3, evap_start=0, inplace=inplace)
            sim = lbm.Simulation([cfg])
            sim.set_substrate_pattern(0, theta)
            sim.set_tiling(tiling)
            sim.step(25)
            sim.sync()
            out[(inplace, tiling)] = (sim.read(0, "populations"), sim.read(0, "accum"))
            sim.close()
    tol = 1e-6 if prec == "fp32" else 5e-3
    for tiling in (2, 6):
        (pa, aa), (pb, ab) = out[(0, tiling)], out[(1, tiling)]
        assert pop_err(pb, pa[0], pa[1]) < tol, tiling
        assert np.allclose(ab, aa, rtol=1e-6, atol=0), tiling


def test_inplace_restore_continues_the_run_across_parities(lbm, oracle):
    """Populations read after an odd number of steps and written into a fresh in-place handle
    whose step counter is set first continue exactly as the original run does."""
    cfg = droplet_cfg(lbm, prec="fp64", J0=1e-3, evap_start=0, inplace=1, top_bc=0)
    a = lbm.Simulation([cfg])
    a.step(5)
    acc = a.read(0, "accum")
    pops = a.read(0, "populations")
    b = lbm.Simulation([cfg])
    b.write(0, "accum", acc)
    b.write(0, "populations", pops)
    assert np.array_equal(b.read(0, "populations"), pops)
    a.step(4)
    b.step(4)
    assert a.status() == 0 and b.status() == 0
    assert np.max(np.abs(a.read(0, "populations") - b.read(0, "populations"))) < 1e-13


def test_inplace_every_tiling_on_a_batch(lbm, oracle):
    cfgs = [droplet_cfg(lbm, nx=96, ny=40, nz=6, prec="fp64", a=30.0, b=12.0, c=5.0, theta_deg=60.0,
                        J0=1e-3, evap_start=0, inplace=1),
            droplet_cfg(lbm, nx=48, ny=32, nz=20, prec="fp64", max_beads=40, xi=0.02, a=18, b=11, c=14,
                        J0=2e-3, evap_start=0, inplace=1)]
    states = [oracle_state(oracle, c, 2) for c in cfgs]
    start = [np.stack([fR, fB]) for (p, fR, fB, cot) in states]
    fil, pos, X = bead_case(cfgs[1], seed=41, n_fil=4)
    cen = X.reshape(4, 4, 3).mean(axis=1)
    dirs = X.reshape(4, 4, 3)[:, -1] - X.reshape(4, 4, 3)[:, 0]
    import oracle as O
    ob = O.Beads(fil, pos, sim_free_positions(cen, dirs, 4, cfgs[1]))
    accs = [O.Acc() for _ in cfgs]
    for _ in range(3):
        for k, ((p, fR, fB, cot), acc) in enumerate(zip(states, accs)):
            oracle.step(p, fR, fB, cot, acc, ob if k == 1 else None)
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
            assert sim.read(k, "accum")[2] == pytest.approx(acc.evaporated, rel=1e-11), (t, k)
        assert np.allclose(sim.read(1, "bead_x"), ob.X, rtol=0, atol=1e-11), t
        del sim


def test_inplace_halves_the_population_memory(lbm):
    from paper_2607_06794_b300 import workspace_bytes, workloads
    for mk in (workloads.droplet_c2, workloads.droplet_c5):
        c = mk("fp32").cfgs[0]
        two = workspace_bytes([c])
        c.inplace = 1
        one = workspace_bytes([c])
        pops = 2 * 19 * c.nx * c.ny * c.nz * 4
        assert two - one == pytest.approx(pops - 2 * 10 * c.nx * c.ny * 4, abs=4096)
