"""GPU parity of the deposit analysis (Sec. II.B, Eqs. (13)-(18)) through the C ABI.

The bead topology is created through lbm_add_nanowires with explicit centres,
then the test's own bead positions are written into the handle, so that the
library and the FP64 oracle (oracle/network.py) analyse the same deposit.
"""
import dataclasses

import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu

# the CG solve stops at ||r|| <= 1e-13 ||b||; potentials are O(1)
TOL_V = 1e-9
TOL_REL = 1e-9


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_06794_b300 import build

    build.build()
    import paper_2607_06794_b300 as P

    return P


@pytest.fixture(scope="module")
def net():
    from oracle import network

    return network


def deposit_sim(P, nx, ny, fil_sets, x_src, x_snk, nz=12, prec="fp32"):
    """One handle with one instance per (cen, dirs, n_beads, X) set; positions written as given."""
    cfgs = []
    for cen, dirs, nb, X in fil_sets:
        cfgs.append(P.Config(nx, ny, nz, prec=prec, cx=nx / 2 - 0.5, cy=ny / 2 - 0.5, cz=-0.5, a=nx * 0.4,
                             b=ny * 0.4, c=nz * 0.8, theta_deg=90.0, top_bc=1, max_beads=len(X) + 8,
                             x_src=x_src, x_snk=x_snk))
    sim = P.Simulation(cfgs)
    for k, (cen, dirs, nb, X) in enumerate(fil_sets):
        sim.add_nanowires(k, len(cen), nb * cfgs[k].d0, cen, dirs)
        sim.write(k, "bead_x", np.ascontiguousarray(X, np.float64))
    return sim


def wrap(X, nx, ny):
    X = np.array(X, np.float64)
    X[:, 0] %= nx
    X[:, 1] %= ny
    return X


def check_conductivity(sim, k, net, fil, pos, X, nx, ny, x_src, x_snk):
    got = sim.conductivity(k, tol=1e-13)
    ref = net.conductivity(fil, pos, X, nx, ny, x_src, x_snk)
    assert got["n_src"] == ref["n_src"] and got["n_snk"] == ref["n_snk"]
    assert got["n_edges"] == ref["n_edges"]
    assert got["I_ref"] == pytest.approx(ref["I_ref"], rel=1e-15)
    assert got["kappa"] == pytest.approx(ref["kappa"], rel=TOL_REL, abs=1e-12)
    assert got["I_tot"] == pytest.approx(ref["I_tot"], rel=TOL_REL, abs=1e-12)
    assert got["I_sink"] == pytest.approx(ref["I_sink"], rel=TOL_REL, abs=1e-12)
    V = sim.read(k, "bead_potential")
    Ist = sim.read(k, "bead_current")
    assert np.max(np.abs(V - ref["V"])) < TOL_V
    assert np.max(np.abs(Ist - ref["I_node"])) < TOL_V * max(1.0, np.max(ref["I_node"]))
    return got, ref


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_conductivity_matches_oracle_on_random_deposits(lbm, net, seed):
    nx, ny = 64, 40
    cen, dirs, fil, pos, X = inputs.flat_deposit(seed, 120, 6, (14, 50, 8, 32))
    X = wrap(X, nx, ny)
    sim = deposit_sim(lbm, nx, ny, [(cen, dirs, 6, X)], 20.0, 44.0)
    got, ref = check_conductivity(sim, 0, net, fil, pos, X, nx, ny, 20.0, 44.0)
    assert ref["kappa"] > 0 and got["iterations"] > 0 and got["residual"] <= 1e-13


def test_conductivity_straight_chain_and_symmetric_bridge(lbm, net):
    nx, ny = 64, 40
    # chain of 11 beads 2 apart from x = 10 to 30: kappa* = 18 / 20
    X1 = np.array([[10.0 + 2 * k, 10.0, 1.0] for k in range(11)])
    cen1, dirs1 = np.array([[20.0, 10.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
    # four single beads forming a mirror-symmetric bridge between x_src = 10.5 and x_snk = 13
    X2 = np.array([(10.0, 20.0, 1.0), (11.8, 21.0, 1.0), (11.8, 19.2, 1.0), (13.6, 20.0, 1.0)])
    dirs2 = np.tile([1.0, 0.0, 0.0], (4, 1))
    sim = deposit_sim(lbm, nx, ny, [(cen1, dirs1, 11, X1)], 11.0, 29.0)
    got = sim.conductivity(0, tol=1e-14)
    assert got["kappa"] == pytest.approx(0.9, rel=1e-12)
    Ist = sim.read(0, "bead_current")
    assert np.allclose(Ist[1:-1], 0.9, rtol=1e-12) and np.allclose(Ist[[0, -1]], 0.45, rtol=1e-12)
    sim2 = deposit_sim(lbm, nx, ny, [(X2, dirs2, 1, X2)], 10.5, 13.0)
    got2 = sim2.conductivity(0, tol=1e-14)
    V = sim2.read(0, "bead_potential")
    assert V[1] == pytest.approx(0.5, abs=1e-13) and V[2] == pytest.approx(0.5, abs=1e-13)
    gab, gac = 1 / np.hypot(1.8, 1.0), 1 / np.hypot(1.8, 0.8)
    assert got2["I_tot"] == pytest.approx(0.5 * (gab + gac), rel=1e-12)


def test_conductivity_floating_and_one_sided_components(lbm, net):
    nx, ny = 64, 40
    X = np.concatenate([[[10.0 + 2 * k, 10.0, 1.0] for k in range(11)],
                        [[16.0 + 2 * k, 30.0, 1.0] for k in range(3)],
                        [[6.0 + 2 * k, 20.0, 1.0] for k in range(4)]])
    fil = np.repeat([0, 1, 2], [11, 3, 4])
    pos = np.concatenate([np.arange(11), np.arange(3), np.arange(4)])
    # three filaments of different lengths: add them one by one
    cfg = lbm.Config(nx, ny, 12, prec="fp32", cx=31.5, cy=19.5, cz=-0.5, a=25, b=16, c=9, theta_deg=90.0,
                     top_bc=1, max_beads=32, x_src=11.0, x_snk=29.0)
    sim = lbm.Simulation([cfg])
    for nb, c in ((11, (20.0, 10.0, 1.0)), (3, (18.0, 30.0, 1.0)), (4, (9.0, 20.0, 1.0))):
        sim.add_nanowires(0, 1, nb * cfg.d0, np.array([c]), np.array([[1.0, 0.0, 0.0]]))
    sim.write(0, "bead_x", X)
    got, ref = check_conductivity(sim, 0, net, fil, pos, X, nx, ny, 11.0, 29.0)
    assert got["kappa"] == pytest.approx(0.9, rel=1e-12)
    V = sim.read(0, "bead_potential")
    assert np.all(V[11:14] == 0.0) and np.allclose(V[14:], 1.0, atol=1e-13)


def test_conductivity_batched_instances_solve_independently(lbm, net):
    nx, ny = 64, 40
    sets, refs = [], []
    for seed in (3, 4):
        cen, dirs, fil, pos, X = inputs.flat_deposit(seed, 100, 5, (14, 50, 8, 32))
        X = wrap(X, nx, ny)
        sets.append((cen, dirs, 5, X))
        refs.append((fil, pos, X))
    sim = deposit_sim(lbm, nx, ny, sets, 20.0, 44.0)
    for k, (fil, pos, X) in enumerate(refs):
        check_conductivity(sim, k, net, fil, pos, X, nx, ny, 20.0, 44.0)


def test_conductivity_full_size_deposit(lbm, net):
    # 2000 filaments of 8 beads on a 512 x 256 substrate (16,000 beads)
    nx, ny = 512, 256
    cen, dirs, fil, pos, X = inputs.flat_deposit(7, 2000, 8, (100, 412, 90, 166))
    X = wrap(X, nx, ny)
    sim = deposit_sim(lbm, nx, ny, [(cen, dirs, 8, X)], 156.0, 356.0, nz=8)
    got, ref = check_conductivity(sim, 0, net, fil, pos, X, nx, ny, 156.0, 356.0)
    assert got["n_edges"] > 80000


def test_conductivity_rejects_bad_arguments(lbm):
    cen, dirs, fil, pos, X = inputs.flat_deposit(0, 10, 4, (14, 50, 8, 32))
    sim = deposit_sim(lbm, 64, 40, [(cen, dirs, 4, wrap(X, 64, 40))], 20.0, 44.0)
    for kw in (dict(tol=0.0), dict(max_iter=0)):
        with pytest.raises(lbm.LBMError):
            sim.conductivity(0, **kw)
    with pytest.raises(lbm.LBMError):
        sim.profiles(0, 2, 0.0, 10.0, 4, 20.0, 5.0)
    with pytest.raises(lbm.LBMError):
        sim.profiles(0, 0, 10.0, 0.0, 4, 20.0, 5.0)
    with pytest.raises(lbm.LBMError):
        sim.profiles(0, 0, 0.0, 10.0, 0, 20.0, 5.0)


def test_empty_deposits_give_zero_descriptors_network_and_profiles(lbm):
    """A lattice with bead capacity but no wires, and one without capacity: no bonds, no
    clusters, no current (kappa* = 0 with a converged solve), empty bins."""
    cfgs = [lbm.Config(48, 32, 12, prec="fp32", cx=23.5, cy=15.5, cz=-0.5, a=18, b=12, c=9,
                       max_beads=64, x_src=12.0, x_snk=36.0),
            lbm.Config(48, 32, 12, prec="fp32", cx=23.5, cy=15.5, cz=-0.5, a=18, b=12, c=9,
                       x_src=12.0, x_snk=36.0)]
    sim = lbm.Simulation(cfgs)
    sim.step(2)
    for k in range(2):
        d = sim.descriptors(k)
        assert d["n_beads"] == 0 and d["n_clusters"] == 0 and d["percolates"] == 0
        assert d["S_x"] == 0.0
        c = sim.conductivity(k)
        assert c["kappa"] == 0.0 and c["I_tot"] == 0.0 and c["n_edges"] == 0
        assert c["I_ref"] == pytest.approx(1.0 / 24.0, rel=1e-15)
        S, g, nb, nd = sim.profiles(k, 0, 0.0, 48.0, 6, 15.5, 8.0)
        assert np.all(S == 0.0) and np.all(g == 0.0) and np.all(nb == 0) and np.all(nd == 0)
    assert sim.status() == 0


@pytest.mark.parametrize("axis", [0, 1])
def test_profiles_match_oracle(lbm, net, axis):
    nx, ny = 64, 40
    cen, dirs, fil, pos, X = inputs.flat_deposit(5, 120, 6, (10, 54, 4, 36), spread=0.9)
    X = wrap(X, nx, ny)
    sim = deposit_sim(lbm, nx, ny, [(cen, dirs, 6, X)], 20.0, 44.0)
    lo, hi, nb, centre, hw = (8.0, 56.0, 12, 20.0, 6.0) if axis == 0 else (2.0, 38.0, 9, 32.0, 8.0)
    S, g, nbond, nbead = sim.profiles(0, axis, lo, hi, nb, centre, hw)
    rS, rg, rnbond, rnbead = net.profiles(fil, pos, X, nx, ny, axis, lo, hi, nb, centre, hw)
    assert np.array_equal(nbond, rnbond) and np.array_equal(nbead, rnbead)
    assert nbead.sum() > 20 and nbond.sum() > 20
    assert np.max(np.abs(S - rS)) < 1e-12
    assert np.max(np.abs(g - rg)) < 1e-12
