"""Pins of the deposit-analysis oracle (Sec. II.B, Eqs. (13)-(18)) against closed forms.

Every expected value here comes from hand analysis of a small network or bin
layout (series and parallel resistors, a mirror-symmetric bridge, nodal
analysis of a two-node bridge by Cramer's rule, bins with known counts), not
from the oracle's own matrix assembly or solver.
"""
import numpy as np
import pytest

from oracle import network as net

NX, NY = 64, 40


def chain(x0, n, y, z=1.0, dx=2.0):
    return np.array([[x0 + k * dx, y, z] for k in range(n)])


def test_straight_chain_spanning_the_electrodes():
    # 11 beads 2 apart from x=10 to x=30: ten bonds of resistance 2 in series
    X = chain(10.0, 11, 10.0)
    fil = np.zeros(11, int)
    pos = np.arange(11)
    r = net.conductivity(fil, pos, X, NX, NY, x_src=11.0, x_snk=29.0)
    assert r["n_src"] == 1 and r["n_snk"] == 1 and r["n_edges"] == 10
    assert r["I_tot"] == pytest.approx(1.0 / 20.0, rel=1e-12)
    assert r["I_sink"] == pytest.approx(1.0 / 20.0, rel=1e-12)
    assert r["I_ref"] == pytest.approx(1.0 / 18.0, rel=1e-14)
    assert r["kappa"] == pytest.approx(18.0 / 20.0, rel=1e-12)
    # linear potential, the same current through every interior node, half at the ends
    assert np.allclose(r["V"], 1.0 - (X[:, 0] - 10.0) / 20.0, atol=1e-12)
    assert np.allclose(r["I_node"][1:-1], 0.9, rtol=1e-12)
    assert np.allclose(r["I_node"][[0, -1]], 0.45, rtol=1e-12)


def test_parallel_chains_add_their_conductances():
    X = np.concatenate([chain(10.0, 11, 10.0), chain(10.0, 11, 20.0)])
    fil = np.repeat([0, 1], 11)
    pos = np.tile(np.arange(11), 2)
    r = net.conductivity(fil, pos, X, NX, NY, x_src=11.0, x_snk=29.0)
    assert r["kappa"] == pytest.approx(2 * 0.9, rel=1e-12)


def test_chain_across_the_periodic_y_boundary_uses_the_nearest_image():
    # a chain along y crossing y = 0, source below x=11, sink above x=29 via a zig-zag
    X = chain(10.0, 11, 10.0)
    X[:, 1] = (np.arange(11) % 2) * (NY - 0.4) + 0.2  # alternate y = 0.2 and y = NY - 0.2
    fil = np.zeros(11, int)
    pos = np.arange(11)
    r = net.conductivity(fil, pos, X, NX, NY, x_src=11.0, x_snk=29.0)
    bond = np.hypot(2.0, 0.4)
    assert r["kappa"] == pytest.approx(18.0 / (10 * bond), rel=1e-12)


def test_symmetric_bridge_carries_no_current():
    # A (source) and D (sink) mirror each other about x = 11.8; so do the paths via B and C
    A, B, C, D = (10.0, 20.0, 1.0), (11.8, 21.0, 1.0), (11.8, 19.2, 1.0), (13.6, 20.0, 1.0)
    X = np.array([A, B, C, D])
    fil = np.arange(4)
    pos = np.zeros(4, int)
    r = net.conductivity(fil, pos, X, NX, NY, x_src=10.5, x_snk=13.0)
    assert r["n_edges"] == 5  # A-B, A-C, B-C, B-D, C-D; A-D is 3.6 apart
    assert r["V"][1] == pytest.approx(0.5, abs=1e-13)
    assert r["V"][2] == pytest.approx(0.5, abs=1e-13)
    gab, gac = 1 / np.hypot(1.8, 1.0), 1 / np.hypot(1.8, 0.8)
    assert r["I_tot"] == pytest.approx(0.5 * (gab + gac), rel=1e-12)
    assert r["kappa"] == pytest.approx(0.5 * (gab + gac) * 2.5, rel=1e-12)


def test_asymmetric_bridge_by_nodal_analysis():
    A, B, C, D = (10.0, 20.0, 1.0), (11.8, 20.6, 1.0), (11.95, 19.4, 1.0), (13.8, 20.0, 1.0)
    X = np.array([A, B, C, D])
    d = lambda p, q: np.linalg.norm(np.subtract(p, q))
    gAB, gAC, gBC, gBD, gCD = 1 / d(A, B), 1 / d(A, C), 1 / d(B, C), 1 / d(B, D), 1 / d(C, D)
    assert d(A, D) > 2.1 and max(d(A, B), d(A, C), d(B, C), d(B, D), d(C, D)) < 2.1
    # KCL at B and C with V_A = 1, V_D = 0, solved by Cramer's rule
    a11, a12, b1 = gAB + gBC + gBD, -gBC, gAB
    a21, a22, b2 = -gBC, gAC + gBC + gCD, gAC
    det = a11 * a22 - a12 * a21
    VB = (b1 * a22 - a12 * b2) / det
    VC = (a11 * b2 - b1 * a21) / det
    I_tot = gAB * (1 - VB) + gAC * (1 - VC)
    r = net.conductivity(np.arange(4), np.zeros(4, int), X, NX, NY, x_src=10.5, x_snk=13.5)
    assert r["V"][1] == pytest.approx(VB, rel=1e-12)
    assert r["V"][2] == pytest.approx(VC, rel=1e-12)
    assert r["I_tot"] == pytest.approx(I_tot, rel=1e-12)
    assert r["I_sink"] == pytest.approx(gBD * VB + gCD * VC, rel=1e-12)
    assert r["kappa"] == pytest.approx(I_tot * 3.0, rel=1e-12)
    # Eq. (15) at B: half the sum of |edge currents|
    IB = 0.5 * (gAB * abs(1 - VB) + gBC * abs(VB - VC) + gBD * abs(VB))
    assert r["I_node"][1] == pytest.approx(IB / r["I_ref"], rel=1e-12)


def test_floating_and_one_sided_components_carry_no_current():
    span = chain(10.0, 11, 10.0)
    floating = chain(16.0, 3, 30.0)          # touches no electrode
    source_only = chain(6.0, 4, 20.0)        # x from 6 to 12: one free bead, source only
    X = np.concatenate([span, floating, source_only])
    fil = np.repeat([0, 1, 2], [11, 3, 4])
    pos = np.concatenate([np.arange(11), np.arange(3), np.arange(4)])
    r = net.conductivity(fil, pos, X, NX, NY, x_src=11.0, x_snk=29.0)
    assert r["kappa"] == pytest.approx(0.9, rel=1e-12)
    assert np.all(r["V"][11:14] == 0.0) and np.all(r["I_node"][11:14] == 0.0)
    assert np.allclose(r["V"][14:], 1.0, rtol=0, atol=1e-13)
    assert np.allclose(r["I_node"][14:], 0.0, rtol=0, atol=1e-12)


def random_deposit(seed, nw=120, nb=6, box=(14.0, 50.0, 8.0, 32.0)):
    g = np.random.default_rng(seed)
    x0, x1, y0, y1 = box
    cen = np.c_[g.uniform(x0, x1, nw), g.uniform(y0, y1, nw)]
    ang = g.normal(0.0, 0.6, nw)
    d = np.c_[np.cos(ang), np.sin(ang)]
    X = np.array([[*(c + (k - (nb - 1) / 2) * 2.0 * dd), 1.0] for c, dd in zip(cen, d) for k in range(nb)])
    return np.repeat(np.arange(nw), nb), np.tile(np.arange(nb), nw), X


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kirchhoff_law_and_current_conservation_on_random_deposits(seed, oracle):
    fil, pos, X = random_deposit(seed)
    r = net.conductivity(fil, pos, X, NX, NY, x_src=20.0, x_snk=44.0)
    i, j, rr = net.edges(fil, pos, X, NX, NY)
    G = 1 / rr
    free = (X[:, 0] >= 20.0) & (X[:, 0] <= 44.0)
    net_in = np.zeros(len(X))
    np.add.at(net_in, i, G * (r["V"][i] - r["V"][j]))
    np.add.at(net_in, j, G * (r["V"][j] - r["V"][i]))
    assert np.max(np.abs(net_in[free])) < 1e-11
    assert r["I_tot"] == pytest.approx(r["I_sink"], rel=1e-9, abs=1e-14)
    assert np.all(r["I_node"] >= 0.0)
    # a current flows exactly when a contact cluster joins the electrodes
    p = oracle.Params(NX, NY, 16)
    _, _, perc, _ = oracle.descriptors(p, fil, pos, X, 2.1, 20.0, 44.0)
    assert (r["I_tot"] > 1e-12) == bool(perc)


# ----------------------------------------------------------------------------- profiles
def test_density_profile_counts_and_normalisation():
    # bead centres: 2, 4, 0, 2 in the four x-bins of width 10 over [0, 40); two beads
    # outside the strip |y - 20| <= 5 and one beyond the range do not count
    xs = [1, 9, 11, 12, 15, 19, 31, 39]
    X = np.array([[x, 20.0 + (k % 3) - 1, 1.0] for k, x in enumerate(xs)]
                 + [[5.0, 26.0, 1.0], [15.0, 13.9, 1.0], [45.0, 20.0, 1.0]])
    fil = np.arange(len(X))
    pos = np.zeros(len(X), int)
    S, g, nbond, nbead = net.profiles(fil, pos, X, NX, NY, 0, 0.0, 40.0, 4, 20.0, 5.0)
    assert list(nbead) == [2, 4, 0, 2]
    assert np.allclose(g, [1.0, 2.0, 0.0, 1.0], rtol=0, atol=1e-15)
    assert list(nbond) == [0, 0, 0, 0] and np.all(S == 0.0)


def test_nematic_profile_of_aligned_perpendicular_and_diagonal_bonds():
    # bin 0: bonds along x (S = 1); bin 1: along y (S = -1); bin 2: at 45 deg in x-y (S = 0);
    # bin 3: one along x and one along z (S = 0)
    pairs = [((1, 20, 1), (3, 20, 1)), ((5, 19, 1), (7, 19, 1)),
             ((15, 19, 1), (15, 21, 1)),
             ((24, 19, 1), (25.41421356237310, 20.41421356237310, 1)),
             ((31, 18, 1), (33, 18, 1)), ((36, 22, 1), (36, 22, 3))]
    X = np.array([p for pr in pairs for p in pr], np.float64)
    fil = np.repeat(np.arange(len(pairs)), 2)
    pos = np.tile([0, 1], len(pairs))
    S, g, nbond, nbead = net.profiles(fil, pos, X, NX, NY, 0, 0.0, 40.0, 4, 20.0, 5.0)
    assert list(nbond) == [2, 1, 1, 2]
    assert S[0] == pytest.approx(1.0, abs=1e-14)
    assert S[1] == pytest.approx(-1.0, abs=1e-14)
    assert S[2] == pytest.approx(0.0, abs=1e-12)
    assert S[3] == pytest.approx(0.0, abs=1e-14)


def test_transverse_profile_uses_the_strip_in_x_and_bins_in_y():
    X = np.array([[20.0, 2.0, 1.0], [20.0, 4.0, 1.0],    # bond along y, midpoint y = 3
                  [21.0, 12.0, 1.0], [23.0, 12.0, 1.0],  # bond along x, midpoint y = 12
                  [40.0, 12.0, 1.0], [42.0, 12.0, 1.0]])  # outside the strip |x - 20| <= 4
    fil = np.repeat([0, 1, 2], 2)
    pos = np.tile([0, 1], 3)
    S, g, nbond, nbead = net.profiles(fil, pos, X, NX, NY, 1, 0.0, 20.0, 2, 20.0, 4.0)
    assert list(nbond) == [1, 1] and list(nbead) == [2, 2]
    assert S[0] == pytest.approx(-1.0) and S[1] == pytest.approx(1.0)
    assert np.allclose(g, [1.0, 1.0])
