"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a conservation law, a finite difference of the energy, an independent
library (scipy root finder, networkx components) or the constants printed in
the paper.  A plausible slip (a dropped term, a sign, a swapped index) fails
at least one of them.
"""
import os

import numpy as np
import pytest

from tests import inputs

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def uniform_liquid(nx, ny, nz):
    fR = np.ascontiguousarray(np.broadcast_to(W[:, None, None, None], (19, nz, ny, nx)).copy())
    return fR, np.zeros_like(fR)


# ---------------------------------------------------------------- constants
def test_defaults_are_the_printed_constants(oracle):
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            vals[k] = float(v)
    p = oracle.Params(4, 4, 4)
    for k in ("ks", "Rm", "d0", "eps_wca", "kb", "eps_s", "K", "substeps"):
        assert getattr(p, k) == vals[k], k
    import inspect
    assert inspect.signature(oracle.descriptors).parameters["rcon"].default == vals["rcon"]


# ---------------------------------------------------------------- fluid
def test_component_mass_is_conserved_exactly(oracle):
    p = oracle.Params(24, 16, 16, top_bc=0, sigma=0.02, beta=0.7)
    fR, fB = oracle.init_droplet(p, 0, 11.5, 7.5, 7.5, 8, 5, 5, 2.0)
    cot = oracle.cot_map(np.full((16, 24), 70.0))
    m0 = oracle.mass(fR, fB)
    acc = oracle.Acc()
    for _ in range(30):
        assert oracle.step(p, fR, fB, cot, acc) == 0
    m1 = oracle.mass(fR, fB)
    assert abs(m1[0] - m0[0]) < 1e-12 * m0[0]
    assert abs(m1[1] - m0[1]) < 1e-12 * m0[1]


def test_top_plane_flux_balances_total_mass(oracle):
    p = oracle.Params(16, 12, 12, top_bc=1, sigma=0.01)
    fR, fB = oracle.init_droplet(p, 0, 7.5, 5.5, -0.5, 6, 4, 8, 2.0)
    cot = oracle.cot_map(np.full((12, 16), 90.0))
    acc = oracle.Acc()
    m0 = sum(oracle.mass(fR, fB))
    for _ in range(20):
        oracle.step(p, fR, fB, cot, acc)
    m1 = sum(oracle.mass(fR, fB))
    assert acc.top_in > 0 and acc.top_out > 0
    assert abs((m1 - m0) - (acc.top_in - acc.top_out)) < 1e-12 * m0


def test_colour_gradient_is_exact_for_a_linear_field(oracle):
    nx, ny, nz = 4, 16, 12
    a, b = 0.03, -0.05
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    C = a * (y - 7.5) + b * (z - 5.5) + 0.0 * np.arange(nx)[None, None, :]
    fR = (W[:, None, None, None] * (1 + C) / 2).copy()
    fB = (W[:, None, None, None] * (1 - C) / 2).copy()
    p = oracle.Params(nx, ny, nz, top_bc=0)
    f = oracle.fields(p, fR, fB, np.zeros((ny, nx)))
    G = f["G"][2:nz - 2, 2:ny - 2]
    assert np.allclose(G[..., 0], 0.0, atol=1e-15)
    assert np.allclose(G[..., 1], a, rtol=0, atol=1e-14)
    assert np.allclose(G[..., 2], b, rtol=0, atol=1e-14)


def test_curvature_of_a_sphere(oracle):
    n, R = 32, 10.0
    p = oracle.Params(n, n, n, top_bc=0)
    fR, fB = oracle.init_droplet(p, 0, 15.5, 15.5, 15.5, R, R, R, 2.0)
    f = oracle.fields(p, fR, fB, np.zeros((n, n)))
    g = np.linalg.norm(f["G"], axis=-1)
    m = np.abs(f["C"]) < 0.5
    kap = (f["kappa"] * g)[m].sum() / g[m].sum()
    assert abs(kap - 2.0 / R) < 0.03 * (2.0 / R)
    # the force points into the drop (towards higher C), magnitude sigma/2 kappa |G|
    Fs = f["Fs"]
    assert np.all(np.einsum("...i,...i->...", Fs, f["G"])[m] > 0)


def _laplace(oracle, R, sigma, steps=800):
    n = 32
    p = oracle.Params(n, n, n, top_bc=0, sigma=sigma)
    fR, fB = oracle.init_droplet(p, 0, 15.5, 15.5, 15.5, R, R, R, 2.0)
    cot = np.zeros((n, n))
    acc = oracle.Acc()
    for _ in range(steps):
        oracle.step(p, fR, fB, cot, acc)
    f = oracle.fields(p, fR, fB, cot)
    rho, C = f["rhoR"] + f["rhoB"], f["C"]
    dp = (rho[C > 0.99].mean() - rho[C < -0.99].mean()) / 3.0
    Rv = (3 * ((1 + C) / 2).sum() / (4 * np.pi)) ** (1 / 3)
    return dp, Rv


def test_laplace_law(oracle):
    """Static drop: dp = c_s^2 drho = 2 sigma / R (diffuse-interface bias shrinks with R)."""
    dp10, R10 = _laplace(oracle, 10.0, 0.01)
    dp6, R6 = _laplace(oracle, 6.0, 0.01)
    r10 = dp10 * R10 / (2 * 0.01)
    r6 = dp6 * R6 / (2 * 0.01)
    assert 0.97 < r10 < 1.10
    assert r10 < r6 < 1.25


def test_poiseuille_profile_is_exact_at_the_magic_relaxation_time(oracle):
    """BGK + half-way bounce-back + Guo force reproduce the parabola exactly at tau=1/2+sqrt(3/16)."""
    nz, g = 10, 1e-6
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    p = oracle.Params(1, 1, nz, top_bc=0, sigma=0.0, tau_R=tau, tau_B=tau, body=(g, 0.0, 0.0))
    fR, fB = uniform_liquid(1, 1, nz)
    acc = oracle.Acc()
    for _ in range(4000):
        oracle.step(p, fR, fB, np.zeros((1, 1)), acc)
    f = oracle.fields(p, fR, fB, np.zeros((1, 1)))
    u = (f["j"][:, 0, 0, 0] + g / 2) / (f["rhoR"] + f["rhoB"])[:, 0, 0]
    z = np.arange(nz) + 0.5
    nu = (tau - 0.5) / 3.0
    ue = g / (2 * nu) * z * (nz - z)
    assert np.max(np.abs(u - ue)) < 1e-9 * ue.max()
    # at tau=1 the known second-order slip remains (a real effect, not round-off)
    p.tau_R = p.tau_B = 1.0
    fR, fB = uniform_liquid(1, 1, nz)
    acc = oracle.Acc()
    for _ in range(3000):
        oracle.step(p, fR, fB, np.zeros((1, 1)), acc)
    f = oracle.fields(p, fR, fB, np.zeros((1, 1)))
    u = (f["j"][:, 0, 0, 0] + g / 2) / (f["rhoR"] + f["rhoB"])[:, 0, 0]
    ue = g / (2 * (0.5 / 3.0)) * z * (nz - z)
    err = np.max(np.abs(u - ue)) / ue.max()
    assert 1e-4 < err < 1e-2


def test_body_force_adds_exactly_F_momentum(oracle):
    nx, ny, nz = 6, 5, 7
    F = (2e-5, -1e-5, 3e-6)
    p = oracle.Params(nx, ny, nz, top_bc=0, sigma=0.0, body=F)
    fR, fB = uniform_liquid(nx, ny, nz)
    oracle.step(p, fR, fB, np.zeros((ny, nx)), oracle.Acc())
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                  [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
    mom = c.T @ (fR + fB).reshape(19, -1).sum(axis=1)
    assert np.allclose(mom, np.array(F) * nx * ny * nz, rtol=1e-10, atol=0)


def _fit_angle(C, zmin=2.0):
    nz, ny, nx = C.shape
    C2 = 0.5 * (C[:, ny // 2, :] + C[:, ny // 2 - 1, :])
    pts = []
    for z in range(nz):
        r = C2[z]
        for x in range(nx - 1):
            if r[x] * r[x + 1] < 0:
                pts.append((x + r[x] / (r[x] - r[x + 1]), z))
    for x in range(nx):
        col = C2[:, x]
        for z in range(nz - 1):
            if col[z] * col[z + 1] < 0:
                pts.append((x, z + col[z] / (col[z] - col[z + 1])))
    P = np.array(pts)
    P = P[P[:, 1] >= zmin]
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    s = np.linalg.lstsq(A, P[:, 0] ** 2 + P[:, 1] ** 2, rcond=None)[0]
    R = np.sqrt(s[2] + s[0] ** 2 + s[1] ** 2)
    return np.degrees(np.arccos(np.clip(-(s[1] + 0.5) / R, -1, 1)))


@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_contact_angle_follows_the_wetting_parameter(oracle, theta):
    n, nz = 32, 16
    p = oracle.Params(n, n, nz, top_bc=0, sigma=0.01)
    R0 = 7.5
    fR, fB = oracle.init_droplet(p, 0, 15.5, 15.5, -0.5 - R0 * np.cos(np.radians(theta)),
                                 R0, R0, R0, 2.0)
    cot = oracle.cot_map(np.full((n, n), theta))
    acc = oracle.Acc()
    for _ in range(1500):
        oracle.step(p, fR, fB, cot, acc)
    f = oracle.fields(p, fR, fB, cot)
    assert abs(_fit_angle(f["C"]) - theta) < 4.0


def test_evaporation_converts_liquid_to_gas_exactly(oracle):
    p = oracle.Params(24, 16, 12, top_bc=0, sigma=0.01, J0=2e-3, evap_start=3)
    fR, fB = oracle.init_droplet(p, 0, 11.5, 7.5, -0.5, 8, 5, 6, 2.0)
    cot = oracle.cot_map(np.full((16, 24), 80.0))
    acc = oracle.Acc()
    m0 = oracle.mass(fR, fB)
    for k in range(8):
        if k == 3:
            h_before = oracle.fields(p, fR, fB, cot)["h"]
        oracle.step(p, fR, fB, cot, acc)
        if k < 3:
            assert acc.evaporated == 0.0
    m1 = oracle.mass(fR, fB)
    assert acc.evaporated > 0
    assert acc.h0 == h_before.max()
    assert abs((m0[0] - m1[0]) - acc.evaporated) < 1e-12 * m0[0]
    assert abs((m1[1] - m0[1]) - acc.evaporated) < 1e-12 * m0[0]


def test_evaporation_sink_is_capped_by_the_resting_population(oracle):
    p = oracle.Params(20, 12, 10, top_bc=0, sigma=0.01, J0=1e3, evap_start=0)
    fR, fB = oracle.init_droplet(p, 0, 9.5, 5.5, -0.5, 6, 4, 5, 2.0)
    cot = oracle.cot_map(np.full((12, 20), 90.0))
    g = np.linalg.norm(oracle.fields(p, fR, fB, cot)["G"], axis=-1)
    acc = oracle.Acc()
    oracle.step(p, fR, fB, cot, acc)
    rest = fR[0]
    assert np.all(rest[g > 1e-6] == 0.0)
    assert np.all(rest >= 0.0)


def test_evaporation_rate_follows_the_height_law(oracle):
    """Uncapped sink: doubling J0 doubles the converted mass; larger h~ evaporates less."""
    base = dict(top_bc=0, sigma=0.01, evap_start=0)
    out = []
    for J0 in (1e-5, 2e-5):
        p = oracle.Params(20, 12, 10, J0=J0, **base)
        fR, fB = oracle.init_droplet(p, 0, 9.5, 5.5, -0.5, 6, 4, 5, 2.0)
        cot = oracle.cot_map(np.full((12, 20), 90.0))
        f0R = fR.copy()
        acc = oracle.Acc()
        p0 = oracle.Params(20, 12, 10, J0=0.0, **base)
        gR, gB = fR.copy(), fB.copy()
        oracle.step(p0, gR, gB, cot, oracle.Acc())
        oracle.step(p, fR, fB, cot, acc)
        out.append((gR[0] - fR[0], acc.evaporated))
        del f0R
    (d1, e1), (d2, e2) = out
    assert e2 == pytest.approx(2 * e1, rel=1e-12)
    assert np.allclose(d2, 2 * d1, rtol=1e-9, atol=1e-20)


# ---------------------------------------------------------------- filaments
def test_bead_forces_are_minus_energy_gradient(oracle):
    p = oracle.Params(32, 32, 16, eps_coh=1.0 * 0.006, eps_s=0.006, rc=4.0)
    fil, pos, X = inputs.straight_filaments([[10.0, 10.0, 1.2], [10.5, 12.6, 1.6]],
                                            [[1, 0.1, 0.05], [1, -0.2, 0.1]], 4, 1.9)
    X = X + inputs.rng(3).normal(scale=0.05, size=X.shape)
    F, err = oracle.bead_conservative_forces(p, fil, pos, X)
    assert err == 0
    h = 1e-6
    Fn = np.zeros_like(X)
    for a in range(X.shape[0]):
        for d in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, d] += h
            Xm[a, d] -= h
            Fn[a, d] = -(oracle.bead_energy(p, fil, pos, Xp) - oracle.bead_energy(p, fil, pos, Xm)) / (2 * h)
    assert np.allclose(F, Fn, rtol=1e-6, atol=1e-8)
    # every term contributed: pairs across filaments, bending, wall
    assert np.abs(F).max() > 1e-3


def test_fene_overstretch_is_reported_not_fatal(oracle):
    p = oracle.Params(16, 16, 16)
    fil, pos, X = inputs.straight_filaments([[8.0, 8.0, 8.0]], [[1, 0, 0]], 2, 2.5)
    F, err = oracle.bead_conservative_forces(p, fil, pos, X)
    assert err & 2
    assert np.all(np.isfinite(F))


def test_relaxed_filament_bond_matches_force_balance(oracle):
    from scipy.optimize import brentq
    n = 12
    p = oracle.Params(n, n, n, top_bc=0, sigma=0.0, eps_s=0.0, gamma=1.0, xi=0.0)
    fR, fB = uniform_liquid(n, n, n)
    fil, pos, X = inputs.straight_filaments([[5.5, 5.5, 5.5]], [[1, 0, 0]], 3, 1.7)
    B = oracle.Beads(fil, pos, X)
    acc = oracle.Acc()
    for _ in range(600):
        assert oracle.step(p, fR, fB, np.zeros((n, n)), acc, B) == 0
    d = np.linalg.norm(B.X[1] - B.X[0])

    def end_force(r):  # along the chain on the outer bead
        fene = -p.ks * r / (1 - r * r / p.Rm ** 2)
        s6 = (p.d0 / r) ** 6
        wca = -p.eps_wca * (-12 * s6 * s6 + 12 * s6) / r if r <= p.d0 else 0.0
        bend = -p.kb * (2 * r - 2 * p.d0)
        return fene + wca + bend

    root = brentq(end_force, 1.5, 2.3)
    assert abs(d - root) < 1e-6


def test_verlet_energy_error_is_second_order(oracle):
    n = 10

    def drift(sub):
        p = oracle.Params(n, n, n, top_bc=0, sigma=0.0, eps_s=0.0, gamma=0.0, xi=0.0, substeps=sub)
        fR, fB = uniform_liquid(n, n, n)
        fil, pos, X = inputs.straight_filaments([[4.5, 4.5, 4.5]], [[1, 0.3, 0.2]], 3, 1.8)
        V = inputs.rng(5).normal(scale=0.02, size=X.shape)
        V -= V.mean(axis=0)
        B = oracle.Beads(fil, pos, X, V)
        F0, _ = oracle.bead_conservative_forces(p, fil, pos, B.X)
        B.F[:] = F0
        e0 = oracle.bead_energy(p, fil, pos, B.X) + 0.5 * np.sum(B.V ** 2)
        dev = 0.0
        acc = oracle.Acc()
        for _ in range(60):
            oracle.step(p, fR, fB, np.zeros((n, n)), acc, B)
            e = oracle.bead_energy(p, fil, pos, B.X) + 0.5 * np.sum(B.V ** 2)
            dev = max(dev, abs(e - e0))
        return dev

    d5, d10 = drift(5), drift(10)
    assert 3.0 < d5 / d10 < 5.5


def test_fluid_plus_bead_momentum_is_conserved(oracle):
    """With only drag and pair forces: M_fluid + P_beads + dt/2 sum F_carried is invariant."""
    n = 16
    p = oracle.Params(n, n, n, top_bc=0, sigma=0.0, eps_s=0.0, gamma=1.0, xi=0.0)
    fR, fB = uniform_liquid(n, n, n)
    fil, pos, X = inputs.straight_filaments([[7.5, 7.5, 8.0]], [[1, 0.5, 0.2]], 4, 1.9)
    V = np.tile([0.01, -0.005, 0.002], (4, 1))
    B = oracle.Beads(fil, pos, X, V)
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                  [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
    dt = 1.0 / p.substeps

    def invariant():
        return (c.T @ (fR + fB).reshape(19, -1).sum(axis=1) + B.V.sum(axis=0) * p.mass
                + 0.5 * dt * B.F.sum(axis=0))

    P0 = invariant()
    acc = oracle.Acc()
    for _ in range(5):
        assert oracle.step(p, fR, fB, np.zeros((n, n)), acc, B) == 0
    P1 = invariant()
    assert np.abs(B.V - V).max() > 1e-4  # the drag did act
    assert np.allclose(P1, P0, rtol=0, atol=1e-12)  # round-off of ~8e4 population sums


def test_drag_reaction_sums_to_minus_bead_impulse(oracle):
    n = 12
    p = oracle.Params(n, n, n, top_bc=0, sigma=0.0, eps_s=0.0, gamma=1.0)
    fR, fB = uniform_liquid(n, n, n)
    fil, pos, X = inputs.straight_filaments([[5.3, 6.1, 5.7]], [[1, 0, 0]], 2, 1.9)
    B = oracle.Beads(fil, pos, X, np.tile([0.02, 0.0, -0.01], (2, 1)))
    err, fext = oracle.step(p, fR, fB, np.zeros((n, n)), oracle.Acc(), B, return_fext=True)
    # fluid receives -gamma(u - V) dt per sub-step; with the fluid at rest that is gamma V dt
    tot = fext.reshape(-1, 3).sum(axis=0)
    assert tot[0] > 0 and tot[2] < 0
    assert abs(tot[1]) < 1e-15


# ---------------------------------------------------------------- descriptors
def test_nematic_order_extremes(oracle):
    p = oracle.Params(64, 64, 16)
    for d, want in (([1, 0, 0], 1.0), ([0, 1, 0], -1.0), ([0, 0, 1], -1.0)):
        fil, pos, X = inputs.straight_filaments([[10, 10, 5], [30, 30, 5]], [d, d], 4, 1.9)
        sx, nc, perc, _ = oracle.descriptors(p, fil, pos, X)
        assert sx == pytest.approx(want, abs=1e-14)
        assert nc == 2


def test_nematic_order_of_isotropic_in_plane_segments(oracle):
    g = inputs.rng(11)
    n = 4000
    ang = g.uniform(0, np.pi, n)
    d = np.c_[np.cos(ang), np.sin(ang), np.zeros(n)]
    cen = np.c_[g.uniform(0, 5000, n), g.uniform(0, 5000, n), np.full(n, 3.0)]
    fil, pos, X = inputs.straight_filaments(cen, d, 2, 1.9)
    p = oracle.Params(5000, 5000, 16)
    sx, *_ = oracle.descriptors(p, fil, pos, X, rcon=0.0)
    assert abs(sx) < 4.0 / np.sqrt(n)


def test_clusters_and_percolation_by_hand(oracle):
    p = oracle.Params(64, 32, 16)
    fil, pos, X = inputs.straight_filaments([[10, 10, 3], [10, 15, 3]], [[1, 0, 0]] * 2, 4, 1.9)
    assert oracle.descriptors(p, fil, pos, X)[1] == 2
    fil, pos, X = inputs.straight_filaments([[10, 10, 3], [10, 12.0, 3]], [[1, 0, 0]] * 2, 4, 1.9)
    assert oracle.descriptors(p, fil, pos, X)[1] == 1
    # a stretched bond (2.3 > 2.1) still connects its filament
    fil, pos, X = inputs.straight_filaments([[10, 10, 3]], [[1, 0, 0]], 3, 2.3)
    assert oracle.descriptors(p, fil, pos, X)[1] == 1
    # overlapping chain from x~3 to x~45 percolates between 8 and 40; a gap breaks it
    cen = [[6 + 5.5 * k, 10, 3] for k in range(8)]
    fil, pos, X = inputs.straight_filaments(cen, [[1, 0, 0]] * 8, 4, 1.9)
    assert oracle.descriptors(p, fil, pos, X, xsrc=8, xsnk=40)[2]
    X2 = X.copy()
    X2[fil >= 4, 0] += 5.0
    assert not oracle.descriptors(p, fil, pos, X2, xsrc=8, xsnk=40)[2]


def test_clusters_match_networkx_on_random_configurations(oracle):
    import networkx as nx
    p = oracle.Params(40, 40, 12)
    for seed in range(3):
        g = inputs.rng(100 + seed)
        nf = 30
        cen = np.c_[g.uniform(0, 40, nf), g.uniform(0, 40, nf), g.uniform(1, 6, nf)]
        d = g.normal(size=(nf, 3))
        fil, pos, X = inputs.straight_filaments(cen, d, 4, 1.9)
        X[:, 0] %= 40
        X[:, 1] %= 40
        sx, nc, perc, lab = oracle.descriptors(p, fil, pos, X)
        G = nx.Graph()
        G.add_nodes_from(range(len(X)))
        for a in range(len(X)):
            for b in range(a + 1, len(X)):
                dd = X[b] - X[a]
                dd[0] -= 40 * np.round(dd[0] / 40)
                dd[1] -= 40 * np.round(dd[1] / 40)
                if (fil[a] == fil[b] and abs(pos[a] - pos[b]) == 1) or np.dot(dd, dd) < 2.1 ** 2:
                    G.add_edge(a, b)
        comps = list(nx.connected_components(G))
        assert nc == len(comps)
        for comp in comps:
            assert len({lab[i] for i in comp}) == 1
            assert lab[min(comp)] == min(comp)


# ------------------------------------------------ coupling, solvation, friction, recolouring
C19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], float)


def _node_coords(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x, y, z], axis=-1).astype(float)  # [nz, ny, nx, 3]


def _streams_to(field_of_position, nx, ny, nz):
    """Post-collision populations f_i(y) = g_i(y + c_i): after the pull every interior
    node x holds g_i(x) (Sec. II.A, Eq. (1) streaming)."""
    P = _node_coords(nx, ny, nz)
    return np.stack([field_of_position(i, P + C19[i]) for i in range(19)])


def _one_bead(oracle, X, V=(0, 0, 0), F=(0, 0, 0)):
    return oracle.Beads(np.array([0], np.int32), np.array([0], np.int32), np.array([X], float),
                        np.array([V], float), np.array([F], float))


def test_drag_interpolates_a_linear_velocity_field_exactly(oracle):
    """Trilinear coupling (Sec. II.A, Ahlrichs-Duenweg drag): a bead at rest in a fluid
    whose velocity is linear in space, u(x) = A x + b, feels exactly gamma (A X + b);
    the reaction spread back has total -F and first moment -F (x) X, as the weights of
    linear interpolation reproduce the position."""
    nx, ny, nz = 12, 12, 10
    A = np.array([[0.0011, -0.0007, 0.0005], [0.0004, 0.0009, -0.0012], [-0.0006, 0.0003, 0.0008]])
    b = np.array([0.002, -0.001, 0.0015])
    # single liquid component, f_i = w_i (1 + 3 c_i.u): rho = 1 and j = u at every interior node
    fR = _streams_to(lambda i, P: W[i] * (1.0 + 3.0 * (P @ A.T + b) @ C19[i]), nx, ny, nz)
    fR = np.ascontiguousarray(fR)
    fB = np.zeros_like(fR)
    p = oracle.Params(nx, ny, nz, top_bc=0, sigma=0.0, eps_s=0.0, gamma=0.7, xi=0.0, substeps=1)
    X = np.array([5.3, 6.8, 4.35])
    B = _one_bead(oracle, X)
    err, fext = oracle.step(p, fR, fB, np.zeros((ny, nx)), oracle.Acc(), B, return_fext=True)
    assert err == 0
    want = 0.7 * (A @ X + b)
    assert np.allclose(B.F[0], want, rtol=0, atol=1e-16)
    assert np.abs(want).min() > 1e-4
    P = _node_coords(nx, ny, nz).reshape(-1, 3)
    fe = fext.reshape(-1, 3)
    assert np.allclose(fe.sum(axis=0), -want, rtol=0, atol=1e-17)
    assert np.allclose(P.T @ fe, -np.outer(X, want), rtol=0, atol=1e-15)
    assert np.count_nonzero(np.abs(fe).sum(axis=1)) == 8


def test_solvation_force_pushes_beads_up_the_colour_gradient(oracle):
    """Solvation (Sec. II.A): F = xi grad C, towards the liquid (C = +1).  With C linear
    in x the colour gradient is exact (G = s e_x), so a free bead feels exactly xi s e_x."""
    nx, ny, nz = 16, 10, 10
    s = 0.02
    col = lambda P: s * (P[..., 0] - 7.5)
    fR = np.ascontiguousarray(_streams_to(lambda i, P: W[i] * (1.0 + col(P)) / 2, nx, ny, nz))
    fB = np.ascontiguousarray(_streams_to(lambda i, P: W[i] * (1.0 - col(P)) / 2, nx, ny, nz))
    p = oracle.Params(nx, ny, nz, top_bc=0, sigma=0.0, eps_s=0.0, gamma=0.0, xi=0.6, substeps=1)
    B = _one_bead(oracle, [7.2, 4.6, 4.3])
    assert oracle.step(p, fR, fB, np.zeros((ny, nx)), oracle.Acc(), B) == 0
    assert np.allclose(B.F[0], [0.6 * s, 0.0, 0.0], rtol=0, atol=1e-16)


def test_substrate_friction_both_branches(oracle):
    """Load-dependent friction (Sec. II.A): |F_t| = min(gamma_t |v_t|, mu N) against the
    half-step tangential velocity, N the downward pull of adhesion and of every other force.
    One sub-step (dt = 1, mass 1): v_h = V + F_carried / 2, the bead drifts by v_h, then
    the force is evaluated there."""
    n = 12
    fR, fB = uniform_liquid(n, n, n)  # fluid at rest: u* = 0, grad C = 0
    mu, gt = 0.5, 1.0

    def run(V, F0, z=1.0, gamma=0.0):
        p = oracle.Params(n, n, n, top_bc=0, sigma=0.0, eps_s=0.006, gamma=gamma, xi=0.0,
                          mu=mu, gamma_t=gt, substeps=1)
        X = np.array([5.3, 6.7, z])
        B = _one_bead(oracle, X, V, F0)
        assert oracle.step(p, fR.copy(), fB.copy(), np.zeros((n, n)), oracle.Acc(), B) == 0
        vh = np.asarray(V, float) + 0.5 * np.asarray(F0, float)
        Fc, _ = oracle.bead_conservative_forces(p, [0], [0], (X + vh)[None, :])
        return B.F[0], vh, Fc[0, 2]

    # viscous branch: gamma_t |v_h| < mu N, the force is -gamma_t v_h (not -gamma_t V)
    F, vh, fw = run([0.0004, -0.0003, 0.0], [0.0006, 0.0002, 0.0])
    assert fw < -1e-3 and gt * np.hypot(*vh[:2]) < mu * -fw
    assert np.allclose(F, [-gt * vh[0], -gt * vh[1], fw], rtol=0, atol=1e-18)
    # Coulomb branch: mu N along -v_h / |v_h|
    F, vh, fw = run([0.02, 0.01, 0.0], [0.004, -0.002, 0.0])
    vt = np.hypot(*vh[:2])
    assert gt * vt > mu * -fw
    assert np.allclose(F, [-mu * -fw * vh[0] / vt, -mu * -fw * vh[1] / vt, fw], rtol=0, atol=1e-18)
    # a downward drag (bead rising through fluid at rest) adds to the load
    F, vh, fw = run([0.02, 0.0, 0.001], [0.0, 0.0, 0.0], gamma=1.0)
    N = 1.0 * vh[2] - fw
    assert np.allclose(F, [-vh[0] - mu * N, 0.0, -vh[2] + fw], rtol=0, atol=1e-18)
    # out of the adhesion range (2(z + 1/2) >= r_c) there is no friction at all
    F, vh, fw = run([0.02, 0.01, 0.0], [0.0, 0.0, 0.0], z=3.0)
    assert fw == 0.0 and np.all(F == 0.0)


def test_recolouring_term_moments(oracle):
    """Recolouring (Sec. II.A, Latva-Kokko/Rothman form with strength beta): against the
    same step at beta = 0, the red populations change by d_i with d_i = -(blue change),
    sum_i d_i = 0 (component mass) and sum_i c_i d_i = beta rho_R rho_B / rho (1 + sqrt 2)/9 n,
    n the unit colour gradient: the lattice sum sum_i w_i c_i c_i / |c_i| is (1 + sqrt 2)/9 I."""
    p1 = oracle.Params(20, 14, 12, top_bc=0, sigma=0.02, beta=0.7)
    p0 = oracle.Params(20, 14, 12, top_bc=0, sigma=0.02, beta=0.0)
    fR, fB = oracle.init_droplet(p1, 0, 9.5, 6.5, 3.0, 6, 4, 5, 2.0)
    # give it a flow so that the collision is not trivial
    fR *= 1.0 + 0.03 * np.sin(np.arange(19))[:, None, None, None]
    cot = oracle.cot_map(np.full((14, 20), 75.0))
    f = oracle.fields(p1, fR, fB, cot)
    aR, aB, bR, bB = fR.copy(), fB.copy(), fR.copy(), fB.copy()
    assert oracle.step(p1, aR, aB, cot, oracle.Acc()) == 0
    assert oracle.step(p0, bR, bB, cot, oracle.Acc()) == 0
    d = (aR - bR).reshape(19, -1)
    assert np.allclose(aB - bB, -(aR - bR), rtol=0, atol=1e-16)
    assert np.abs(d.sum(axis=0)).max() < 1e-16
    G = f["G"].reshape(-1, 3)
    g = np.linalg.norm(G, axis=1)
    nrm = np.where(g[:, None] > 1e-8, G / np.where(g > 0, g, 1)[:, None], 0.0)
    rR, rB = f["rhoR"].ravel(), f["rhoB"].ravel()
    want = 0.7 * (rR * rB / (rR + rB))[:, None] * (1 + np.sqrt(2)) / 9 * nrm
    got = (C19.T @ d).T
    assert np.abs(want).max() > 1e-2
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    # even moments vanish (the term is odd in c_i)
    assert np.abs((C19[:, 0] ** 2) @ d).max() < 1e-16


def _slab(oracle, beta, steps):
    nx, ny, nz = 32, 4, 12
    p = oracle.Params(nx, ny, nz, top_bc=0, sigma=0.01, beta=beta)
    fR, fB = oracle.init_droplet(p, 1, 15.5, 1.5, 5.5, 8.0, 1e6, 1e6, 2.0)
    cot = oracle.cot_map(np.full((ny, nx), 90.0))
    acc = oracle.Acc()
    for _ in range(steps):
        assert oracle.step(p, fR, fB, cot, acc) == 0
    return oracle.fields(p, fR, fB, cot)["C"]


def test_flat_interface_stays_flat_and_segregated(oracle):
    """A liquid slab across a 90 deg substrate (Sec. II.A colour-gradient model): the
    interface stays flat and normal to the wall, C stays in [-1, 1], the bulk phases stay
    pure under recolouring and mix without it (beta = 0)."""
    C = _slab(oracle, 0.7, 300)
    assert C.min() >= -1.0 - 1e-12 and C.max() <= 1.0 + 1e-12
    assert C[:, :, 15].min() > 0.99 and C[:, :, 0].max() < -0.99
    # interface position per plane: the C = 0 crossing on the left flank, interpolated
    prof = C[:, 0, :16]
    k = np.argmax(prof > 0, axis=1)
    xs = k - 1 + (-prof[np.arange(len(k)), k - 1]) / (prof[np.arange(len(k)), k] - prof[np.arange(len(k)), k - 1])
    assert xs.max() - xs.min() < 0.02
    assert np.abs(C - C[:, :1, :]).max() < 1e-12  # y-invariant
    C0 = _slab(oracle, 0.0, 300)
    assert C0[:, :, 15].min() < 0.9  # without recolouring the components diffuse
