"""FP64 CPU oracle of the deposit analysis (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this module; it shares nothing with the CUDA library.

Electrical network model (Sec. II.B, Eqs. (15)-(18)):
  * every bead is a node; two beads are connected when they are bonded
    neighbours of one filament or closer than r_c = 2.1 (minimum image in the
    periodic x and y directions), with conductance G_ij = 1 / r_ij;
  * Delta V = 1: beads with x < x_src are held at V = 1 (source electrode),
    beads with x > x_snk at V = 0 (sink electrode); the other potentials obey
    Kirchhoff's current law  sum_j G_ij (V_i - V_j) = 0;
  * node current I_i = 1/2 sum_j |G_ij (V_i - V_j)|                 (Eq. (15));
  * I_tot = current leaving the source electrode;
  * I_ref = Delta V / (x_snk - x_src): a straight filament of conductance
    1/r per unit length spanning the electrodes                     (Eq. (16));
  * I_i* = I_i / I_ref (Eq. (17)),  kappa* = I_tot / I_ref            (Eq. (18)).
A node in a component that touches no electrode has no defined potential; it
is reported at V = 0 and carries no current.  A component that touches one
electrode only sits at that electrode's potential.

Morphology profiles (Sec. II.B, Eqs. (13)-(14)):
  * S_x^b = mean of 2 cos^2(zeta_x) - 1 over the bonds whose midpoints lie in bin b;
  * g^b   = N_b / mean_b(N_b), N_b the bead centres in bin b (equal bins);
  * only bonds / beads inside the central strip |other coordinate - centre| <= half_width
    count (axial profile: bins along x, strip in y; transverse: bins along y, strip in x).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla


def min_image(d, L):
    """Nearest periodic image of a separation along a direction of period L."""
    return d - L * np.round(d / L)


def bonds(fil, pos):
    """Index pairs (a, a+1) of consecutive beads of one filament."""
    fil = np.asarray(fil)
    pos = np.asarray(pos)
    a = np.nonzero((fil[:-1] == fil[1:]) & (pos[1:] == pos[:-1] + 1))[0]
    return a, a + 1


def edges(fil, pos, X, nx, ny, rcon=2.1, chunk=2048):
    """Edges (i < j) of the contact graph with their lengths r_ij: bonds plus pairs r < rcon."""
    X = np.asarray(X, np.float64)
    n = len(X)
    fil = np.asarray(fil)
    pos = np.asarray(pos)
    I, J, R = [], [], []
    for a0 in range(0, n, chunk):
        a = np.arange(a0, min(n, a0 + chunk))
        d = X[None, :, :] - X[a, None, :]
        d[..., 0] = min_image(d[..., 0], nx)
        d[..., 1] = min_image(d[..., 1], ny)
        r2 = (d * d).sum(-1)
        bonded = (fil[None, :] == fil[a, None]) & (np.abs(pos[None, :] - pos[a, None]) == 1)
        keep = (bonded | (r2 < rcon * rcon)) & (np.arange(n)[None, :] > a[:, None])
        ii, jj = np.nonzero(keep)
        I.append(a[ii])
        J.append(jj)
        R.append(np.sqrt(r2[ii, jj]))
    if not I:
        return np.zeros(0, int), np.zeros(0, int), np.zeros(0)
    return np.concatenate(I), np.concatenate(J), np.concatenate(R)


def conductivity(fil, pos, X, nx, ny, x_src, x_snk, rcon=2.1):
    """Potentials, node currents and kappa* of the bead network (Eqs. (15)-(18))."""
    X = np.asarray(X, np.float64)
    n = len(X)
    i, j, r = edges(fil, pos, X, nx, ny, rcon)
    G = 1.0 / r
    src = X[:, 0] < x_src
    snk = X[:, 0] > x_snk
    fixed = src | snk
    V = np.where(src, 1.0, 0.0)
    W = sp.coo_matrix((np.concatenate([G, G]), (np.concatenate([i, j]), np.concatenate([j, i]))),
                      shape=(n, n)).tocsr()
    # components: only those holding an electrode node have a defined potential
    ncomp, lab = csg.connected_components(W, directed=False)
    has_src = np.zeros(ncomp, bool)
    has_snk = np.zeros(ncomp, bool)
    has_src[lab[src]] = True
    has_snk[lab[snk]] = True
    free = ~fixed
    solve = free & has_src[lab] & has_snk[lab]
    one = free & has_src[lab] & ~has_snk[lab]
    V[one] = 1.0
    if solve.any():
        deg = np.asarray(W.sum(axis=1)).ravel()
        L = sp.diags(deg) - W  # graph Laplacian
        f = np.nonzero(solve)[0]
        s = np.nonzero(fixed)[0]
        A = L[f][:, f].tocsc()
        b = -(L[f][:, s] @ V[s])
        V[f] = spla.spsolve(A, b)
    dV = V[i] - V[j]
    Iij = G * dV
    node_I = np.zeros(n)
    np.add.at(node_I, i, 0.5 * np.abs(Iij))
    np.add.at(node_I, j, 0.5 * np.abs(Iij))
    # current leaving the source and entering the sink
    out_src = np.where(src[i] & ~src[j], Iij, 0.0) + np.where(src[j] & ~src[i], -Iij, 0.0)
    in_snk = np.where(snk[j] & ~snk[i], Iij, 0.0) + np.where(snk[i] & ~snk[j], -Iij, 0.0)
    I_tot = out_src.sum()
    I_snk = in_snk.sum()
    I_ref = 1.0 / (x_snk - x_src)
    return dict(V=V, I_node=node_I / I_ref, I_tot=I_tot, I_sink=I_snk, I_ref=I_ref,
                kappa=I_tot / I_ref, n_src=int(src.sum()), n_snk=int(snk.sum()),
                n_edges=len(i))


def profiles(fil, pos, X, nx, ny, axis, lo, hi, nbins, centre, half_width):
    """Per-bin nematic order S_x^b (Eq. (13)) and normalised bead density g^b (Eq. (14)).

    axis 0: bins along x over [lo, hi), strip |y - centre| <= half_width;
    axis 1: bins along y, strip |x - centre| <= half_width.
    Returns (S_x^b, g^b, bond counts, bead counts); empty bins give S_x^b = 0."""
    X = np.asarray(X, np.float64)
    other = 1 - axis
    w = (hi - lo) / nbins
    # beads
    inside = np.abs(X[:, other] - centre) <= half_width
    kb = np.floor((X[:, axis] - lo) / w).astype(int)
    ok = inside & (kb >= 0) & (kb < nbins)
    Nb = np.bincount(kb[ok], minlength=nbins).astype(np.float64)
    mean = Nb.mean()
    g = Nb / mean if mean > 0 else np.zeros(nbins)
    # bonds by midpoint (the bond vector and midpoint use the nearest image)
    a, b = bonds(fil, pos)
    d = X[b] - X[a]
    d[:, 0] = min_image(d[:, 0], nx)
    d[:, 1] = min_image(d[:, 1], ny)
    mid = X[a] + 0.5 * d
    c2 = d[:, 0] ** 2 / (d * d).sum(1)
    ins = np.abs(mid[:, other] - centre) <= half_width
    km = np.floor((mid[:, axis] - lo) / w).astype(int)
    okb = ins & (km >= 0) & (km < nbins)
    Sb = np.bincount(km[okb], weights=2.0 * c2[okb] - 1.0, minlength=nbins)
    Cb = np.bincount(km[okb], minlength=nbins).astype(np.float64)
    S = np.where(Cb > 0, Sb / np.maximum(Cb, 1), 0.0)
    return S, g, Cb.astype(int), Nb.astype(int)
