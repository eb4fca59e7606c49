"""Seeded synthetic inputs shared by the oracle and the GPU tests.

Holds no arithmetic of the method: only random numbers and geometric
placements that both sides receive as inputs.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def stripe_angles(nx, ny, width, inside_deg, outside_deg, period=None):
    """Contact-angle map [ny, nx]: a stripe of `width` centred in y (or a periodic set)."""
    y = np.arange(ny)[:, None] + 0.0 * np.arange(nx)[None, :]
    if period is None:
        inside = np.abs(y - (ny - 1) / 2.0) < width / 2.0
    else:
        inside = (np.mod(y, period) < width)
    return np.where(inside, inside_deg, outside_deg).astype(np.float64)


def straight_filaments(centres, dirs, n_beads, spacing):
    """Bead positions of straight filaments; returns fil, pos, X."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 3)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    fil, pos, X = [], [], []
    for f, (c, d) in enumerate(zip(centres, dirs)):
        for k in range(n_beads):
            fil.append(f)
            pos.append(k)
            X.append(c + (k - (n_beads - 1) / 2.0) * spacing * d)
    return np.array(fil, np.int32), np.array(pos, np.int32), np.array(X)


def random_filaments(seed, n_fil, n_beads, spacing, box_lo, box_hi, min_dist=2.0, max_tries=100000):
    """Non-overlapping straight filaments with uniform centres and isotropic directions."""
    g = rng(seed)
    box_lo = np.asarray(box_lo, float)
    box_hi = np.asarray(box_hi, float)
    cs, ds, placed = [], [], np.zeros((0, 3))
    tries = 0
    while len(cs) < n_fil and tries < max_tries:
        tries += 1
        c = g.uniform(box_lo, box_hi)
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        _, _, X = straight_filaments([c], [d], n_beads, spacing)
        if np.any(X < box_lo) or np.any(X > box_hi):
            continue
        if len(placed):
            dd = np.linalg.norm(placed[:, None, :] - X[None, :, :], axis=-1)
            if dd.min() <= min_dist:
                continue
        cs.append(c)
        ds.append(d)
        placed = np.vstack([placed, X])
    return np.array(cs), np.array(ds)


def flat_deposit(seed, n_fil, n_beads, box, z=1.0, spread=0.6, spacing=2.0):
    """A dried deposit: straight filaments lying flat at height z with uniform centres in
    box = (x0, x1, y0, y1) and directions scattered by `spread` (radians) about the x axis.
    Returns centres, directions and fil, pos, X of the beads (overlaps allowed)."""
    g = rng(seed)
    x0, x1, y0, y1 = box
    cen = np.c_[g.uniform(x0, x1, n_fil), g.uniform(y0, y1, n_fil), np.full(n_fil, z)]
    ang = g.normal(0.0, spread, n_fil)
    dirs = np.c_[np.cos(ang), np.sin(ang), np.zeros(n_fil)]
    fil, pos, X = straight_filaments(cen, dirs, n_beads, spacing)
    return cen, dirs, fil, pos, X
