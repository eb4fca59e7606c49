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


_PLACE = None


def _place_lib():
    """The placement loop in C (tests/place_wires.c), built with gcc on first use."""
    global _PLACE
    if _PLACE is None:
        import ctypes as C
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src, lib = os.path.join(here, "place_wires.c"), os.path.join(here, "libplace_wires.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", lib, src, "-lm"])
        L = C.CDLL(lib)
        dp = C.POINTER(C.c_double)
        L.place_wires.restype = C.c_int
        L.place_wires.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                  dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_longlong, dp, dp]
        _PLACE = L
    return _PLACE


def wires_in_droplet(seed, n_wires, n_beads, spacing, lattice, centre, semi_axes, q_max,
                     min_dist=2.0, z_range=None, max_tries=None):
    """Straight wires placed at random (uniform centres, isotropic directions) with every
    bead inside the ellipsoid of `semi_axes` about `centre` scaled by q_max (ellipsoidal
    radius q < q_max, minimum image in x and y), beads of different wires further apart
    than `min_dist`, beads in z_range (default 1 <= z <= nz - 2).  Candidates are taken
    in order, each against every wire accepted before it.  Positions wrap in x and y.
    Returns centres (unwrapped) and unit directions, [n, 3] each (fewer rows when the
    droplet is full before max_tries candidates)."""
    import ctypes as C
    nx, ny, nz = lattice
    zlo, zhi = (1.0, nz - 2.0) if z_range is None else z_range
    c = np.ascontiguousarray(centre, np.float64)
    ax = np.ascontiguousarray(semi_axes, np.float64)
    cen = np.zeros((n_wires, 3))
    dr = np.zeros((n_wires, 3))
    dp = C.POINTER(C.c_double)
    lim = 200000 + 2000 * n_wires if max_tries is None else max_tries
    got = _place_lib().place_wires(int(seed), n_wires, n_beads, float(spacing), nx, ny, nz,
                                   c.ctypes.data_as(dp), ax.ctypes.data_as(dp), float(q_max),
                                   float(min_dist), float(zlo), float(zhi), int(lim),
                                   cen.ctypes.data_as(dp), dr.ctypes.data_as(dp))
    if got < 0:
        raise RuntimeError("wire placement: cell overflow")
    return cen[:got], dr[:got]
