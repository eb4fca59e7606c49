"""FP64 CPU oracle of the droplet-shape observables of the drying runs (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this module; it shares nothing with the CUDA library.

The paper tracks, for the pure droplet on a patch (Sec. III.A, Fig. 2), the
droplet height, the footprint radii along x and y, the contact angles along
both axes and the mean flow speeds at half the footprint radius.  It does not
say how they are measured; the readings taken here:
  * liquid column height h(x,y) = sum_z (1 + C)/2 (as in the sink of Eq. (8));
    the droplet height H is its maximum, the volume V its sum;
  * centre (x_c, y_c) = h-weighted centroid of the footprint;
  * footprint radius r_x = half the length of the positive run of C(x, y_c, 0)
    around x_c, its ends at the C = 0 crossings (linear interpolation); r_y alike
    along y at x_c (indices rounded to the nearest node);
  * contact angles theta_x = 2 atan(H / r_x), theta_y = 2 atan(H / r_y): the
    spherical-cap relation in each principal section;
  * v_x = mean of u_x = j_x / rho over the liquid nodes (C > 0) of the column at
    (x_c + r_x/2, y_c); v_y = mean of u_y over the column at (x_c, y_c + r_y/2).
"""
from __future__ import annotations

import numpy as np


def colour(rhoR, rhoB):
    return (rhoR - rhoB) / (rhoR + rhoB)


def crossing_run(profile, i0):
    """(left, right) C = 0 crossings of the positive run of `profile` around index i0."""
    n = len(profile)
    if not (0 <= i0 < n) or profile[i0] <= 0:
        return float(i0), float(i0)
    lo = i0
    while lo - 1 >= 0 and profile[lo - 1] > 0:
        lo -= 1
    hi = i0
    while hi + 1 < n and profile[hi + 1] > 0:
        hi += 1
    left = lo - profile[lo] / (profile[lo] - profile[lo - 1]) if lo > 0 else float(lo)
    right = hi + profile[hi] / (profile[hi] - profile[hi + 1]) if hi + 1 < n else float(hi)
    return left, right


def shape(rhoR, rhoB, j):
    """Observables from the moments [nz, ny, nx] (rho_R, rho_B) and j [nz, ny, nx, 3]."""
    C = colour(rhoR, rhoB)
    nz, ny, nx = C.shape
    h = ((1.0 + C) / 2.0).sum(axis=0)
    V = h.sum()
    H = h.max()
    xs = np.arange(nx)[None, :]
    ys = np.arange(ny)[:, None]
    xc = float((h * xs).sum() / V)
    yc = float((h * ys).sum() / V)
    ix, iy = int(np.floor(xc + 0.5)), int(np.floor(yc + 0.5))
    lx, rx = crossing_run(C[0, iy, :], ix)
    ly, ry = crossing_run(C[0, :, ix], iy)
    r_x, r_y = (rx - lx) / 2.0, (ry - ly) / 2.0
    th_x = float(np.degrees(2.0 * np.arctan2(H, r_x)))
    th_y = float(np.degrees(2.0 * np.arctan2(H, r_y)))
    rho = rhoR + rhoB

    def column_mean(x, y, d):
        x, y = int(np.floor(x + 0.5)) % nx, int(np.floor(y + 0.5)) % ny
        liq = C[:, y, x] > 0
        if not liq.any():
            return 0.0
        return float((j[:, y, x, d][liq] / rho[:, y, x][liq]).mean())

    v_x = column_mean(xc + r_x / 2.0, yc, 0)
    v_y = column_mean(xc, yc + r_y / 2.0, 1)
    return dict(volume=float(V), height=float(H), xc=xc, yc=yc, r_x=float(r_x), r_y=float(r_y),
                theta_x=th_x, theta_y=th_y, v_x=v_x, v_y=v_y)
