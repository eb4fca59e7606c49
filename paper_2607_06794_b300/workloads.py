"""Synthetic workloads with the shapes of the paper's runs (Sec. III) and of the
benchmark configurations: droplet geometry, substrate wetting pattern,
nanowire load.  Every input is generated here from a seed; no dataset is used.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import Config


def stripe(nx, ny, width, inside, outside, period=None):
    """Contact angles [ny, nx]: one stripe of `width` centred in y, or stripes of `period`."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    if period is None:
        ins = np.abs(y - (ny - 1) / 2.0) < width / 2.0
    else:
        ins = np.mod(y - (ny - 1) / 2.0 + width / 2.0, period) < width
    return np.where(ins, inside, outside)


def patch(nx, ny, cx, cy, hx, hy, inside, outside):
    """Rectangular wetting patch of half-lengths hx, hy (Fig. 1 set-up)."""
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ins = (np.abs(x - cx) <= hx) & (np.abs(y - cy) <= hy)
    return np.where(ins, inside, outside)


@dataclasses.dataclass
class Workload:
    name: str
    cfgs: list
    thetas: list          # per instance [ny, nx] or None
    wires: list           # per instance (n_wires, length) or None
    steps_nominal: int

    @property
    def nodes(self):
        return sum(c.nx * c.ny * c.nz for c in self.cfgs)

    def setup(self, sim):
        for k, (th, w) in enumerate(zip(self.thetas, self.wires)):
            if th is not None:
                sim.set_substrate_pattern(k, th)
            if w is not None and w[0] > 0:
                sim.add_nanowires(k, w[0], w[1], seed=self.cfgs[k].seed)


def droplet_c1(prec="fp64"):
    """64x32x32, cap 24x8x10 on a homogeneous 90 deg substrate, no wires, sink on."""
    c = Config(64, 32, 32, prec=prec, cx=31.5, cy=15.5, cz=-0.5, a=24, b=8, c=10, width=2.0,
               theta_deg=90.0, J0=1e-4, evap_start=0, top_bc=1)
    return Workload("c1_64x32x32_droplet", [c], [None], [None], 1000)


def droplet_c2(prec="fp32", wires=200):
    """256x128x64, aspect-4 cap 96x24x24 on a 48-wide 60/110 deg stripe, 200 wires L=8."""
    c = Config(256, 128, 64, prec=prec, cx=127.5, cy=63.5, cz=-0.5, a=96, b=24, c=24, width=2.0,
               theta_deg=110.0, J0=5e-4, evap_start=0, top_bc=1, max_beads=4 * wires + 64,
               eps_coh=1.0 * 0.006, xi=0.05, gamma=1.0, x_src=127.5 - 0.26 * 192,
               x_snk=127.5 + 0.26 * 192, seed=1234)
    th = stripe(256, 128, 48, 60.0, 110.0)
    return Workload("c2_256x128x64_stripe_200wires", [c], [th], [(wires, 8.0)], 20000)


def droplet_c5(prec="fp16", wires=2000):
    """512x256x128, aspect-6 cap 192x32x48 on periodic stripes (64/32), 2000 wires L=16."""
    c = Config(512, 256, 128, prec=prec, cx=255.5, cy=127.5, cz=-0.5, a=192, b=32, c=48,
               width=2.0, theta_deg=110.0, J0=2e-4, evap_start=0, top_bc=1,
               max_beads=8 * wires + 64, eps_coh=0.006, xi=0.05, gamma=1.0,
               x_src=255.5 - 0.26 * 384, x_snk=255.5 + 0.26 * 384, seed=4321)
    th = stripe(512, 256, 32, 60.0, 110.0, period=64)
    return Workload("c5_512x256x128_periodic_stripes_2000wires", [c], [th], [(wires, 16.0)], 50000)


def paper_droplet(prec="fp32", theta_r=30.0):
    """The paper's pure-droplet domain 256x104x36 with a 116x42 patch (Fig. 1, Sec. III.A)."""
    c = Config(256, 104, 36, prec=prec, cx=127.5, cy=51.5, cz=-0.5, a=116, b=42, c=30, width=2.0,
               theta_deg=90.0, J0=2e-4, evap_start=0, top_bc=1)
    th = patch(256, 104, 127.5, 51.5, 116, 42, theta_r, 90.0)
    return Workload("paper_256x104x36_patch", [c], [th], [None], 20000)


def batched_c4(prec="fp16", n=64):
    """64 uneven lattices (64..192) x 64 x 48: aspect ratio x eps* x wire length grid.

    Wire counts follow the droplet volume (about 1% of it in beads, 10..400 wires)
    so that straight wires of every length fit inside the liquid."""
    ars = [1.0, 2.67, 4.33, 6.0]
    epss = [0.0, 0.5, 1.0, 2.0]
    lens = [4.0, 8.0, 12.0, 16.0]
    cfgs, ths, ws = [], [], []
    k = 0
    for ar in ars:
        for e in epss:
            for L in lens:
                if k >= n:
                    break
                b = 14.0
                a = b * ar
                nx = int(min(192, max(64, 32 * np.ceil((2 * a + 24) / 32))))
                ny, nz = 64, 48
                vol = 2.0 / 3.0 * np.pi * a * b * 20.0
                nbpw = max(1, int(round(L / 2.0)))
                nw = int(np.clip(vol * 0.01 / nbpw, 10, 400))
                c = Config(nx, ny, nz, prec=prec, cx=nx / 2 - 0.5, cy=ny / 2 - 0.5, cz=-0.5, a=a, b=b,
                           c=20.0, width=2.0, theta_deg=110.0, J0=5e-4, evap_start=0, top_bc=1,
                           max_beads=nw * nbpw + 64, eps_coh=e * 0.006, xi=0.05, gamma=1.0,
                           substeps=5, x_src=nx / 2 - 0.26 * 2 * a, x_snk=nx / 2 + 0.26 * 2 * a,
                           seed=1000 + k)
                cfgs.append(c)
                ths.append(stripe(nx, ny, 2 * b, 60.0, 110.0))
                ws.append((nw, L))
                k += 1
    return Workload(f"c4_batched_{n}_instances", cfgs, ths, ws, 10000)


def deposit_c5(seed=7, n_wires=2000, n_beads=8, spread=0.6):
    """A dried deposit with the c5 wire load for the analysis kernels: 2000 straight
    filaments of 8 beads lying flat (z = 1) on the 512 x 256 substrate, centres uniform
    in the droplet's central region, directions scattered by `spread` radians about x,
    electrodes at x_c -/+ 0.26 (2a) of the aspect-6 cap.  Returns (cfg, centres, dirs, X)
    with X the bead positions wrapped into the lattice."""
    g = np.random.default_rng(seed)
    nx, ny = 512, 256
    cen = np.c_[g.uniform(100, 412, n_wires), g.uniform(90, 166, n_wires), np.ones(n_wires)]
    ang = g.normal(0.0, spread, n_wires)
    dirs = np.c_[np.cos(ang), np.sin(ang), np.zeros(n_wires)]
    k = np.arange(n_beads) - (n_beads - 1) / 2.0
    X = (cen[:, None, :] + 2.0 * k[None, :, None] * dirs[:, None, :]).reshape(-1, 3)
    X[:, 0] %= nx
    X[:, 1] %= ny
    c = Config(nx, ny, 8, prec="fp32", cx=255.5, cy=127.5, cz=-0.5, a=200, b=100, c=6.0, width=2.0,
               theta_deg=90.0, top_bc=1, max_beads=n_wires * n_beads + 64,
               x_src=255.5 - 0.26 * 384, x_snk=255.5 + 0.26 * 384, seed=seed)
    return c, cen, dirs, X


WORKLOADS = {"c1": droplet_c1, "c2": droplet_c2, "c5": droplet_c5, "paper": paper_droplet,
             "c4": batched_c4}
