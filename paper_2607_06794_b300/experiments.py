"""Experiment drivers built on the library (Sec. III).

e1_drying: the pure droplet on a rectangular patch (Sec. III.A, Fig. 2) -- the
paper's 256x104x36 domain with a 116x42 patch of receding angle theta_r in a 90
deg surround -- evaporating from step 0, with the droplet height, footprint
radii, contact angles and mean flow recorded every `every` steps, normalised by
the initial height h0 as in the paper (h~ = h/h0, r~ = r/h0).
"""
from __future__ import annotations

import numpy as np

from . import Simulation, workloads


def e1_drying(steps=20000, every=500, prec="fp32", theta_r=30.0, J0=None):
    wl = workloads.paper_droplet(prec, theta_r)
    if J0 is not None:
        wl.cfgs[0].J0 = J0
    sim = Simulation(wl.cfgs)
    wl.setup(sim)
    keys = ("volume", "height", "r_x", "r_y", "theta_x", "theta_y", "v_x", "v_y")
    rec = {k: [] for k in keys}
    t = []
    done = 0
    while True:
        s = sim.shape(0)
        t.append(done)
        for k in keys:
            rec[k].append(s[k])
        if done >= steps or s["volume"] <= 0.0:
            break
        n = min(every, steps - done)
        sim.step(n)
        done += n
    sim.sync()
    sim.close()
    out = {k: np.array(v) for k, v in rec.items()}
    out["step"] = np.array(t)
    h0 = out["height"][0]
    out["h_tilde"] = out["height"] / h0
    out["rx_tilde"] = out["r_x"] / h0
    out["ry_tilde"] = out["r_y"] / h0
    return out
