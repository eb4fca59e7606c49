"""Experiment drivers built on the library (Sec. III).

e1_drying: the pure droplet on a rectangular patch (Sec. III.A, Fig. 2) -- the
paper's 256x104x36 domain with a 116x42 patch of receding angle theta_r in a 90
deg surround -- evaporating from step 0, with the droplet height, footprint
radii, contact angles and mean flow recorded every `every` steps, normalised by
the initial height h0 as in the paper (h~ = h/h0, r~ = r/h0).

storage_comparison: one workload run at several storage precisions from the
same initial state and the same wires, recording the droplet observables over
the run and the deposit descriptors (S_x of Eq. (13), contact clusters and
percolation of Sec. II.B) at the end, for the error of reduced-precision
storage against FP64.
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


def storage_comparison(make, precs=("fp64", "fp16", "bf16"), steps=1000, every=None, wires=None, report=None):
    """Run the workload `make(prec)` at each precision for `steps` steps.

    wires: per instance (centres, directions, beads per wire) placed identically in
    every run (None: the workload's own seeded placement).  Returns, per precision,
    the shape observables every `every` steps (and at the end) and the descriptors
    and shape at the end, of instance 0 and, under "instances", of every instance.  A run
    whose device status latches a failure stops at the next record; its status and step
    are reported and the state where it stopped is measured."""
    out = {}
    for prec in precs:
        wl = make(prec)
        sim = Simulation(wl.cfgs)
        for k, th in enumerate(wl.thetas):
            if th is not None:
                sim.set_substrate_pattern(k, th)
        if wires is None:
            # the first run places the wires (seeded, inside its liquid); the later runs take
            # the same wires, rebuilt from the first run's bead positions
            for k, w in enumerate(wl.wires):
                if w is not None and w[0] > 0:
                    sim.add_nanowires(k, w[0], w[1], seed=wl.cfgs[k].seed)
            wires = [None] * len(wl.cfgs)
            for k, w in enumerate(wl.wires):
                if w is not None and w[0] > 0:
                    c = wl.cfgs[k]
                    nbf = max(1, int(round(w[1] / c.d0)))
                    X = sim.read(k, "bead_x").reshape(w[0], nbf, 3)
                    d = X[:, -1] - X[:, 0]
                    d[:, 0] -= c.nx * np.round(d[:, 0] / c.nx)
                    d[:, 1] -= c.ny * np.round(d[:, 1] / c.ny)
                    cen = X[:, 0] + 0.5 * d
                    wires[k] = (cen, d, nbf)
        else:
            for k, pw in enumerate(wires):
                if pw is not None:
                    sim.add_nanowires(k, len(pw[0]), pw[2] * wl.cfgs[k].d0, pw[0], pw[1])
        ninst = len(wl.cfgs)
        rec = [[] for _ in range(ninst)]
        done = 0
        every_ = steps if not every else every
        status = 0
        while True:
            status = sim.status()
            if status != 0:
                # a latched failure (say a bead pushed out of the fluid at the top late in the
                # drying): the run stops here and reports it; the error is cleared so that the
                # state where it stopped can still be measured
                sim.clear_error()
                for k in range(ninst):
                    rec[k].append(dict(step=done, **sim.shape(k)))
                break
            if done % every_ == 0 or done == steps:
                for k in range(ninst):
                    rec[k].append(dict(step=done, **sim.shape(k)))
            if done >= steps:
                break
            n = min(every_ - done % every_, steps - done)
            sim.step(n)
            done += n
        sim.sync()
        placed = wires or wl.wires
        desc = [sim.descriptors(k) if placed[k] is not None else None for k in range(ninst)]
        # instance 0 at the top level; every instance under "instances"
        out[prec] = {"series": rec[0], "final": rec[0][-1], "descriptors": desc[0], "status": status,
                     "stopped_at": done if status != 0 else None,
                     "instances": [{"series": rec[k], "final": rec[k][-1], "descriptors": desc[k]}
                                   for k in range(ninst)]}
        sim.close()
        if report is not None:
            report(prec, out[prec])
    return out


def main(argv=None):
    """python -m paper_2607_06794_b300.experiments [--steps N] [--every K] [--J0 J] [--theta_r T]:
    prints one JSON line per record of the E1 drying run.
    python -m paper_2607_06794_b300.experiments --compare c5 [--precs fp64,fp32,fp16] --steps N:
    runs that workload at each storage precision with the same wires and prints, per
    precision, the droplet observables along the run and the deposit descriptors."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--compare", default=None)
    ap.add_argument("--precs", default="fp64,fp32,fp16")
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--theta_r", type=float, default=30.0)
    ap.add_argument("--J0", type=float, default=None)
    a = ap.parse_args(argv)
    if a.compare:
        def show(prec, r):
            print(json.dumps({"precision": prec, "status": r["status"], "stopped_at": r["stopped_at"],
                              "descriptors": r["descriptors"],
                              "series": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in e.items()}
                                         for e in r["series"]]}), flush=True)
        storage_comparison(workloads.WORKLOADS[a.compare], tuple(a.precs.split(",")), a.steps, a.every,
                           report=show)
        return
    r = e1_drying(a.steps, a.every, a.prec, a.theta_r, a.J0)
    for k in range(len(r["step"])):
        print(json.dumps({key: (int(r[key][k]) if key == "step" else round(float(r[key][k]), 6))
                          for key in ("step", "volume", "h_tilde", "rx_tilde", "ry_tilde", "theta_x",
                                      "theta_y", "v_x", "v_y")}))


if __name__ == "__main__":
    main()
