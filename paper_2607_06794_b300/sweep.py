"""Parameter sweeps over batched lattices and the learned sweep proposer.

The paper explores droplet geometry, filament cohesion and filament length by
running ensembles at enumerated parameter values (Sec. III).  Here a sweep
point p = (aspect ratio, eps*, length L, stripe width) becomes one lattice of
a batch; all points of a batch advance together in one launch per step
(`batched_points`).  The proposer is a small MLP trained on the GPU through
the library's own forward/backward/Adam kernels on the descriptors the runs
produce (S_x, cluster count, percolation); it picks which points to simulate
next, and every proposal is judged by running it.  Plain enumeration of the
grid is the fallback and the comparison.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import Config, LBMError, Simulation, _lib
from .workloads import stripe

N_IN, N_HIDDEN, N_OUT = 4, 64, 3


# ----------------------------------------------------------------------------- simulation side
def point_config(p, prec="fp16", nz=32, seed=0):
    """Lattice, droplet and wires of one sweep point (aspect, eps*, L, stripe width)."""
    ar, eps_star, L, sw = p
    b = 10.0
    a = b * ar
    nx = int(max(32, 16 * np.ceil((2 * a + 16) / 16)))
    ny = int(max(32, 16 * np.ceil((2 * b + 24) / 16)))
    c = Config(nx, ny, nz, prec=prec, cx=nx / 2 - 0.5, cy=ny / 2 - 0.5, cz=-0.5, a=a, b=b, c=16.0,
               width=2.0, theta_deg=110.0, J0=1e-3, evap_start=0, top_bc=1, eps_coh=eps_star * 0.006,
               xi=0.05, gamma=1.0, x_src=nx / 2 - 0.26 * 2 * a, x_snk=nx / 2 + 0.26 * 2 * a, seed=seed)
    nbw = max(1, int(round(L / c.d0)))
    vol = 2.0 / 3.0 * np.pi * a * b * 16.0
    nw = int(np.clip(vol * 0.005 / nbw, 4, 200))
    c.max_beads = nw * nbw + 16
    theta = stripe(nx, ny, sw, 60.0, 110.0)
    return c, theta, nw


def batched_points(points, steps, prec="fp16", seed=0, autotune=False):
    """Run every point as one lattice of a single batch; returns descriptor rows."""
    cfgs, thetas, nws = [], [], []
    for k, p in enumerate(points):
        c, th, nw = point_config(p, prec, seed=seed + k)
        cfgs.append(c)
        thetas.append(th)
        nws.append(nw)
    sim = Simulation(cfgs)
    for k, (p, th, nw) in enumerate(zip(points, thetas, nws)):
        sim.set_substrate_pattern(k, th)
        sim.add_nanowires(k, nw, p[2], seed=1 + seed + k)
    if autotune:
        sim.autotune(2)
    sim.step(steps)
    sim.sync()
    rows = []
    for k in range(len(points)):
        d = sim.descriptors(k)
        rows.append([d["S_x"], d["n_clusters"] / max(1, nws[k]), float(d["percolates"])])
    sim.close()
    return np.array(rows)


def deposit_table(points, seeds=(0,), prec="fp16", max_steps=20000, every=500, autotune=True):
    """Descriptors of the dried deposits of every sweep point: all (point, seed) pairs
    advance as one batch until every droplet has evaporated (no liquid left) or
    max_steps.  Returns (rows [n_points, 3] = mean S_x, mean cluster count per wire,
    percolation fraction over the seeds, NaN where no wire fits the droplet; steps
    taken; per-run raw rows)."""
    runs = [(k, s) for k in range(len(points)) for s in seeds]
    cfgs, thetas, nws = [], [], []
    for k, s in runs:
        c, th, nw = point_config(points[k], prec, seed=1009 * s + k)
        cfgs.append(c)
        thetas.append(th)
        nws.append(nw)
    sim = Simulation(cfgs)
    for j, ((k, s), th, nw) in enumerate(zip(runs, thetas, nws)):
        sim.set_substrate_pattern(j, th)
        # long wires in a small droplet: halve the count until they fit straight inside;
        # a point where not even one fits has no deposit (its row is NaN)
        while nw > 0:
            try:
                sim.add_nanowires(j, nw, points[k][2], seed=1 + 1009 * s + k)
                break
            except LBMError as e:
                if e.code != _lib.EINVAL:
                    raise
                nw //= 2
        nws[j] = nw
    if autotune:
        sim.autotune(2)
    done = 0
    while done < max_steps:
        sim.step(every)
        done += every
        if all(sim.shape(j)["volume"] <= 0.0 for j in range(len(runs))):
            break
    sim.sync()
    raw = np.full((len(runs), 3), np.nan)
    for j in range(len(runs)):
        if nws[j] > 0:
            d = sim.descriptors(j)
            raw[j] = (d["S_x"], d["n_clusters"] / nws[j], float(d["percolates"]))
    sim.close()
    r3 = raw.reshape(len(points), len(seeds), 3)
    rows = np.full((len(points), 3), np.nan)
    ok = ~np.all(np.isnan(r3[:, :, 0]), axis=1)
    rows[ok] = np.nanmean(r3[ok], axis=1)
    return rows, done, raw


# ----------------------------------------------------------------------------- proposer
class Proposer:
    """Ensemble of small MLPs on the GPU (parameters, Adam moments and batches in
    device memory); the spread of the members' predictions measures uncertainty."""

    def __init__(self, seed=0, device="cuda:0", lr=3e-3, members=4):
        import torch
        self.torch = torch
        self.L = _lib.load()
        self.dev = torch.device(device)
        self.P = int(self.L.lbm_mlp_param_count(N_IN, N_HIDDEN, N_OUT))
        self.lr = lr
        self.nets = []
        for k in range(members):
            g = np.random.default_rng(1000 * seed + k)
            parts = []
            for (fan_out, fan_in) in ((N_HIDDEN, N_IN), (N_HIDDEN, N_HIDDEN), (N_OUT, N_HIDDEN)):
                parts.append(g.normal(scale=1.0 / np.sqrt(fan_in), size=fan_out * fan_in))
                parts.append(np.zeros(fan_out))
            p = np.concatenate(parts)
            assert p.size == self.P
            self.nets.append(torch.tensor(p, dtype=torch.float32, device=self.dev))
        self.grad = torch.zeros(self.P, dtype=torch.float32, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.xmu = self.xsd = self.ymu = self.ysd = None

    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream(self.dev).cuda_stream)

    @staticmethod
    def _p(t):
        return C.c_void_p(t.data_ptr())

    def fit(self, X, Y, epochs=400):
        """Refit every member on (X, Y) (inputs and targets standardised); returns the mean loss."""
        torch = self.torch
        X = np.asarray(X, np.float64)
        Y = np.asarray(Y, np.float64)
        self.xmu, self.xsd = X.mean(0), X.std(0) + 1e-9
        self.ymu, self.ysd = Y.mean(0), Y.std(0) + 1e-9
        x = torch.tensor((X - self.xmu) / self.xsd, dtype=torch.float32, device=self.dev)
        t = torch.tensor((Y - self.ymu) / self.ysd, dtype=torch.float32, device=self.dev)
        B = x.shape[0]
        y = torch.zeros((B, N_OUT), dtype=torch.float32, device=self.dev)
        nsc = int(self.L.lbm_mlp_scratch_bytes(0, N_HIDDEN, B))
        sc = torch.empty(nsc, dtype=torch.uint8, device=self.dev)
        st = self._stream()
        losses = []
        for prm in self.nets:
            m = torch.zeros(self.P, dtype=torch.float32, device=self.dev)
            v = torch.zeros(self.P, dtype=torch.float32, device=self.dev)
            for step in range(1, epochs + 1):
                r = self.L.lbm_mlp_loss_grad(0, self._p(prm), N_IN, N_HIDDEN, N_OUT, self._p(x), self._p(t), B,
                                             self._p(y), self._p(self.grad), self._p(self.loss), self._p(sc),
                                             nsc, st)
                assert r == 0, r
                r = self.L.lbm_mlp_adam(0, self._p(prm), self._p(self.grad), self._p(m), self._p(v), self.P,
                                        self.lr, 0.9, 0.999, 1e-8, step, st)
                assert r == 0, r
            torch.cuda.synchronize(self.dev)
            losses.append(float(self.loss.item()))
        return float(np.mean(losses))

    def predict_members(self, X):
        """[members, n, N_OUT] predictions in the original units."""
        torch = self.torch
        X = np.asarray(X, np.float64)
        x = torch.tensor((X - self.xmu) / self.xsd, dtype=torch.float32, device=self.dev)
        out = []
        for prm in self.nets:
            y = torch.zeros((x.shape[0], N_OUT), dtype=torch.float32, device=self.dev)
            r = self.L.lbm_mlp_forward(0, self._p(prm), N_IN, N_HIDDEN, N_OUT, self._p(x), x.shape[0],
                                       self._p(y), self._stream())
            assert r == 0, r
            out.append(y)
        torch.cuda.synchronize(self.dev)
        return np.stack([o.cpu().numpy().astype(np.float64) * self.ysd + self.ymu for o in out])

    def predict(self, X):
        return self.predict_members(X).mean(axis=0)


@dataclasses.dataclass
class SweepResult:
    evaluated: list          # indices of candidates simulated, in order
    values: list             # objective of each evaluated point
    prediction_error: list   # |predicted - simulated| objective of each proposal

    @property
    def best(self):
        return max(self.values)


def active_sweep(candidates, simulate, objective, budget, seed_points, per_round, seed=0, epochs=400,
                 kappa=1.0, members=4):
    """Spend `budget` simulations: `seed_points` random grid points, then rounds in which
    the ensemble, refit on everything simulated so far, proposes the `per_round`
    unevaluated candidates with the highest mean + kappa * spread of the predicted
    objective; every proposal is simulated and its prediction error recorded."""
    cand = np.asarray(candidates, np.float64)
    g = np.random.default_rng(seed)
    order = g.permutation(len(cand))
    chosen = [int(i) for i in order[:seed_points]]
    Y = list(simulate(cand[chosen]))
    vals = [objective(y) for y in Y]
    err = []
    prop = Proposer(seed=seed, members=members)
    while len(chosen) < budget:
        prop.fit(cand[chosen], np.array(Y), epochs=epochs)
        left = np.array([i for i in range(len(cand)) if i not in set(chosen)])
        pm = prop.predict_members(cand[left])
        objs = np.array([[objective(p) for p in member] for member in pm])
        mean, spread = objs.mean(axis=0), objs.std(axis=0)
        rank = np.argsort(-(mean + kappa * spread))[:min(per_round, budget - len(chosen))]
        take = left[rank]
        Yn = simulate(cand[take])
        for i, y, s in zip(take, Yn, mean[rank]):
            chosen.append(int(i))
            Y.append(y)
            vals.append(objective(y))
            err.append(abs(s - objective(y)))
    return SweepResult(chosen, vals, err)


def grid_sweep(candidates, simulate, objective, budget):
    """Fallback: enumerate the grid in its natural order until the budget is spent."""
    cand = np.asarray(candidates, np.float64)
    idx = list(range(min(budget, len(cand))))
    Y = simulate(cand[idx])
    return SweepResult(idx, [objective(y) for y in Y], [])


def default_grid():
    """Aspect ratio x eps* x length x stripe width grid of the batched sweep."""
    pts = []
    for ar in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0):
        for e in (0.0, 0.5, 1.0, 2.0):
            for L in (4.0, 8.0, 12.0, 16.0):
                for sw in (12.0, 16.0, 24.0):
                    pts.append((ar, e, L, sw))
    return np.array(pts)
