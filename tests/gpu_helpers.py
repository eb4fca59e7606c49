"""Shared helpers of the GPU tests: build matching oracle/library parameter sets."""
import numpy as np

from paper_2607_06794_b300 import Config

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)

SHARED = ("tau_R", "tau_B", "beta", "sigma", "rho0", "J0", "K", "evap_start", "top_bc", "ks",
          "Rm", "d0", "eps_wca", "kb", "eps_coh", "eps_s", "rc", "gamma", "xi", "mu", "gamma_t")


def oracle_params(oracle, cfg: Config):
    kw = {k: getattr(cfg, k) for k in SHARED}
    return oracle.Params(cfg.nx, cfg.ny, cfg.nz, mass=cfg.bead_mass, substeps=cfg.substeps,
                         body=tuple(cfg.body), **kw)


def oracle_state(oracle, cfg: Config, warm_steps=0, theta=None):
    """Oracle initial droplet, optionally advanced without evaporation."""
    p = oracle_params(oracle, cfg)
    fR, fB = oracle.init_droplet(p, cfg.shape, cfg.cx, cfg.cy, cfg.cz, cfg.a, cfg.b, cfg.c, cfg.width)
    th = np.full((cfg.ny, cfg.nx), cfg.theta_deg) if theta is None else theta
    cot = oracle.cot_map(th)
    if warm_steps:
        pw = oracle_params(oracle, cfg)
        pw.J0 = 0.0
        acc = oracle.Acc()
        for _ in range(warm_steps):
            oracle.step(pw, fR, fB, cot, acc)
    return p, fR, fB, cot


def pop_err(gpu, fR, fB):
    """max over populations of |gpu - oracle| / (|oracle| + w_i)."""
    ref = np.stack([fR, fB])
    scale = np.abs(ref) + W[None, :, None, None, None]
    return float(np.max(np.abs(gpu - ref) / scale))
