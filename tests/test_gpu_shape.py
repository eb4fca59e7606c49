"""GPU parity of the droplet-shape observables through the C ABI, and the E1 driver.

The parity case takes a droplet state evolved by the FP64 oracle on a patterned
substrate, writes its populations into the handle and compares every observable
with the oracle's (oracle/shape.py) from the oracle's own moments.
"""
import numpy as np
import pytest

from tests import inputs
from tests.gpu_helpers import oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_06794_b300 import build

    build.build()
    import paper_2607_06794_b300 as P

    return P


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shape_matches_oracle_on_an_evolved_droplet(lbm, oracle, prec):
    from oracle import shape as osh

    cfg = lbm.Config(72, 48, 24, prec=prec, cx=35.5, cy=23.5, cz=-0.5, a=26.0, b=12.0, c=14.0, width=2.0,
                     theta_deg=90.0, top_bc=1)
    theta = inputs.stripe_angles(cfg.nx, cfg.ny, 16, 50.0, 100.0)
    p, fR, fB, cot = oracle_state(oracle, cfg, warm_steps=30, theta=theta)
    f = oracle.fields(p, fR, fB, cot)
    ref = osh.shape(f["rhoR"], f["rhoB"], f["j"])
    sim = lbm.Simulation([cfg])
    sim.set_substrate_pattern(0, theta)
    sim.write(0, "populations", np.stack([fR, fB]))
    got = sim.shape(0)
    tol = 1e-9 if prec == "fp64" else 2e-4
    for k, v in ref.items():
        assert got[k] == pytest.approx(v, rel=tol, abs=tol), k
    assert ref["r_x"] > ref["r_y"] > 5 and 0 < ref["theta_y"] < 180


def test_e1_drying_run_shrinks_the_droplet(lbm):
    from paper_2607_06794_b300 import experiments

    r = experiments.e1_drying(steps=600, every=200, J0=2e-3)
    assert len(r["step"]) == 4
    assert np.all(np.diff(r["volume"]) < 0)            # the sink removes liquid
    assert r["h_tilde"][0] == pytest.approx(1.0)
    assert r["r_x"][0] > 2 * r["r_y"][0]               # elongated along the 116 x 42 patch
    assert np.all((r["theta_x"] > 0) & (r["theta_x"] < 180))
