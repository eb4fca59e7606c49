"""The 512x256x128 benchmark workload at full size against the FP64 oracle.

The whole lattice does not fit the oracle's few-second budget, so the GPU runs one step of
the whole lattice (FP32 and FP16 storage, the 2000 wires placed by the benchmark's rule, the
tilings the autotuner chooses from on this lattice) and the oracle one step of a 160-column x-slab
through the droplet centre holding the wires that lie wholly inside it.  Both start from
the initial droplet, each side computing it from the formula.

What one step can carry from the slab's ends (its periodic wrap, the wires it leaves out)
into the slab bounds the comparison.  The fluid alone reaches 4 columns (colour gradient,
unit normals and curvature 3, the pull 1), but the beads reach farther: in each of the 5
sub-steps a force change moves on by up to r_c = 4 through a cohesion contact or a bond,
so 20 cells of beads and 2-3 more of the fluid they push; a left-out wire that crosses a
slab end reaches up to 14 cells into the slab.  So compared are:

* every population of the slab columns at least 38 from its ends and farther than 24 cells
  from every bead of a left-out wire;
* the positions, velocities and forces of the slab's beads whose stencil lies in those
  columns and which are farther than 24 from every left-out bead.

(Two oracle slabs of 160 and 224 columns, compared on the narrower one, agree to 1e-13 from
32 columns inwards and differ by up to 0.5 in the outer 14.)  Tolerances are those of the
small-lattice parity tests: per population relative to |f| + w_i, 2e-6 for FP32 arithmetic
(2e-3 for FP16 storage) times 5 for the initial states that each side rounds on its own; bead
positions to 1e-6 (1e-5), velocities and forces to 2e-5 (2e-4).
"""
import dataclasses

import numpy as np
import pytest

from tests import inputs
from tests.gpu_helpers import W, oracle_params

pytestmark = pytest.mark.gpu

SLAB, MARGIN, REACH = 160, 38, 24.0


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import build
    build.build()
    import paper_2607_06794_b300 as P
    return P


@pytest.fixture(scope="module")
def case(lbm, oracle):
    import bench
    from paper_2607_06794_b300 import workloads
    wl = workloads.droplet_c5("fp32")
    cfg = wl.cfgs[0]
    wires = bench.wire_placement(wl)
    cen, dirs, nbf = wires[0]
    assert len(cen) == 2000
    # the slab and its wires (the benchmark's oracle arm), one oracle step
    x0 = int(round(cfg.cx + 0.5 - SLAB / 2.0))
    p = oracle_params(oracle, dataclasses.replace(cfg, nx=SLAB))
    fR, fB = oracle.init_droplet(p, cfg.shape, cfg.cx - x0, cfg.cy, cfg.cz, cfg.a, cfg.b, cfg.c, cfg.width)
    cot = oracle.cot_map(np.ascontiguousarray(wl.thetas[0][:, x0:x0 + SLAB]))
    fil, pos, X = inputs.straight_filaments(cen, dirs, nbf, cfg.d0)
    X[:, 0] %= cfg.nx
    X[:, 1] %= cfg.ny
    xb = X[:, 0].reshape(len(cen), nbf)
    inside = np.all((xb >= x0 + 1.0) & (xb <= x0 + SLAB - 2.0), axis=1)
    keepb = np.repeat(inside, nbf)
    beads = oracle.Beads(np.repeat(np.arange(int(inside.sum()), dtype=np.int32), nbf), pos[keepb],
                         X[keepb] - [x0, 0.0, 0.0])
    acc = oracle.Acc()
    oracle.step(p, fR, fB, cot, acc, beads)
    # slab nodes and beads that nothing left out of the slab reaches in one step
    out = X[~keepb]
    near = out[(out[:, 0] > x0 + MARGIN - REACH - 1) & (out[:, 0] < x0 + SLAB - MARGIN + REACH + 1)]
    node_ok = np.zeros((cfg.nz, cfg.ny, SLAB), bool)
    node_ok[:, :, MARGIN:SLAB - MARGIN] = True
    zc, yc, xc = np.meshgrid(np.arange(cfg.nz), np.arange(cfg.ny), np.arange(SLAB), indexing="ij")
    for b in near:
        dy = np.abs(yc - b[1])
        dy = np.minimum(dy, cfg.ny - dy)
        node_ok &= (xc + x0 - b[0]) ** 2 + dy ** 2 + (zc - b[2]) ** 2 > REACH ** 2
    d = X[keepb][:, None, :] - near[None, :, :]
    d[..., 1] -= cfg.ny * np.round(d[..., 1] / cfg.ny)
    far = (np.sqrt((d ** 2).sum(-1)).min(axis=1) > REACH) if len(near) else np.ones(keepb.sum(), bool)
    bx = X[keepb][:, 0] - x0
    bead_ok = far & (bx >= MARGIN + 2) & (bx <= SLAB - MARGIN - 3)
    return dict(wl=wl, wires=wires, x0=x0, fR=fR, fB=fB, beads=beads, acc=acc, keepb=keepb,
                node_ok=node_ok, bead_ok=bead_ok)


def test_the_comparison_covers_the_slab_centre(case):
    assert case["node_ok"].mean() > 0.4
    assert case["bead_ok"].sum() > 2000


# per population relative to |f| + w_i (the small-lattice parity bounds, times 5 for the
# initial states each side rounds on its own); bead velocity and force bounds
POP_TOL = {"fp32": 5 * 2e-6, "fp16": 5 * 2e-3}
BEAD_TOL = {"fp32": 2e-5, "fp16": 2e-4}


@pytest.mark.parametrize("prec,tiling", [("fp32", 13), ("fp32", 4), ("fp16", 13)])
def test_full_size_c5_step_on_the_slab(lbm, case, prec, tiling):
    import bench
    from paper_2607_06794_b300 import workloads
    x0 = case["x0"]
    wl = workloads.droplet_c5(prec)  # the same lattice, droplet and wires, stored in `prec`
    sim = bench.make_sim(wl, case["wires"])
    sim.set_tiling(tiling)
    sim.step(1)
    sim.sync()
    assert sim.status() == 0
    got = sim.read(0, "populations")[..., x0:x0 + SLAB]
    ref = np.stack([case["fR"], case["fB"]])
    rel = np.abs(got - ref) / (np.abs(ref) + W[None, :, None, None, None])
    ok = case["node_ok"][None, None]
    assert float(np.max(np.where(ok, rel, 0.0))) < POP_TOL[prec], (prec, tiling)
    del got, rel
    keepb, bok = case["keepb"], case["bead_ok"]
    ob = case["beads"]
    gx = sim.read(0, "bead_x")[keepb] - [x0, 0.0, 0.0]
    assert np.allclose(gx[bok], ob.X[bok], rtol=0, atol=1e-6 if prec == "fp32" else 1e-5), tiling
    # velocities and forces (pair forces in FP32; the drag reads u* of the stored populations)
    assert np.allclose(sim.read(0, "bead_v")[keepb][bok], ob.V[bok], rtol=0, atol=BEAD_TOL[prec]), tiling
    assert np.allclose(sim.read(0, "bead_f")[keepb][bok], ob.F[bok], rtol=0, atol=BEAD_TOL[prec]), tiling
    a = sim.read(0, "accum")
    assert a[1] == pytest.approx(case["acc"].h0, rel=1e-5)
    sim.close()
