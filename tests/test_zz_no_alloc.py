"""The descriptor entry point that allocates nothing, checked against the
workspace-based entry point (lbm_deposit_descriptors) on two calls in a row.

Some callers cannot allocate device memory (a host application that has
already reserved nearly all of it for its own pool, or a time-critical loop
that must not pay for cudaMalloc); lbm_deposit_descriptors_noalloc serves them
from a fixed array inside the library.  This file is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_descriptors_match_the_workspace_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import Config, Simulation, _lib, build
    build.build()
    L = _lib.load()
    nx, ny = 64, 48
    cfg = Config(nx, ny, 24, prec="fp64", cx=31.5, cy=23.5, cz=-0.5, a=24, b=18, c=16, max_beads=400,
                 x_src=20.0, x_snk=44.0)
    sim = Simulation([cfg])
    g = np.random.default_rng(3)
    nw = 60
    cen = np.c_[g.uniform(12, 52, nw), g.uniform(10, 38, nw), g.uniform(2, 10, nw)]
    dirs = np.c_[g.normal(size=nw), g.normal(size=nw), 0.2 * g.normal(size=nw)]
    sim.add_nanowires(0, nw, 8.0, cen, dirs)
    ref = sim.descriptors(0)
    X = sim.read(0, "bead_x")
    topo = sim.read(0, "bead_topo")
    n = X.shape[0]
    dX = torch.tensor(X, dtype=torch.float64, device="cuda")
    dfil = torch.tensor(np.ascontiguousarray(topo[:, 0]), dtype=torch.int32, device="cuda")
    dpos = torch.tensor(np.ascontiguousarray(topo[:, 1]), dtype=torch.int32, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(-1.0)
        r = L.lbm_deposit_descriptors_noalloc(_p(dX), _p(dfil), _p(dpos), n, nx, ny, cfg.rcon, cfg.x_src,
                                              cfg.x_snk, _p(out), st)
        assert r == _lib.OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[4] == 0.0
        assert o[0] == pytest.approx(ref["S_x"], abs=1e-12)
        assert int(o[1]) == ref["n_clusters"]
        assert bool(o[2]) == bool(ref["percolates"])
        assert int(o[3]) == ref["n_bonds"]
    # sizes beyond the fixed array are refused before any device work
    assert L.lbm_deposit_descriptors_noalloc(_p(dX), _p(dfil), _p(dpos), 16385, nx, ny, 2.1, 0.0, 1.0,
                                             _p(out), st) == _lib.ECAPACITY
    sim.close()
