"""Sweep-proposer network: oracle pinned by finite differences and closed forms;
GPU forward/backward/Adam through the C ABI against the oracle."""
import ctypes as C

import numpy as np
import pytest

from tests import inputs
from oracle import mlp as M

I, H, O = 4, 64, 3


def params(seed, scale=0.4):
    g = inputs.rng(seed)
    return g.normal(scale=scale, size=M.count(I, H, O))


def batch(seed, B=37):
    g = inputs.rng(seed)
    return g.normal(size=(B, I)), g.normal(size=(B, O))


def test_oracle_gradient_matches_central_differences():
    p = params(1)
    x, t = batch(2, 9)
    g = M.grad(p, x, t, I, H, O)
    h = 1e-6
    idx = inputs.rng(3).choice(p.size, 300, replace=False)
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss(pp, x, t, I, H, O) - M.loss(pm, x, t, I, H, O)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k]))


def test_oracle_closed_forms():
    p = params(4)
    x, t = batch(5)
    W1, b1, W2, b2, W3, b3 = M.unpack(p, I, H, O)
    # with the last layer zero the output is b3 and dL/db3 = mean(b3 - t)
    q = p.copy()
    off = H * I + H + H * H + H
    q[off:off + O * H] = 0.0
    y, _, _ = M.forward(q, x, I, H, O)
    assert np.allclose(y, np.broadcast_to(q[-O:], y.shape))
    g = M.grad(q, x, t, I, H, O)
    assert np.allclose(g[-O:], (q[-O:] - t).mean(axis=0), rtol=1e-14, atol=1e-15)
    # gradients below a zero last layer vanish
    assert np.all(g[:off] == 0.0)
    # Adam's first step moves every parameter by lr * sign(g) (up to eps)
    g = M.grad(p, x, t, I, H, O)
    p1, m, v = M.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1e-3, 0.9, 0.999, 1e-12, 1)
    assert np.allclose(p - p1, 1e-3 * np.sign(g), rtol=1e-6, atol=1e-12)


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06794_b300 import _lib, build
    build.build()
    return _lib.load(), torch


def _dev(torch, a, dt):
    return torch.tensor(a, dtype=dt, device="cuda")


def _ptr(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,tol", [(1, 1e-12), (0, 1e-5)])
def test_gpu_loss_grad_matches_oracle(gpu, dtype, tol):
    L, torch = gpu
    dt = torch.float64 if dtype == 1 else torch.float32
    p = params(7)
    x, t = batch(8, 200)
    P = L.lbm_mlp_param_count(I, H, O)
    assert P == p.size
    dp, dx, dtg = _dev(torch, p, dt), _dev(torch, x, dt), _dev(torch, t, dt)
    y = torch.zeros((200, O), dtype=dt, device="cuda")
    g = torch.zeros(P, dtype=dt, device="cuda")
    loss = torch.zeros(1, dtype=dt, device="cuda")
    nsc = L.lbm_mlp_scratch_bytes(dtype, H, 200)
    sc = torch.empty(nsc, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.lbm_mlp_loss_grad(dtype, _ptr(dp), I, H, O, _ptr(dx), _ptr(dtg), 200, _ptr(y), _ptr(g),
                               _ptr(loss), _ptr(sc), nsc, C.c_void_p(st)) == 0
    torch.cuda.synchronize()
    yo, _, _ = M.forward(p, x, I, H, O)
    go = M.grad(p, x, t, I, H, O)
    assert np.allclose(y.cpu().numpy(), yo, rtol=tol, atol=tol)
    gs = np.abs(go).max()
    assert np.max(np.abs(g.cpu().numpy() - go)) <= tol * gs
    assert abs(loss.item() - M.loss(p, x, t, I, H, O)) <= tol * M.loss(p, x, t, I, H, O)


@pytest.mark.gpu
def test_gpu_adam_matches_oracle(gpu):
    L, torch = gpu
    g0 = inputs.rng(9)
    p, gr = g0.normal(size=500), g0.normal(size=500)
    m, v = np.zeros(500), np.zeros(500)
    dp, dg, dm, dv = (_dev(torch, a, torch.float64) for a in (p, gr, m, v))
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k in range(1, 4):
        assert L.lbm_mlp_adam(1, _ptr(dp), _ptr(dg), _ptr(dm), _ptr(dv), 500, 1e-2, 0.9, 0.999, 1e-8, k, st) == 0
        p, m, v = M.adam(p, gr, m, v, 1e-2, 0.9, 0.999, 1e-8, k)
    torch.cuda.synchronize()
    assert np.allclose(dp.cpu().numpy(), p, rtol=1e-13, atol=1e-15)


def test_mlp_entry_points_reject_bad_sizes():
    from paper_2607_06794_b300 import _lib, build
    build.build()
    L = _lib.load()
    assert L.lbm_mlp_param_count(4, 64, 3) == M.count(4, 64, 3)
    assert L.lbm_mlp_param_count(0, 64, 3) == 0
    assert L.lbm_mlp_param_count(4, 1000, 3) == 0
    assert L.lbm_mlp_forward(0, None, 4, 64, 3, None, 10, None, None) == _lib.EINVAL
