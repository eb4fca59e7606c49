"""FP64 CPU oracle of the fluid-filament time step (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It loads ``liboracle.so`` built from ``lbm_oracle.c``
(plain C, gcc, OpenMP) and shares nothing with the CUDA library.

Arrays follow the oracle's own layout: populations ``[19, nz, ny, nx]``,
node fields ``[nz, ny, nx]`` (vectors ``[nz, ny, nx, 3]``), substrate maps
``[ny, nx]``, bead vectors ``[n, 3]``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("tau_R", C.c_double), ("tau_B", C.c_double), ("beta", C.c_double),
        ("sigma", C.c_double), ("rho0", C.c_double), ("J0", C.c_double), ("K", C.c_double),
        ("evap_start", C.c_longlong), ("top_bc", C.c_int),
        ("ks", C.c_double), ("Rm", C.c_double), ("d0", C.c_double), ("eps_wca", C.c_double),
        ("kb", C.c_double), ("eps_coh", C.c_double), ("eps_s", C.c_double), ("rc", C.c_double),
        ("gamma", C.c_double), ("xi", C.c_double), ("mu", C.c_double), ("gamma_t", C.c_double),
        ("mass", C.c_double), ("substeps", C.c_int), ("body", C.c_double * 3),
    ]


class _Acc(C.Structure):
    _fields_ = [("step", C.c_longlong), ("h0", C.c_double), ("evaporated", C.c_double),
                ("top_in", C.c_double), ("top_out", C.c_double), ("err", C.c_int)]


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters (lattice units).

    Filament constants default to the values printed in Sec. II.A:
    k_s=0.3, R_m=2.4 (Eq. (9)); d0=2, eps=0.03 (Eq. (10)); k_b=8 (Eq. (11));
    eps_s=0.006 (substrate adhesion); K=0.01 (Eq. (8)); 5 sub-steps.
    ``eps_coh`` is the physical well depth eps = eps* x eps_s.
    """
    nx: int
    ny: int
    nz: int
    tau_R: float = 1.0
    tau_B: float = 1.0
    beta: float = 0.7
    sigma: float = 0.01
    rho0: float = 1.0
    J0: float = 0.0
    K: float = 0.01
    evap_start: int = -1
    top_bc: int = 1
    ks: float = 0.3
    Rm: float = 2.4
    d0: float = 2.0
    eps_wca: float = 0.03
    kb: float = 8.0
    eps_coh: float = 0.0
    eps_s: float = 0.006
    rc: float = 4.0
    gamma: float = 1.0
    xi: float = 0.0
    mu: float = 0.5
    gamma_t: float = 1.0
    mass: float = 1.0
    substeps: int = 5
    body: tuple = (0.0, 0.0, 0.0)

    def c(self) -> _Params:
        vals = []
        for f in _Params._fields_:
            v = getattr(self, f[0])
            vals.append((C.c_double * 3)(*v) if f[0] == "body" else v)
        return _Params(*vals)


@dataclasses.dataclass
class Acc:
    step: int = 0
    h0: float = 0.0
    evaporated: float = 0.0
    top_in: float = 0.0
    top_out: float = 0.0
    err: int = 0


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        _lib.orc_step.restype = C.c_int
        _lib.orc_step.argtypes = [C.POINTER(_Params), dp, dp, dp, C.c_int, ip, ip, dp, dp, dp,
                                  C.POINTER(_Acc), dp]
        _lib.orc_init_droplet.restype = None
        _lib.orc_init_droplet.argtypes = [C.POINTER(_Params), C.c_int] + [C.c_double] * 7 + [dp, dp]
        _lib.orc_fields.restype = None
        _lib.orc_fields.argtypes = [C.POINTER(_Params), dp, dp, dp] + [dp] * 8
        _lib.orc_bead_energy.restype = C.c_double
        _lib.orc_bead_energy.argtypes = [C.POINTER(_Params), C.c_int, ip, ip, dp]
        _lib.orc_bead_conservative_forces.restype = C.c_int
        _lib.orc_bead_conservative_forces.argtypes = [C.POINTER(_Params), C.c_int, ip, ip, dp, dp]
        _lib.orc_descriptors.restype = None
        _lib.orc_descriptors.argtypes = [C.POINTER(_Params), C.c_int, ip, ip, dp, C.c_double,
                                         C.c_double, C.c_double, dp, ip, ip, ip]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def init_droplet(p: Params, shape: int, cx, cy, cz, a, b, c, width):
    """Equilibrium-at-rest populations of a droplet (shape 0 ellipsoid, 1 cylinder)."""
    n = p.nx * p.ny * p.nz
    fR = np.empty((19, p.nz, p.ny, p.nx))
    fB = np.empty_like(fR)
    pc = p.c()
    lib().orc_init_droplet(C.byref(pc), shape, cx, cy, cz, a, b, c, width, _dp(fR), _dp(fB))
    assert fR.size == 19 * n
    return fR, fB


def cot_map(theta_deg) -> np.ndarray:
    """cot(theta) per substrate cell from contact angles in degrees."""
    t = np.radians(np.asarray(theta_deg, dtype=np.float64))
    return np.cos(t) / np.sin(t)


class Beads:
    """Bead-spring filaments: bead arrays in filament order."""

    def __init__(self, fil, pos, X, V=None, F=None):
        self.fil = _i32(fil)
        self.pos = _i32(pos)
        self.X = _f64(X).reshape(-1, 3).copy()
        n = self.X.shape[0]
        self.V = np.zeros((n, 3)) if V is None else _f64(V).reshape(-1, 3).copy()
        self.F = np.zeros((n, 3)) if F is None else _f64(F).reshape(-1, 3).copy()

    @property
    def n(self):
        return self.X.shape[0]

    def copy(self):
        return Beads(self.fil, self.pos, self.X, self.V, self.F)


def step(p: Params, fR, fB, cot, acc: Acc, beads: Beads | None = None, return_fext=False):
    """Advance (fR, fB, beads, acc) by one time step in place; returns error bits."""
    assert fR.dtype == np.float64 and fR.flags.c_contiguous
    assert fB.dtype == np.float64 and fB.flags.c_contiguous
    cot = _f64(cot)
    a = _Acc(acc.step, acc.h0, acc.evaporated, acc.top_in, acc.top_out, acc.err)
    pc = p.c()
    fext = np.zeros((p.nz, p.ny, p.nx, 3)) if return_fext else None
    if beads is not None and beads.n > 0:
        err = lib().orc_step(C.byref(pc), _dp(fR), _dp(fB), _dp(cot), beads.n, _ip(beads.fil),
                             _ip(beads.pos), _dp(beads.X), _dp(beads.V), _dp(beads.F), C.byref(a),
                             _dp(fext))
    else:
        err = lib().orc_step(C.byref(pc), _dp(fR), _dp(fB), _dp(cot), 0, None, None, None, None,
                             None, C.byref(a), _dp(fext))
    acc.step, acc.h0, acc.evaporated = a.step, a.h0, a.evaporated
    acc.top_in, acc.top_out, acc.err = a.top_in, a.top_out, a.err
    return (err, fext) if return_fext else err


def fields(p: Params, fR, fB, cot):
    """Moments, colour gradient, curvature, CSF force and column height of a state."""
    N = (p.nz, p.ny, p.nx)
    out = dict(rhoR=np.empty(N), rhoB=np.empty(N), C=np.empty(N), j=np.empty(N + (3,)),
               G=np.empty(N + (3,)), kappa=np.empty(N), Fs=np.empty(N + (3,)),
               h=np.empty((p.ny, p.nx)))
    pc = p.c()
    lib().orc_fields(C.byref(pc), _dp(_f64(fR)), _dp(_f64(fB)), _dp(_f64(cot)), _dp(out["rhoR"]),
                     _dp(out["rhoB"]), _dp(out["C"]), _dp(out["j"]), _dp(out["G"]),
                     _dp(out["kappa"]), _dp(out["Fs"]), _dp(out["h"]))
    return out


def bead_energy(p: Params, fil, pos, X) -> float:
    X = _f64(X).reshape(-1, 3).copy()
    pc = p.c()
    return lib().orc_bead_energy(C.byref(pc), X.shape[0], _ip(_i32(fil)), _ip(_i32(pos)), _dp(X))


def bead_conservative_forces(p: Params, fil, pos, X):
    X = _f64(X).reshape(-1, 3).copy()
    F = np.zeros_like(X)
    pc = p.c()
    err = lib().orc_bead_conservative_forces(C.byref(pc), X.shape[0], _ip(_i32(fil)),
                                             _ip(_i32(pos)), _dp(X), _dp(F))
    return F, err


def descriptors(p: Params, fil, pos, X, rcon=2.1, xsrc=None, xsnk=None):
    """(S_x, cluster count, percolates, labels) of a bead configuration."""
    X = _f64(X).reshape(-1, 3)
    n = X.shape[0]
    sx = C.c_double()
    nc = C.c_int()
    pc_ = C.c_int()
    lab = np.empty(n, dtype=np.int32)
    pc = p.c()
    lib().orc_descriptors(C.byref(pc), n, _ip(_i32(fil)), _ip(_i32(pos)), _dp(X), rcon,
                          -1e300 if xsrc is None else xsrc, 1e300 if xsnk is None else xsnk,
                          C.byref(sx), C.byref(nc), C.byref(pc_), _ip(lab))
    return sx.value, nc.value, bool(pc_.value), lab


def mass(fR, fB):
    """Total mass of each component (exact sums in FP64)."""
    return float(np.sum(fR)), float(np.sum(fB))
