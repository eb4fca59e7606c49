"""B300-native lattice Boltzmann library for evaporating, nanowire-laden droplets.

Python face of the C ABI in ``include/lbm.h``: it marshals arguments, lets
PyTorch own the device workspace and supplies the CUDA stream.  Every step of
the method runs in the library's sm_103a kernels; there is no CPU path.

    from paper_2607_06794_b300 import Config, Simulation
    sim = Simulation([Config(nx=64, ny=32, nz=32, a=24, b=8, c=10, cx=32, cy=16)])
    sim.step(100)
    C = sim.read(0, "colour")
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math

import numpy as np

from . import _lib

PRECISIONS = {"fp64": _lib.FP64, "fp32": _lib.FP32, "fp16": _lib.FP16_SHIFTED,
              "bf16": _lib.BF16_SHIFTED}
FIELDS = {"populations": _lib.FIELD_POPULATIONS, "moments": _lib.FIELD_MOMENTS,
          "colour": _lib.FIELD_COLOUR, "bead_x": _lib.FIELD_BEAD_X, "bead_v": _lib.FIELD_BEAD_V,
          "bead_f": _lib.FIELD_BEAD_F, "bead_topo": _lib.FIELD_BEAD_TOPO,
          "accum": _lib.FIELD_ACCUM, "fext": _lib.FIELD_FEXT, "cot": _lib.FIELD_THETA_COT,
          "bead_potential": _lib.FIELD_BEAD_POTENTIAL, "bead_current": _lib.FIELD_BEAD_CURRENT}


class LBMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.load().lbm_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")


def _check(code, where):
    if code != _lib.OK:
        raise LBMError(code, where)


@dataclasses.dataclass
class Config:
    """One lattice instance (lattice units).  Defaults: paper constants (Sec. II.A)."""
    nx: int
    ny: int
    nz: int
    prec: str = "fp32"
    tau_R: float = 1.0
    tau_B: float = 1.0
    beta: float = 0.7
    sigma: float = 0.01
    rho0: float = 1.0
    J0: float = 0.0
    K: float = 0.01
    evap_start: int = -1
    top_bc: int = 1
    body: tuple = (0.0, 0.0, 0.0)
    shape: int = 0
    cx: float = 0.0
    cy: float = 0.0
    cz: float = -0.5
    a: float = 8.0
    b: float = 8.0
    c: float = 8.0
    width: float = 2.0
    theta_deg: float = 90.0
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
    bead_mass: float = 1.0
    substeps: int = 5
    max_beads: int = 0
    rcon: float = 2.1
    x_src: float = -math.inf
    x_snk: float = math.inf
    seed: int = 1234
    inplace: int = 0  # 1: esoteric-pull in-place population storage

    def to_c(self) -> _lib.lbm_config:
        c = _lib.lbm_config()
        for name, _ in _lib.lbm_config._fields_:
            v = getattr(self, name)
            if name == "prec":
                v = PRECISIONS[v] if isinstance(v, str) else int(v)
            if name == "body":
                v = (C.c_double * 3)(*v)
            setattr(c, name, v)
        return c


def workspace_bytes(cfgs) -> int:
    arr = (_lib.lbm_config * len(cfgs))(*[c.to_c() for c in cfgs])
    return int(_lib.load().lbm_workspace_bytes(arr, len(cfgs)))


def tiling_count() -> int:
    """Number of candidate tilings of the fused kernel."""
    return int(_lib.load().lbm_tiling_count())


def tiling_table(cfgs, index):
    """Blocks of tiling `index` for a batch (host only): (n_blocks, 7) int array of
    instance, x0, y0, z0, z1, width, height."""
    L = _lib.load()
    arr = (_lib.lbm_config * len(cfgs))(*[c.to_c() for c in cfgs])
    nbl = C.c_int()
    st = L.lbm_tiling_table(arr, len(cfgs), int(index), None, 0, C.byref(nbl))
    if st not in (_lib.OK, _lib.ENOMEM_WS):
        _check(st, "lbm_tiling_table")
    out = np.zeros((max(nbl.value, 1), 7), np.int32)
    _check(L.lbm_tiling_table(arr, len(cfgs), int(index), out.ctypes.data_as(C.POINTER(C.c_int)),
                              int(nbl.value), C.byref(nbl)), "lbm_tiling_table")
    return out[:nbl.value]


class Simulation:
    """A batch of lattice instances advancing together on one CUDA stream."""

    def __init__(self, cfgs, device="cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Simulation needs a CUDA device (B300); there is no CPU path")
        self.L = _lib.load()
        self.cfgs = list(cfgs)
        self.device = torch.device(device)
        arr = (_lib.lbm_config * len(self.cfgs))(*[c.to_c() for c in self.cfgs])
        nbytes = int(self.L.lbm_workspace_bytes(arr, len(self.cfgs)))
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(self.L.lbm_create(arr, len(self.cfgs), C.c_void_p(self.ws.data_ptr()), nbytes,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h)), "lbm_create")
        self.h = h
        self.nb = [0] * len(self.cfgs)

    # ---------------------------------------------------------------- set-up
    def set_substrate_pattern(self, inst, theta_deg):
        c = self.cfgs[inst]
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(theta_deg, np.float64), (c.ny, c.nx)))
        _check(self.L.lbm_set_substrate_pattern(self.h, inst, t.ctypes.data_as(C.POINTER(C.c_double))),
               "lbm_set_substrate_pattern")

    def add_nanowires(self, inst, n_wires, length, centers=None, dirs=None, seed=0):
        dp = C.POINTER(C.c_double)
        if centers is not None:
            cen = np.ascontiguousarray(centers, np.float64).reshape(-1, 3)
            dr = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
            assert cen.shape[0] == n_wires and dr.shape[0] == n_wires
            pc, pd = cen.ctypes.data_as(dp), dr.ctypes.data_as(dp)
        else:
            pc = pd = None
        _check(self.L.lbm_add_nanowires(self.h, inst, n_wires, float(length), pc, pd, seed),
               "lbm_add_nanowires")
        self.nb[inst] = int(self.read(inst, "accum")[5])

    # ---------------------------------------------------------------- stepping
    def step(self, n=1):
        _check(self.L.lbm_step(self.h, int(n)), "lbm_step")

    def profile_steps(self, n):
        """(ms per fused fluid-kernel launch, ms per step) over n directly launched steps."""
        a, b = C.c_double(), C.c_double()
        _check(self.L.lbm_profile_steps(self.h, int(n), C.byref(a), C.byref(b)), "lbm_profile_steps")
        return a.value, b.value

    def autotune(self, steps_per_candidate=5):
        """Pick the fastest fused-kernel tiling on real steps; returns (index, ms)."""
        k, ms = C.c_int(), C.c_double()
        _check(self.L.lbm_autotune(self.h, int(steps_per_candidate), C.byref(k), C.byref(ms)),
               "lbm_autotune")
        return k.value, ms.value

    def tiling_count(self) -> int:
        """Number of candidate tilings of the fused kernel."""
        return int(self.L.lbm_tiling_count())

    def set_tiling(self, index):
        """Use candidate tiling `index` from the next step on (same results, other blocking)."""
        _check(self.L.lbm_set_tiling(self.h, int(index)), "lbm_set_tiling")

    def sync(self):
        _check(self.L.lbm_sync(self.h), "lbm_sync")

    def status(self) -> int:
        """Latched device status without raising."""
        return int(self.L.lbm_sync(self.h))

    def clear_error(self):
        _check(self.L.lbm_clear_error(self.h), "lbm_clear_error")

    # ---------------------------------------------------------------- fields
    def _shape(self, inst, field):
        c = self.cfgs[inst]
        nb = self.nb[inst]
        return {
            "populations": ((2, 19, c.nz, c.ny, c.nx), np.float64),
            "moments": ((c.nz, c.ny, c.nx, 5), np.float64),
            "colour": ((c.nz, c.ny, c.nx), np.float64),
            "bead_x": ((nb, 3), np.float64), "bead_v": ((nb, 3), np.float64),
            "bead_f": ((nb, 3), np.float64), "bead_topo": ((nb, 2), np.int32),
            "accum": ((6,), np.float64), "fext": ((c.nz, c.ny, c.nx, 3), np.float64),
            "cot": ((c.ny, c.nx), np.float64),
            "bead_potential": ((nb,), np.float64), "bead_current": ((nb,), np.float64),
        }[field]

    def read(self, inst, field, out=None):
        shape, dt = self._shape(inst, field)
        if out is None:
            out = np.empty(shape, dt)
        assert out.shape == shape and out.dtype == dt and out.flags.c_contiguous
        _check(self.L.lbm_read_fields(self.h, inst, FIELDS[field], C.c_void_p(out.ctypes.data),
                                      out.nbytes), f"lbm_read_fields({field})")
        return out

    def read_into(self, inst, field, host_tensor):
        """Read into a (pinned) host torch tensor of the right size."""
        _check(self.L.lbm_read_fields(self.h, inst, FIELDS[field], C.c_void_p(host_tensor.data_ptr()),
                                      host_tensor.numel() * host_tensor.element_size()),
               f"lbm_read_fields({field})")
        return host_tensor

    def read_accum_async(self, inst, host_tensor):
        """Enqueue a copy of the budget record (the 'accum' field layout) into a pinned
        float64 host tensor of 6; its values hold after the next sync."""
        import torch
        assert host_tensor.dtype == torch.float64 and host_tensor.numel() == 6 and host_tensor.is_pinned()
        _check(self.L.lbm_read_accum_async(self.h, inst, C.cast(C.c_void_p(host_tensor.data_ptr()),
                                                                 C.POINTER(C.c_double))),
               "lbm_read_accum_async")
        return host_tensor

    def write(self, inst, field, arr):
        shape, dt = self._shape(inst, field)
        a = np.ascontiguousarray(arr, dt).reshape(shape)
        _check(self.L.lbm_write_fields(self.h, inst, FIELDS[field], C.c_void_p(a.ctypes.data), a.nbytes),
               f"lbm_write_fields({field})")

    def write_from(self, inst, field, host_tensor):
        _check(self.L.lbm_write_fields(self.h, inst, FIELDS[field], C.c_void_p(host_tensor.data_ptr()),
                                       host_tensor.numel() * host_tensor.element_size()),
               f"lbm_write_fields({field})")

    def descriptors(self, inst) -> dict:
        d = _lib.lbm_descriptors()
        _check(self.L.lbm_deposit_descriptors(self.h, inst, C.byref(d)), "lbm_deposit_descriptors")
        return {k: getattr(d, k) for k, _ in _lib.lbm_descriptors._fields_}

    def conductivity(self, inst, tol=1e-12, max_iter=200000) -> dict:
        """Kirchhoff network of the deposit (kappa*, currents); potentials and node
        currents are then readable as the 'bead_potential' / 'bead_current' fields."""
        d = _lib.lbm_conductivity()
        _check(self.L.lbm_deposit_conductivity(self.h, inst, tol, max_iter, C.byref(d)),
               "lbm_deposit_conductivity")
        return {k: getattr(d, k) for k, _ in _lib.lbm_conductivity._fields_}

    def profiles(self, inst, axis, lo, hi, nbins, centre, half_width):
        """Per-bin S_x^b and g^b (axis 0: bins along x, strip in y; axis 1: the reverse);
        returns (S_x, g, bond counts, bead counts)."""
        S = np.zeros(nbins)
        g = np.zeros(nbins)
        nb = np.zeros(nbins, np.int32)
        nd = np.zeros(nbins, np.int32)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        _check(self.L.lbm_deposit_profiles(self.h, inst, axis, lo, hi, nbins, centre, half_width,
                                           S.ctypes.data_as(dp), g.ctypes.data_as(dp),
                                           nb.ctypes.data_as(ip), nd.ctypes.data_as(ip)),
               "lbm_deposit_profiles")
        return S, g, nb, nd

    def shape(self, inst) -> dict:
        """Droplet height, volume, centre, footprint radii, contact angles and mean flow."""
        d = _lib.lbm_shape()
        _check(self.L.lbm_droplet_shape(self.h, inst, C.byref(d)), "lbm_droplet_shape")
        return {k: getattr(d, k) for k, _ in _lib.lbm_shape._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
