"""The C-ABI library loads and exports everything include/lbm.h declares (CPU only)."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_06794_b300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))


def test_header_and_binding_agree():
    from paper_2607_06794_b300 import _lib
    assert declared_functions() == set(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(10):
        assert lib.lbm_status_string(code)
    assert lib.lbm_status_string(0) == b"ok"


def test_config_struct_matches_header_order():
    from paper_2607_06794_b300 import _lib
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = src[src.index("typedef struct lbm_config"):src.index("} lbm_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";")[:-1]:
        decl = decl.split("{")[-1].strip()
        if not decl:
            continue
        parts = decl.split()
        for n in " ".join(parts[1:] if parts[0] != "long" else parts[2:]).split(","):
            names.append(n.strip().split("[")[0])
    assert names == [f[0] for f in _lib.lbm_config._fields_]


def test_workspace_size_needs_no_gpu(lib):
    from paper_2607_06794_b300 import Config, workspace_bytes
    small = workspace_bytes([Config(32, 16, 16)])
    big = workspace_bytes([Config(64, 32, 32)])
    assert 0 < small < big
    # two populations buffers of 2x19 floats per node at least
    assert big >= 2 * 2 * 19 * 4 * 64 * 32 * 32
    with_beads = workspace_bytes([Config(32, 16, 16, max_beads=100)])
    assert with_beads > small
    batch = workspace_bytes([Config(32, 16, 16), Config(64, 32, 32)])
    assert big < batch < small + big  # the staging area is shared by the batch


@pytest.mark.parametrize("bad", [dict(nz=1), dict(tau_R=0.5), dict(prec=7), dict(theta_deg=0.0),
                                 dict(top_bc=3), dict(a=0.0), dict(K=0.0), dict(beta=2.0),
                                 dict(max_beads=10, Rm=1.0), dict(inplace=2)])
def test_invalid_configs_are_rejected_before_any_device_call(lib, bad):
    from paper_2607_06794_b300 import Config, _lib
    import dataclasses
    cfg = dataclasses.replace(Config(16, 16, 16), **bad)
    arr = (_lib.lbm_config * 1)(cfg.to_c())
    h = C.c_void_p()
    fake_ws = C.c_void_p(1 << 20)  # never touched: validation fails first
    st = lib.lbm_create(arr, 1, fake_ws, 1 << 40, None, C.byref(h))
    assert st == _lib.EINVAL
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2607_06794_b300 import _lib
    assert lib.lbm_step(None, 1) == _lib.EINVAL
    assert lib.lbm_sync(None) == _lib.EINVAL
    assert lib.lbm_destroy(None) == _lib.EINVAL
    assert lib.lbm_workspace_bytes(None, 1) == 0
    assert not math.isnan(0.0)


def test_inplace_storage_takes_one_population_buffer(lib):
    """Esoteric-pull storage needs one population buffer plus the wall ghost slots instead of
    two buffers (workspace size, computed without a GPU)."""
    from paper_2607_06794_b300 import Config, workspace_bytes
    for prec, eb in (("fp64", 8), ("fp32", 4), ("fp16", 2)):
        c = Config(64, 48, 40, prec=prec)
        two = workspace_bytes([c])
        c.inplace = 1
        one = workspace_bytes([c])
        assert abs((two - one) - (2 * 19 * 64 * 48 * 40 * eb - 2 * 10 * 64 * 48 * eb)) <= 1024


def test_largest_lattice_is_accepted_and_one_plane_more_is_rejected(lib):
    """Element offsets inside one population buffer are 32-bit: 2 x 19 x N must stay below
    2^32 (N < 113,025,456 nodes); the check runs on the host, before any device call."""
    from paper_2607_06794_b300 import Config, tiling_table
    assert 38 * 1024 * 1024 * 107 < 2 ** 32 <= 38 * 1024 * 1024 * 108
    tab = tiling_table([Config(1024, 1024, 107)], 0)
    assert len(tab) > 0 and tab[:, 4].max() == 107
    with pytest.raises(RuntimeError):
        tiling_table([Config(1024, 1024, 108)], 0)
