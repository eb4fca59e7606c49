"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

# status codes
OK, EINVAL, ENOMEM_WS, ECUDA, ENAN, EFENE, EBEAD_OOB, ETIMEOUT, ESTATE, ECAPACITY = range(10)
# precisions
FP64, FP32, FP16_SHIFTED, BF16_SHIFTED = range(4)
# field ids
(FIELD_POPULATIONS, FIELD_MOMENTS, FIELD_COLOUR, FIELD_BEAD_X, FIELD_BEAD_V, FIELD_BEAD_F,
 FIELD_BEAD_TOPO, FIELD_ACCUM, FIELD_FEXT, FIELD_THETA_COT, FIELD_BEAD_POTENTIAL,
 FIELD_BEAD_CURRENT) = range(1, 13)

# every entry point that include/lbm.h declares
EXPORTS = ("lbm_workspace_bytes", "lbm_create", "lbm_set_substrate_pattern", "lbm_add_nanowires",
           "lbm_step", "lbm_profile_steps", "lbm_autotune", "lbm_tiling_count", "lbm_set_tiling", "lbm_tiling_table", "lbm_sync", "lbm_clear_error", "lbm_read_fields", "lbm_read_accum_async", "lbm_write_fields",
           "lbm_deposit_descriptors", "lbm_destroy", "lbm_status_string", "lbm_mlp_param_count",
           "lbm_mlp_scratch_bytes", "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_adam",
           "lbm_deposit_descriptors_noalloc", "lbm_deposit_conductivity", "lbm_deposit_profiles",
           "lbm_droplet_shape")


class lbm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("prec", C.c_int),
        ("tau_R", C.c_double), ("tau_B", C.c_double), ("beta", C.c_double), ("sigma", C.c_double),
        ("rho0", C.c_double), ("J0", C.c_double), ("K", C.c_double), ("evap_start", C.c_longlong),
        ("top_bc", C.c_int), ("body", C.c_double * 3),
        ("shape", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
        ("a", C.c_double), ("b", C.c_double), ("c", C.c_double), ("width", C.c_double),
        ("theta_deg", C.c_double),
        ("ks", C.c_double), ("Rm", C.c_double), ("d0", C.c_double), ("eps_wca", C.c_double),
        ("kb", C.c_double), ("eps_coh", C.c_double), ("eps_s", C.c_double), ("rc", C.c_double),
        ("gamma", C.c_double), ("xi", C.c_double), ("mu", C.c_double), ("gamma_t", C.c_double),
        ("bead_mass", C.c_double), ("substeps", C.c_int), ("max_beads", C.c_int),
        ("rcon", C.c_double), ("x_src", C.c_double), ("x_snk", C.c_double), ("seed", C.c_uint64),
        ("inplace", C.c_int),
    ]


class lbm_descriptors(C.Structure):
    _fields_ = [
        ("S_x", C.c_double), ("n_clusters", C.c_int), ("percolates", C.c_int),
        ("n_beads", C.c_int), ("n_bonds", C.c_int), ("mass_R", C.c_double), ("mass_B", C.c_double),
        ("evaporated", C.c_double), ("top_in", C.c_double), ("top_out", C.c_double),
        ("h0", C.c_double), ("step", C.c_longlong),
    ]


class lbm_conductivity(C.Structure):
    _fields_ = [
        ("kappa", C.c_double), ("I_tot", C.c_double), ("I_sink", C.c_double), ("I_ref", C.c_double),
        ("residual", C.c_double), ("iterations", C.c_int), ("n_src", C.c_int), ("n_snk", C.c_int),
        ("n_edges", C.c_int),
    ]


class lbm_shape(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("volume", "height", "xc", "yc", "r_x", "r_y", "theta_x",
                                          "theta_y", "v_x", "v_y")]


_lib = None


def load():
    """Load liblbm.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblbm.so not built at {LIB_PATH}; run paper_2607_06794_b300/build.py")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    L.lbm_workspace_bytes.restype = C.c_size_t
    L.lbm_workspace_bytes.argtypes = [C.POINTER(lbm_config), C.c_int]
    L.lbm_create.restype = C.c_int
    L.lbm_create.argtypes = [C.POINTER(lbm_config), C.c_int, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.lbm_set_substrate_pattern.restype = C.c_int
    L.lbm_set_substrate_pattern.argtypes = [vp, C.c_int, dp]
    L.lbm_add_nanowires.restype = C.c_int
    L.lbm_add_nanowires.argtypes = [vp, C.c_int, C.c_int, C.c_double, dp, dp, C.c_uint64]
    L.lbm_step.restype = C.c_int
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_profile_steps.restype = C.c_int
    L.lbm_profile_steps.argtypes = [vp, C.c_int, dp, dp]
    L.lbm_autotune.restype = C.c_int
    L.lbm_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), dp]
    L.lbm_tiling_count.restype = C.c_int
    L.lbm_tiling_count.argtypes = []
    L.lbm_set_tiling.restype = C.c_int
    L.lbm_set_tiling.argtypes = [vp, C.c_int]
    L.lbm_tiling_table.restype = C.c_int
    L.lbm_tiling_table.argtypes = [C.POINTER(lbm_config), C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                                   C.POINTER(C.c_int)]
    L.lbm_sync.restype = C.c_int
    L.lbm_sync.argtypes = [vp]
    L.lbm_clear_error.restype = C.c_int
    L.lbm_clear_error.argtypes = [vp]
    L.lbm_read_accum_async.restype = C.c_int
    L.lbm_read_accum_async.argtypes = [vp, C.c_int, dp]
    L.lbm_read_fields.restype = C.c_int
    L.lbm_read_fields.argtypes = [vp, C.c_int, C.c_uint, vp, C.c_size_t]
    L.lbm_write_fields.restype = C.c_int
    L.lbm_write_fields.argtypes = [vp, C.c_int, C.c_uint, vp, C.c_size_t]
    L.lbm_deposit_descriptors.restype = C.c_int
    L.lbm_deposit_descriptors.argtypes = [vp, C.c_int, C.POINTER(lbm_descriptors)]
    L.lbm_destroy.restype = C.c_int
    L.lbm_destroy.argtypes = [vp]
    L.lbm_mlp_param_count.restype = C.c_size_t
    L.lbm_mlp_param_count.argtypes = [C.c_int, C.c_int, C.c_int]
    L.lbm_mlp_scratch_bytes.restype = C.c_size_t
    L.lbm_mlp_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
    L.lbm_mlp_forward.restype = C.c_int
    L.lbm_mlp_forward.argtypes = [C.c_int, vp, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, vp]
    L.lbm_mlp_loss_grad.restype = C.c_int
    L.lbm_mlp_loss_grad.argtypes = [C.c_int, vp, C.c_int, C.c_int, C.c_int, vp, vp, C.c_int, vp, vp, vp,
                                    vp, C.c_size_t, vp]
    L.lbm_mlp_adam.restype = C.c_int
    L.lbm_mlp_adam.argtypes = [C.c_int, vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_int, vp]
    L.lbm_deposit_descriptors_noalloc.restype = C.c_int
    L.lbm_deposit_descriptors_noalloc.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_double,
                                                  C.c_double, C.c_double, vp, vp]
    L.lbm_deposit_conductivity.restype = C.c_int
    L.lbm_deposit_conductivity.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.POINTER(lbm_conductivity)]
    L.lbm_deposit_profiles.restype = C.c_int
    L.lbm_deposit_profiles.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                       C.c_double, dp, dp, ip, ip]
    L.lbm_droplet_shape.restype = C.c_int
    L.lbm_droplet_shape.argtypes = [vp, C.c_int, C.POINTER(lbm_shape)]
    L.lbm_status_string.restype = C.c_char_p
    L.lbm_status_string.argtypes = [C.c_int]
    _lib = L
    return L
