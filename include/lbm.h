/*
 * lbm.h — C ABI of the B300 library for the fluid–filament method of
 * "Evaporation-Driven Nanowire Self-Assembly in an Elongated Droplet"
 * (Schoettner, Xie, Harting), Sec. II.
 *
 * One handle holds one or more lattice instances (a batch) that advance
 * together on one CUDA stream.  Each time step of each instance is
 *   stream (Eq. (1), left side)  ->  moments (Eq. (3))
 *   -> wetting ghost layer + colour gradient + curvature + CSF force (Sec. II.A)
 *   -> filament sub-steps with two-way drag coupling (Eqs. (9)-(12))
 *   -> colour-blind forced BGK (Eqs. (1)-(2)) -> recolouring
 *   -> evaporation sink (Eq. (8))
 * computed by hand-written sm_103a kernels.  There is no CPU fallback.
 *
 * Conventions
 *  - The caller owns all device memory: it allocates one workspace of
 *    lbm_workspace_bytes() bytes (16-byte aligned) and passes it to
 *    lbm_create().  The library never allocates device memory.
 *  - Host arrays passed to a call are borrowed for that call only.
 *  - Every call returns a status.  Kernel-side failures (NaN density, FENE
 *    overstretch, bead out of range, capacity overflow) are latched in a
 *    device flag word; lbm_sync() and every call that reads data back
 *    report them.  Once latched, a failure stays until lbm_clear_error().
 *  - lbm_step() only enqueues work on the handle's stream and returns.
 *  - Lattice arrays are x-fastest: index = (z*ny + y)*nx + x.
 *  - Units are lattice units; rho0 = 1 is the reference density.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* invalid argument or configuration */
    LBM_ENOMEM_WS = 2,   /* workspace smaller than lbm_workspace_bytes() */
    LBM_ECUDA = 3,       /* a CUDA runtime call failed */
    LBM_ENAN = 4,        /* non-finite or non-positive density met in a step */
    LBM_EFENE = 5,       /* a FENE bond reached R_m (Eq. (9) undefined there) */
    LBM_EBEAD_OOB = 6,   /* a bead left the fluid or moved > 0.5 in one step */
    LBM_ETIMEOUT = 7,    /* a bounded device-side wait gave up */
    LBM_ESTATE = 8,      /* call not valid in the handle's current state */
    LBM_ECAPACITY = 9    /* bead, neighbour or contact capacity exceeded */
} lbm_status;

/* Storage precision of the populations.  FP64 and FP32 store f^R and f^B.
 * The two shifted forms store, per direction, the total population as its
 * deviation from rest, F_i - w_i rho0, and the liquid fraction f^R_i/F_i - 1/2,
 * both as 16-bit numbers; collision, forcing and moments run in FP32, mass
 * and evaporation sums and the bead integration stay FP64. */
typedef enum {
    LBM_FP64 = 0,
    LBM_FP32 = 1,
    LBM_FP16_SHIFTED = 2,
    LBM_BF16_SHIFTED = 3
} lbm_precision;

typedef struct lbm_config {
    int nx, ny, nz;        /* lattice size; x, y periodic; wall below z = 0 */
    int prec;              /* lbm_precision (must be equal across a batch) */
    double tau_R, tau_B;   /* relaxation times of liquid (R) and gas (B), Eq. (1) */
    double beta;           /* recolouring strength (Sec. II.A, colour-gradient method) */
    double sigma;          /* surface tension of the CSF force F = sigma/2 kappa grad C */
    double rho0;           /* reference density, Eq. (3) */
    double J0;             /* evaporation rate scale, Eq. (8); 0 disables evaporation */
    double K;              /* kinetic resistance, Eq. (8) (paper: 0.01) */
    long long evap_start;  /* first step with the sink on; < 0 never */
    int top_bc;            /* 0: bounce-back wall at the top; 1: pure-gas equilibrium inflow */
    double body[3];        /* uniform body-force density (0 for the paper's runs) */
    /* initial droplet (Sec. III): C = tanh(-(q-1) min(a,b,c)/width) */
    int shape;             /* 0 ellipsoid (cap if cz < 0), 1 elliptic cylinder along x */
    double cx, cy, cz;     /* centre */
    double a, b, c;        /* semi-axes (for shape 1, a is the half-length) */
    double width;          /* interface width of the tanh profile */
    double theta_deg;      /* uniform contact angle until lbm_set_substrate_pattern() */
    /* filaments, Eqs. (9)-(12) and the filament paragraph of Sec. II.A */
    double ks, Rm;         /* FENE (paper: 0.3, 2.4) */
    double d0, eps_wca;    /* bead diameter and WCA strength (paper: 2, 0.03) */
    double kb;             /* bending constant (paper: 8) */
    double eps_coh;        /* cohesive LJ well depth between filaments (eps* x eps_s) */
    double eps_s;          /* substrate adhesion (paper: 0.006) */
    double rc;             /* cut-off of the cohesive and substrate LJ (shifted) */
    double gamma;          /* drag coefficient of the dissipative coupling */
    double xi;             /* solvation strength: F = xi grad C */
    double mu, gamma_t;    /* substrate friction: |F_t| = min(gamma_t |v_t|, mu N) */
    double bead_mass;
    int substeps;          /* MD sub-steps per LB step (paper: 5) */
    int max_beads;         /* bead capacity of this instance */
    double rcon;           /* contact cut-off of the network model (paper: 2.1) */
    double x_src, x_snk;   /* electrodes: beads with x < x_src / x > x_snk */
    uint64_t seed;         /* seed of lbm_add_nanowires' random placement */
    int inplace;           /* population storage: 0 two buffers (read one, write the other);
                              1 esoteric pull, one buffer read and written in place plus wall
                              ghost slots (half the population memory, same bytes moved per
                              step); equal across a batch */
} lbm_config;

typedef struct lbm_descriptors {
    double S_x;            /* mean over bonds of 2 cos^2(zeta_x) - 1 (Eq. (13), one bin) */
    int n_clusters;        /* connected components of bonds + contacts r < rcon */
    int percolates;        /* 1 if one component touches both electrodes */
    int n_beads, n_bonds;
    double mass_R, mass_B; /* total populations of each component (FP64 sums) */
    double evaporated;     /* total mass converted liquid -> gas */
    double top_in, top_out;/* total mass that entered / left through the top plane */
    double h0;             /* maximum liquid column height at the first evaporating step */
    long long step;        /* steps taken */
} lbm_descriptors;

/* Field ids of lbm_read_fields / lbm_write_fields.  Every field moves as FP64
 * on the host side except LBM_FIELD_BEAD_TOPO (int32). */
enum {
    LBM_FIELD_POPULATIONS = 1, /* [2][19][nz][ny][nx]: post-collision f^R, then f^B (rw) */
    LBM_FIELD_MOMENTS = 2,     /* [nz][ny][nx][5]: rho_R, rho_B, j_x, j_y, j_z of the
                                  streamed populations of the next step (r) */
    LBM_FIELD_COLOUR = 3,      /* [nz][ny][nx]: C of the next step (r) */
    LBM_FIELD_BEAD_X = 4,      /* [n_beads][3] positions (rw) */
    LBM_FIELD_BEAD_V = 5,      /* [n_beads][3] velocities (rw) */
    LBM_FIELD_BEAD_F = 6,      /* [n_beads][3] force of the last sub-step (rw) */
    LBM_FIELD_BEAD_TOPO = 7,   /* int32 [n_beads][2]: filament id, index in filament (r) */
    LBM_FIELD_ACCUM = 8,       /* [6]: step, h0, evaporated, top_in, top_out, n_beads (rw) */
    LBM_FIELD_FEXT = 9,        /* [nz][ny][nx][3]: force the beads put on the fluid in
                                  the last step (r; zero where no bead is near) */
    LBM_FIELD_THETA_COT = 10,  /* [ny][nx]: cot(theta) of the substrate (r) */
    LBM_FIELD_BEAD_POTENTIAL = 11, /* [n_beads]: node potentials V of the last
                                      lbm_deposit_conductivity() call (r) */
    LBM_FIELD_BEAD_CURRENT = 12    /* [n_beads]: node currents I_i* = I_i / I_ref
                                      (Eqs. (15), (17)) of the same call (r) */
};

typedef struct lbm_handle lbm_handle;

/* Bytes of device workspace needed by lbm_create() for these instances. */
size_t lbm_workspace_bytes(const lbm_config* cfgs, int n_instances);

/* Build a handle over caller-owned device memory `dev_ws` (ws_bytes long,
 * 16-byte aligned) working on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  Validates every config, lays out the workspace,
 * initialises each droplet at rest in equilibrium and the derived moment
 * buffers.  On error *out is NULL and nothing is kept. */
lbm_status lbm_create(const lbm_config* cfgs, int n_instances, void* dev_ws, size_t ws_bytes,
                      void* stream, lbm_handle** out);

/* Contact-angle map of instance `inst`: theta_deg_xy[ny*nx] in degrees,
 * 0 < theta < 180, measured through the liquid (Sec. II.A wetting model,
 * Fig. 1 patch pattern).  Host array, copied. */
lbm_status lbm_set_substrate_pattern(lbm_handle* h, int inst, const double* theta_deg_xy);

/* Add n_wires straight filaments of length `length` (n_b = round(length/d0)
 * beads spaced d0, Sec. II.A).  centers/dirs are host arrays [n_wires][3];
 * pass NULL for both to place them at random (seeded, uniform centres,
 * isotropic directions, every bead where C > 0.9, beads of different
 * filaments further apart than d0; Sec. III.B set-up).  Velocities and
 * carried forces start at zero.  Fails with LBM_ECAPACITY past max_beads and
 * LBM_EINVAL if random placement finds no room after many tries. */
lbm_status lbm_add_nanowires(lbm_handle* h, int inst, int n_wires, double length,
                             const double* centers, const double* dirs, uint64_t seed);

/* Enqueue n_steps time steps of every instance on the handle's stream. */
lbm_status lbm_step(lbm_handle* h, int n_steps);

/* Measurement aid (the paper has no counterpart): advance n_steps like
 * lbm_step() but with direct launches, recording CUDA events on the handle's
 * stream around every fused fluid-kernel launch and around every whole step.
 * Synchronises; *ms_fluid and *ms_step receive the mean milliseconds per
 * fluid launch and per step. */
lbm_status lbm_profile_steps(lbm_handle* h, int n_steps, double* ms_fluid, double* ms_step);

/* Autotuner of the fused kernel's blocking (no paper counterpart): times
 * every candidate tiling (columns of nodes per block in x and y, times a
 * z-chunk per block) on steps_per_candidate real time steps of this batch and
 * keeps the fastest.  Every candidate computes the same step, so the steps
 * taken are ordinary steps of the run.  *chosen receives the candidate index
 * and *best_ms the mean milliseconds of one fused launch (either may be NULL). */
lbm_status lbm_autotune(lbm_handle* h, int steps_per_candidate, int* chosen, double* best_ms);

/* Number of candidate tilings (no paper counterpart); a constant of the build. */
int lbm_tiling_count(void);

/* Select candidate tiling `index` (0 <= index < lbm_tiling_count()) without
 * timing it (no paper counterpart).  Synchronises the stream and rebuilds the
 * moments the next step reads, so the run continues unchanged.  Returns
 * LBM_EINVAL for an index out of range. */
lbm_status lbm_set_tiling(lbm_handle* h, int index);

/* Host-only view of candidate tiling `index` for a batch (no paper
 * counterpart; no CUDA call is made): one column piece per block of the fused
 * kernel.  out (host, cap x 7 ints, may be NULL when cap is 0) receives per
 * block: instance, x0, y0, z0, z1 and the piece's width and height in nodes
 * (planes z0 <= z < z1 of the nodes x0 <= x < x0 + width, y0 <= y < y0 +
 * height).  *n_blocks receives the number of blocks.  Returns LBM_EINVAL for
 * a bad index or config, and LBM_ENOMEM_WS when cap is below *n_blocks (the
 * count is still set). */
lbm_status lbm_tiling_table(const lbm_config* cfgs, int n, int index, int* out, int cap, int* n_blocks);

/* Wait for the stream and return the first latched device-side failure. */
lbm_status lbm_sync(lbm_handle* h);

/* Reset the latched device-side failure word. */
lbm_status lbm_clear_error(lbm_handle* h);

/* Copy one field of instance `inst` to host memory (layouts above);
 * `bytes` must equal the field's size.  Synchronises the stream. */
lbm_status lbm_read_fields(lbm_handle* h, int inst, unsigned field, void* host_dst, size_t bytes);

/* Budget record of instance `inst` without waiting (no paper counterpart; the
 * FP64 budgets of Eq. (8) and of the top boundary, for monitoring a run step by
 * step): host_dst (6 doubles, the layout of LBM_FIELD_ACCUM: step, h0,
 * evaporated, top_in, top_out, n_beads) must be page-locked host memory that
 * the caller owns; entries 1-4 are copied on the handle's stream behind the
 * steps already enqueued and hold their values once the stream has reached the
 * copy (after lbm_sync or any synchronising call); entries 0 and 5 are written
 * before the call returns.  Returns LBM_EINVAL for a bad instance or NULL. */
lbm_status lbm_read_accum_async(lbm_handle* h, int inst, double* host_dst);

/* Overwrite one writable field from host memory (checkpoint restore).
 * Writing populations recomputes the derived moment buffers.  Synchronous. */
lbm_status lbm_write_fields(lbm_handle* h, int inst, unsigned field, const void* host_src,
                            size_t bytes);

/* Deposit descriptors of instance `inst` (Sec. II.B): nematic order, contact
 * clusters, percolation between the electrodes, plus mass budgets.
 * Synchronises the stream. */
lbm_status lbm_deposit_descriptors(lbm_handle* h, int inst, lbm_descriptors* out);

/* Electrical network of the deposit (Sec. II.B, Eqs. (15)-(18)).
 * Nodes are the beads; edges are the bonds and the pairs closer than rcon
 * (the contact graph of lbm_deposit_descriptors, minimum image in x and y),
 * each with conductance G_ij = 1 / r_ij.  With Delta V = 1, beads with
 * x < x_src are held at V = 1 and beads with x > x_snk at V = 0; Kirchhoff's
 * current law fixes the other potentials, solved on the GPU by Jacobi-
 * preconditioned conjugate gradients in FP64 until ||r|| <= tol ||b||.
 * Nodes of a component that touches no electrode keep V = 0 and carry no
 * current.  I_ref = 1 / (x_snk - x_src), the current of a straight filament
 * of conductance 1/r per unit length spanning the electrodes. */
typedef struct {
    double kappa;    /* kappa* = I_tot / I_ref (Eq. (18), one run) */
    double I_tot;    /* current leaving the source electrode */
    double I_sink;   /* current entering the sink electrode (= I_tot once converged) */
    double I_ref;    /* reference current (Eq. (16)) */
    double residual; /* ||r|| / ||b|| at exit (0 when no free node touches an electrode) */
    int iterations;  /* conjugate-gradient iterations taken */
    int n_src;       /* beads held at V = 1 */
    int n_snk;       /* beads held at V = 0 */
    int n_edges;     /* edges of the network */
} lbm_conductivity;

/* Solve the network of instance `inst` (tol > 0; max_iter >= 1 iterations at
 * most).  Node potentials and currents are then readable as
 * LBM_FIELD_BEAD_POTENTIAL / LBM_FIELD_BEAD_CURRENT.  Returns LBM_ETIMEOUT,
 * with the partial result written, when max_iter is reached first, and
 * LBM_ECAPACITY when the contact graph overflows its 8 edges per bead.
 * Synchronises the stream. */
lbm_status lbm_deposit_conductivity(lbm_handle* h, int inst, double tol, int max_iter,
                                    lbm_conductivity* out);

/* Axial or transverse profiles of the deposit (Sec. II.B, Eqs. (13)-(14)).
 * axis 0: nbins equal bins along x over [lo, hi), counting only what lies in
 * the strip |y - centre| <= half_width; axis 1: bins along y, strip in x.
 * S_x[b] = mean of 2 cos^2(zeta_x) - 1 over the bonds whose midpoint (nearest
 * image) falls in bin b, 0 for a bin without bonds (Eq. (13));
 * g[b] = N_b / mean_b N_b with N_b the bead centres in bin b (Eq. (14), equal
 * bins), 0 everywhere when no bead is counted.  Host outputs of nbins
 * entries (n_bonds, n_beads may be NULL); 1 <= nbins <= 65536, hi > lo,
 * half_width >= 0.  Synchronises the stream. */
lbm_status lbm_deposit_profiles(lbm_handle* h, int inst, int axis, double lo, double hi, int nbins,
                                double centre, double half_width, double* S_x, double* g,
                                int* n_bonds, int* n_beads);

/* Droplet-shape observables of instance `inst` at its current step, the
 * quantities tracked for the pure droplet on a patch (Sec. III.A, Fig. 2):
 * liquid column height h(x,y) = sum_z (1 + C)/2; volume = sum h; height = max h;
 * centre = h-weighted centroid; footprint radii r_x, r_y = half the positive
 * runs of C on the first fluid layer (z = 0) through the centre along x and y,
 * ends at the linearly interpolated C = 0 crossings; contact angles
 * theta = 2 atan(height / r) in degrees (spherical-cap relation in each
 * principal section); v_x (v_y) = mean of j_x/rho (j_y/rho) over the liquid
 * nodes (C > 0) of the column at (x_c + r_x/2, y_c) ((x_c, y_c + r_y/2)).
 * Synchronises the stream. */
typedef struct {
    double volume, height, xc, yc, r_x, r_y, theta_x, theta_y, v_x, v_y;
} lbm_shape;
lbm_status lbm_droplet_shape(lbm_handle* h, int inst, lbm_shape* out);

/* Release the handle (the workspace stays the caller's). */
lbm_status lbm_destroy(lbm_handle* h);

const char* lbm_status_string(lbm_status s);

/* Largest bead count lbm_deposit_descriptors_noalloc() accepts. */
#define LBM_NOALLOC_MAX_BEADS 16384

/* Deposit descriptors for callers that cannot allocate device memory (no
 * counterpart in the paper).  Some callers have no room to allocate: a host
 * application that has already reserved almost all device memory for its own
 * pool, or a time-critical loop that must not pay for cudaMalloc/cudaFree.
 * This entry point allocates nothing: its scratch (instance table, labels,
 * flags, edge list, counters, about 1.2 MB) is a fixed array in the library
 * that every GPU loading the library holds until the process exits.
 * Inputs are DEVICE arrays: bead_x [n_beads][3] FP64 positions (x in [0,nx),
 * y in [0,ny)), bead_fil and bead_pos [n_beads] int32 (filament id, index in
 * the filament; beads of a filament consecutive).  Output is a DEVICE array
 * out[5] = {S_x, n_clusters, percolates, n_bonds, error bits (0 = ok)},
 * written asynchronously on `stream`.  n_beads above LBM_NOALLOC_MAX_BEADS
 * fails with LBM_ECAPACITY before any device work.  The first call on a
 * device looks up the array's device address once (cudaGetSymbolAddress).
 * Calls share the array: counters are cleared on every call, and two calls
 * whose work overlaps on the GPU (other streams, other threads) race. */
lbm_status lbm_deposit_descriptors_noalloc(const double* bead_x, const int* bead_fil,
                                           const int* bead_pos, int n_beads, int nx, int ny,
                                           double rcon, double x_src, double x_snk, double* out,
                                           void* stream);

/* ---------------------------------------------------------------------------
 * Sweep proposer: a small multilayer perceptron trained on deposit
 * descriptors of batched runs (no paper counterpart; the paper sweeps its
 * parameters by enumeration, Sec. III).  Network: x[n_in] -> tanh(W1 x + b1)
 * -> tanh(W2 h1 + b2) -> y = W3 h2 + b3.  Parameters are one flat array
 * [W1 (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2,
 *  W3 (n_out x n_hidden), b3].  Loss L = 1/(2B) sum_b sum_k (y_bk - t_bk)^2.
 * All arrays are caller-owned DEVICE memory of dtype 0 (float) or 1 (double),
 * row-major [batch][n_in] / [batch][n_out]; calls are asynchronous on
 * `stream` (a cudaStream_t).  Limits: n_in, n_out <= 16, n_hidden <= 256.
 * ------------------------------------------------------------------------- */
size_t lbm_mlp_param_count(int n_in, int n_hidden, int n_out);
/* Device scratch that lbm_mlp_loss_grad() needs for activations and deltas. */
size_t lbm_mlp_scratch_bytes(int dtype, int n_hidden, int batch);
lbm_status lbm_mlp_forward(int dtype, const void* params, int n_in, int n_hidden, int n_out,
                           const void* x, int batch, void* y, void* stream);
/* Forward pass into y, loss into *loss (device scalar, may be NULL) and dL/dparams into grad. */
lbm_status lbm_mlp_loss_grad(int dtype, const void* params, int n_in, int n_hidden, int n_out,
                             const void* x, const void* targets, int batch, void* y, void* grad,
                             void* loss, void* scratch, size_t scratch_bytes, void* stream);
/* One Adam update with bias correction; `step` counts from 1. */
lbm_status lbm_mlp_adam(int dtype, void* params, const void* grad, void* m, void* v, int n_params,
                        double lr, double beta1, double beta2, double eps, int step, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
