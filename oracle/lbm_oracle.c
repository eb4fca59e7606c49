/*
 * Plain FP64 CPU oracle of one time step of the fluid–filament method of
 * "Evaporation-Driven Nanowire Self-Assembly in an Elongated Droplet"
 * (Schoettner, Xie, Harting), Sec. II.A.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  It shares no code, header,
 * table or constant with the CUDA path; only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Every loop is written node by node, direction by direction, in the order
 * the method is described: stream, moments, wetting ghost layer, colour
 * gradient / curvature / CSF force, filament sub-steps with two-way drag
 * coupling, colour-blind forced BGK collision, recolouring, evaporation sink.
 * OpenMP only splits independent nodes; every sum whose order matters is
 * taken serially in a fixed order so results are deterministic.
 *
 * Readings of points the paper leaves open (each is a parameter or a choice
 * listed with its reason in the design notes):
 *   - velocity set D3Q19, c_s^2 = 1/3, populations in density units, rho0 = 1
 *   - both components share one velocity and the bulk density (Eq. (2) has no
 *     density-ratio term)
 *   - forcing: Guo source with u = (sum c_i f_i + F/2)/rho
 *   - recolouring: Latva-Kokko/Rothman split with parameter beta
 *   - wetting: flat-wall geometric ghost colour C(-1) = C(0) + cot(theta)|grad_par C|
 *   - evaporation: sink |grad C|/2 * J0/(K + h~) on the resting liquid population,
 *     h~ = local liquid column height / its maximum at the first evaporating step
 *   - top plane: pure-gas equilibrium inflow (or bounce-back wall)
 *   - filaments: FENE + WCA(all pairs) + bending(2nd neighbours) + cohesive LJ
 *     tail between filaments + substrate LJ at image distance + load-dependent
 *     friction + solvation xi*grad C + drag gamma(u - V); velocity Verlet with
 *     `substeps` sub-steps per LB step, fluid frozen during the sub-steps.
 *
 * Parity status: the fluid step is pinned by closed forms and invariants
 * (Poiseuille, Laplace law, exact linear-field gradient, mass/momentum
 * conservation, hand-computed evaporation, the lattice moments of the
 * recolouring term, a flat interface that stays flat and segregated);
 * conservative bead forces by finite differences of the energy; the coupling
 * stencil by exact interpolation of a linear velocity field and the first
 * moment of the spread reaction; solvation by its exact value in a linear
 * colour field; friction by both branches of its law at known loads;
 * descriptors by hand-made configurations.  The long drying trajectory of
 * Sec. III (Fig. 2) is qualitative only: parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* ---- D3Q19 (Sec. II.A, Eq. (1); the paper does not name the set) ---- */
static const int ex[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int ey[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int ez[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static double wgt(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* the direction pointing the other way, found by search */
static int reverse_of(int i) {
    for (int k = 0; k < Q; ++k)
        if (ex[k] == -ex[i] && ey[k] == -ey[i] && ez[k] == -ez[i]) return k;
    return -1;
}

/* error bits (mirrors the meaning of the library's status codes) */
#define ORC_ERR_NAN 1
#define ORC_ERR_FENE 2
#define ORC_ERR_BEAD 4

typedef struct {
    int nx, ny, nz;
    double tau_R, tau_B;   /* relaxation times, Eq. (1) */
    double beta;           /* recolouring strength */
    double sigma;          /* CSF surface tension */
    double rho0;           /* reference density, Eq. (3) */
    double J0, K;          /* evaporation, Eq. (8) */
    long long evap_start;  /* first step with the sink on; <0 = never */
    int top_bc;            /* 0 bounce-back wall, 1 pure-gas equilibrium */
    /* filaments, Eqs. (9)-(12) */
    double ks, Rm, d0, eps_wca, kb, eps_coh, eps_s, rc, gamma, xi, mu, gamma_t, mass;
    int substeps;
    double body[3]; /* uniform body-force density (0 in the paper's runs; used by pins) */
} orc_params;

typedef struct {
    long long step;
    double h0;         /* initial (first evaporating step) maximum column height */
    double evaporated; /* sum of converted resting mass */
    double top_in;     /* mass entering through the top plane */
    double top_out;    /* mass leaving through the top plane */
    int err;
} orc_acc;

typedef struct {
    int n;            /* beads */
    const int* fil;   /* filament id per bead */
    const int* pos;   /* index within its filament */
    double* X;        /* positions, 3 per bead */
    double* V;        /* velocities */
    double* F;        /* force of the last evaluation (carried between steps) */
} orc_beads;

static inline long long nid(const orc_params* p, int x, int y, int z) {
    return ((long long)z * p->ny + y) * p->nx + x;
}
static inline long long pid(const orc_params* p, int i, int x, int y, int z) {
    return (long long)i * p->nx * p->ny * p->nz + nid(p, x, y, z);
}
static inline int wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

/* ------------------------------------------------------------------ */
/* Initial droplet: C = tanh(-s/width), s = (q-1)*min(a,b,c), q the    */
/* ellipsoidal (shape 0) or elliptic-cylinder (shape 1) radius; both   */
/* components at rest in equilibrium, rho = rho0 (Sec. III.B set-up).  */
/* ------------------------------------------------------------------ */
void orc_init_droplet(const orc_params* p, int shape, double cx, double cy, double cz,
                      double a, double b, double c, double width, double* fR, double* fB) {
    double m = a < b ? a : b;
    m = m < c ? m : c;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double dx = (x - cx) / a, dy = (y - cy) / b, dz = (z - cz) / c;
                double q;
                if (shape == 0) {
                    q = sqrt(dx * dx + dy * dy + dz * dz);
                } else {
                    double r = sqrt(dy * dy + dz * dz);
                    q = fabs(dx) > r ? fabs(dx) : r;
                }
                double C = tanh(-(q - 1.0) * m / width);
                for (int i = 0; i < Q; ++i) {
                    fR[pid(p, i, x, y, z)] = wgt(i) * p->rho0 * (1.0 + C) / 2.0;
                    fB[pid(p, i, x, y, z)] = wgt(i) * p->rho0 * (1.0 - C) / 2.0;
                }
            }
}

/* ------------------------------------------------------------------ */
/* Streaming with boundaries (Eq. (1) left-hand side).                 */
/* fRs/fBs receive the streamed (pre-collision) populations.           */
/* ------------------------------------------------------------------ */
static void stream(const orc_params* p, const double* fR, const double* fB, double* fRs,
                   double* fBs, double* top_in, double* top_out) {
#pragma omp parallel for
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                for (int i = 0; i < Q; ++i) {
                    int sx = wrap(x - ex[i], p->nx), sy = wrap(y - ey[i], p->ny), sz = z - ez[i];
                    double r, bl;
                    if (sz < 0 || (sz >= p->nz && p->top_bc == 0)) {
                        /* half-way bounce-back: what left this node towards the wall returns */
                        int j = reverse_of(i);
                        r = fR[pid(p, j, x, y, z)];
                        bl = fB[pid(p, j, x, y, z)];
                    } else if (sz >= p->nz) {
                        /* pure-gas equilibrium at rest above the top plane */
                        r = 0.0;
                        bl = wgt(i) * p->rho0;
                    } else {
                        r = fR[pid(p, i, sx, sy, sz)];
                        bl = fB[pid(p, i, sx, sy, sz)];
                    }
                    fRs[pid(p, i, x, y, z)] = r;
                    fBs[pid(p, i, x, y, z)] = bl;
                }
    if (p->top_bc == 1) {
        int z = p->nz - 1;
        double in = 0.0, out = 0.0;
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                for (int i = 0; i < Q; ++i) {
                    if (ez[i] < 0) in += wgt(i) * p->rho0;
                    if (ez[i] > 0) out += fR[pid(p, i, x, y, z)] + fB[pid(p, i, x, y, z)];
                }
        *top_in += in;
        *top_out += out;
    }
}

/* ------------------------------------------------------------------ */
/* Macroscopic fields of the streamed populations (Eq. (3)) plus the   */
/* colour field C = (rho_R - rho_B)/(rho_R + rho_B) (Sec. II.A).       */
/* ------------------------------------------------------------------ */
typedef struct {
    double *rR, *rB, *C, *j; /* j: 3 per node */
} orc_mom;

static void moments(const orc_params* p, const double* fRs, const double* fBs, orc_mom* m) {
    long long N = (long long)p->nx * p->ny * p->nz;
#pragma omp parallel for
    for (long long n = 0; n < N; ++n) {
        double sR = 0, sB = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < Q; ++i) {
            double a = fRs[i * N + n], b = fBs[i * N + n];
            sR += a;
            sB += b;
            jx += ex[i] * (a + b);
            jy += ey[i] * (a + b);
            jz += ez[i] * (a + b);
        }
        /* Eq. (3) writes rho_k = rho0 sum_i f_i; the populations here carry
         * density units (rho0 is their unit), so the sum is the density. */
        m->rR[n] = sR;
        m->rB[n] = sB;
        m->C[n] = (m->rR[n] - m->rB[n]) / (m->rR[n] + m->rB[n]);
        m->j[3 * n + 0] = jx;
        m->j[3 * n + 1] = jy;
        m->j[3 * n + 2] = jz;
    }
}

/* ------------------------------------------------------------------ */
/* Wetting ghost layer (Sec. II.A, Akai's geometric formulation on a   */
/* flat wall).  With the liquid at C = +1, theta measured through the  */
/* liquid and wall normal +z, the interface normal satisfies           */
/* n_z = -cos(theta), |n_par| = sin(theta), hence                     */
/*   C(x,y,-1) = C(x,y,0) + cot(theta) |grad_par C(x,y,0)|,            */
/* clipped to [-1,1]; grad_par uses the isotropic D2Q9 weights.        */
/* ------------------------------------------------------------------ */
static void ghost_colour(const orc_params* p, const double* C, const double* cot, double* Cg) {
    static const double w2[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double gx = 0, gy = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int k = abs(dx) + abs(dy); /* 0 rest, 1 axis, 2 diagonal */
                    double Cn = C[nid(p, wrap(x + dx, p->nx), wrap(y + dy, p->ny), 0)];
                    gx += w2[k] * dx * Cn;
                    gy += w2[k] * dy * Cn;
                }
            gx *= 3.0;
            gy *= 3.0;
            double g = C[nid(p, x, y, 0)] + cot[y * p->nx + x] * sqrt(gx * gx + gy * gy);
            if (g > 1.0) g = 1.0;
            if (g < -1.0) g = -1.0;
            Cg[y * p->nx + x] = g;
        }
}

/* C extended by the ghost layer below z = 0 and a copy of the top plane above */
static inline double C_ext(const orc_params* p, const double* C, const double* Cg, int x, int y,
                           int z) {
    x = wrap(x, p->nx);
    y = wrap(y, p->ny);
    if (z < 0) return Cg[y * p->nx + x];
    if (z >= p->nz) z = p->nz - 1;
    return C[nid(p, x, y, z)];
}

/* ------------------------------------------------------------------ */
/* Colour gradient G = 3 sum_i w_i c_i C(x+c_i), unit normal n and     */
/* curvature kappa = -3 sum_i w_i c_i . n(x+c_i); CSF force            */
/* F_s = (sigma/2) kappa G applied before the collision (Sec. II.A).   */
/* Normals outside the fluid copy the nearest fluid plane.             */
/* ------------------------------------------------------------------ */
static void csf(const orc_params* p, const double* C, const double* Cg, double* G, double* nrm,
                double* kap, double* Fs) {
    long long N = (long long)p->nx * p->ny * p->nz;
#pragma omp parallel for
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double gx = 0, gy = 0, gz = 0;
                for (int i = 1; i < Q; ++i) {
                    double Cn = C_ext(p, C, Cg, x + ex[i], y + ey[i], z + ez[i]);
                    gx += wgt(i) * ex[i] * Cn;
                    gy += wgt(i) * ey[i] * Cn;
                    gz += wgt(i) * ez[i] * Cn;
                }
                gx *= 3.0;
                gy *= 3.0;
                gz *= 3.0;
                long long n = nid(p, x, y, z);
                G[3 * n] = gx;
                G[3 * n + 1] = gy;
                G[3 * n + 2] = gz;
                double g = sqrt(gx * gx + gy * gy + gz * gz);
                if (g > 1e-8) {
                    nrm[3 * n] = gx / g;
                    nrm[3 * n + 1] = gy / g;
                    nrm[3 * n + 2] = gz / g;
                } else {
                    nrm[3 * n] = nrm[3 * n + 1] = nrm[3 * n + 2] = 0.0;
                }
            }
#pragma omp parallel for
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double k = 0;
                for (int i = 1; i < Q; ++i) {
                    int zz = z + ez[i];
                    if (zz < 0) zz = 0;
                    if (zz >= p->nz) zz = p->nz - 1;
                    long long m = nid(p, wrap(x + ex[i], p->nx), wrap(y + ey[i], p->ny), zz);
                    k += wgt(i) * (ex[i] * nrm[3 * m] + ey[i] * nrm[3 * m + 1] + ez[i] * nrm[3 * m + 2]);
                }
                k *= -3.0;
                long long n = nid(p, x, y, z);
                kap[n] = k;
                for (int d = 0; d < 3; ++d) Fs[3 * n + d] = 0.5 * p->sigma * k * G[3 * n + d];
            }
    (void)N;
}

/* ------------------------------------------------------------------ */
/* Filaments (Sec. II.A, Eqs. (9)-(12)).                               */
/* ------------------------------------------------------------------ */

/* LJ shape of Eq. (12) without the prefactor: (d0/r)^12 - 2 (d0/r)^6 */
static double lj_shape(double d0, double r) {
    double s6 = pow(d0 / r, 6.0);
    return s6 * s6 - 2.0 * s6;
}
/* d/dr of lj_shape */
static double lj_shape_dr(double d0, double r) {
    double s6 = pow(d0 / r, 6.0);
    return (-12.0 * s6 * s6 + 12.0 * s6) / r;
}

/* minimum image of a separation along a periodic axis of length L */
static double min_image(double d, int L) {
    return d - L * floor(d / L + 0.5);
}

/* pair dU/dr for beads a<b; also adds the pair energy to *U when U != NULL */
static double pair_dUdr(const orc_params* p, const orc_beads* B, int a, int b, double r, double* U,
                        int* err) {
    int same = B->fil[a] == B->fil[b];
    int sep = same ? abs(B->pos[a] - B->pos[b]) : 0;
    double dUdr = 0.0, e = 0.0;
    if (same && sep == 1) { /* FENE, Eq. (9) */
        double q = r * r / (p->Rm * p->Rm);
        if (q >= 1.0) {
            *err |= ORC_ERR_FENE;
            q = 0.99;
        }
        dUdr += p->ks * r / (1.0 - q);
        e += -0.5 * p->ks * p->Rm * p->Rm * log(1.0 - q);
    }
    if (same && sep == 2) { /* bending on second neighbours, Eq. (11) */
        dUdr += p->kb * (r - 2.0 * p->d0);
        e += 0.5 * p->kb * (r - 2.0 * p->d0) * (r - 2.0 * p->d0);
    }
    if (r <= p->d0) { /* WCA, Eq. (10): every pair, bonded ones included */
        dUdr += p->eps_wca * lj_shape_dr(p->d0, r);
        e += p->eps_wca * (lj_shape(p->d0, r) + 1.0);
    }
    if (!same && p->eps_coh > 0.0 && r < p->rc) { /* cohesive tail of Eq. (12), shifted */
        double shift = lj_shape(p->d0, p->rc);
        if (r > p->d0) {
            dUdr += p->eps_coh * lj_shape_dr(p->d0, r);
            e += p->eps_coh * (lj_shape(p->d0, r) - shift);
        } else {
            e += p->eps_coh * (-1.0 - shift);
        }
    }
    if (U) *U += e;
    return dUdr;
}

/* substrate adhesion: LJ of Eq. (12) with eps_s at the image distance 2(z+1/2) */
static double wall_Fz(const orc_params* p, double z, double* U) {
    double r = 2.0 * (z + 0.5);
    if (p->eps_s <= 0.0 || r >= p->rc || r <= 0.0) return 0.0;
    if (U) *U += p->eps_s * (lj_shape(p->d0, r) - lj_shape(p->d0, p->rc));
    return -2.0 * p->eps_s * lj_shape_dr(p->d0, r);
}

/* conservative forces (pairs + wall) on every bead, brute force over all pairs */
static void conservative_forces(const orc_params* p, const orc_beads* B, double* Fc, double* Fw,
                                double* U, int* err) {
    int n = B->n;
    for (int a = 0; a < 3 * n; ++a) Fc[a] = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            double d[3];
            d[0] = min_image(B->X[3 * b] - B->X[3 * a], p->nx);
            d[1] = min_image(B->X[3 * b + 1] - B->X[3 * a + 1], p->ny);
            d[2] = B->X[3 * b + 2] - B->X[3 * a + 2];
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double f = pair_dUdr(p, B, a, b, r, U, err);
            if (f != 0.0)
                for (int k = 0; k < 3; ++k) {
                    Fc[3 * b + k] -= f * d[k] / r;
                    Fc[3 * a + k] += f * d[k] / r;
                }
        }
    for (int a = 0; a < n; ++a) Fw[a] = wall_Fz(p, B->X[3 * a + 2], U);
}

/* trilinear stencil: 8 node ids and weights around a position */
static void stencil(const orc_params* p, const double* X, long long* id, double* w) {
    double px = X[0], py = X[1], pz = X[2];
    if (pz < 0.0) pz = 0.0;
    if (pz > p->nz - 1) pz = p->nz - 1;
    int x0 = (int)floor(px), y0 = (int)floor(py), z0 = (int)floor(pz);
    if (p->nz >= 2 && z0 > p->nz - 2) z0 = p->nz - 2;
    double fx = px - x0, fy = py - y0, fz = pz - z0;
    int z1 = p->nz >= 2 ? z0 + 1 : z0;
    int k = 0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int xx = wrap(x0 + a, p->nx), yy = wrap(y0 + b, p->ny), zz = c ? z1 : z0;
                id[k] = nid(p, xx, yy, zz);
                w[k] = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy) * (c ? fz : 1.0 - fz);
                ++k;
            }
}

/* total force on every bead given the frozen fluid fields; drag returned separately */
static void bead_forces(const orc_params* p, const orc_beads* B, const double* Vh,
                        const double* ustar, const double* G, double* Ftot, double* Fdrag,
                        double* Fc, double* Fw, int* err) {
    conservative_forces(p, B, Fc, Fw, NULL, err);
    for (int a = 0; a < B->n; ++a) {
        long long id[8];
        double w[8], u[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        stencil(p, &B->X[3 * a], id, w);
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d) {
                u[d] += w[k] * ustar[3 * id[k] + d];
                g[d] += w[k] * G[3 * id[k] + d];
            }
        double f[3];
        for (int d = 0; d < 3; ++d) {
            Fdrag[3 * a + d] = p->gamma * (u[d] - Vh[3 * a + d]); /* Ahlrichs-Duenweg drag */
            f[d] = Fc[3 * a + d] + Fdrag[3 * a + d] + p->xi * g[d]; /* + solvation */
        }
        /* load-dependent substrate friction on beads within range of the substrate */
        double rw = 2.0 * (B->X[3 * a + 2] + 0.5);
        double fw = Fw[a];
        if (p->eps_s > 0.0 && rw < p->rc) {
            double load = (f[2] < 0.0 ? -f[2] : 0.0) + (fw < 0.0 ? -fw : 0.0);
            double vx = Vh[3 * a], vy = Vh[3 * a + 1];
            double vt = sqrt(vx * vx + vy * vy);
            if (vt > 0.0) {
                double mag = p->gamma_t * vt;
                if (mag > p->mu * load) mag = p->mu * load;
                f[0] -= mag * vx / vt;
                f[1] -= mag * vy / vt;
            }
        }
        f[2] += fw;
        for (int d = 0; d < 3; ++d) Ftot[3 * a + d] = f[d];
    }
}

/* energy of the conservative part; used by the finite-difference pins */
double orc_bead_energy(const orc_params* p, int n, const int* fil, const int* pos, double* X) {
    orc_beads B = {n, fil, pos, X, NULL, NULL};
    double* Fc = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* Fw = malloc(sizeof(double) * (n > 0 ? n : 1));
    double U = 0.0;
    int err = 0;
    conservative_forces(p, &B, Fc, Fw, &U, &err);
    free(Fc);
    free(Fw);
    return U;
}

/* conservative force on each bead (pairs + wall), for the finite-difference pins */
int orc_bead_conservative_forces(const orc_params* p, int n, const int* fil, const int* pos,
                                 double* X, double* F) {
    orc_beads B = {n, fil, pos, X, NULL, NULL};
    double* Fw = malloc(sizeof(double) * (n > 0 ? n : 1));
    int err = 0;
    conservative_forces(p, &B, F, Fw, NULL, &err);
    for (int a = 0; a < n; ++a) F[3 * a + 2] += Fw[a];
    free(Fw);
    return err;
}

/* ------------------------------------------------------------------ */
/* Diagnostic fields of the current state without advancing it.        */
/* out (each may be NULL): rR, rB, C, j(3N), G(3N), kappa(N), Fs(3N),   */
/* h(nx*ny).                                                           */
/* ------------------------------------------------------------------ */
void orc_fields(const orc_params* p, const double* fR, const double* fB, const double* cot,
                double* rR, double* rB, double* Cout, double* jout, double* Gout, double* kout,
                double* Fsout, double* hout) {
    long long N = (long long)p->nx * p->ny * p->nz;
    double* fRs = malloc(sizeof(double) * Q * N);
    double* fBs = malloc(sizeof(double) * Q * N);
    double ti = 0, to = 0;
    stream(p, fR, fB, fRs, fBs, &ti, &to);
    orc_mom m;
    m.rR = malloc(sizeof(double) * N);
    m.rB = malloc(sizeof(double) * N);
    m.C = malloc(sizeof(double) * N);
    m.j = malloc(sizeof(double) * 3 * N);
    moments(p, fRs, fBs, &m);
    double* Cg = malloc(sizeof(double) * p->nx * p->ny);
    ghost_colour(p, m.C, cot, Cg);
    double* G = malloc(sizeof(double) * 3 * N);
    double* nr = malloc(sizeof(double) * 3 * N);
    double* k = malloc(sizeof(double) * N);
    double* Fs = malloc(sizeof(double) * 3 * N);
    csf(p, m.C, Cg, G, nr, k, Fs);
    if (rR) memcpy(rR, m.rR, sizeof(double) * N);
    if (rB) memcpy(rB, m.rB, sizeof(double) * N);
    if (Cout) memcpy(Cout, m.C, sizeof(double) * N);
    if (jout) memcpy(jout, m.j, sizeof(double) * 3 * N);
    if (Gout) memcpy(Gout, G, sizeof(double) * 3 * N);
    if (kout) memcpy(kout, k, sizeof(double) * N);
    if (Fsout) memcpy(Fsout, Fs, sizeof(double) * 3 * N);
    if (hout)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double h = 0;
                for (int z = 0; z < p->nz; ++z) h += (1.0 + m.C[nid(p, x, y, z)]) / 2.0;
                hout[y * p->nx + x] = h;
            }
    free(fRs); free(fBs); free(m.rR); free(m.rB); free(m.C); free(m.j);
    free(Cg); free(G); free(nr); free(k); free(Fs);
}

/* ------------------------------------------------------------------ */
/* One full time step, in place on (fR, fB) and the beads.              */
/* fR/fB hold post-collision populations [19][nz][ny][nx]; cot holds    */
/* cot(theta) per substrate cell [ny][nx].  Returns the error bits.     */
/* fext_out (3N, may be NULL) receives the force the beads put on the   */
/* fluid in this step.                                                  */
/* ------------------------------------------------------------------ */
int orc_step(const orc_params* p, double* fR, double* fB, const double* cot, int nbeads,
             const int* fil, const int* pos, double* X, double* V, double* Fb, orc_acc* acc,
             double* fext_out) {
    long long N = (long long)p->nx * p->ny * p->nz;
    int nxy = p->nx * p->ny;
    int err = 0;
    double* fRs = malloc(sizeof(double) * Q * N);
    double* fBs = malloc(sizeof(double) * Q * N);
    stream(p, fR, fB, fRs, fBs, &acc->top_in, &acc->top_out);

    orc_mom m;
    m.rR = malloc(sizeof(double) * N);
    m.rB = malloc(sizeof(double) * N);
    m.C = malloc(sizeof(double) * N);
    m.j = malloc(sizeof(double) * 3 * N);
    moments(p, fRs, fBs, &m);

    /* liquid column height h(x,y) = sum_z (1+C)/2 and its normalisation (Eq. (8)) */
    int evap = p->evap_start >= 0 && acc->step >= p->evap_start && p->J0 > 0.0;
    double* h = malloc(sizeof(double) * nxy);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double s = 0;
            for (int z = 0; z < p->nz; ++z) s += (1.0 + m.C[nid(p, x, y, z)]) / 2.0;
            h[y * p->nx + x] = s;
        }
    if (p->evap_start >= 0 && acc->step == p->evap_start) {
        double mx = 0.0;
        for (int a = 0; a < nxy; ++a) mx = h[a] > mx ? h[a] : mx;
        acc->h0 = mx;
    }

    double* Cg = malloc(sizeof(double) * nxy);
    ghost_colour(p, m.C, cot, Cg);
    double* G = malloc(sizeof(double) * 3 * N);
    double* nr = malloc(sizeof(double) * 3 * N);
    double* kap = malloc(sizeof(double) * N);
    double* Fs = malloc(sizeof(double) * 3 * N);
    csf(p, m.C, Cg, G, nr, kap, Fs);

    /* filaments: `substeps` velocity-Verlet sub-steps on the frozen fluid */
    double* Fext = calloc(3 * N, sizeof(double));
    if (nbeads > 0) {
        double* ust = malloc(sizeof(double) * 3 * N);
        for (long long n = 0; n < N; ++n) {
            double rho = m.rR[n] + m.rB[n];
            for (int d = 0; d < 3; ++d)
                ust[3 * n + d] = (m.j[3 * n + d] + 0.5 * (Fs[3 * n + d] + p->body[d])) / rho;
        }
        orc_beads B = {nbeads, fil, pos, X, V, Fb};
        double dt = 1.0 / p->substeps;
        double* Vh = malloc(sizeof(double) * 3 * nbeads);
        double* Fd = malloc(sizeof(double) * 3 * nbeads);
        double* Fc = malloc(sizeof(double) * 3 * nbeads);
        double* Fw = malloc(sizeof(double) * nbeads);
        double* X0 = malloc(sizeof(double) * 3 * nbeads);
        memcpy(X0, X, sizeof(double) * 3 * nbeads);
        for (int s = 0; s < p->substeps; ++s) {
            for (int a = 0; a < nbeads; ++a) {
                for (int d = 0; d < 3; ++d) {
                    Vh[3 * a + d] = V[3 * a + d] + 0.5 * dt / p->mass * Fb[3 * a + d];
                    X[3 * a + d] += dt * Vh[3 * a + d];
                }
                X[3 * a] -= p->nx * floor(X[3 * a] / p->nx);
                X[3 * a + 1] -= p->ny * floor(X[3 * a + 1] / p->ny);
                if (!(X[3 * a + 2] > -0.5 && X[3 * a + 2] < p->nz - 0.5)) err |= ORC_ERR_BEAD;
            }
            bead_forces(p, &B, Vh, ust, G, Fb, Fd, Fc, Fw, &err);
            for (int a = 0; a < nbeads; ++a) {
                for (int d = 0; d < 3; ++d) V[3 * a + d] = Vh[3 * a + d] + 0.5 * dt / p->mass * Fb[3 * a + d];
                long long id[8];
                double w[8];
                stencil(p, &X[3 * a], id, w);
                for (int k = 0; k < 8; ++k)
                    for (int d = 0; d < 3; ++d) Fext[3 * id[k] + d] -= dt * w[k] * Fd[3 * a + d];
            }
        }
        for (int a = 0; a < nbeads; ++a) {
            double dx = min_image(X[3 * a] - X0[3 * a], p->nx);
            double dy = min_image(X[3 * a + 1] - X0[3 * a + 1], p->ny);
            double dz = X[3 * a + 2] - X0[3 * a + 2];
            if (dx * dx + dy * dy + dz * dz > 0.25) err |= ORC_ERR_BEAD;
        }
        free(ust); free(Vh); free(Fd); free(Fc); free(Fw); free(X0);
    }
    if (fext_out) memcpy(fext_out, Fext, sizeof(double) * 3 * N);

    /* colour-blind forced BGK, recolouring, evaporation sink */
    double* evap_z = calloc(p->nz, sizeof(double));
    int* err_z = calloc(p->nz, sizeof(int));
#pragma omp parallel for
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long long n = nid(p, x, y, z);
                double rR = m.rR[n], rB = m.rB[n], rho = rR + rB;
                if (!(rho > 0.0) || rho != rho) err_z[z] |= ORC_ERR_NAN;
                double F[3], u[3];
                for (int d = 0; d < 3; ++d) {
                    F[d] = Fs[3 * n + d] + Fext[3 * n + d] + p->body[d];
                    u[d] = (m.j[3 * n + d] + 0.5 * F[d]) / rho;
                }
                double omega = (rR / rho) / p->tau_R + (rB / rho) / p->tau_B;
                double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                double g[3] = {G[3 * n], G[3 * n + 1], G[3 * n + 2]};
                double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                double phi = rR / rho;
                double post[Q];
                for (int i = 0; i < Q; ++i) {
                    double fi = fRs[i * N + n] + fBs[i * N + n];
                    double cu = ex[i] * u[0] + ey[i] * u[1] + ez[i] * u[2];
                    double feq = wgt(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                    double cF = ex[i] * F[0] + ey[i] * F[1] + ez[i] * F[2];
                    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
                    double S = (1.0 - 0.5 * omega) * wgt(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
                    post[i] = fi - omega * (fi - feq) + S;
                }
                for (int i = 0; i < Q; ++i) {
                    double cosphi = 0.0;
                    if (i > 0 && gm > 1e-8) {
                        double cl = sqrt((double)(ex[i] * ex[i] + ey[i] * ey[i] + ez[i] * ez[i]));
                        cosphi = (ex[i] * g[0] + ey[i] * g[1] + ez[i] * g[2]) / (cl * gm);
                    }
                    double r = phi * post[i] + p->beta * (rR * rB / rho) * wgt(i) * cosphi;
                    fR[pid(p, i, x, y, z)] = r;
                    fB[pid(p, i, x, y, z)] = post[i] - r;
                }
                if (evap && acc->h0 > 0.0) {
                    double ht = h[y * p->nx + x] / acc->h0;
                    if (ht > 0.0) {
                        double dm = p->J0 / (p->K + ht) * 0.5 * gm;
                        double avail = fR[pid(p, 0, x, y, z)];
                        if (dm > avail) dm = avail;
                        if (dm < 0.0) dm = 0.0;
                        fR[pid(p, 0, x, y, z)] -= dm;
                        fB[pid(p, 0, x, y, z)] += dm;
                        evap_z[z] += dm;
                    }
                }
            }
    for (int z = 0; z < p->nz; ++z) {
        acc->evaporated += evap_z[z];
        err |= err_z[z];
    }
    acc->step += 1;
    acc->err |= err;
    free(evap_z); free(err_z);
    free(fRs); free(fBs); free(m.rR); free(m.rB); free(m.C); free(m.j); free(h);
    free(Cg); free(G); free(nr); free(kap); free(Fs); free(Fext);
    return err;
}

/* ------------------------------------------------------------------ */
/* Deposit descriptors (Sec. II.B).                                    */
/*  S_x: mean over all bonds of 2 cos^2(zeta_x) - 1 (Eq. (13), one bin) */
/*  clusters: connected components of bonds and contacts r < rcon       */
/*  percolation: a component holds beads with x < xsrc and x > xsnk     */
/* ------------------------------------------------------------------ */
static int uf_find(int* par, int a) {
    while (par[a] != a) a = par[a];
    return a;
}

void orc_descriptors(const orc_params* p, int n, const int* fil, const int* pos, const double* X,
                     double rcon, double xsrc, double xsnk, double* Sx, int* nclusters,
                     int* percolates, int* label) {
    double s = 0.0;
    int nb = 0;
    for (int a = 0; a + 1 < n; ++a)
        if (fil[a] == fil[a + 1] && pos[a + 1] == pos[a] + 1) {
            double dx = min_image(X[3 * (a + 1)] - X[3 * a], p->nx);
            double dy = min_image(X[3 * (a + 1) + 1] - X[3 * a + 1], p->ny);
            double dz = X[3 * (a + 1) + 2] - X[3 * a + 2];
            double c2 = dx * dx / (dx * dx + dy * dy + dz * dz);
            s += 2.0 * c2 - 1.0;
            ++nb;
        }
    *Sx = nb ? s / nb : 0.0;
    int* par = malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int a = 0; a < n; ++a) par[a] = a;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            int bonded = fil[a] == fil[b] && abs(pos[a] - pos[b]) == 1;
            double dx = min_image(X[3 * b] - X[3 * a], p->nx);
            double dy = min_image(X[3 * b + 1] - X[3 * a + 1], p->ny);
            double dz = X[3 * b + 2] - X[3 * a + 2];
            if (bonded || dx * dx + dy * dy + dz * dz < rcon * rcon) {
                int ra = uf_find(par, a), rb = uf_find(par, b);
                if (ra != rb) {
                    if (ra < rb) par[rb] = ra; else par[ra] = rb;
                }
            }
        }
    int nc = 0;
    for (int a = 0; a < n; ++a) {
        label[a] = uf_find(par, a);
        if (label[a] == a) ++nc;
    }
    *nclusters = nc;
    int perc = 0;
    for (int r = 0; r < n && !perc; ++r) {
        if (label[r] != r) continue;
        int lo = 0, hi = 0;
        for (int a = 0; a < n; ++a)
            if (label[a] == r) {
                if (X[3 * a] < xsrc) lo = 1;
                if (X[3 * a] > xsnk) hi = 1;
            }
        perc = lo && hi;
    }
    *percolates = perc;
    free(par);
}
