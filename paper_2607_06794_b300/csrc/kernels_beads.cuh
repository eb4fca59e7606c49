// Filament kernels: bead-spring chains (Eqs. (9)-(12)) coupled to the fluid
// by a dissipative drag with equal and opposite reaction (Sec. II.A,
// Ahlrichs-Duenweg scheme), a solvation force xi grad C, substrate adhesion
// and load-dependent friction; `substeps` velocity-Verlet sub-steps per LB
// step on a frozen fluid.  Beads are FP64 throughout.
#pragma once

#include "kernels_fluid.cuh"

namespace lbm {

// beads a neighbour-search cell can hold (cells are at least rlist wide)
constexpr int CELL_CAP = 64;

// a coordinate as its nearest lattice point and the FP32 offset from it; a
// non-finite coordinate (already an error) maps to the origin
__device__ __forceinline__ void split_pos(double x, int& K, float& r) {
    if (!isfinite(x)) {
        K = 0;
        r = 0.0f;
        return;
    }
    const double k = rint(x);
    K = (int)k;
    r = (float)(x - k);
}

// minimum image of a separation of two wrapped coordinates (|d| <= L)
__device__ __forceinline__ double min_image(double d, int L) {
    const double h = 0.5 * L;
    return d > h ? d - L : (d < -h ? d + L : d);
}

// (d0/r)^12 - 2 (d0/r)^6 and its r-derivative (Eq. (12) without prefactor)
template <typename T>
__device__ __forceinline__ T lj_shape_dr(T d0, T r) {
    const T s = d0 / r, s2 = s * s, s6 = s2 * s2 * s2;
    return (T(-12) * s6 * s6 + T(12) * s6) / r;
}

// Force parameters of an instance in the compute type: the FP64 values, or their
// FP32 roundings made on the host (the same values a conversion here would give).
// has_coh / has_s: cohesion / substrate adhesion on (tested in FP64).
template <typename T>
struct BeadPar {
    T ks, Rm2, d0, eps_wca, kb, eps_coh, eps_s, rc, gamma, xi, mu, gamma_t, dt;
    bool has_coh, has_s;
    __device__ __forceinline__ explicit BeadPar(const InstDev& I) {
        if constexpr (sizeof(T) == 8) {
            ks = I.ks, Rm2 = I.Rm * I.Rm, d0 = I.d0, eps_wca = I.eps_wca, kb = I.kb, eps_coh = I.eps_coh;
            eps_s = I.eps_s, rc = I.rc, gamma = I.gamma, xi = I.xi, mu = I.mu, gamma_t = I.gamma_t;
            dt = I.dt_sub;
        } else {
            ks = I.f_ks, Rm2 = I.f_Rm2, d0 = I.f_d0, eps_wca = I.f_eps_wca, kb = I.f_kb;
            eps_coh = I.f_eps_coh, eps_s = I.f_eps_s, rc = I.f_rc, gamma = I.f_gamma, xi = I.f_xi;
            mu = I.f_mu, gamma_t = I.f_gamma_t, dt = I.f_dt_sub;
        }
        has_coh = I.eps_coh > 0.0;
        has_s = I.eps_s > 0.0;
    }
};

// dU/dr of a bead pair; `sep` = |index difference| if same filament, else 0
template <typename T>
__device__ __forceinline__ T pair_dUdr(const BeadPar<T>& bp, bool same, int sep, T r, int& err) {
    T f = 0;
    const T d0 = bp.d0;
    if (same && sep == 1) {  // FENE, Eq. (9)
        T q = r * r / bp.Rm2;
        if (q >= T(1)) {
            err |= ERR_FENE;
            q = T(0.99);
        }
        f += bp.ks * r / (T(1) - q);
    }
    if (same && sep == 2) f += bp.kb * (r - T(2) * d0);  // bending, Eq. (11)
    if (r <= d0) f += bp.eps_wca * lj_shape_dr<T>(d0, r);  // WCA, Eq. (10)
    if (!same && bp.has_coh && r > d0 && r < bp.rc) f += bp.eps_coh * lj_shape_dr<T>(d0, r);
    return f;
}

// index within one period of a coordinate that left [0, n) by less than n
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ double wrap1(double a, int n) { return a < 0.0 ? a + n : (a >= n ? a - n : a); }

// The trilinear stencil around a position (z clamped into the fluid): its lower
// corner cell and the fractions.  Positions are kept inside the periodic box by the
// integrator; a non-finite position (already an error) is mapped to the origin so
// that no index is ever formed from it.  W = double computes the fractions in FP64;
// W = float takes the cell and its fraction in FP64 and rounds the fraction to FP32.
template <typename W>
struct StencilCell {
    int x0, y0, z0;
    W fx, fy, fz;
};
template <typename W>
__device__ __forceinline__ StencilCell<W> stencil_cell(const InstDev& I, const double* X) {
    double px = X[0], py = X[1], pz = X[2];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) px = py = pz = 0.0;
    px = wrap1(px, I.nx);
    py = wrap1(py, I.ny);
    pz = pz < 0.0 ? 0.0 : (pz > I.nz - 1 ? (double)(I.nz - 1) : pz);
    StencilCell<W> sc;
    sc.x0 = min(max((int)floor(px), 0), I.nx - 1);
    sc.y0 = min(max((int)floor(py), 0), I.ny - 1);
    sc.z0 = (int)floor(pz);
    if (I.nz >= 2 && sc.z0 > I.nz - 2) sc.z0 = I.nz - 2;
    sc.fx = (W)(px - sc.x0);
    sc.fy = (W)(py - sc.y0);
    sc.fz = (W)(pz - sc.z0);
    return sc;
}

// The same from a split position (x = K + r): floor and fraction without FP64
// arithmetic, with the clamps of the FP64 form (z into [0, nz - 1], the cell at
// most nz - 2; x, y into the box)
__device__ __forceinline__ StencilCell<float> stencil_cell_split(const InstDev& I, int4 K, float4 R) {
    StencilCell<float> sc;
    const int fx = K.x - (R.x < 0.0f), fy = K.y - (R.y < 0.0f), fz = K.z - (R.z < 0.0f);
    const float rx = R.x < 0.0f ? R.x + 1.0f : R.x, ry = R.y < 0.0f ? R.y + 1.0f : R.y;
    const float rz = R.z < 0.0f ? R.z + 1.0f : R.z;
    sc.x0 = min(max(fx, 0), I.nx - 1);
    sc.y0 = min(max(fy, 0), I.ny - 1);
    sc.fx = rx;
    sc.fy = ry;
    if (fz < 0) {
        sc.z0 = 0;
        sc.fz = 0.0f;
    } else if (fz >= I.nz - 1) {
        sc.z0 = I.nz - 2;
        sc.fz = 1.0f;
    } else {
        sc.z0 = fz;
        sc.fz = rz;
    }
    return sc;
}

// Corner c (bit 0: x, bit 1: y, bit 2: z) of a stencil: node index, weight and
// 8^3 coupling tile.
template <typename W>
__device__ __forceinline__ void stencil_corner(const InstDev& I, const StencilCell<W>& sc, int c, long long& id,
                                               W& w, int& tile) {
    const int a = c & 1, b = (c >> 1) & 1, e = c >> 2;
    const int xx = wrap1(sc.x0 + a, I.nx), yy = wrap1(sc.y0 + b, I.ny), zz = (e && I.nz >= 2) ? sc.z0 + 1 : sc.z0;
    id = ((long long)zz * I.ny + yy) * I.nx + xx;
    w = (a ? sc.fx : W(1) - sc.fx) * (b ? sc.fy : W(1) - sc.fy) * (e ? sc.fz : W(1) - sc.fz);
    tile = ((zz >> 3) * I.t8y + (yy >> 3)) * I.t8x + (xx >> 3);
}
// cell of a (finite, wrapped) position; cells are at least rlist wide
__device__ __forceinline__ int cell_of(const InstDev& I, float x, float y, float z) {
    int cx_ = (int)(x * I.cgx / I.nx), cy_ = (int)(y * I.cgy / I.ny), cz_ = (int)((z + 0.5f) * I.cgz / I.nz);
    cx_ = min(max(cx_, 0), I.cgx - 1);
    cy_ = min(max(cy_, 0), I.cgy - 1);
    cz_ = min(max(cz_, 0), I.cgz - 1);
    return (cz_ * I.cgy + cy_) * I.cgx + cx_;
}

// Flag set of the step a bead start prepares: the current step (ahead = 0), or
// the step after the one whose sub-steps just ran (ahead = 1: the sub-step pass
// recorded it, so the answer does not depend on whether the fused kernel,
// which advances the step counter, has finished)
__device__ __forceinline__ int start_parity(const StepGlobals* glob, int ahead) {
    return (int)((ahead ? __ldcg(&glob->bead_next) : __ldcg(&glob->step)) & 1);
}

// Clear the coupling-tile flags (and the flagged-tile count behind them), the
// reach bits and the cell counts of every instance with beads, before its bead start.
__global__ void k_bead_clear(const InstDev* __restrict__ insts, const StepGlobals* __restrict__ glob, int ahead) {
    const InstDev& I = insts[blockIdx.y];
    if (I.tflag == nullptr) return;
    const int p = start_parity(glob, ahead);
    unsigned* tflag = tflag_of(I, p);
    unsigned* nbit = nbit_of(I, p);
    const int nt = I.ntile + 1, nc = I.cgx * I.cgy * I.cgz, nw = I.nword;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt + nc + nw; i += gridDim.x * blockDim.x) {
        if (i < nt)
            tflag[i] = 0u;
        else if (i < nt + nc)
            I.ccount[i - nt] = 0;
        else
            nbit[i - nt - nc] = 0u;
    }
}

// Step start, one warp per bead: remember the position, keep an FP32 copy
// for the neighbour search, file the bead in its cell, take the first half
// kick and drift of the step (FP64, lane 0; lanes 0..2 then split the drifted
// position into lattice point and FP32 offset for the first sub-step), and flag
// the coupling tiles its trilinear stencil can reach during the step (lane = one
// corner of the 4x4x2 reach; duplicates are harmless).
__global__ void k_bead_begin(const InstDev* __restrict__ insts, const StepGlobals* __restrict__ glob, int ahead) {
    const InstDev I = insts[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= I.nb) return;
    double X[3];
    for (int d = 0; d < 3; ++d) X[d] = I.bx[3 * a + d];
    if (!(isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2]))) {
        if (lane == 0) atomicOr(I.err, ERR_BEAD);
        return;
    }
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            I.bx0[3 * a + d] = X[d];
            I.bxf[3 * a + d] = (float)X[d];
        }
        const int c = cell_of(I, (float)X[0], (float)X[1], (float)X[2]);
        const int slot = atomicAdd(I.ccount + c, 1);
        if (slot < CELL_CAP)
            I.cbeads[(size_t)c * CELL_CAP + slot] = a;
        else
            atomicOr(I.err, ERR_CAP);
        const double dt = I.dt_sub, hk = I.hk_sub;
        double Y[3];
        for (int d = 0; d < 3; ++d) {
            const double vh = I.bv[3 * a + d] + hk * I.bF[3 * a + d];
            I.bvh[3 * a + d] = vh;
            Y[d] = X[d] + dt * vh;
        }
        Y[0] = wrap1(Y[0], I.nx);
        Y[1] = wrap1(Y[1], I.ny);
        if (!(Y[2] > -0.5 && Y[2] < I.nz - 0.5)) atomicOr(I.err, ERR_BEAD);
        for (int d = 0; d < 3; ++d) I.bx2[3 * a + d] = Y[d];
    }
    {
        // the split form of the sub-step-1 positions, one component per lane
        const int d = lane < 3 ? lane : 0;
        __syncwarp();
        const double y = I.bx2[3 * a + d];
        if (lane < 3) {
            int K;
            float r;
            split_pos(y, K, r);
            ((int*)(I.bK[0] + a))[d] = K;
            ((float*)(I.bR[0] + a))[d] = r;
        }
    }
    const double zc = X[2] < -1.0 ? -1.0 : (X[2] > I.nz ? (double)I.nz : X[2]);
    const int fx = wrap_near((int)floor(X[0]), I.nx), fy = wrap_near((int)floor(X[1]), I.ny), fz = (int)floor(zc);
    const int dx = (lane & 3) - 1, dy = ((lane >> 2) & 3) - 1, dz = (lane >> 4) ? 2 : -1;
    const int x = wrap_near(fx + dx, I.nx), y = wrap_near(fy + dy, I.ny);
    int z = fz + dz;
    z = z < 0 ? 0 : (z >= I.nz ? I.nz - 1 : z);
    const int t = ((z >> 3) * I.t8y + (y >> 3)) * I.t8x + (x >> 3);
    // one lane per distinct tile of the warp; most tiles are already flagged by a
    // neighbour, so the flag is read before the atomic; new tiles are appended
    // with one counter update per warp
    const int p = start_parity(glob, ahead);
    unsigned* tflag = tflag_of(I, p);
    unsigned* nbit = nbit_of(I, p);
    const unsigned same_t = __match_any_sync(0xffffffffu, t);
    bool fresh = false;
    if (lane == __ffs(same_t) - 1)
        fresh = !((volatile unsigned*)tflag)[t] && atomicExch(tflag + t, 1u) == 0u;
    const unsigned fresh_m = __ballot_sync(0xffffffffu, fresh);
    if (fresh_m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(tcount_of(I, p), __popc(fresh_m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) tlist_of(I, p)[base + __popc(fresh_m & ((1u << lane) - 1u))] = t;
    }
    // the 4x4x4 nodes the stencil can reach during the step, two per lane; the bits of
    // one 32-node word are gathered in the warp and set by one lane
    for (int k = 0; k < 2; ++k) {
        const int zr = fz + (lane >> 4) * 2 + k - 1;
        const int zz = zr < 0 ? 0 : (zr >= I.nz ? I.nz - 1 : zr);
        const long long node = ((long long)zz * I.ny + y) * I.nx + x;
        const unsigned word = (unsigned)(node >> 5);
        const unsigned same_w = __match_any_sync(0xffffffffu, word);
        const unsigned bits = __reduce_or_sync(same_w, 1u << (node & 31));
        if (lane == __ffs(same_w) - 1 && (((volatile unsigned*)nbit)[word] & bits) != bits)
            atomicOr(nbit + word, bits);
    }
}

// u* = (j + (F_s + body)/2)/rho and grad C on the nodes of flagged tiles.
template <class S, bool EP>
__device__ void bead_field_tile(const InstDev* __restrict__ Ip, const StepGlobals* __restrict__ glob, int t);

// EP: the populations are stored in place (esoteric pull), else in two buffers.
// Three blocks per SM (40 registers a thread): the pass waits on global loads twice
// per tile (colour block, pulls), and a third resident block hides more of that than
// the few spilled registers cost (four blocks spill ~250 bytes a thread)
template <class S, bool EP>
__global__ void __launch_bounds__(512, 3) k_bead_field(const InstDev* __restrict__ insts,
                                                    const StepGlobals* __restrict__ glob) {
    using T = typename S::T;
    using E = typename S::E;
    const InstDev* Ip = insts + blockIdx.y;
    if (Ip->tflag == nullptr || Ip->nb == 0) return;
    const int p = (int)(__ldcg(&glob->step) & 1);
    const int ntl = *tcount_of(*Ip, p);
    for (int it = blockIdx.x; it < ntl; it += gridDim.x) {
        bead_field_tile<S, EP>(Ip, glob, tlist_of(*Ip, p)[it]);
        __syncthreads();
    }
}

template <class S, bool EP>
__device__ void bead_field_tile(const InstDev* __restrict__ Ip, const StepGlobals* __restrict__ glob, int t) {
    using T = typename S::T;
    using E = typename S::E;
    const InstDev& I = *Ip;
    using V4 = typename Vec4<T>::type;
    __shared__ T sC[12][12][12];
    __shared__ V4 sN[10][10][10];  // unit normals (w unused): one 16/32-byte access each
    const long long step = __ldcg(&glob->step);
    const T* rho = (const T*)I.rho[step % 3];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const int X0 = (t % I.t8x) * 8, Y0 = ((t / I.t8x) % I.t8y) * 8, Z0 = (t / (I.t8x * I.t8y)) * 8;
    const int tid = threadIdx.x;
    __syncthreads();  // shared blocks of the previous tile are free
    // colour of the planes in the fluid (z = nz copies the top plane), then the
    // wetting ghost plane z = -1 from the shared plane z = 0 where it holds the
    // 3x3 neighbourhood, else from memory
    for (int s = tid; s < 12 * 12 * 12; s += 512) {
        const int lx = s % 12, ly = (s / 12) % 12, lz = s / 144;
        const int z = Z0 - 2 + lz;
        T c = T(0);
        if (z >= 0 && z <= nz) {
            const int x = wrap_near(X0 - 2 + lx, nx), y = wrap_near(Y0 - 2 + ly, ny);
            c = colour_of(rho, N, ((long long)(z < nz ? z : nz - 1) * ny + y) * nx + x);
        }
        sC[lz][ly][lx] = c;
    }
    __syncthreads();
    if (Z0 == 0) {
        for (int s = tid; s < 12 * 12; s += 512) {
            const int lx = s % 12, ly = s / 12;
            const int x = wrap_near(X0 - 2 + lx, nx), y = wrap_near(Y0 - 2 + ly, ny);
            T g;
            if (lx >= 1 && lx <= 10 && ly >= 1 && ly <= 10) {
                T ax = 0, ay = 0;
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int k = (dx != 0) + (dy != 0);
                        const T w = k == 0 ? T(4.0 / 9.0) : (k == 1 ? T(1.0 / 9.0) : T(1.0 / 36.0));
                        const T c = sC[2][ly + dy][lx + dx];
                        ax += w * dx * c;
                        ay += w * dy * c;
                    }
                ax *= T(3);
                ay *= T(3);
                g = sC[2][ly][lx] + (T)I.cot[y * nx + x] * sqrt(ax * ax + ay * ay);
                g = g > T(1) ? T(1) : (g < T(-1) ? T(-1) : g);
            } else {
                g = ghost_colour<T>(I, rho, x, y);
            }
            sC[1][ly][lx] = g;
        }
        __syncthreads();
    }
    for (int s = tid; s < 1000; s += 512) {
        const int lx = s % 10, ly = (s / 10) % 10, lz = s / 100;
        const int z = Z0 - 1 + lz;
        if (z < 0 || z >= nz) continue;
        T gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const T c = sC[lz + 1 + cz(i)][ly + 1 + cy(i)][lx + 1 + cx(i)];
            const T w = (T)wq(i);
            gx += w * cx(i) * c;
            gy += w * cy(i) * c;
            gz += w * cz(i) * c;
        }
        gx *= T(3);
        gy *= T(3);
        gz *= T(3);
        const T g2 = gx * gx + gy * gy + gz * gz;
        V4 nn;
        if (g2 > T(1e-16)) {
            const T ig = inv_norm<T>(g2);
            nn.x = gx * ig;
            nn.y = gy * ig;
            nn.z = gz * ig;
        } else {
            nn.x = nn.y = nn.z = T(0);
        }
        nn.w = T(0);
        sN[lz][ly][lx] = nn;
    }
    __syncthreads();
    // normals outside the fluid copy the nearest fluid plane
    for (int s = tid; s < 100; s += 512) {
        const int lx = s % 10, ly = s / 10;
        if (Z0 - 1 < 0) sN[0][ly][lx] = sN[1][ly][lx];
        for (int lz = 0; lz < 10; ++lz)
            if (Z0 - 1 + lz == nz) sN[lz][ly][lx] = sN[lz - 1][ly][lx];
    }
    __syncthreads();
    const int lx = tid % 8, ly = (tid / 8) % 8, lz = tid / 64;
    const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
    if (x >= nx || y >= ny || z >= nz) return;  // the caller's barrier follows
    const long long node = ((long long)z * ny + y) * nx + x;
    // the sub-steps of this step accumulate the drag reaction here from zero
    T* fe = (T*)I.fext + 3 * node;
    fe[0] = fe[1] = fe[2] = T(0);
    // u* and grad C are read only inside the beads' reach (marked at the step start)
    if (!((nbit_of(I, (int)(step & 1))[node >> 5] >> (node & 31)) & 1u)) return;
    T gx = 0, gy = 0, gz = 0, kap = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const T c = sC[lz + 2 + cz(i)][ly + 2 + cy(i)][lx + 2 + cx(i)];
        const T w = (T)wq(i);
        gx += w * cx(i) * c;
        gy += w * cy(i) * c;
        gz += w * cz(i) * c;
    }
    gx *= T(3);
    gy *= T(3);
    gz *= T(3);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const V4 nn = sN[lz + 1 + cz(i)][ly + 1 + cy(i)][lx + 1 + cx(i)];
        T d = 0;
        if (cx(i) != 0) d += cx(i) * nn.x;
        if (cy(i) != 0) d += cy(i) * nn.y;
        if (cz(i) != 0) d += cz(i) * nn.z;
        kap += (T)wq(i) * d;
    }
    kap *= T(-3);
    const T hs = T(0.5) * (T)I.sigma;
    const T rho0 = (T)I.rho0;
    T rR = 0, rB = 0, jx = 0, jy = 0, jz = 0;
    const NodePull<S, EP> pl(I, step, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        T r, b;
        pl.pull(i, r, b);
        rR += r;
        rB += b;
        const T F = r + b;
        jx += cx(i) * F;
        jy += cy(i) * F;
        jz += cz(i) * F;
    }
    const T irr = T(1) / (rR + rB);
    T* u = (T*)I.ust + 3 * node;
    T* g = (T*)I.gcol + 3 * node;
    u[0] = (jx + T(0.5) * (hs * kap * gx + (T)I.body[0])) * irr;
    u[1] = (jy + T(0.5) * (hs * kap * gy + (T)I.body[1])) * irr;
    u[2] = (jz + T(0.5) * (hs * kap * gz + (T)I.body[2])) * irr;
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

// Verlet neighbour list of the step, one warp per bead (FP32 positions; the
// skin absorbs the rounding).  Lanes 0..26 read the counts of the 27 (distinct
// periodic) neighbour cells at once; the candidates of all cells are then
// numbered cell by cell and taken 32 at a time, each lane finding its cell by a
// binary search over the lanes' prefix counts.  The list keeps the cell-major
// order of a plain cell-by-cell scan.
__global__ void k_bead_nlist(const InstDev* __restrict__ insts) {
    const InstDev I = insts[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (a >= I.nb) return;
    const float xa = I.bxf[3 * a], ya = I.bxf[3 * a + 1], za = I.bxf[3 * a + 2];
    if (!(isfinite(xa) && isfinite(ya) && isfinite(za))) return;
    const int c0 = cell_of(I, xa, ya, za);
    const int ix = c0 % I.cgx, iy = (c0 / I.cgx) % I.cgy, iz = c0 / (I.cgx * I.cgy);
    const int fa = I.bfil[a], pa = I.bpos[a];
    const float r2 = (float)(I.rlist * I.rlist);
    const float Lx = (float)I.nx, Ly = (float)I.ny;
    const int nxo = min(3, I.cgx), nyo = min(3, I.cgy);  // distinct periodic neighbour cells
    // this lane's cell: lane = (dz + 1) * 9 + oy * 3 + ox
    int cell = 0, m = 0;
    if (lane < 27) {
        const int dz = lane / 9 - 1, oy = (lane / 3) % 3, ox = lane % 3;
        const int zz = iz + dz;
        if (zz >= 0 && zz < I.cgz && oy < nyo && ox < nxo) {
            const int yy = wrap_near(iy + (nyo == 3 ? oy - 1 : oy), I.cgy);
            const int xx = wrap_near(ix + (nxo == 3 ? ox - 1 : ox), I.cgx);
            cell = (zz * I.cgy + yy) * I.cgx + xx;
            m = min(I.ccount[cell], CELL_CAP);
        }
    }
    int incl = m;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - m;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int cnt = 0;
    for (int base = 0; base < total; base += 32) {
        const int k = base + lane;
        // owner: the last lane whose exclusive prefix is <= k
        int lo = 0;
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, lo + step);
            if (lo + step < 32 && e <= k) lo += step;
        }
        const int oc = __shfl_sync(0xffffffffu, cell, lo);
        const int oe = __shfl_sync(0xffffffffu, excl, lo);
        bool hit = false;
        int b = -1;
        if (k < total) {
            b = I.cbeads[(size_t)oc * CELL_CAP + (k - oe)];
            if (b != a && !(I.bfil[b] == fa && abs(I.bpos[b] - pa) <= 2)) {
                float ex = I.bxf[3 * b] - xa, ey = I.bxf[3 * b + 1] - ya;
                const float ez = I.bxf[3 * b + 2] - za;
                ex = ex > 0.5f * Lx ? ex - Lx : (ex < -0.5f * Lx ? ex + Lx : ex);
                ey = ey > 0.5f * Ly ? ey - Ly : (ey < -0.5f * Ly ? ey + Ly : ey);
                hit = ex * ex + ey * ey + ez * ez < r2;
            }
        }
        const unsigned msk = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int kk = cnt + __popc(msk & ((1u << lane) - 1u));
            if (kk < I.max_nbr) I.nbr[(long long)a * I.max_nbr + kk] = b;
        }
        cnt += __popc(msk);
    }
    if (lane == 0) {
        if (cnt > I.max_nbr) {
            atomicOr(I.err, ERR_CAP);
            cnt = I.max_nbr;
        }
        I.nnbr[a] = cnt;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the L lanes of one bead's group (mask: the group's lanes)
template <int L, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Force evaluation of sub-step s (1-based), L lanes per bead (4, 8 or 16): the
// lanes share the bonded partners and the neighbour list (pair forces in the
// compute type) and the eight nodes of the trilinear stencil (8 / L each below
// eight lanes, else lanes 0..7 one each) for the interpolation of u* and grad C
// and for the reaction spread; every lane adds drag, solvation, adhesion and
// friction, and lanes 0..2 integrate one component each in FP64 (second half
// kick; if not last, the next first half kick and drift).  B300's FP64 pipe is
// narrow, so the FP64 work per bead is what sets the pace: fewer lanes per bead
// share the per-bead FP64 steps (stencil cell, constants, integration) among
// more beads per warp.
template <typename T, int L>
__global__ void k_bead_force(const InstDev* __restrict__ insts, StepGlobals* __restrict__ glob, int s) {
    static_assert(L >= 4 && L <= 32 && (L & (L - 1)) == 0, "4, 8, 16 or 32 lanes per bead");
    constexpr int CPL = L >= 8 ? 1 : 8 / L;  // stencil corners per lane
    const InstDev I = insts[blockIdx.y];
    const long long step = __ldcg(&glob->step);
    if (s == I.substeps && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) glob->bead_next = step + 1;
    const int lane = threadIdx.x & (L - 1);
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (threadIdx.x & (32 - L)));
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) / L;
    if (a >= I.nb) return;  // a whole group leaves together
    const bool last = s == I.substeps;
    const double* cur = (s & 1) ? I.bx2 : I.bx;
    double* nxt = (s & 1) ? I.bx : I.bx2;
    const double dt = I.dt_sub, hk = I.hk_sub;
    const BeadPar<T> bp(I);
    int err = 0;
    const double P[3] = {cur[3 * a], cur[3 * a + 1], cur[3 * a + 2]};
    // FP32 path: the split form of the current positions ([0] mirrors bx2, [1] bx)
    constexpr bool SPLIT = sizeof(T) == 4;
    // (selected, not indexed: a runtime index into the record would put it in local memory)
    const int4* Kc = (s & 1) ? I.bK[0] : I.bK[1];
    const float4* Rc = (s & 1) ? I.bR[0] : I.bR[1];
    int4* Kn = (s & 1) ? I.bK[1] : I.bK[0];
    float4* Rn = (s & 1) ? I.bR[1] : I.bR[0];
    int4 Ka = make_int4(0, 0, 0, 0);
    float4 Ra = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (SPLIT) {
        Ka = Kc[a];
        Ra = Rc[a];
    }
    const int fa = I.bfil[a], pa = I.bpos[a];
    const int nn = I.nnbr[a];
    // loads that do not depend on the pair loop go first, so that their latency overlaps it:
    // this lane's stencil corners with u*, grad C and the tile flag there, the half-step velocity
    long long idl[CPL];
    T wdl[CPL], uc[CPL][3], gcc[CPL][3];
    unsigned flagged[CPL];
    StencilCell<T> sc;  // once per lane, whatever its corners
    if constexpr (SPLIT)
        sc = stencil_cell_split(I, Ka, Ra);
    else
        sc = stencil_cell<T>(I, P);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int c = lane + k * L;
        idl[k] = 0;
        wdl[k] = 0;
        flagged[k] = 1u;
        for (int d = 0; d < 3; ++d) uc[k][d] = gcc[k][d] = 0;
        if (c < 8) {
            int tl = 0;
            stencil_corner(I, sc, c, idl[k], wdl[k], tl);
            const T* ust = (const T*)I.ust + 3 * idl[k];
            const T* gcl = (const T*)I.gcol + 3 * idl[k];
            for (int d = 0; d < 3; ++d) {
                uc[k][d] = ust[d];
                gcc[k][d] = gcl[d];
            }
            flagged[k] = tflag_of(I, (int)(step & 1))[tl];
        }
    }
    const double vh[3] = {I.bvh[3 * a], I.bvh[3 * a + 1], I.bvh[3 * a + 2]};
    // ---- pair forces, candidates spread over the lanes ----
    T fx = 0, fy = 0, fz = 0;
    // candidate c >= 4 is list entry c - 4; the next candidate's index is loaded one
    // iteration ahead, so that its latency overlaps the loads of the current pair
    const int* nl = I.nbr + (long long)a * I.max_nbr - 4;
    int bn = (lane >= 4 && lane < 4 + nn) ? nl[lane] : -1;
    for (int c = lane; c < 4 + nn; c += L) {
        const int bl = bn;
        bn = (c + L >= 4 && c + L < 4 + nn) ? nl[c + L] : -1;
        int b;
        bool same;
        int sep;
        if (c < 4) {
            const int k = c < 2 ? c - 2 : c - 1;  // -2, -1, +1, +2
            b = a + k;
            if (b < 0 || b >= I.nb || I.bfil[b] != fa || I.bpos[b] - pa != k) continue;
            same = true;
            sep = k < 0 ? -k : k;
        } else {
            b = bl;
            same = I.bfil[b] == fa;
            sep = same ? abs(I.bpos[b] - pa) : 0;
        }
        T d0, d1, d2;
        if constexpr (!SPLIT) {
            d0 = (T)min_image(cur[3 * b] - P[0], I.nx);
            d1 = (T)min_image(cur[3 * b + 1] - P[1], I.ny);
            d2 = (T)(cur[3 * b + 2] - P[2]);
        } else {
            // lattice-point difference (periodic image taken on the integers) plus the
            // difference of the offsets: one FP32 rounding, as the FP64 difference rounded
            const int4 Kb = Kc[b];
            const float4 Rb = Rc[b];
            int dx = Kb.x - Ka.x, dy = Kb.y - Ka.y;
            dx = 2 * dx > I.nx ? dx - I.nx : (2 * dx < -I.nx ? dx + I.nx : dx);
            dy = 2 * dy > I.ny ? dy - I.ny : (2 * dy < -I.ny ? dy + I.ny : dy);
            d0 = (T)dx + (Rb.x - Ra.x);
            d1 = (T)dy + (Rb.y - Ra.y);
            d2 = (T)(Kb.z - Ka.z) + (Rb.z - Ra.z);
        }
        const T r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const T g = pair_dUdr<T>(bp, same, sep, r, err);
        if (g != T(0)) {
            const T gr = g / r;
            fx += gr * d0;
            fy += gr * d1;
            fz += gr * d2;
        }
    }
    fx = group_sum<L>(fx, gmask);
    fy = group_sum<L>(fy, gmask);
    fz = group_sum<L>(fz, gmask);
    // ---- interpolation of u* and grad C over the lanes' stencil corners ----
    T u[3], gc[3];
    for (int d = 0; d < 3; ++d) {
        T su = 0, sg = 0;
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            su += wdl[k] * uc[k][d];
            sg += wdl[k] * gcc[k][d];
        }
        u[d] = group_sum<L>(su, gmask);
        gc[d] = group_sum<L>(sg, gmask);
    }
    const T vt3[3] = {(T)vh[0], (T)vh[1], (T)vh[2]};
    T drag[3];
    for (int d = 0; d < 3; ++d) drag[d] = bp.gamma * (u[d] - vt3[d]);
    T f[3] = {fx + drag[0] + bp.xi * gc[0], fy + drag[1] + bp.xi * gc[1], fz + drag[2] + bp.xi * gc[2]};
    // ---- substrate adhesion (LJ at the image distance) and load-dependent friction ----
    T rw;  // twice the height above the substrate's image plane z = -1/2
    if constexpr (SPLIT)
        rw = T(2) * (((T)Ka.z + T(0.5)) + Ra.z);
    else
        rw = T(2) * ((T)P[2] + T(0.5));
    T fw = 0;
    if (bp.has_s && rw < bp.rc && rw > T(0)) fw = T(-2) * bp.eps_s * lj_shape_dr<T>(bp.d0, rw);
    if (bp.has_s && rw < bp.rc) {
        const T load = (f[2] < T(0) ? -f[2] : T(0)) + (fw < T(0) ? -fw : T(0));
        const T vx = vt3[0], vy = vt3[1];
        const T vt = sqrt(vx * vx + vy * vy);
        if (vt > T(0)) {
            T mag = bp.gamma_t * vt;
            if (mag > bp.mu * load) mag = bp.mu * load;
            f[0] -= mag * vx / vt;
            f[1] -= mag * vy / vt;
        }
    }
    f[2] += fw;
    // ---- reaction of the drag onto the fluid, over the lanes' stencil corners ----
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        if (lane + k * L < 8) {
            if (flagged[k]) {
                T* fe = (T*)I.fext + 3 * idl[k];
                const T c = -bp.dt * wdl[k];
                for (int d = 0; d < 3; ++d) atomicAdd(fe + d, c * drag[d]);
            } else {
                err |= ERR_BEAD;
            }
        }
    }
    // ---- FP64 integration, component d on lane d ----
    double disp2 = 0.0;
    if (lane < 3) {
        const int d = lane;
        const double fd = (double)(d == 0 ? f[0] : (d == 1 ? f[1] : f[2]));
        const double vhd = d == 0 ? vh[0] : (d == 1 ? vh[1] : vh[2]);
        const double Pd = d == 0 ? P[0] : (d == 1 ? P[1] : P[2]);
        I.bF[3 * a + d] = fd;
        const double v = vhd + hk * fd;
        if (!last) {
            const double v2 = v + hk * fd;
            I.bvh[3 * a + d] = v2;
            double X = Pd + dt * v2;
            if (d == 0)
                X = wrap1(X, I.nx);
            else if (d == 1)
                X = wrap1(X, I.ny);
            else if (!(X > -0.5 && X < I.nz - 0.5))
                err |= ERR_BEAD;
            nxt[3 * a + d] = X;
            if constexpr (SPLIT) {  // the next sub-step's split form (the other buffer)
                int K;
                float r;
                split_pos(X, K, r);
                ((int*)(Kn + a))[d] = K;
                ((float*)(Rn + a))[d] = r;
            }
        } else {
            I.bv[3 * a + d] = v;
            if (cur != I.bx) I.bx[3 * a + d] = Pd;
            double dd = Pd - I.bx0[3 * a + d];
            if (d == 0)
                dd = min_image(dd, I.nx);
            else if (d == 1)
                dd = min_image(dd, I.ny);
            disp2 = dd * dd;
        }
    }
    if (last) {
        // a bead that moved more than half a cell since its neighbour list was built
        disp2 = group_sum<L>(disp2, gmask);
        if (lane == 0 && disp2 > 0.25) err |= ERR_BEAD;
    }
    if (err) atomicOr(I.err, err);
}

// ---------------------------------------------------------------------------
// Deposit descriptors (Sec. II.B): contact graph edges, then one block per
// instance labels components by min-label propagation with pointer jumping,
// and reduces S_x, cluster count and percolation.
// ---------------------------------------------------------------------------
__global__ void k_desc_edges(const InstDev* __restrict__ insts, int only) {
    const InstDev I = insts[only];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= I.nb) return;
    const double r2 = I.rcon * I.rcon;
    for (int b = a + 1; b < I.nb; ++b) {
        const bool bonded = I.bfil[b] == I.bfil[a] && abs(I.bpos[b] - I.bpos[a]) == 1;
        const double dx = min_image(I.bx[3 * b] - I.bx[3 * a], I.nx),
                     dy = min_image(I.bx[3 * b + 1] - I.bx[3 * a + 1], I.ny),
                     dz = I.bx[3 * b + 2] - I.bx[3 * a + 2];
        if (bonded || dx * dx + dy * dy + dz * dz < r2) {
            const int e = atomicAdd(I.nedges, 1);
            if (e < I.max_edges)
                I.edges[e] = make_int2(a, b);
            else
                atomicOr(I.err, ERR_CAP);
        }
    }
}

__global__ void __launch_bounds__(1024) k_desc_solve(const InstDev* __restrict__ insts, int only) {
    const InstDev I = insts[only];
    const int n = I.nb;
    int* lab = I.lab;
    int* srcf = I.lab + I.nb_max;
    int* snkf = I.lab + 2 * I.nb_max;
    const int ne = min(*I.nedges, I.max_edges);
    __shared__ int changed;
    __shared__ double sred[32];
    __shared__ int ired[32][3];
    const int tid = threadIdx.x;
    for (int a = tid; a < n; a += blockDim.x) {
        lab[a] = a;
        srcf[a] = 0;
        snkf[a] = 0;
    }
    __syncthreads();
    int it = 0;
    for (; it <= n + 1; ++it) {
        if (tid == 0) changed = 0;
        __syncthreads();
        for (int e = tid; e < ne; e += blockDim.x) {
            const int2 ed = I.edges[e];
            const int la = lab[ed.x], lb = lab[ed.y];
            if (la != lb) {
                const int m = la < lb ? la : lb;
                atomicMin(lab + ed.x, m);
                atomicMin(lab + ed.y, m);
                atomicMin(lab + la, m);
                atomicMin(lab + lb, m);
                changed = 1;
            }
        }
        __syncthreads();
        for (int a = tid; a < n; a += blockDim.x) {
            int l = lab[a];
            for (int k = 0; k < 64 && lab[l] < l; ++k) l = lab[l];
            atomicMin(lab + a, l);
        }
        __syncthreads();
        if (!changed) break;
        __syncthreads();
    }
    if (it > n + 1 && tid == 0) atomicOr(I.err, ERR_TIMEOUT);
    // resolve every label to its root
    for (int a = tid; a < n; a += blockDim.x) {
        int l = lab[a];
        for (int k = 0; k < n && lab[l] != l; ++k) l = lab[l];
        lab[a] = l;
    }
    __syncthreads();
    double s = 0.0;
    int nb = 0, nc = 0;
    for (int a = tid; a < n; a += blockDim.x) {
        if (lab[a] == a) ++nc;
        if (I.bx[3 * a] < I.x_src) srcf[lab[a]] = 1;
        if (I.bx[3 * a] > I.x_snk) snkf[lab[a]] = 1;
        if (a + 1 < n && I.bfil[a + 1] == I.bfil[a] && I.bpos[a + 1] == I.bpos[a] + 1) {
            const double dx = min_image(I.bx[3 * (a + 1)] - I.bx[3 * a], I.nx),
                         dy = min_image(I.bx[3 * (a + 1) + 1] - I.bx[3 * a + 1], I.ny),
                         dz = I.bx[3 * (a + 1) + 2] - I.bx[3 * a + 2];
            s += 2.0 * dx * dx / (dx * dx + dy * dy + dz * dz) - 1.0;
            ++nb;
        }
    }
    __syncthreads();
    int perc = 0;
    for (int a = tid; a < n; a += blockDim.x) perc |= (srcf[a] && snkf[a]);
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
        perc |= __shfl_xor_sync(0xffffffffu, perc, o);
    }
    if ((tid & 31) == 0) {
        sred[tid >> 5] = s;
        ired[tid >> 5][0] = nb;
        ired[tid >> 5][1] = nc;
        ired[tid >> 5][2] = perc;
    }
    __syncthreads();
    if (tid == 0) {
        double ss = 0.0;
        int b = 0, c = 0, p = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            ss += sred[w];
            b += ired[w][0];
            c += ired[w][1];
            p |= ired[w][2];
        }
        I.desc[0] = b ? ss / b : 0.0;
        I.desc[1] = c;
        I.desc[2] = p;
        I.desc[3] = b;
    }
}

}  // namespace lbm
