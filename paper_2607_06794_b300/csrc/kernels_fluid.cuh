// Fluid kernels: one fused pass per time step (pull-stream, moments, CSF,
// forced BGK, recolouring, evaporation, store, push of the next moments),
// plus initialisation, moment recomputation and diagnostics.
// Method: Sec. II.A of "Evaporation-Driven Nanowire Self-Assembly in an
// Elongated Droplet" (Eqs. (1)-(3), (8) and the colour-gradient / CSF /
// wetting paragraphs).
#pragma once

#include <cstring>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

template <typename T>
__device__ __forceinline__ T colour_of(const T* __restrict__ rho, long long N, long long n) {
    T a = rho[n], b = rho[N + n];
    return (a - b) / (a + b);
}

// Wetting ghost layer below z = 0 (Sec. II.A, Akai's geometric scheme on a
// flat wall): C(x,y,-1) = C(x,y,0) + cot(theta) |grad_par C(x,y,0)|, clipped
// to [-1, 1]; grad_par with the isotropic 2-D weights 4/9, 1/9, 1/36.
template <typename T>
__device__ T ghost_colour(const InstDev& I, const T* __restrict__ rho, int x, int y) {
    const int nx = I.nx, ny = I.ny;
    const long long N = I.N;
    T gx = 0, gy = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int k = (dx != 0) + (dy != 0);
            const T w = k == 0 ? T(4.0 / 9.0) : (k == 1 ? T(1.0 / 9.0) : T(1.0 / 36.0));
            const T c = colour_of(rho, N, (long long)wrapi(y + dy, ny) * nx + wrapi(x + dx, nx));
            gx += w * dx * c;
            gy += w * dy * c;
        }
    gx *= T(3);
    gy *= T(3);
    T g = colour_of(rho, N, (long long)y * nx + x) + (T)I.cot[y * nx + x] * sqrt(gx * gx + gy * gy);
    return g > T(1) ? T(1) : (g < T(-1) ? T(-1) : g);
}

// Colour at an extended position: z = -1 is the ghost layer, z = nz copies the top plane.
template <typename T>
__device__ T colour_ext(const InstDev& I, const T* __restrict__ rho, int x, int y, int z) {
    x = wrapi(x, I.nx);
    y = wrapi(y, I.ny);
    if (z < 0) return ghost_colour<T>(I, rho, x, y);
    if (z >= I.nz) z = I.nz - 1;
    return colour_of(rho, I.N, ((long long)z * I.ny + y) * I.nx + x);
}

// ---------------------------------------------------------------------------
// Fused time step over one tile (TX x TY columns, planes z0..z1-1), marching
// upwards in z.  Shared memory holds a 3-plane ring of C with a 2-cell halo,
// a 3-plane ring of unit normals with a 1-cell halo and the core gradient of
// the next two planes.  Every stored population is pushed to the node it
// streams to next step: a warp is one row of the tile, so the x-neighbour's
// share moves by a lane shuffle, the share of the planes above and below
// waits in the thread's registers, and only the sum over the three source
// rows goes through shared memory (plain stores, no shared atomics).  Fully
// interior nodes are stored plainly; tile-edge and halo nodes are added
// atomically (their buffer was zeroed one step earlier).
// Per plane z, separated by barriers:
//   1. flush plane z-2, store the prefetched C of plane z+2 (and vote whether it
//      is pure gas, C = -1 throughout the ring), prefetch C of plane z+3; the
//      pull of plane z is already in flight (FP64: its register loads go out here)
//   2. gradient and normals of plane z+1, or zeros where planes z..z+2 are pure gas
//   3. decode the pulled pairs, curvature (zero without the stencil where the normals
//      of planes z-1..z+1 are), collide, recolour, evaporate, store, push; a warp of
//      16-bit storage without red takes the red-free form of the collision; the pull
//      of plane z+1 goes out after the decode (16-bit storage, 32x4 tiles) or at the end
// ---------------------------------------------------------------------------
// slot of a push that leaves the tile sideways, by its (c_y, c_z); |c_y| + |c_z| <= 1
__host__ __device__ constexpr int side_slot(int dy, int dz) {
    return dz == 0 ? (dy == 0 ? 0 : (dy > 0 ? 1 : 2)) : (dz > 0 ? 3 : 4);
}
__host__ __device__ constexpr int slot_dy(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
__host__ __device__ constexpr int slot_dz(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }

__device__ __forceinline__ int wrap_near(int a, int n) {
    while (a < 0) a += n;
    while (a >= n) a -= n;
    return a;
}

// compile-time loop over lattice directions: f(std::integral_constant<int, I>)
// for I in [B, E); every c_i and w_i folds to a constant in the body
template <int B, int E, int STEP = 1, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + STEP, E, STEP>(f);
    }
}

// 4-byte asynchronous global->shared copies (completion tracked per thread)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N_>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N_) : "memory");
}

// Bulk asynchronous copies (the tensor-memory-access engine's 1-D form) into shared
// memory, completion counted in bytes on a shared-memory mbarrier.  Source and
// destination 16-byte aligned, sizes multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// one arrival that also announces `bytes` of copies to come in the current phase
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// the waiting thread may be suspended up to MBAR_SUSPEND_NS before the poll returns
// false, so that waiting warps sleep rather than take issue slots
constexpr unsigned MBAR_SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, "
        "p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "n"(MBAR_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// order this thread's earlier generic-proxy shared accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(smem)),
                 "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// try_wait polls before a wait is declared lost
constexpr int MBAR_POLLS = 1 << 16;

// Colour C = (rho_R - rho_B)/(rho_R + rho_B) of component densities a, b.  FP64
// divides.  FP32 takes the fast reciprocal, through the smaller fraction:
// C = 2 min(a, b)/(a + b) - 1 (or 1 - that), so that a pure or nearly pure phase
// (the smaller density below half an ulp of the sum) comes out exactly -1 or +1, as
// correctly rounded division gives, where a quotient of two equal numbers from the
// fast reciprocal may miss 1 by an ulp.  Uniform pure regions then have exactly zero
// colour gradient.
template <typename T>
__device__ __forceinline__ T colour_q(T a, T b) { return (a - b) / (a + b); }
// (1 + C)/2 = rho_R/(rho_R + rho_B): exactly 0 where there is no red
template <typename T>
__device__ __forceinline__ T liquid_fraction(T a, T b) { return a / (a + b); }
template <>
__device__ __forceinline__ float liquid_fraction<float>(float a, float b) { return __fdividef(a, a + b); }
template <>
__device__ __forceinline__ float colour_q<float>(float a, float b) {
    const float t = __fdividef(2.0f * fminf(a, b), a + b);
    return a < b ? t - 1.0f : 1.0f - t;
}

template <typename T>
__device__ __forceinline__ T inv_norm(T g2);
template <>
__device__ __forceinline__ float inv_norm<float>(float g2) { return rsqrtf(g2); }
template <>
__device__ __forceinline__ double inv_norm<double>(double g2) { return 1.0 / sqrt(g2); }
// smallest normal number of the compute type (below it a square is treated as zero)
template <typename T>
__device__ __forceinline__ constexpr T min_normal();
template <>
__device__ __forceinline__ constexpr float min_normal<float>() { return 1.17549435e-38f; }
template <>
__device__ __forceinline__ constexpr double min_normal<double>() { return 2.2250738585072014e-308; }

// Liquid column height h(x,y) = sum_z (1 + C)/2 = sum_z rho_R/rho of the current moments (Eq. (8))
// for instances whose sink is on in this step.  A block takes 32 columns with 8
// threads per column, each summing every 8th plane; the 8 partial sums are then
// added in a fixed order.
constexpr int HCOL_X = 32, HCOL_Z = 8;
template <typename T>
__global__ void __launch_bounds__(HCOL_X * HCOL_Z) k_column_height(const InstDev* __restrict__ insts,
                                                                   const StepGlobals* __restrict__ glob) {
    const InstDev& I = insts[blockIdx.y];
    const long long step = __ldcg(&glob->step);
    if (!(I.J0 > 0.0 && I.evap_start >= 0 && step >= I.evap_start) || I.hcol == nullptr) return;
    __shared__ T part[HCOL_Z][HCOL_X];
    const int c = blockIdx.x * HCOL_X + threadIdx.x;
    const unsigned nxy = (unsigned)I.nx * I.ny;
    if (blockIdx.x * HCOL_X >= nxy) return;  // whole block past the last column
    const T* __restrict__ rho = (const T*)I.rho[step % 3];
    const unsigned N = (unsigned)I.N;
    T h = 0;
    if (c < (int)nxy)
        for (int z = threadIdx.y; z < I.nz; z += HCOL_Z) {
            const T a = rho[(unsigned)z * nxy + c], b = rho[N + (unsigned)z * nxy + c];
            h += liquid_fraction<T>(a, b);
        }
    part[threadIdx.y][threadIdx.x] = h;
    __syncthreads();
    if (threadIdx.y == 0 && c < (int)nxy) {
        T s = part[0][threadIdx.x];
        for (int k = 1; k < HCOL_Z; ++k) s += part[k][threadIdx.x];
        ((T*)I.hcol)[c] = s;
    }
}

// MINB: resident blocks per SM the register budget is sized for (4 blocks of 128
// threads: 128 registers a thread; 5 blocks: 96), a choice of the tiling autotuner
// BULK (32- and 16-bit storage, every lattice nx % 4 == 0): the pull of a plane
// arrives as bulk row copies, one per (direction and component, tile row): the
// tile's row of that direction's source plane, widened by 4 columns on the side
// it is shifted to so that it starts and ends on 16-byte boundaries (split in two
// where it crosses the periodic x boundary), landing so that the node reads its
// element at column 4 - c_x of the staged row.  Otherwise per-element 4-byte
// asynchronous copies.
// EP: esoteric-pull in-place storage (one buffer and the wall ghost slots; the
// slot rules are ep_load / ep_store / ep_outflow); per-element or register pulls.
template <class S, int TX, int TY, int MINB, bool BULK, bool EP>
__global__ void __launch_bounds__(TX * TY, MINB)
    k_stream_collide(const InstDev* __restrict__ insts, const TileDesc* __restrict__ tiles,
                     StepGlobals* __restrict__ glob) {
    using T = typename S::T;
    using E = typename S::E;
    static_assert(TX == 32, "a warp is one row of the tile");
    constexpr int NT = TX * TY;
    constexpr int HX2 = TX + 4, HY2 = TY + 4, HX1 = TX + 2, HY1 = TY + 2;
    static_assert(NT >= 2 * TX + 2 * HY1, "one thread per halo slot of the flush");
    constexpr int NPF = (HX2 * HY2 + NT - 1) / NT;  // C-halo slots per thread
    __shared__ T sC[3][HY2][HX2];
    using V4 = typename Vec4<T>::type;
    __shared__ V4 sN[3][HY1][HX1];
    __shared__ V4 sG[2][TY][TX];
    // next-step moments of one plane by source row offset: [c_y + 1][comp][row + 1][x]
    __shared__ T sB[3][2][HY1][TX];
    // pushes that leave the tile sideways: [source plane ring][left/right][slot][comp][row]
    __shared__ T sE[3][2][5][2][TY];
    __shared__ double sRed[NT / 32][3];
    __shared__ int sErr;
    // pulled populations of the next plane (16- and 32-bit storage; FP64 keeps them
    // in registers): per-element copies [19 WORDS][NT] words, or bulk row copies
    // [NBUF][19 WORDS][TY][RW] words; 16-bit bulk staging is double-buffered, so the
    // copies of a plane go out a whole plane ahead
    constexpr bool ASYNC = S::WORDS > 0;
    // next plane's pull issued mid-plane: 16-bit storage on 32x4 tiles (on 32x8 tiles it
    // spilled and ran slower)
    constexpr bool EARLY_PULL = ASYNC && !BULK && S::WORDS == 1 && TY == 4;
    static_assert(!BULK || ASYNC, "bulk staging needs word storage");
    static_assert(!(BULK && EP), "in-place storage pulls element by element");
    constexpr int RW = TX + 8;  // staged row: the tile row and 4 columns each side
    constexpr int NBUF = (BULK && S::WORDS == 1) ? 2 : 1;
    constexpr int BUFW = 19 * S::WORDS * TY * RW;  // words of one bulk stage buffer
    extern __shared__ __align__(128) unsigned stage_dyn[];
    __shared__ __align__(8) unsigned long long sBar[NBUF];
    // bulk copies of an interior plane, per (direction-component, row) pair: source word
    // offset without the plane term, staged word offset, first and second segment
    // (source column, words) - the second empty unless the row wraps in x
    constexpr int NPAIR = BULK ? 19 * S::WORDS * TY : 1;
    __shared__ int4 sCopy[NPAIR];
    __shared__ int2 sCopy2[NPAIR];

    const TileDesc td = tiles[blockIdx.x];
    const InstDev& Ig = insts[td.inst];
    const int nx = Ig.nx, ny = Ig.ny, nz = Ig.nz, top_bc = Ig.top_bc;
    const unsigned nxy = (unsigned)nx * ny;
    const unsigned N = (unsigned)Ig.N;
    const unsigned cs = 19u * N;
    const long long step = __ldcg(&glob->step);
    const int pa = (int)(step & 1);
    const int pr = (int)(step % 3);
    // two buffers: read one, write the other.  In place both name the one buffer: each
    // slot is read and written by one node of the step, its pull loads (phase 1 or the
    // previous plane) are separated from its stores (phase 3) by block barriers, and the
    // outflow read of phase 3 touches a slot that no store of that node writes
    const E* __restrict__ src = (const E*)Ig.pop[pa];
    E* __restrict__ dst = (E*)Ig.pop[pa ^ 1];
    E* gslot = (E*)Ig.ghost;  // in place: the wall ghost slots
    const unsigned gcs = 10u * nxy;  // component stride of the ghost slots
    const T* __restrict__ rho_r = (const T*)Ig.rho[pr];
    T* __restrict__ rho_w = (T*)Ig.rho[(pr + 1) % 3];
    T* __restrict__ rho_z = (T*)Ig.rho[(pr + 2) % 3];
    const T* __restrict__ fext = (const T*)Ig.fext;
    const unsigned* __restrict__ tflag = Ig.tflag ? tflag_of(Ig, (int)(step & 1)) : nullptr;
    const double* __restrict__ cotm = Ig.cot;
    const T* __restrict__ hcolm = (const T*)Ig.hcol;
    double* accp = Ig.acc;
    int* errp = Ig.err;
    const int t8x = Ig.t8x, t8y = Ig.t8y;

    const int x0 = td.x0, y0 = td.y0, z0 = td.z0, z1 = td.z1;
    const int tw = min(TX, nx - x0), th = min(TY, ny - y0);
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const bool active = tx < tw && ty < th;
    const unsigned lanes = __ballot_sync(0xffffffffu, active);  // a prefix of the row
    const int x = x0 + tx, y = y0 + ty;

    const T rho0 = (T)Ig.rho0, itR = T(1) / (T)Ig.tau_R, itB = T(1) / (T)Ig.tau_B;
    const unsigned step_key = hash32((unsigned)step * 0x9e3779b9u + (unsigned)td.inst);
    const T beta = (T)Ig.beta;
    const T hsig = T(0.5) * (T)Ig.sigma;
    const T bfx = (T)Ig.body[0], bfy = (T)Ig.body[1], bfz = (T)Ig.body[2];
    const double h0 = accp[1];
    const bool evap_on = Ig.J0 > 0.0 && Ig.evap_start >= 0 && step >= Ig.evap_start && h0 > 0.0;
    const T J0 = (T)Ig.J0, Kk = (T)Ig.K, inv_h0 = evap_on ? (T)(1.0 / h0) : T(0);

    auto ring = [](int q) { return ((q % 3) + 3) % 3; };
    auto colour = [&](unsigned n) { return colour_q<T>(rho_r[n], rho_r[N + n]); };
    // wetting ghost colour below z = 0 (flat-wall geometric form, D2Q9 weights)
    auto ghost = [&](int gx, int gy) {
        T ax = 0, ay = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int k = (dx != 0) + (dy != 0);
                const T w = k == 0 ? T(4.0 / 9.0) : (k == 1 ? T(1.0 / 9.0) : T(1.0 / 36.0));
                const T c = colour((unsigned)wrap_near(gy + dy, ny) * nx + wrap_near(gx + dx, nx));
                ax += w * dx * c;
                ay += w * dy * c;
            }
        ax *= T(3);
        ay *= T(3);
        T g = colour((unsigned)gy * nx + gx) + (T)cotm[gy * nx + gx] * sqrt(ax * ax + ay * ay);
        return g > T(1) ? T(1) : (g < T(-1) ? T(-1) : g);
    };

    const T hcol = (evap_on && active) ? hcolm[y * nx + x] : T(0);
    // coupling-tile flags of this thread's column for the 8-plane slabs of the chunk,
    // read once (bit s: slab (z0 >> 3) + s), so that no plane waits on a flag load
    unsigned tbits = 0u;
    if (tflag != nullptr && active) {
        const int s0 = z0 >> 3, s1 = min((z1 - 1) >> 3, s0 + 31);
        for (int sl = s0; sl <= s1; ++sl)
            if (tflag[(sl * t8y + (y >> 3)) * t8x + (x >> 3)]) tbits |= 1u << (sl - s0);
    }

    for (int s = tid; s < 3 * 2 * HY1 * TX; s += NT) (&sB[0][0][0][0])[s] = T(0);
    if (tid == 0) sErr = 0;
    if constexpr (BULK) {
        if (tid < NBUF) mbar_init(&sBar[tid], NT);  // every thread arrives with the bytes it copies
    }

    // C of plane p into the ring over the tile plus 2 cells (synchronous form)
    auto loadC = [&](int p) {
        if (p < -1 || p > nz) return;
        const int r = ring(p);
        const int pz = p >= nz ? nz - 1 : p;
        for (int s = tid; s < HX2 * HY2; s += NT) {
            const int sy = s / HX2, sx = s - sy * HX2;
            if (sx > tw + 3 || sy > th + 3) continue;
            const int gx = wrap_near(x0 - 2 + sx, nx), gy = wrap_near(y0 - 2 + sy, ny);
            sC[r][sy][sx] = p < 0 ? ghost(gx, gy) : colour((unsigned)pz * nxy + (unsigned)gy * nx + gx);
        }
    };
    // prefetched form for planes p >= 0: raw moments into registers now, colour into the ring later;
    // slot tid + k NT of the ring plane has the same in-plane source offset on every plane
    unsigned pfo[NPF];
#pragma unroll
    for (int k = 0; k < NPF; ++k) {
        const int s = tid + k * NT;
        const int sy = s / HX2, sx = s - sy * HX2;
        pfo[k] = ~0u;
        if (s < HX2 * HY2 && sx <= tw + 3 && sy <= th + 3)
            pfo[k] = (unsigned)wrap_near(y0 - 2 + sy, ny) * nx + wrap_near(x0 - 2 + sx, nx);
    }
    T pfa[NPF], pfb[NPF];
    int pfp = -100;
    auto prefetchC = [&](int p) {
        pfp = p;
        if (p < 0 || p > nz) return;
        const unsigned pb = (unsigned)(p >= nz ? nz - 1 : p) * nxy;
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            pfa[k] = T(1);
            pfb[k] = T(0);
            if (pfo[k] != ~0u) {
                pfa[k] = rho_r[pb + pfo[k]];
                pfb[k] = rho_r[N + pb + pfo[k]];
            }
        }
    };
    // commit the prefetched plane; true when every slot this thread wrote is pure gas (C = -1)
    auto commitC = [&]() -> bool {
        if (pfp < 0 || pfp > nz) return false;
        T* ringp = &sC[ring(pfp)][0][0];
        bool gas = true;
#pragma unroll
        for (int k = 0; k < NPF; ++k)
            if (pfo[k] != ~0u) {
                const T c = colour_q<T>(pfa[k], pfb[k]);
                ringp[tid + k * NT] = c;
                gas = gas && c == T(-1);
            }
        return gas;
    };
    // gradient and unit normal of plane q over the tile plus 1 cell: every thread
    // takes its own node, the first 2 HX1 + 2 TY threads one node of the ring around
    // the tile as well (slots as indices into a [HY1][HX1] plane)
    static_assert(NT >= 2 * HX1 + 2 * TY, "one thread per ring node of the normals");
    int nring = -1;
    {
        int sx = -1, sy = -1;
        if (tid < HX1) {
            sx = tid, sy = 0;
        } else if (tid < 2 * HX1) {
            sx = tid - HX1, sy = th + 1;
        } else if (tid < 2 * HX1 + TY) {
            sx = 0, sy = 1 + tid - 2 * HX1;
        } else if (tid < 2 * HX1 + 2 * TY) {
            sx = tw + 1, sy = 1 + tid - 2 * HX1 - TY;
        }
        if (sx >= 0 && sx <= tw + 1 && sy <= th + 1) nring = sy * HX1 + sx;
    }
    auto normal_at = [&](int rm, int r0, int rp, int sy, int sx, T& gx, T& gy, T& gz) {
        gx = gy = gz = T(0);
        static_for<1, 19>([&](auto I_) {
            constexpr int i = decltype(I_)::value;
            const int rr = cz(i) < 0 ? rm : (cz(i) > 0 ? rp : r0);
            const T c = sC[rr][sy + 1 + cy(i)][sx + 1 + cx(i)];
            constexpr T w = (T)wq(i);
            if constexpr (cx(i) != 0) gx += w * cx(i) * c;
            if constexpr (cy(i) != 0) gy += w * cy(i) * c;
            if constexpr (cz(i) != 0) gz += w * cz(i) * c;
        });
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
        return nn;
    };
    // skip: the colour of planes q-1..q+1 is -1 over the whole ring, so every gradient and
    // normal of plane q is exactly zero (opposite directions cancel term by term)
    auto computeN = [&](int q, bool skip) {
        const int rq = ring(q);
        if (skip) {
            V4 zero;
            zero.x = zero.y = zero.z = zero.w = T(0);
            if (active) {
                sN[rq][ty + 1][tx + 1] = zero;
                sG[q & 1][ty][tx] = zero;
            }
            if (nring >= 0) (&sN[rq][0][0])[nring] = zero;
        } else if (q >= 0 && q < nz) {
            const int rm = ring(q - 1), r0 = ring(q), rp = ring(q + 1);
            T gx, gy, gz;
            if (active) {
                sN[rq][ty + 1][tx + 1] = normal_at(rm, r0, rp, ty + 1, tx + 1, gx, gy, gz);
                V4 G;
                G.x = gx;
                G.y = gy;
                G.z = gz;
                G.w = T(0);
                sG[q & 1][ty][tx] = G;
            }
            if (nring >= 0) {
                const int sy = nring / HX1, sx = nring - sy * HX1;
                (&sN[rq][0][0])[nring] = normal_at(rm, r0, rp, sy, sx, gx, gy, gz);
            }
        } else if (q == -1 || q == nz) {
            // outside the fluid the normal copies the nearest fluid plane
            const int rf = ring(q == -1 ? 0 : nz - 1);
            for (int s = tid; s < HX1 * HY1; s += NT) (&sN[rq][0][0])[s] = (&sN[rf][0][0])[s];
        }
    };

    // per-thread partial budgets in the compute type; FP64 from the block sum on
    T evap_sum = 0, top_in = 0, top_out = 0;
    int err = 0;

    // next-step moment shares of this thread's column for planes z-1 and z: [c_y + 1][comp]
    T acm[3][2], ac0[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) acm[d][0] = acm[d][1] = ac0[d][0] = ac0[d][1] = T(0);

    // in-plane offset of this thread's halo node in the flush (halo rows, then halo columns)
    unsigned hoff = ~0u;
    if (tid < 2 * TX) {
        const int side = tid / TX, hx = tid - side * TX;
        if (hx < tw) hoff = (unsigned)wrap_near(side ? y0 + th : y0 - 1, ny) * nx + (x0 + hx);
    } else if (tid < 2 * TX + 2 * HY1) {
        const int k2 = tid - 2 * TX;
        const int side = k2 / HY1, sy = k2 - side * HY1;
        if (sy <= th + 1)
            hoff = (unsigned)wrap_near(y0 - 1 + sy, ny) * nx + wrap_near(side ? x0 + tw : x0 - 1, nx);
    }
    // flush the completed plane q (its row shares are in sB) to global memory
    auto flush = [&](int q) {
        if (q < z0 - 1 || q < 0 || q >= nz) return;  // nothing was pushed below the halo plane
        const bool own = q >= z0 && q < z1;
        if (active) {
            const T a0 = sB[0][0][ty + 1][tx] + sB[1][0][ty + 1][tx] + sB[2][0][ty + 1][tx];
            const T a1 = sB[0][1][ty + 1][tx] + sB[1][1][ty + 1][tx] + sB[2][1][ty + 1][tx];
            const unsigned n = (unsigned)q * nxy + (unsigned)y * nx + x;
            const bool interior = own && tx > 0 && tx < tw - 1 && ty > 0 && ty < th - 1 &&
                                  !(q == z0 && z0 > 0) && !(q == z1 - 1 && z1 < nz);
            if (interior) {
                rho_w[n] = a0;
                rho_w[N + n] = a1;
            } else {
                atomicAdd(rho_w + n, a0);
                atomicAdd(rho_w + N + n, a1);
                if (own) {
                    rho_z[n] = T(0);
                    rho_z[N + n] = T(0);
                }
            }
        }
        if (tid < 2 * TX) {
            // halo rows y0-1 and y0+th: only row 0 pushes down, only row th-1 up
            const int side = tid / TX, hx = tid - side * TX;
            if (hoff != ~0u) {
                const T a0 = side ? sB[2][0][th + 1][hx] : sB[0][0][0][hx];
                const T a1 = side ? sB[2][1][th + 1][hx] : sB[0][1][0][hx];
                const unsigned n = (unsigned)q * nxy + hoff;
                atomicAdd(rho_w + n, a0);
                atomicAdd(rho_w + N + n, a1);
            }
        } else if (tid < 2 * TX + 2 * HY1) {
            // halo columns x0-1 and x0+tw: sideways pushes of the edge lanes, planes q-1..q+1
            const int k2 = tid - 2 * TX;
            const int side = k2 / HY1, sy = k2 - side * HY1;
            if (hoff != ~0u) {
                T a0 = 0, a1 = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int ys = sy - 1 - slot_dy(k), sp = q - slot_dz(k);
                    if (ys >= 0 && ys < th && sp >= z0 && sp < z1) {
                        const int r = ring(sp);
                        a0 += sE[r][side][k][0][ys];
                        a1 += sE[r][side][k][1][ys];
                    }
                }
                const unsigned n = (unsigned)q * nxy + hoff;
                atomicAdd(rho_w + n, a0);
                atomicAdd(rho_w + N + n, a1);
            }
        }
    };
    // hand the completed share of plane z-1 to the row reduction, then move the shares up one plane
    auto retire = [&](T (&up)[3][2]) {
        if (active) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sB[d][0][ty + d][tx] = acm[d][0];
                sB[d][1][ty + d][tx] = acm[d][1];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acm[d][0] = ac0[d][0];
            acm[d][1] = ac0[d][1];
            ac0[d][0] = up[d][0];
            ac0[d][1] = up[d][1];
        }
    };

    // neighbour columns of this thread (pull sources) as row/column offsets
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const unsigned rowm = (unsigned)ym * nx, row0 = (unsigned)y * nx, rowp = (unsigned)yp * nx;

    // in place: where direction i of this thread's node of plane z is read (interior
    // planes: no ghost slot, no gas inflow)
    auto pull_ep = [&](int z, auto I_, auto EDGE_) -> PopLoc {
        constexpr int i = decltype(I_)::value;
        if constexpr (decltype(EDGE_)::value) {
            PopLoc L;
            ep_load(i, x, y, z, pa, nx, ny, nz, top_bc, L);
            return L;
        } else {
            const unsigned node = (unsigned)z * nxy + row0 + x;
            if constexpr (i == 0) return {node, false};
            if constexpr (i & 1) return {(pa ? (unsigned)i : (unsigned)(i + 1)) * N + node, false};
            // the even member comes from n + c_{i-1}, the two-buffer source node
            const int sx = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : x);
            const unsigned row = cy(i) == 1 ? rowm : (cy(i) == -1 ? rowp : row0);
            return {(pa ? (unsigned)i : (unsigned)(i - 1)) * N + (unsigned)(z - cz(i)) * nxy + row + sx, false};
        }
    };
    // element of direction i that streams into this thread's node of plane z; EDGE:
    // z may be the bottom or the top plane (interior planes need no boundary test)
    auto pull_index = [&](int z, int i, auto EDGE_) -> unsigned {
        const int sz = z - cz(i);
        if constexpr (decltype(EDGE_)::value) {
            const unsigned node = (unsigned)z * nxy + row0 + x;
            if (sz < 0 || (sz >= nz && top_bc == 0)) return (unsigned)opp(i) * N + node;  // bounce-back
            if (sz >= nz) return (unsigned)i * N + node;  // replaced by the gas inflow
        }
        const int sx = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : x);
        const unsigned row = cy(i) == 1 ? rowm : (cy(i) == -1 ? rowp : row0);
        return (unsigned)i * N + (unsigned)sz * nxy + row + sx;
    };
    // asynchronous pull of plane z into the stage (one commit group per plane);
    // every slot is read and written by its own thread only
    auto issue_pull_t = [&](int z, auto EDGE_) {
        if (active && z < z1) {
            unsigned* st = stage_dyn + tid;
            static_for<0, 19>([&](auto I_) {
                constexpr int i = decltype(I_)::value;
                const E* base = src;
                unsigned k, kc = cs;
                (void)kc;
                if constexpr (EP) {
                    const PopLoc L = pull_ep(z, I_, EDGE_);
                    k = L.k;
                    if (L.ghost) {
                        base = gslot;
                        kc = gcs;
                    }
                } else {
                    k = pull_index(z, i, EDGE_);
                }
                if constexpr (S::WORDS == 2) {
                    cp_async4(st + (size_t)i * NT, base + k);
                    cp_async4(st + (size_t)(19 + i) * NT, base + kc + k);
                } else {
                    cp_async4(st + (size_t)i * NT, (const unsigned*)base + k);
                }
            });
        }
        cp_async_commit();
    };
    auto issue_pull = [&](int z) {
        if (z == 0 || z == nz - 1)
            issue_pull_t(z, std::true_type{});
        else
            issue_pull_t(z, std::false_type{});
    };
    // bulk pull of plane z (called by every thread between barriers, the stage free):
    // the (direction-component, row) pairs are spread over the block, each thread
    // arriving on the mbarrier with the bytes of its copies.  A row shifted by c_x = +1
    // is read from 4 columns left of the tile and lands at staged column 0, one with
    // c_x = -1 or 0 from the tile's first column landing at column 4; a bounced-back
    // pair (z = 0 or the top wall) copies the opposite direction's own row of plane z
    // to column 4; a gas-inflow pair copies its own row of plane z in the shifted
    // layout (the value is replaced, but every staged slot read was written).
    // Interior planes take the per-pair offsets tabulated in shared memory.
    auto pair_copy = [&](int p, int z, bool edge, int& sofs, int& dofs, int& cA, int& nA, int& cB, int& nB) {
        const int j = p / th, r = p - j * th;
        const int i = j >= 19 ? j - 19 : j, comp = j >= 19 ? 1 : 0;
        int sz = z - cz(i), di = i, ys = y0 + r - cy(i), sh = cx(i);
        if (edge && (sz < 0 || (sz >= nz && top_bc == 0))) {
            sz = z;
            di = opp(i);
            ys = y0 + r;
            sh = 0;
        } else if (edge && sz >= nz) {
            sz = z;
            ys = y0 + r;
        }
        ys = wrap_near(ys, ny);
        sofs = (int)(comp * cs + (unsigned)di * N + (unsigned)ys * nx) + (sz - z) * (int)nxy;
        const int len = sh != 0 ? tw + 4 : tw;
        const int d = sh > 0 ? 0 : 4;
        dofs = (j * TY + r) * RW + d;
        int c0 = sh > 0 ? x0 - 4 : x0;
        if (c0 < 0) c0 += nx;
        cA = c0;
        nA = min(len, nx - c0);
        cB = 0;
        nB = len - nA;
    };
    if constexpr (BULK) {
        for (int p = tid; p < 19 * S::WORDS * th; p += NT) {
            int sofs, dofs, cA, nA, cB, nB;
            pair_copy(p, 1, false, sofs, dofs, cA, nA, cB, nB);
            sCopy[p] = make_int4(sofs, dofs, cA, nA);
            sCopy2[p] = make_int2(cB, nB);
        }
    }
    auto issue_bulk = [&](int z) {
        if (z >= z1) return;
        const int b = (z - z0) % NBUF;
        unsigned* stg = stage_dyn + (size_t)b * BUFW;
        const unsigned* srcz = (const unsigned*)src + (size_t)z * nxy;
        const bool edge = z == 0 || z == nz - 1;
        unsigned bytes = 0;
        bool fenced = false;
        for (int p = tid; p < 19 * S::WORDS * th; p += NT) {
            if (!fenced) {
                fence_proxy_async();
                fenced = true;
            }
            int sofs, dofs, cA, nA, cB, nB;
            if (edge) {
                pair_copy(p, z, true, sofs, dofs, cA, nA, cB, nB);
            } else {
                const int4 a = sCopy[p];
                const int2 b = sCopy2[p];
                sofs = a.x;
                dofs = a.y;
                cA = a.z;
                nA = a.w;
                cB = b.x;
                nB = b.y;
            }
            const unsigned* row = srcz + sofs;
            bulk_g2s(stg + dofs, row + cA, (unsigned)nA * 4u, &sBar[b]);
            if (nB > 0) bulk_g2s(stg + dofs + nA, row + cB, (unsigned)nB * 4u, &sBar[b]);
            bytes += (unsigned)(nA + nB) * 4u;
        }
        mbar_arrive_expect(&sBar[b], bytes);
    };
    // wait for the bulk pull of plane z (bounded: a lost wait is reported): plane z sits
    // in buffer (z - z0) % NBUF, whose barrier completes one phase per plane it carries
    auto wait_bulk = [&](int z) {
        const int k = z - z0;
        const unsigned parity = (unsigned)(k / NBUF) & 1u;
        int polls = 0;
        while (!mbar_try_wait(&sBar[k % NBUF], parity)) {
            if (++polls >= MBAR_POLLS) {
                err |= ERR_TIMEOUT;
                break;
            }
        }
    };

    // ---- prologue: C planes and normals below the first plane ----
    if (z0 == 0) {
        loadC(-1);
        loadC(0);
        loadC(1);
        __syncthreads();
        computeN(0, false);
        __syncthreads();
        computeN(-1, false);
    } else {
        loadC(z0 - 2);
        loadC(z0 - 1);
        loadC(z0);
        __syncthreads();
        computeN(z0 - 1, false);
        __syncthreads();
        loadC(z0 + 1);
        __syncthreads();
        computeN(z0, false);
    }
    prefetchC(z0 + 2);
    if constexpr (ASYNC && !BULK) issue_pull(z0);
    __syncthreads();
    if constexpr (BULK) {
        issue_bulk(z0);
        if constexpr (NBUF == 2) issue_bulk(z0 + 1);
    }

    // block-uniform plane flags, shifted up one plane per iteration: gasC bit k = the
    // colour ring of plane z+2-k is -1 throughout (planes the loop committed); zeroN bit
    // k = the normals (and core gradient) of plane z+1-k were skipped as zero
    unsigned gasC = 0u, zeroN = 0u;
    for (int z = z0; z < z1; ++z) {
        const unsigned node = (unsigned)z * nxy + row0 + x;
        const int rz[3] = {ring(z - 1), ring(z), ring(z + 1)};  // ring slots of planes z-1, z, z+1
        // ---- phase 1: raw pull loads of plane z, flush, C ring upkeep ----
        E rawR[ASYNC ? 1 : 19], rawB[ASYNC ? 1 : 19];
        if constexpr (ASYNC) {
            // plane z was issued at the end of the previous plane (or before the loop)
        } else if (active) {
            static_for<0, 19>([&](auto I_) {
                constexpr int i = decltype(I_)::value;
                if constexpr (EP) {
                    const PopLoc L = pull_ep(z, I_, std::true_type{});
                    const E* base = L.ghost ? gslot : src;
                    const unsigned kc = L.ghost ? gcs : cs;
                    rawR[i] = base[L.k];
                    rawB[i] = base[kc + L.k];
                } else {
                    const unsigned k = pull_index(z, i, std::true_type{});
                    rawR[i] = __ldg(src + k);
                    rawB[i] = __ldg(src + cs + k);
                }
            });
        }
        flush(z - 2);
        const bool cgas = commitC();
        prefetchC(z + 3);
        gasC = (gasC << 1) | (__syncthreads_and(cgas) ? 1u : 0u);
        // ---- phase 2: normals of plane z+1 (zero without computing where planes z..z+2 are pure gas) ----
        const bool skipN = (gasC & 7u) == 7u;
        computeN(z + 1, skipN);
        zeroN = (zeroN << 1) | (skipN ? 1u : 0u);
        __syncthreads();
        // ---- phase 3: decode, collide, recolour, evaporate, store, push ----
        T ac1[3][2] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};  // shares of plane z+1
        // EDGE: the bottom or the top plane, where streaming meets the walls or the gas
        auto phase3 = [&](auto EDGE_) {
            constexpr bool EDGE = decltype(EDGE_)::value;
            T Fi[19];
            T rR = 0, rho = 0, jx = 0, jy = 0, jz = 0;
            const bool top_gas = EDGE && z == nz - 1 && top_bc == 1;
            if constexpr (BULK)
                wait_bulk(z);  // plane z landed
            else if constexpr (ASYNC)
                cp_async_wait<0>();
            static_for<0, 19>([&](auto I_) {
                constexpr int i = decltype(I_)::value;
                // total F_i and f^R_i (a bounced-back element has the same weight: w_opp(i) = w_i)
                T F, r;
                if constexpr (BULK) {
                    // column of this node's source in the staged row; a bounced-back
                    // element sits in the node's own column
                    int o = 4 - cx(i);
                    if constexpr (EDGE && cz(i) > 0) o = z == 0 ? 4 : o;
                    if constexpr (EDGE && cz(i) < 0) o = (z == nz - 1 && top_bc == 0) ? 4 : o;
                    const unsigned* st = stage_dyn + (size_t)((z - z0) % NBUF) * BUFW + (size_t)ty * RW + tx + o;
                    if constexpr (S::WORDS == 2)
                        S::decode_total(__uint_as_float(st[(size_t)i * TY * RW]),
                                        __uint_as_float(st[(size_t)(19 + i) * TY * RW]), (T)wq(i), rho0, F, r);
                    else
                        S::decode_word_total(st[(size_t)i * TY * RW], (T)wq(i), rho0, F, r);
                } else if constexpr (ASYNC) {
                    const unsigned* st = stage_dyn + tid;
                    if constexpr (S::WORDS == 2)
                        S::decode_total(__uint_as_float(st[(size_t)i * NT]),
                                        __uint_as_float(st[(size_t)(19 + i) * NT]), (T)wq(i), rho0, F, r);
                    else
                        S::decode_word_total(st[(size_t)i * NT], (T)wq(i), rho0, F, r);
                } else {
                    S::decode_total(rawR[i], rawB[i], (T)wq(i), rho0, F, r);
                }
                if (top_gas && cz(i) < 0) {
                    // pure-gas equilibrium streams in; what streamed out is booked
                    r = T(0);
                    F = (T)wq(i) * rho0;
                    top_in += F;
                }
                rR += r;
                rho += F;
                Fi[i] = F;
                if constexpr (cx(i) != 0) jx += cx(i) * Fi[i];
                if constexpr (cy(i) != 0) jy += cy(i) * Fi[i];
                if constexpr (cz(i) != 0) jz += cz(i) * Fi[i];
            });
            if (top_gas) {
                static_for<0, 19>([&](auto I_) {
                    constexpr int i = decltype(I_)::value;
                    if constexpr (cz(i) > 0) {
                        T r, b;
                        if constexpr (EP) {
                            const PopLoc L = ep_outflow(i, x, y, pa, nx, ny, nz);
                            S::load(L.ghost ? gslot : src, L.ghost ? gcs : cs, L.k, (T)wq(i), rho0, r, b);
                        } else {
                            S::load(src, cs, (unsigned)i * N + node, (T)wq(i), rho0, r, b);
                        }
                        top_out += r + b;
                    }
                });
            }
            // 16-bit storage: this thread has read its staged slots, so the pull of the next
            // plane goes out now, a collision and a store earlier than at the end of the plane
            // (FP16 fused kernel 0.91 -> 0.87 ms on the 512x256x128 lattice; FP32, whose
            // collision holds twice the staged words' worth of registers, gained nothing there
            // and lost 2 % on the 64-lattice batch, so it issues at the end of the plane)
            if constexpr (EARLY_PULL) issue_pull(z + 1);
            T kap = 0;
            if ((zeroN & 7u) != 7u) {  // else every normal of planes z-1..z+1 is zero
                static_for<1, 19>([&](auto I_) {
                    constexpr int i = decltype(I_)::value;
                    const V4 nn = sN[rz[cz(i) + 1]][ty + 1 + cy(i)][tx + 1 + cx(i)];
                    T d = 0;
                    if constexpr (cx(i) != 0) d += cx(i) * nn.x;
                    if constexpr (cy(i) != 0) d += cy(i) * nn.y;
                    if constexpr (cz(i) != 0) d += cz(i) * nn.z;
                    kap += (T)wq(i) * d;
                });
            }
            kap *= T(-3);
            const V4 G = sG[z & 1][ty][tx];
            const T Gx = G.x, Gy = G.y, Gz = G.z;
            T Fx = hsig * kap * Gx + bfx, Fy = hsig * kap * Gy + bfy, Fz = hsig * kap * Gz + bfz;
            if ((tbits >> ((z >> 3) - (z0 >> 3))) & 1u) {
                const T* fe = fext + 3 * (size_t)node;
                Fx += fe[0];
                Fy += fe[1];
                Fz += fe[2];
            }
            const T rB = rho - rR;
            if (!(rho > T(0))) err |= ERR_NAN;
            const T irho = T(1) / rho;
            const T ux = (jx + T(0.5) * Fx) * irho, uy = (jy + T(0.5) * Fy) * irho,
                    uz = (jz + T(0.5) * Fz) * irho;
            const T phi = rR * irho;
            const T omega = phi * itR + (rB * irho) * itB;
            const T usq = ux * ux + uy * uy + uz * uz;
            const T uF = ux * Fx + uy * Fy + uz * Fz;
            const T gsrc = T(1) - T(0.5) * omega;
            const T g2 = Gx * Gx + Gy * Gy + Gz * Gz;
            const bool hasg = g2 > T(1e-16);
            // 1/|G| wherever |G| is a normal number; the unit vector of the recolouring
            // takes it above the threshold only, the sink takes |G| itself (Eq. (8))
            const T ign = g2 > min_normal<T>() ? inv_norm<T>(g2) : T(0);
            const T ig = hasg ? ign : T(0);
            const T coef = beta * (rR * rB * irho);
            T dm = 0;
            if (evap_on) {
                const T ht = hcol * inv_h0;
                if (ht > T(0)) dm = J0 / (Kk + ht) * T(0.5) * (g2 * ign);
            }
            const T rGx = Gx * ig, rGy = Gy * ig, rGz = Gz * ig;
            const T base0 = T(1) - T(1.5) * usq;
            const T omc = T(1) - omega;
            // recolouring weight beta (rho_R rho_B / rho) w_i / |c_i| of the two direction classes
            const T cw_axis = coef * T(1.0 / 18.0), cw_diag = coef * T(1.0 / 36.0 / 1.4142135623730951);
            // post = the colour-blind post-collision population of direction i;
            // cG = c_i . G / |G| (sign included).  RED0: the warp's nodes hold no red
            // (rho_R = 0 exactly), so phi = 0 and the recolouring weight is 0: every red
            // population leaves as 0, the blue one as post, and the sink takes nothing
            auto emit = [&](auto I_, T post, T cG, auto RED0_) {
                constexpr int i = decltype(I_)::value;
                constexpr bool R0 = decltype(RED0_)::value;
                constexpr T w = (T)wq(i);
                constexpr bool axis = (cx(i) != 0) + (cy(i) != 0) + (cz(i) != 0) == 1;
                T rq, bq;
                if constexpr (R0) {
                    rq = T(0);
                    bq = post;
                    unsigned k = (unsigned)i * N + node;
                    if constexpr (EP && i != 0) {  // interior planes: no ghost slot
                        if constexpr (i & 1) {
                            const int tx_ = cx(i) == 1 ? xp : (cx(i) == -1 ? xm : x);
                            const unsigned trow = cy(i) == 1 ? rowp : (cy(i) == -1 ? rowm : row0);
                            k = (pa ? (unsigned)(i + 1) : (unsigned)i) * N + (unsigned)(z + cz(i)) * nxy + trow + tx_;
                        } else {
                            k = (pa ? (unsigned)(i - 1) : (unsigned)i) * N + node;
                        }
                    }
                    S::store_gas(dst, cs, k, w, rho0, bq);
                } else {
                    T r = phi * post;
                    if constexpr (i != 0) r += (axis ? cw_axis : cw_diag) * cG;
                    T b = post - r;
                    if (i == 0 && evap_on) {
                        T d = dm > r ? r : dm;
                        d = d < T(0) ? T(0) : d;
                        r -= d;
                        b += d;
                        evap_sum += d;
                    }
                    if constexpr (i == 0) {  // the sink's population: stochastic rounding in 16-bit storage
                        S::store_sr(dst, cs, node, w, rho0, r, b, rq, bq, hash32(node ^ step_key));
                    } else if constexpr (EP) {
                        // in place: the odd member goes to its destination n + c_i (a ghost slot
                        // beyond a wall or the gas top), the even member stays at its node
                        if constexpr (i & 1) {
                            if (EDGE && (z + cz(i) < 0 || z + cz(i) >= nz)) {
                                const PopLoc L = ep_store(i, x, y, z, pa, nx, ny, nz);
                                S::store(gslot, gcs, L.k, w, rho0, r, b, rq, bq);
                            } else {
                                const int tx_ = cx(i) == 1 ? xp : (cx(i) == -1 ? xm : x);
                                const unsigned trow = cy(i) == 1 ? rowp : (cy(i) == -1 ? rowm : row0);
                                S::store(dst, cs,
                                         (pa ? (unsigned)(i + 1) : (unsigned)i) * N + (unsigned)(z + cz(i)) * nxy + trow + tx_,
                                         w, rho0, r, b, rq, bq);
                            }
                        } else {
                            S::store(dst, cs, (pa ? (unsigned)(i - 1) : (unsigned)i) * N + node, w, rho0, r, b, rq, bq);
                        }
                    } else {
                        S::store(dst, cs, (unsigned)i * N + node, w, rho0, r, b, rq, bq);
                    }
                }
                const int tz = z + cz(i);  // the same for the whole block
                if (EDGE && (tz < 0 || (tz >= nz && top_bc == 0))) {
                    ac0[1][0] += rq;  // bounces back to this node
                    ac0[1][1] += bq;
                } else if (!EDGE || tz < nz) {
                    constexpr int d = cy(i) + 1;
                    T vr = rq, vb = bq;
                    if constexpr (cx(i) != 0) {
                        // the share for this lane's column comes from the lane at x - c_x;
                        // the edge lane's own share leaves the tile sideways
                        constexpr int side = cx(i) > 0 ? 1 : 0;
                        constexpr int k = side_slot(cy(i), cz(i));
                        if (tx == (side ? tw - 1 : 0)) {
                            sE[rz[1]][side][k][0][ty] = rq;
                            sE[rz[1]][side][k][1][ty] = bq;
                        }
                        if constexpr (cx(i) > 0) {
                            if constexpr (!R0) vr = __shfl_up_sync(lanes, rq, 1);
                            vb = __shfl_up_sync(lanes, bq, 1);
                        } else {
                            if constexpr (!R0) vr = __shfl_down_sync(lanes, rq, 1);
                            vb = __shfl_down_sync(lanes, bq, 1);
                        }
                        if (tx == (side ? 0 : tw - 1)) vr = vb = T(0);  // source outside the tile
                    }
                    // RED0: every red share of the warp is 0 and its accumulators stay as they are
                    if constexpr (cz(i) < 0) {
                        if constexpr (!R0) acm[d][0] += vr;
                        acm[d][1] += vb;
                    } else if constexpr (cz(i) == 0) {
                        if constexpr (!R0) ac0[d][0] += vr;
                        ac0[d][1] += vb;
                    } else {
                        if constexpr (!R0) ac1[d][0] += vr;
                        ac1[d][1] += vb;
                    }
                }
            };
            // BGK with the Guo source, post_i = (1 - omega) F_i + omega F_i^eq + S_i, written per
            // direction pair (i, opp(i)): F^eq = even +- odd, S = se +- so with
            //   even = w rho (1 - 1.5 u.u + 4.5 (c.u)^2), odd = 3 w rho c.u,
            //   se = (1 - omega/2) w (9 (c.u)(c.F) - 3 u.F), so = 3 (1 - omega/2) w c.F
            auto collide = [&](auto RED0_) {
                {  // rest direction
                    constexpr T w = (T)wq(0);
                    const T pre = omega * (w * rho * base0) + gsrc * w * (T(-3) * uF);
                    emit(std::integral_constant<int, 0>{}, omc * Fi[0] + pre, T(0), RED0_);
                }
                static_for<1, 19, 2>([&](auto I_) {
                    // the pair (i, opp(i) = i+1) shares c.u, c.F and c.G up to sign
                    constexpr int i = decltype(I_)::value;
                    constexpr T w = (T)wq(i);
                    T cu = 0, cF = 0, cG = 0;
                    if constexpr (cx(i) != 0) { cu += cx(i) * ux; cF += cx(i) * Fx; cG += cx(i) * rGx; }
                    if constexpr (cy(i) != 0) { cu += cy(i) * uy; cF += cy(i) * Fy; cG += cy(i) * rGy; }
                    if constexpr (cz(i) != 0) { cu += cz(i) * uz; cF += cz(i) * Fz; cG += cz(i) * rGz; }
                    const T ow = omega * (w * rho), gw = gsrc * w;
                    const T A = ow * (base0 + T(4.5) * cu * cu) + gw * (T(9) * cu * cF - T(3) * uF);
                    const T B = ow * (T(3) * cu) + gw * (T(3) * cF);
                    emit(std::integral_constant<int, i>{}, omc * Fi[i] + (A + B), cG, RED0_);
                    emit(std::integral_constant<int, i + 1>{}, omc * Fi[i + 1] + (A - B), -cG, RED0_);
                });
            };
            // interior planes of 16-bit storage: a warp whose nodes hold no red takes the
            // red-free form (the choice is per warp, no block vote needed), which drops the
            // division and rounding of the liquid fraction and half the push.  Measured: FP16
            // 1.014 -> 0.915 ms on the 512x256x128 lattice; FP32, which has no encode to drop,
            // ran 1-1.5 % slower with it (the second form's registers), so it keeps one form
            if constexpr (!EDGE && S::WORDS == 1) {
                if (__all_sync(lanes, rR == T(0)))
                    collide(std::true_type{});
                else
                    collide(std::false_type{});
            } else {
                collide(std::false_type{});
            }
            if (top_gas) {
                // gas inflow that the next stream brings to this node
                T inB = 0;
                static_for<0, 19>([&](auto I_) {
                    constexpr int i = decltype(I_)::value;
                    if constexpr (cz(i) < 0) inB += (T)wq(i) * rho0;
                });
                ac0[1][1] += inB;
            }
        };
        if (active) {
            if (z == 0 || z == nz - 1)
                phase3(std::true_type{});
            else
                phase3(std::false_type{});
        }
        retire(ac1);
        if constexpr (ASYNC && !BULK && !EARLY_PULL) issue_pull(z + 1);  // its slots were consumed above by this thread
        __syncthreads();
        if constexpr (BULK) {
            issue_bulk(z + NBUF);  // plane z's buffer is free once every thread passed the barrier
        }
    }
    if constexpr (ASYNC && !BULK) cp_async_wait<0>();
    // the last two planes: shares still in registers
    T none[3][2] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    flush(z1 - 2);
    __syncthreads();
    retire(none);
    __syncthreads();
    flush(z1 - 1);
    __syncthreads();
    retire(none);
    __syncthreads();
    flush(z1);

    // ---- block sums of the FP64 budgets ----
    double v[3] = {(double)evap_sum, (double)top_in, (double)top_out};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((tid & 31) == 0)
        for (int k = 0; k < 3; ++k) sRed[tid >> 5][k] = v[k];
    if (err) atomicOr(&sErr, err);
    __syncthreads();
    if (tid < 3) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += sRed[w][tid];
        if (s != 0.0) atomicAdd(accp + 2 + tid, s);
    }
    if (tid == 0) {
        if (sErr) atomicOr(errp, sErr);
        // the last block to finish advances the step counter
        __threadfence();
        const unsigned t = atomicAdd(&glob->done, 1u);
        if (t == gridDim.x - 1) {
            glob->done = 0u;
            glob->step = step + 1;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Moments of the streamed populations (pull + sum), used after initialisation
// and after populations are written from the host.  Writes rho[pr] (both
// components) and clears the next buffer.
// ---------------------------------------------------------------------------
// The streamed populations of node (x, y, z) at `step` in the compute type, under
// either storage layout (two buffers: pulled from x - c_i of the buffer of the step's
// parity, bounced back at the walls, gas equilibrium from above the gas top; in place:
// ep_load, chosen at compile time by EP).  The instance's fields are read once per
// node, then pull(i) per direction.
template <class S, bool EP>
struct NodePull {
    using T = typename S::T;
    using E = typename S::E;
    const E* src;
    const E* gslot;
    unsigned N, cs, gcs, node;
    int nx, ny, nz, top_bc, x, y, z, p;
    T rho0;
    __device__ __forceinline__ NodePull(const InstDev& I, long long step, int x_, int y_, int z_)
        : x(x_), y(y_), z(z_) {
        nx = I.nx;
        ny = I.ny;
        nz = I.nz;
        top_bc = I.top_bc;
        N = (unsigned)I.N;
        cs = 19u * N;
        gcs = 10u * (unsigned)nx * ny;
        p = (int)(step & 1);
        src = (const E*)I.pop[EP ? 0 : p];
        gslot = (const E*)I.ghost;
        rho0 = (T)I.rho0;
        node = ((unsigned)z * ny + y) * nx + x;
    }
    __device__ __forceinline__ void pull(int i, T& r, T& b) const {
        if constexpr (EP) {
            PopLoc L;
            if (!ep_load(i, x, y, z, p, nx, ny, nz, top_bc, L)) {
                r = T(0);
                b = (T)wq(i) * rho0;
                return;
            }
            S::load(L.ghost ? gslot : src, L.ghost ? gcs : cs, L.k, (T)wq(i), rho0, r, b);
            return;
        }
        const int sz = z - cz(i);
        if (sz < 0 || (sz >= nz && top_bc == 0)) {
            S::load(src, cs, (unsigned)opp(i) * N + node, (T)wq(opp(i)), rho0, r, b);
        } else if (sz >= nz) {
            r = T(0);
            b = (T)wq(i) * rho0;
        } else {
            const int sx = wrap_one(x - cx(i), nx), sy = wrap_one(y - cy(i), ny);  // shifts of one cell
            S::load(src, cs, (unsigned)i * N + ((unsigned)sz * ny + sy) * nx + sx, (T)wq(i), rho0, r, b);
        }
    }
};

// Where the post-collision population i of node n, as left by the step before
// `step`, is stored: base pointer, component stride and element index.
template <class S>
__device__ __forceinline__ void post_place(const InstDev& I, long long step, int i, long long n,
                                           typename S::E*& base, long long& cs, long long& k) {
    using E = typename S::E;
    if (I.inplace) {
        const int nx = I.nx, ny = I.ny;
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
        const PopLoc L = ep_store(i, x, y, z, (int)((step - 1) & 1), nx, ny, I.nz);
        base = L.ghost ? (E*)I.ghost : (E*)I.pop[0];
        cs = L.ghost ? 10LL * nx * ny : 19 * I.N;
        k = L.k;
        return;
    }
    base = (E*)I.pop[step & 1];
    cs = 19 * I.N;
    k = (long long)i * I.N + n;
}

// rho_R, rho_B, j of node n from the populations that stream into it at `step`
template <class S, bool EP>
__device__ void stream_moments_t(const InstDev& I, long long step, int x, int y, int z,
                                 typename S::T* m) {
    using T = typename S::T;
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
    m[0] = rR;
    m[1] = rB;
    m[2] = jx;
    m[3] = jy;
    m[4] = jz;
}

template <class S>
__device__ void stream_moments(const InstDev& I, long long step, long long n, typename S::T* m) {
    const int nx = I.nx, ny = I.ny;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    if (I.inplace)
        stream_moments_t<S, true>(I, step, x, y, z, m);
    else
        stream_moments_t<S, false>(I, step, x, y, z, m);
}

template <class S>
__global__ void k_moments(InstDev I, long long step, long long n0, long long len,
                          double* __restrict__ diag) {
    using T = typename S::T;
    const long long N = I.N;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= len) return;
    const long long n = n0 + u;
    T m[5];
    stream_moments<S>(I, step, n, m);
    const T rR = m[0], rB = m[1], jx = m[2], jy = m[3], jz = m[4];
    if (diag) {
        double* d = diag + 5 * u;
        d[0] = rR;
        d[1] = rB;
        d[2] = jx;
        d[3] = jy;
        d[4] = jz;
        return;
    }
    T* rho = (T*)I.rho[step % 3];
    rho[n] = rR;
    rho[N + n] = rB;
    T* nxt = (T*)I.rho[(step + 1) % 3];
    nxt[n] = T(0);
    nxt[N + n] = T(0);
    T* nn = (T*)I.rho[(step + 2) % 3];
    nn[n] = T(0);
    nn[N + n] = T(0);
}

// Initial droplet at rest in equilibrium: C = tanh(-(q-1) min(a,b,c)/width).
template <class S>
__global__ void k_init_droplet(InstDev I, int shape, double cx_, double cy_, double cz_, double a,
                               double b, double c, double width) {
    using E = typename S::E;
    const long long N = I.N;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int nx = I.nx, ny = I.ny;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    double m = a < b ? a : b;
    m = m < c ? m : c;
    const double dx = (x - cx_) / a, dy = (y - cy_) / b, dz = (z - cz_) / c;
    double q;
    if (shape == 0) {
        q = sqrt(dx * dx + dy * dy + dz * dz);
    } else {
        const double r = sqrt(dy * dy + dz * dz);
        q = fabs(dx) > r ? fabs(dx) : r;
    }
    const double C = tanh(-(q - 1.0) * m / width);
    for (int i = 0; i < 19; ++i) {
        E* p;
        long long cs, k;
        post_place<S>(I, 0, i, n, p, cs, k);
        S::from_f64(p, cs, k, i, I.rho0, wq(i) * I.rho0 * (1.0 + C) / 2.0, wq(i) * I.rho0 * (1.0 - C) / 2.0);
    }
}

// Populations <-> FP64 staging: elements t0..t0+len of [19][N]; staging
// holds len values of f^R followed by len values of f^B.
template <class S>
__global__ void k_pop_to_f64(InstDev I, long long step, long long t0, long long len,
                             double* __restrict__ out) {
    using E = typename S::E;
    const long long N = I.N;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= len) return;
    const long long t = t0 + u;
    double r, b;
    E* p;
    long long cs, k;
    post_place<S>(I, step, (int)(t / N), t % N, p, cs, k);
    S::to_f64(p, cs, k, (int)(t / N), I.rho0, r, b);
    out[u] = r;
    out[len + u] = b;
}
template <class S>
__global__ void k_pop_from_f64(InstDev I, long long step, long long t0, long long len,
                               const double* __restrict__ in) {
    using E = typename S::E;
    const long long N = I.N;
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= len) return;
    const long long t = t0 + u;
    E* p;
    long long cs, k;
    post_place<S>(I, step, (int)(t / N), t % N, p, cs, k);
    S::from_f64(p, cs, k, (int)(t / N), I.rho0, in[u], in[len + u]);
}

// Colour field of the next step, FP64
template <typename T>
__global__ void k_colour(InstDev I, long long step, long long n0, long long len,
                         double* __restrict__ out) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= len) return;
    out[u] = (double)colour_of((const T*)I.rho[step % 3], I.N, n0 + u);
}

// Bead force on the fluid, FP64 copy of a node range
template <typename T>
__global__ void k_fext(InstDev I, int parity, long long n0, long long len, double* __restrict__ out) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= 3 * len || I.fext == nullptr) return;
    const long long n = n0 + u / 3;
    const int x = (int)(n % I.nx), y = (int)((n / I.nx) % I.ny), z = (int)(n / ((long long)I.nx * I.ny));
    const bool live = tflag_of(I, parity)[((long long)(z >> 3) * I.t8y + (y >> 3)) * I.t8x + (x >> 3)] != 0;
    out[u] = live ? (double)((const T*)I.fext)[3 * n0 + u] : 0.0;
}

// Liquid column heights and their maximum -> h0 (first evaporating step)
template <typename T>
__global__ void k_h0(InstDev I, long long step) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncol = I.nx * I.ny;
    double h = 0.0;
    if (c < ncol) {
        const T* rho = (const T*)I.rho[step % 3];
        T s = 0;
        for (int z = 0; z < I.nz; ++z) s += (T(1) + colour_of(rho, I.N, (long long)z * ncol + c)) / T(2);
        h = (double)s;
    }
    for (int o = 16; o > 0; o >>= 1) h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
    if ((threadIdx.x & 31) == 0 && h > 0.0)
        atomicMax((unsigned long long*)(I.acc + 1), (unsigned long long)__double_as_longlong(h));
}

// Component masses: sums of all stored populations (FP64 block sums)
template <class S>
__global__ void k_mass(InstDev I, long long step, double* __restrict__ out) {
    using E = typename S::E;
    const long long N = I.N;
    double sr = 0.0, sb = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 19 * N;
         t += (long long)gridDim.x * blockDim.x) {
        double r, b;
        E* p;
        long long cs, k;
        post_place<S>(I, step, (int)(t / N), t % N, p, cs, k);
        S::to_f64(p, cs, k, (int)(t / N), I.rho0, r, b);
        sr += r;
        sb += b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, sr);
        atomicAdd(out + 1, sb);
    }
}

}  // namespace lbm
