// Internal device-side definitions of the B300 library: lattice constants,
// population storage formats, per-instance tables.  Paper references are to
// "Evaporation-Driven Nanowire Self-Assembly in an Elongated Droplet", Sec. II.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <type_traits>

namespace lbm {

// ---------------------------------------------------------------------------
// D3Q19 velocity set (Sec. II.A, Eq. (1)): rest, 6 axis links, 12 face
// diagonals.  Directions come in opposite pairs (2k-1, 2k).  Written as
// constexpr functions so that fully unrolled loops fold every c_i and w_i.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wq(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// 1/|c_i| for the recolouring direction cosine
__host__ __device__ constexpr double inv_len(int i) {
    return i == 0 ? 0.0 : (i <= 6 ? 1.0 : 0.70710678118654752440);
}

// error bits latched per instance
enum : int { ERR_NAN = 1, ERR_FENE = 2, ERR_BEAD = 4, ERR_TIMEOUT = 8, ERR_CAP = 16 };

// ---------------------------------------------------------------------------
// Population storage.  Element k = i N + node of direction i.  FP64 and FP32
// lay a buffer out as [comp][dir][z][y][x] (comp stride cs = 19 N); the 16-bit
// forms keep both numbers of an element in one 4-byte word, [dir][z][y][x].
// WORDS = 4-byte words per element and component layout (2: two planes of
// 4-byte values, 1: one word per element; 0: not staged in words).  load()
// returns (f^R, f^B) in the compute type; store() writes a post-collision pair
// and returns in (rq, bq) the pair that the push of the next step's moments
// adds up.  FP64 and FP32 store exactly, so there the pushed moments are the
// moments of the stored populations.  The 16-bit forms return the pair before
// rounding: the next step's colour field and column heights then differ from
// the moments of the stored words by the rounding of those words, while the
// populations (and hence the mass) are always the stored words.  A restore
// from stored words rebuilds the moments from the words themselves, so a
// restored 16-bit run continues the unbroken one only up to that rounding.
// ---------------------------------------------------------------------------
// 32-bit integer hash (Wellons' "lowbias32"): the counter-based uniform source
// of the stochastic rounding below
__host__ __device__ __forceinline__ unsigned hash32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

struct StoreF64 {
    using T = double;
    using E = double;
    static constexpr int WORDS = 0;
    static __device__ __forceinline__ void decode(E a, E c, T w, T rho0, T& r, T& b) {
        r = a;
        b = c;
    }
    // total F = f^R + f^B and f^R
    static __device__ __forceinline__ void decode_total(E a, E c, T w, T rho0, T& F, T& r) {
        r = a;
        F = a + c;
    }
    static __device__ __forceinline__ void load(const E* __restrict__ p, unsigned cs, unsigned k,
                                                T w, T rho0, T& r, T& b) {
        r = __ldg(p + k);
        b = __ldg(p + cs + k);
    }
    static __device__ __forceinline__ void store(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                 T rho0, T r, T b, T& rq, T& bq) {
        p[k] = r;
        p[cs + k] = b;
        rq = r;
        bq = b;
    }
    static __device__ __forceinline__ void store_sr(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                    T rho0, T r, T b, T& rq, T& bq, unsigned) {
        store(p, cs, k, w, rho0, r, b, rq, bq);
    }
    // an element without the red component (f^R = 0): what store gives for r = 0
    static __device__ __forceinline__ void store_gas(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                     T rho0, T b) {
        p[k] = E(0);
        p[cs + k] = b;
    }
    static __host__ __device__ void to_f64(const E* p, long long cs, long long k, int i, double rho0,
                                           double& r, double& b) {
        r = p[k];
        b = p[cs + k];
    }
    static __host__ __device__ void from_f64(E* p, long long cs, long long k, int i, double rho0,
                                             double r, double b) {
        p[k] = r;
        p[cs + k] = b;
    }
};

struct StoreF32 {
    using T = float;
    using E = float;
    static constexpr int WORDS = 2;
    static __device__ __forceinline__ void decode(E a, E c, T w, T rho0, T& r, T& b) {
        r = a;
        b = c;
    }
    // total F = f^R + f^B and f^R
    static __device__ __forceinline__ void decode_total(E a, E c, T w, T rho0, T& F, T& r) {
        r = a;
        F = a + c;
    }
    static __device__ __forceinline__ void load(const E* __restrict__ p, unsigned cs, unsigned k,
                                                T w, T rho0, T& r, T& b) {
        r = __ldg(p + k);
        b = __ldg(p + cs + k);
    }
    static __device__ __forceinline__ void store(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                 T rho0, T r, T b, T& rq, T& bq) {
        p[k] = r;
        p[cs + k] = b;
        rq = r;
        bq = b;
    }
    static __device__ __forceinline__ void store_sr(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                    T rho0, T r, T b, T& rq, T& bq, unsigned) {
        store(p, cs, k, w, rho0, r, b, rq, bq);
    }
    // an element without the red component (f^R = 0): what store gives for r = 0
    static __device__ __forceinline__ void store_gas(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                     T rho0, T b) {
        p[k] = E(0);
        p[cs + k] = b;
    }
    static __host__ __device__ void to_f64(const E* p, long long cs, long long k, int i, double rho0,
                                           double& r, double& b) {
        r = p[k];
        b = p[cs + k];
    }
    static __host__ __device__ void from_f64(E* p, long long cs, long long k, int i, double rho0,
                                             double r, double b) {
        p[k] = (float)r;
        p[cs + k] = (float)b;
    }
};

// Shifted 16-bit storage: comp 0 holds F_i - w_i rho0 (total population as a
// deviation from rest) in HP, comp 1 holds f^R_i/F_i - 1/2 (liquid fraction;
// exactly +-1/2 in pure phases) in HQ.  FP16 storage keeps both halves in
// __half; BF16 storage keeps the deviation in __nv_bfloat16 and the fraction,
// bounded by 1/2, in __half, whose 10 fraction bits resolve it 8 times finer
// than bfloat16's 7 (bfloat16's exponent range is of no use to a bounded number).
template <class H>
struct Cvt;
template <>
struct Cvt<__half> {
    static __device__ __forceinline__ float f(__half h) { return __half2float(h); }
    static __device__ __forceinline__ __half h(float f) { return __float2half_rn(f); }
    static __device__ __forceinline__ __half rd(float f) { return __float2half_rd(f); }
    static __device__ __forceinline__ __half ru(float f) { return __float2half_ru(f); }
    static __host__ __device__ float fh(__half h) { return __half2float(h); }
    static __host__ __device__ __half hf(float f) { return __float2half_rn(f); }
    // a pair in one word (lo in the low half) and back, with the packed conversions
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        const __half2 v = __floats2half2_rn(lo, hi);
        unsigned w;
        memcpy(&w, &v, 4);
        return w;
    }
    static __device__ __forceinline__ float2 unpack(unsigned w) {
        __half2 v;
        memcpy(&v, &w, 4);
        return __half22float2(v);
    }
    // one value as the bits of a half-word and back
    static __device__ __forceinline__ unsigned bits(float f) { return __half_as_ushort(__float2half_rn(f)); }
    static __device__ __forceinline__ float from_bits(unsigned b) {
        return __half2float(__ushort_as_half((unsigned short)b));
    }
};
template <>
struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ float f(__nv_bfloat16 h) { return __bfloat162float(h); }
    static __device__ __forceinline__ __nv_bfloat16 h(float f) { return __float2bfloat16_rn(f); }
    static __device__ __forceinline__ __nv_bfloat16 rd(float f) { return __float2bfloat16_rd(f); }
    static __device__ __forceinline__ __nv_bfloat16 ru(float f) { return __float2bfloat16_ru(f); }
    static __host__ __device__ float fh(__nv_bfloat16 h) { return __bfloat162float(h); }
    static __host__ __device__ __nv_bfloat16 hf(float f) { return __float2bfloat16_rn(f); }
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        unsigned w;
        memcpy(&w, &v, 4);
        return w;
    }
    static __device__ __forceinline__ float2 unpack(unsigned w) {
        __nv_bfloat162 v;
        memcpy(&v, &w, 4);
        return __bfloat1622float2(v);
    }
    static __device__ __forceinline__ unsigned bits(float f) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    }
    static __device__ __forceinline__ float from_bits(unsigned b) { return __uint_as_float(b << 16); }
};

// the element word of an (HP, HQ) pair: HP in the low half, HQ in the high half
template <class HP, class HQ>
struct Pair16 {
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        if constexpr (std::is_same<HP, HQ>::value)
            return Cvt<HP>::pack(lo, hi);
        else
            return Cvt<HP>::bits(lo) | (Cvt<HQ>::bits(hi) << 16);
    }
    static __device__ __forceinline__ float2 unpack(unsigned w) {
        if constexpr (std::is_same<HP, HQ>::value)
            return Cvt<HP>::unpack(w);
        else
            return make_float2(Cvt<HP>::from_bits(w & 0xffffu), Cvt<HQ>::from_bits(w >> 16));
    }
};

// the bits of -1/2 in IEEE binary16 (sign 1, exponent 14, fraction 0)
constexpr unsigned HALF_MINUS_HALF = 0xB800u;

template <class HP, class HQ>
struct StoreShift16 {
    using T = float;
    using E = HP;  // half-words: the deviation (HP) at even, the fraction (HQ) at odd positions
    using H = HQ;
    static_assert(std::is_same<HQ, __half>::value, "the liquid fraction is stored in binary16");
    static constexpr int WORDS = 1;
    static __host__ __device__ __forceinline__ void decode(float P, float psi, float w, float rho0,
                                                           float& r, float& b) {
        float F = P + w * rho0;
        r = (psi + 0.5f) * F;
        b = F - r;
    }
    // one element as its 4-byte word: low half P, high half psi
    static __device__ __forceinline__ void decode_word(unsigned word, float w, float rho0, float& r,
                                                       float& b) {
        const float2 v = Pair16<HP, HQ>::unpack(word);
        decode(v.x, v.y, w, rho0, r, b);
    }
    // total F = f^R + f^B and f^R of an element word
    static __device__ __forceinline__ void decode_word_total(unsigned word, float w, float rho0, float& F,
                                                             float& r) {
        const float2 v = Pair16<HP, HQ>::unpack(word);
        F = v.x + w * rho0;
        r = (v.y + 0.5f) * F;
    }
    static __device__ __forceinline__ void load(const E* __restrict__ p, unsigned cs, unsigned k,
                                                T w, T rho0, T& r, T& b) {
        decode_word(__ldg((const unsigned*)p + k), w, rho0, r, b);
    }
    // rq, bq: what the next step's moments (colour field, column height) sum: the values
    // before rounding; the populations themselves are the stored words, decoded at the pull
    static __device__ __forceinline__ void store(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                 T rho0, T r, T b, T& rq, T& bq) {
        float F = r + b;
        const unsigned word = Pair16<HP, HQ>::pack(F - w * rho0, F != 0.0f ? __fdividef(r, F) - 0.5f : 0.0f);
        ((unsigned*)p)[k] = word;
        rq = r;
        bq = b;
    }
    // the same with the liquid fraction rounded stochastically (up with probability
    // (x - lo)/(hi - lo), rnd a uniform 32-bit number): per-step changes far below one
    // unit of the last place, such as the evaporation sink's, survive on average
    static __device__ __forceinline__ void store_sr(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                    T rho0, T r, T b, T& rq, T& bq, unsigned rnd) {
        float F = r + b;
        const float x = F != 0.0f ? __fdividef(r, F) - 0.5f : 0.0f;
        const H lo = Cvt<H>::rd(x), hi = Cvt<H>::ru(x);
        const float flo = Cvt<H>::f(lo), fhi = Cvt<H>::f(hi);
        const float u = (float)(rnd >> 8) * (1.0f / 16777216.0f);
        const H q = (u * (fhi - flo) < x - flo) ? hi : lo;
        const unsigned word = Cvt<HP>::bits(F - w * rho0) | ((unsigned)__half_as_ushort(q) << 16);
        ((unsigned*)p)[k] = word;
        rq = r;
        bq = b;
    }
    // an element without the red component (f^R = 0): the liquid fraction -1/2 (store
    // writes 0 where the total is 0; the fraction only ever multiplies the total, so both
    // decode to the same populations)
    static __device__ __forceinline__ void store_gas(E* __restrict__ p, unsigned cs, unsigned k, T w,
                                                     T rho0, T b) {
        ((unsigned*)p)[k] = Cvt<HP>::bits(b - w * rho0) | (HALF_MINUS_HALF << 16);
    }
    static __device__ void to_f64(const E* p, long long cs, long long k, int i, double rho0,
                                  double& r, double& b) {
        float rr, bb;
        const unsigned w = ((const unsigned*)p)[k];
        decode(Cvt<HP>::from_bits(w & 0xffffu), Cvt<HQ>::from_bits(w >> 16), (float)wq(i), (float)rho0, rr, bb);
        r = rr;
        b = bb;
    }
    static __device__ void from_f64(E* p, long long cs, long long k, int i, double rho0, double r,
                                    double b) {
        float F = (float)(r + b);
        ((unsigned*)p)[k] = Cvt<HP>::bits(F - (float)wq(i) * (float)rho0) |
                            (Cvt<HQ>::bits(F != 0.0f ? (float)(r / (r + b)) - 0.5f : 0.0f) << 16);
    }
};
using StoreF16 = StoreShift16<__half, __half>;
using StoreB16 = StoreShift16<__nv_bfloat16, __half>;

// ---------------------------------------------------------------------------
// Device tables
// ---------------------------------------------------------------------------
struct InstDev {
    int nx, ny, nz, top_bc;
    long long N;
    // esoteric-pull in-place storage: one population buffer (pop[0] == pop[1]) plus
    // ghost slots below z = 0 and above the top, [comp][side][5 pairs][ny][nx]
    int inplace, pad3;
    void* ghost;
    int t8x, t8y, t8z;           // 8^3 coupling-tile grid
    int pad0;
    void* pop[2];                // population buffers (storage type)
    void* rho[3];                // moment buffers: [2][N] rho_R, rho_B (compute type)
    void* fext;                  // [N][3] bead force on the fluid (compute type)
    void* ust;                   // [N][3] u* near beads (compute type)
    void* gcol;                  // [N][3] grad C near beads (compute type)
    void* hcol;                  // [ny][nx] liquid column height of the step (compute type)
    // per-step coupling flags in two sets by step parity: the next step's set is
    // filled while the fused kernel still reads this step's
    unsigned* tflag;             // [2][ntile + 1]: [t8z][t8y][t8x] tile flags, then the flagged-tile count
    int* tlist;                  // [2][ntile]: flagged tiles (compact)
    unsigned* nbit;              // [2][nword]: nodes the beads' stencils can reach in the step
    int ntile, nword;            // t8z t8y t8x and N/32 + 1
    double* cot;                 // [ny][nx] cot(theta)
    double* acc;                 // [8]: step, h0, evaporated, top_in, top_out, ...
    int* err;                    // latched error bits
    double tau_R, tau_B, beta, sigma, rho0, J0, K;
    double body[3];
    long long evap_start;
    // filaments
    int nb, nb_max, substeps, max_nbr;
    double* bx;
    double* bv;
    double* bF;
    double* bvh;
    double* bx2;
    double* bx0;
    // sub-step positions split into the nearest lattice point and an FP32 offset
    // (x = K + r, |r| <= 1/2), [0] mirroring bx2, [1] mirroring bx: the FP32 force
    // path forms pair separations and the trilinear stencil from them with no FP64
    // arithmetic (the FP64 path reads the positions themselves)
    int4* bK[2];
    float4* bR[2];
    int* bfil;
    int* bpos;
    int* nbr;
    int* nnbr;
    double ks, Rm, d0, eps_wca, kb, eps_coh, eps_s, rc, gamma, xi, mu, gamma_t, mass, rlist;
    double dt_sub, hk_sub;       // sub-step 1/substeps and half kick dt/(2 m)
    // FP32 roundings of the force parameters (Rm as Rm^2), made on the host: the FP32
    // force path then converts nothing from FP64 per thread
    float f_ks, f_Rm2, f_d0, f_eps_wca, f_kb, f_eps_coh, f_eps_s, f_rc, f_gamma, f_xi, f_mu, f_gamma_t;
    float f_dt_sub, f_pad[3];
    // cell list of large instances (cells at least rlist wide)
    int cgx, cgy, cgz, pad2;
    int* ccount;                 // beads filed per cell this step
    int* cbeads;                 // [cell][CELL_CAP] bead ids
    float* bxf;                  // [n][3] FP32 copy of the step-start positions
    // descriptors
    double rcon, x_src, x_snk;
    int* lab;
    int2* edges;
    int* nedges;
    int max_edges;
    int pad1;
    double* desc;                // [8] descriptor results
    // electrical network of the deposit
    double* net;                 // [6][nb_max]: V, r, p, q, 1/diag, I*
    double* netout;              // [10] network results
    int* csr_row;                // [nb_max + 1]
    int* csr_cnt;                // [2][nb_max]: fill cursors, node classes
    int* csr_col;                // [2 max_edges]
    double* csr_val;             // [2 max_edges] conductances
};

// ---------------------------------------------------------------------------
// Esoteric-pull in-place storage (one buffer, read and written in place).  The
// directions pair up as (i, i+1), i odd, c_{i+1} = -c_i.  At a step of parity
// p = step & 1 a node reads the streamed f_i from its own slot (p ? i : i+1) and
// f_{i+1} from slot (p ? i+1 : i) of its neighbour n + c_i, and writes the
// post-collision f*_i to slot (p ? i+1 : i) of n + c_i and f*_{i+1} to its own
// slot (p ? i : i+1): every slot is read and written by one node per step, so
// the step needs no second buffer.  At the walls the neighbour n + c_i may not
// exist: f*_i then goes to a ghost slot of the node's column (side 0 below z = 0,
// 1 above the top), from which the bounced f_{i+1} is read next step; the f_i
// bounced from the other side is read from the node's other own slot, where the
// previous step left f*_{i+1}.  Under the gas top the inflow replaces the
// downward populations, and the outflow of the previous step is read (for the
// FP64 budget) from the top ghost (odd members) or the other own slot (even).
// ---------------------------------------------------------------------------
// ghost pair of the odd member of a pair with c_z != 0
__host__ __device__ constexpr int ghost_pair(int i) {
    return i == 5 ? 0 : (i == 11 ? 1 : (i == 13 ? 2 : (i == 15 ? 3 : 4)));
}
// a population's place: element index k into the main buffer (comp stride 19 N)
// or, with ghost set, into the ghost array (comp stride 10 nx ny)
struct PopLoc {
    unsigned k;
    bool ghost;
};
__host__ __device__ __forceinline__ int wrap_one(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__host__ __device__ __forceinline__ unsigned ghost_index(int side, int g, int x, int y, int nx, int ny) {
    return (unsigned)((side * 5 + g) * ny + y) * nx + x;
}
// where the post-collision population i of node (x, y, z) goes at a step of parity p
__host__ __device__ __forceinline__ PopLoc ep_store(int i, int x, int y, int z, int p, int nx, int ny, int nz) {
    const unsigned nxy = (unsigned)nx * ny, N = nxy * (unsigned)nz;
    if (i == 0) return {(unsigned)z * nxy + (unsigned)y * nx + x, false};
    if (i & 1) {
        const int tz = z + cz(i);
        if (tz < 0) return {ghost_index(0, ghost_pair(i), x, y, nx, ny), true};
        if (tz >= nz) return {ghost_index(1, ghost_pair(i), x, y, nx, ny), true};
        const unsigned slot = p ? i + 1 : i;
        return {slot * N + (unsigned)tz * nxy + (unsigned)wrap_one(y + cy(i), ny) * nx + wrap_one(x + cx(i), nx),
                false};
    }
    const unsigned slot = p ? i - 1 : i;
    return {slot * N + (unsigned)z * nxy + (unsigned)y * nx + x, false};
}
// where the streamed population i of node (x, y, z) is read at a step of parity p;
// false: replaced by the gas inflow (loc is then a harmless own slot)
__host__ __device__ __forceinline__ bool ep_load(int i, int x, int y, int z, int p, int nx, int ny, int nz,
                                                 int top_bc, PopLoc& loc) {
    const unsigned nxy = (unsigned)nx * ny, N = nxy * (unsigned)nz;
    const unsigned node = (unsigned)z * nxy + (unsigned)y * nx + x;
    loc = {node, false};
    if (i == 0) return true;
    if (i & 1) {
        const int sz = z - cz(i);
        if (sz >= nz && top_bc == 1) return false;
        const bool bounce = sz < 0 || sz >= nz;  // from the node's other own slot
        const unsigned slot = (p != 0) != bounce ? i : i + 1;
        loc = {slot * N + node, false};
        return true;
    }
    const int j = i - 1;  // the odd member: f_i comes from n + c_j
    const int tz = z + cz(j);
    if (tz < 0) {
        loc = {ghost_index(0, ghost_pair(j), x, y, nx, ny), true};
        return true;
    }
    if (tz >= nz) {
        if (top_bc == 1) return false;
        loc = {ghost_index(1, ghost_pair(j), x, y, nx, ny), true};
        return true;
    }
    const unsigned slot = p ? i : j;
    loc = {slot * N + (unsigned)tz * nxy + (unsigned)wrap_one(y + cy(j), ny) * nx + wrap_one(x + cx(j), nx), false};
    return true;
}
// the previous step's outflow through the gas top, direction i (c_z(i) > 0), column (x, y)
__host__ __device__ __forceinline__ PopLoc ep_outflow(int i, int x, int y, int p, int nx, int ny, int nz) {
    if (i & 1) return {ghost_index(1, ghost_pair(i), x, y, nx, ny), true};
    const unsigned nxy = (unsigned)nx * ny;
    const unsigned slot = p ? i : i - 1;
    return {slot * nxy * (unsigned)nz + (unsigned)(nz - 1) * nxy + (unsigned)y * nx + x, false};
}

struct StepGlobals {
    long long step;
    unsigned int done;
    int pad;
    long long bead_next;  // step whose bead start the last sub-step pass enabled (step + 1)
};

__device__ __forceinline__ unsigned* tflag_of(const InstDev& I, int p) {
    return I.tflag + (size_t)p * (I.ntile + 1);
}
__device__ __forceinline__ int* tcount_of(const InstDev& I, int p) { return (int*)(tflag_of(I, p) + I.ntile); }
__device__ __forceinline__ int* tlist_of(const InstDev& I, int p) { return I.tlist + (size_t)p * I.ntile; }
__device__ __forceinline__ unsigned* nbit_of(const InstDev& I, int p) { return I.nbit + (size_t)p * I.nword; }

struct TileDesc {
    int inst, x0, y0, z0, z1, pad0, pad1, pad2;
};

// 4-wide vectors for shared-memory staging (one 16/32-byte access per node)
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4_16a;
};

__host__ __device__ inline int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

}  // namespace lbm
