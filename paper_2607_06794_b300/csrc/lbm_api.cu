// Host side of the C ABI declared in include/lbm.h: configuration checks,
// workspace layout over caller-owned device memory, launch sequence of one
// time step (captured once into a CUDA graph and replayed), field transfer,
// nanowire placement and descriptors.
#include <math.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <random>
#include <vector>

#include "../../include/lbm.h"
#include "kernels_beads.cuh"
#include "kernels_network.cuh"
#include "kernels_shape.cuh"

using namespace lbm;

namespace {

// Tilings of the fused kernel the autotuner chooses from: columns of tx-by-ty
// nodes, then a z-chunk per block (chunk 0 means "split until the whole batch
// fills the GPU"; chunks above nz take the whole column; chunk -1 means whole
// columns in full waves of resident blocks, then the rest of the columns in
// chunks short enough to fill the last waves, see make_tiles), and the register
// budget as resident blocks per SM (128 registers a thread: 4 blocks of 32x4,
// 2 of 32x8; a 96-register form of 32x4 at 5 blocks per SM measured 5-40 %
// slower on every workload, a spill-free 168-register form at 3 blocks 6-16 %
// slower, and both were dropped), and how 32- and 16-bit storage
// stages the pull (0: per-element asynchronous copies; 1: bulk row copies where
// every lattice of the batch has nx % 4 == 0, else per-element).  Blocks of equal
// chunks march up in step, so the halo planes a block re-reads were just read by
// its neighbours and come from L2.
struct Shape {
    int tx, ty, chunk, minb, bulk;
};
const Shape SHAPES[] = {{32, 8, 0, 2, 0}, {32, 8, 16, 2, 0}, {32, 8, 32, 2, 0}, {32, 8, 64, 2, 0},
                        {32, 4, 0, 4, 0}, {32, 4, 16, 4, 0}, {32, 4, 32, 4, 0}, {32, 4, 64, 4, 0},
                        {32, 8, 0, 2, 1}, {32, 8, 32, 2, 1}, {32, 4, 0, 4, 1}, {32, 4, 32, 4, 1},
                        {32, 4, 64, 4, 1}, {32, 4, -1, 4, 0}, {32, 8, -1, 2, 0}};
constexpr int NSHAPES = sizeof(SHAPES) / sizeof(SHAPES[0]);
constexpr int MAX_NBR = 128;
constexpr size_t STAGE_BYTES = size_t(64) << 20;
constexpr int PROFILE_MAX_BINS = 65536;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_bytes(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2); }
int comp_bytes(int prec) { return prec == LBM_FP64 ? 8 : 4; }

// A bump allocator over the workspace; with base == nullptr it only measures.
struct Carver {
    char* base;
    size_t off = 0;
    void* take(size_t bytes) {
        off = align_up(off, 256);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

struct Layout {
    std::vector<InstDev> inst;
    StepGlobals* glob = nullptr;
    InstDev* d_inst = nullptr;
    TileDesc* d_tiles = nullptr;
    double* stage = nullptr;
    size_t stage_bytes = 0;
    int ntiles = 0;
    size_t tile_cap = 0;  // entries the tile table has room for
};

// neighbour-list radius: the longest interaction range plus a skin of one
// lattice unit (beads move less than half a unit per step)
double rlist_of(const lbm_config& c) {
    double rl = c.d0;
    if (c.eps_coh > 0) rl = std::max(rl, c.rc);
    rl = std::max(rl, c.rcon);
    return rl + 1.0;
}

// planes per block: at most 240 (241 with a merged last plane) so that a chunk spans at most 32 coupling-tile
// slabs of 8 planes (the fused kernel keeps their flags in one 32-bit mask)
constexpr int MAX_CHUNK = 240;
// column tiles of all instances (the x-by-y tiles of the fused kernel)
long long column_tiles(const lbm_config* cfgs, int n, const Shape& sh) {
    long long cols = 0;
    for (int k = 0; k < n; ++k)
        cols += (long long)((cfgs[k].nx + sh.tx - 1) / sh.tx) * ((cfgs[k].ny + sh.ty - 1) / sh.ty);
    return cols;
}

int chunk_z(const lbm_config& c, const Shape& sh, long long cols_all) {
    if (sh.chunk > 0) return std::max(2, std::min(std::min(sh.chunk, MAX_CHUNK), c.nz));
    // enough blocks over the whole batch to fill the GPU when the lattices are small
    const long long cols = (long long)((c.nx + sh.tx - 1) / sh.tx) * ((c.ny + sh.ty - 1) / sh.ty);
    int ch = std::min(c.nz, MAX_CHUNK);
    while ((cols_all - cols) + cols * ((c.nz + ch - 1) / ch) < 4 * 148 && ch > 8) ch = (ch + 1) / 2;
    return std::max(2, std::min(ch, c.nz));
}

// z-ranges of the chunks of one column: never a 1-plane chunk
std::vector<std::pair<int, int>> z_chunks(int nz, int ch) {
    std::vector<std::pair<int, int>> zr;
    for (int z0 = 0; z0 < nz;) {
        int z1 = std::min(nz, z0 + ch);
        if (nz - z1 > 0 && nz - z1 < 2) z1 = nz;
        zr.push_back({z0, z1});
        z0 = z1;
    }
    return zr;
}

// Whole columns in full waves, then chunks (chunk -1).  With S = 148 x minb resident
// blocks, a whole wave of column blocks costs nz planes plus the start of a block
// (its first C and normal planes and the flush of its boundary planes, about
// START_PLANES planes of work), and the blocks that do not fill a wave are better
// cut into chunks, so that the last waves end together.  The head (the first
// `head` columns, in column order, marching up in step) and the tail chunk are
// chosen by that cost model; the tail goes out chunk by chunk, the columns of a
// chunk in order, so that neighbouring blocks still march in step.
constexpr int RESIDENT_SMS = 148;
constexpr double START_PLANES = 4.0;
struct MixedPlan {
    long long head = 0;  // columns taken whole
    int tail_chunk = 0;  // planes per block of the other columns (0: none left)
};
MixedPlan mixed_plan(const lbm_config* cfgs, int n, const Shape& sh) {
    const long long cols = column_tiles(cfgs, n, sh);
    const long long S = (long long)RESIDENT_SMS * sh.minb;
    int nzmax = 2;
    for (int k = 0; k < n; ++k) nzmax = std::max(nzmax, std::min(cfgs[k].nz, MAX_CHUNK));
    MixedPlan best;
    double bt = 1e300;
    for (long long w = cols / S; w >= 0 && w >= cols / S - 1; --w) {
        const long long head = w * S, rest = cols - head;
        const int chunks[] = {0, 8, 12, 16, 24, 32, 48, 64};
        for (int c : chunks) {
            if ((c == 0) != (rest == 0) || c >= nzmax) continue;
            double t = (double)w * (nzmax + START_PLANES);
            if (rest > 0) {
                const long long per = (nzmax + c - 1) / c;
                t += (double)((rest * per + S - 1) / S) * (c + START_PLANES);
            }
            if (t < bt) {
                bt = t;
                best.head = head;
                best.tail_chunk = c;
            }
        }
    }
    return best;
}

// the tile table of a tiling: one column piece per block
std::vector<TileDesc> make_tiles(const lbm_config* cfgs, int n, const Shape& sh) {
    const long long cols_all = column_tiles(cfgs, n, sh);
    std::vector<TileDesc> t;
    if (sh.chunk < 0) {
        const MixedPlan mp = mixed_plan(cfgs, n, sh);
        if (mp.head > 0 || mp.tail_chunk > 0) {
            struct Col {
                int inst, x0, y0;
            };
            std::vector<Col> col;
            for (int k = 0; k < n; ++k)
                for (int y0 = 0; y0 < cfgs[k].ny; y0 += sh.ty)
                    for (int x0 = 0; x0 < cfgs[k].nx; x0 += sh.tx) col.push_back(Col{k, x0, y0});
            for (long long j = 0; j < mp.head; ++j)
                for (auto& r : z_chunks(cfgs[col[j].inst].nz, std::min(cfgs[col[j].inst].nz, MAX_CHUNK)))
                    t.push_back(TileDesc{col[j].inst, col[j].x0, col[j].y0, r.first, r.second, 0, 0, 0});
            if (mp.tail_chunk > 0) {
                // chunk index outer, so that the blocks of one chunk level go out together
                int most = 0;
                std::vector<std::vector<std::pair<int, int>>> zr(col.size());
                for (size_t j = (size_t)mp.head; j < col.size(); ++j) {
                    zr[j] = z_chunks(cfgs[col[j].inst].nz, mp.tail_chunk);
                    most = std::max(most, (int)zr[j].size());
                }
                for (int q = 0; q < most; ++q)
                    for (size_t j = (size_t)mp.head; j < col.size(); ++j)
                        if (q < (int)zr[j].size())
                            t.push_back(TileDesc{col[j].inst, col[j].x0, col[j].y0, zr[j][q].first,
                                                 zr[j][q].second, 0, 0, 0});
            }
            return t;
        }
    }
    for (int k = 0; k < n; ++k) {
        const lbm_config& c = cfgs[k];
        for (auto& r : z_chunks(c.nz, chunk_z(c, sh, cols_all)))
            for (int y0 = 0; y0 < c.ny; y0 += sh.ty)
                for (int x0 = 0; x0 < c.nx; x0 += sh.tx)
                    t.push_back(TileDesc{k, x0, y0, r.first, r.second, 0, 0, 0});
    }
    return t;
}

void carve(const lbm_config* cfgs, int n, Carver& cv, Layout& L) {
    L.inst.assign(n, InstDev{});
    L.glob = (StepGlobals*)cv.take(sizeof(StepGlobals));
    L.d_inst = (InstDev*)cv.take(sizeof(InstDev) * n);
    size_t maxt = 0;
    for (int k = 0; k < NSHAPES; ++k) maxt = std::max(maxt, make_tiles(cfgs, n, SHAPES[k]).size());
    L.d_tiles = (TileDesc*)cv.take(sizeof(TileDesc) * maxt);
    L.tile_cap = maxt;
    size_t need_stage = 0;
    for (int k = 0; k < n; ++k) {
        const lbm_config& c = cfgs[k];
        InstDev& I = L.inst[k];
        I.nx = c.nx;
        I.ny = c.ny;
        I.nz = c.nz;
        I.top_bc = c.top_bc;
        I.N = (long long)c.nx * c.ny * c.nz;
        const size_t eb = elem_bytes(c.prec), cb = comp_bytes(c.prec);
        I.inplace = c.inplace;
        if (c.inplace) {
            // one buffer read and written in place, plus the wall ghost slots
            I.pop[0] = I.pop[1] = cv.take(2 * 19 * I.N * eb);
            I.ghost = cv.take(2 * 10 * (size_t)c.nx * c.ny * eb);
        } else {
            for (int p = 0; p < 2; ++p) I.pop[p] = cv.take(2 * 19 * I.N * eb);
            I.ghost = nullptr;
        }
        for (int p = 0; p < 3; ++p) I.rho[p] = cv.take(2 * I.N * cb);
        I.cot = (double*)cv.take(sizeof(double) * c.nx * c.ny);
        I.hcol = cv.take(cb * c.nx * c.ny);
        I.acc = (double*)cv.take(sizeof(double) * 8);
        I.err = (int*)cv.take(sizeof(int));
        I.desc = (double*)cv.take(sizeof(double) * 8);
        I.t8x = (c.nx + 7) / 8;
        I.t8y = (c.ny + 7) / 8;
        I.t8z = (c.nz + 7) / 8;
        I.nb_max = c.max_beads;
        I.max_nbr = MAX_NBR;
        if (c.max_beads > 0) {
            I.fext = cv.take(3 * I.N * cb);
            I.ust = cv.take(3 * I.N * cb);
            I.gcol = cv.take(3 * I.N * cb);
            I.ntile = I.t8x * I.t8y * I.t8z;
            I.nword = (int)(I.N >> 5) + 1;
            I.tflag = (unsigned*)cv.take(sizeof(unsigned) * 2 * ((size_t)I.ntile + 1));
            I.tlist = (int*)cv.take(sizeof(int) * 2 * (size_t)I.ntile);
            I.nbit = (unsigned*)cv.take(sizeof(unsigned) * 2 * (size_t)I.nword);
            const size_t vb = sizeof(double) * 3 * c.max_beads;
            I.bx = (double*)cv.take(vb);
            I.bv = (double*)cv.take(vb);
            I.bF = (double*)cv.take(vb);
            I.bvh = (double*)cv.take(vb);
            I.bx2 = (double*)cv.take(vb);
            I.bx0 = (double*)cv.take(vb);
            for (int b = 0; b < 2; ++b) {
                I.bK[b] = (int4*)cv.take(sizeof(int4) * (size_t)c.max_beads);
                I.bR[b] = (float4*)cv.take(sizeof(float4) * (size_t)c.max_beads);
            }
            I.bfil = (int*)cv.take(sizeof(int) * c.max_beads);
            I.bpos = (int*)cv.take(sizeof(int) * c.max_beads);
            I.nbr = (int*)cv.take(sizeof(int) * (size_t)c.max_beads * MAX_NBR);
            I.nnbr = (int*)cv.take(sizeof(int) * c.max_beads);
            I.lab = (int*)cv.take(sizeof(int) * 3 * (size_t)c.max_beads);
            const double rl = rlist_of(c);
            I.cgx = std::max(1, (int)floor(c.nx / rl));
            I.cgy = std::max(1, (int)floor(c.ny / rl));
            I.cgz = std::max(1, (int)floor(c.nz / rl));
            const size_t ncell = (size_t)I.cgx * I.cgy * I.cgz;
            I.ccount = (int*)cv.take(sizeof(int) * ncell);
            I.cbeads = (int*)cv.take(sizeof(int) * ncell * CELL_CAP);
            I.bxf = (float*)cv.take(sizeof(float) * 3 * (size_t)c.max_beads);
            I.max_edges = 16 * c.max_beads + 64;
            I.edges = (int2*)cv.take(sizeof(int2) * (size_t)I.max_edges);
            I.nedges = (int*)cv.take(sizeof(int));
            I.net = (double*)cv.take(sizeof(double) * 6 * (size_t)c.max_beads);
            I.netout = (double*)cv.take(sizeof(double) * 10);
            I.csr_row = (int*)cv.take(sizeof(int) * ((size_t)c.max_beads + 1));
            I.csr_cnt = (int*)cv.take(sizeof(int) * 2 * (size_t)c.max_beads);
            I.csr_col = (int*)cv.take(sizeof(int) * 2 * (size_t)I.max_edges);
            I.csr_val = (double*)cv.take(sizeof(double) * 2 * (size_t)I.max_edges);
        }
        need_stage = std::max(need_stage, (size_t)(2 * 19 * I.N * sizeof(double)));
        need_stage = std::max(need_stage, (size_t)(5 * I.N * sizeof(double)));
    }
    need_stage = std::max(need_stage, (size_t)PROFILE_MAX_BINS * 24);  // deposit profiles
    L.stage_bytes = std::min(need_stage, STAGE_BYTES);
    L.stage = (double*)cv.take(L.stage_bytes);
}

lbm_status check_config(const lbm_config& c) {
    if (c.nx < 1 || c.ny < 1 || c.nz < 2) return LBM_EINVAL;
    // 32-bit element offsets inside one population buffer: 38 N < 2^32
    if ((long long)c.nx * c.ny * c.nz * 38 >= (1LL << 32)) return LBM_EINVAL;
    if (c.prec < LBM_FP64 || c.prec > LBM_BF16_SHIFTED) return LBM_EINVAL;
    if (!(c.tau_R > 0.5) || !(c.tau_B > 0.5)) return LBM_EINVAL;
    if (!(c.rho0 > 0.0) || c.beta < 0.0 || c.beta > 1.0 || c.sigma < 0.0) return LBM_EINVAL;
    if (c.J0 < 0.0 || c.K <= 0.0) return LBM_EINVAL;
    if (c.top_bc != 0 && c.top_bc != 1) return LBM_EINVAL;
    if (c.inplace != 0 && c.inplace != 1) return LBM_EINVAL;
    if (c.shape != 0 && c.shape != 1) return LBM_EINVAL;
    if (!(c.a > 0 && c.b > 0 && c.c > 0 && c.width > 0)) return LBM_EINVAL;
    if (!(c.theta_deg > 0.0 && c.theta_deg < 180.0)) return LBM_EINVAL;
    if (c.max_beads < 0) return LBM_EINVAL;
    if (c.max_beads > 0) {
        if (c.substeps < 1 || !(c.bead_mass > 0) || !(c.d0 > 0) || !(c.Rm > c.d0)) return LBM_EINVAL;
        if (c.rc <= c.d0 && (c.eps_coh > 0 || c.eps_s > 0)) return LBM_EINVAL;
    }
    return LBM_OK;
}

double cot_deg(double t) {
    const double r = t * (M_PI / 180.0);
    return cos(r) / sin(r);
}

}  // namespace

struct lbm_handle {
    std::vector<lbm_config> cfg;
    Layout L;
    cudaStream_t stream = nullptr;
    long long step = 0;  // host mirror of the device step counter
    int prec = 0;
    bool any_beads_cap = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;
    int max_nb = 0;
    int shape = 0;  // index into SHAPES
    // the fused kernel may pull by bulk row copies (32- and 16-bit storage, every nx % 4 == 0)
    bool bulk = false;
    bool inplace = false;  // esoteric-pull storage (every instance of the batch)
    // second stream of a step: column heights and the neighbour list run beside
    // the coupling-field pass (fork/join by events, captured into the graph)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ev_begun = nullptr, ev_side = nullptr, ev_forced = nullptr, ev_next = nullptr;
    // the bead start (flags, cells, neighbour list, first kick-drift) of the current
    // step has been enqueued; every step then enqueues the start of the next one
    bool beads_ready = false;
    ~lbm_handle() {
        if (side) {
            cudaStreamSynchronize(side);
            cudaStreamDestroy(side);
        }
        for (cudaEvent_t e : {ev_start, ev_begun, ev_side, ev_forced, ev_next})
            if (e) cudaEventDestroy(e);
    }
};

#define CK(x)                                   \
    do {                                        \
        if ((x) != cudaSuccess) {               \
            (void)cudaGetLastError();           \
            return LBM_ECUDA;                   \
        }                                       \
    } while (0)

namespace {

// dynamic shared memory of the fused kernel: the staged pull of one plane (bulk
// rows carry 4 extra columns on each side; 16-bit bulk staging keeps two planes)
template <class S>
constexpr size_t stage_bytes(int tx, int ty, bool bulk) {
    return (size_t)19 * S::WORDS * ty * (bulk ? tx + 8 : tx) * 4 * ((bulk && S::WORDS == 1) ? 2 : 1);
}

// Resident blocks per SM the fused kernel's register budget is sized for.  FP32 and
// 16-bit storage: the tiling's own (128 registers a thread).  FP64: half as many blocks,
// 255 registers a thread: the FP64 form is bound by B300's narrow FP64 pipe, not by
// latency, and at 128 registers it spilled 1.4 KB a thread (44 bytes at 255)
template <class S>
struct MinBlocks {
    static constexpr bool F64 = std::is_same<S, StoreF64>::value;
    static constexpr int of32x8 = F64 ? 1 : 2;
    static constexpr int of32x4 = F64 ? 2 : 4;
};

template <class S, int TX, int TY, int MINB>
lbm_status prepare_one() {
    const size_t dyn = stage_bytes<S>(TX, TY, false);
    if (dyn > 0) {
        CK(cudaFuncSetAttribute(k_stream_collide<S, TX, TY, MINB, false, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        CK(cudaFuncSetAttribute(k_stream_collide<S, TX, TY, MINB, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    }
    if constexpr (S::WORDS > 0)
        CK(cudaFuncSetAttribute(k_stream_collide<S, TX, TY, MINB, true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes<S>(TX, TY, true)));
    return LBM_OK;
}


// per-kernel attributes, set once before any launch or capture
template <class S>
lbm_status prepare_fused() {
    lbm_status st = prepare_one<S, 32, 8, MinBlocks<S>::of32x8>();
    if (st == LBM_OK) st = prepare_one<S, 32, 4, MinBlocks<S>::of32x4>();
    return st;
}

template <class S>
lbm_status launch_fused(lbm_handle* h) {
    const Shape& sh = SHAPES[h->shape];
    const int nb = h->L.ntiles;
    const InstDev* in = h->L.d_inst;
    const TileDesc* td = h->L.d_tiles;
    const bool bulk = S::WORDS > 0 && h->bulk && sh.bulk != 0;
    constexpr bool W = S::WORDS != 0;
    if (sh.tx == 32 && sh.ty == 8 && sh.minb == 2) {
        if (h->inplace)
            k_stream_collide<S, 32, 8, MinBlocks<S>::of32x8, false, true><<<nb, 256, stage_bytes<S>(32, 8, false), h->stream>>>(
                in, td, h->L.glob);
        else if (bulk)
            k_stream_collide<S, 32, 8, MinBlocks<S>::of32x8, W, false><<<nb, 256, stage_bytes<S>(32, 8, true), h->stream>>>(
                in, td, h->L.glob);
        else
            k_stream_collide<S, 32, 8, MinBlocks<S>::of32x8, false, false><<<nb, 256, stage_bytes<S>(32, 8, false), h->stream>>>(
                in, td, h->L.glob);
    } else if (sh.tx == 32 && sh.ty == 4 && sh.minb == 4) {
        if (h->inplace)
            k_stream_collide<S, 32, 4, MinBlocks<S>::of32x4, false, true><<<nb, 128, stage_bytes<S>(32, 4, false), h->stream>>>(
                in, td, h->L.glob);
        else if (bulk)
            k_stream_collide<S, 32, 4, MinBlocks<S>::of32x4, W, false><<<nb, 128, stage_bytes<S>(32, 4, true), h->stream>>>(
                in, td, h->L.glob);
        else
            k_stream_collide<S, 32, 4, MinBlocks<S>::of32x4, false, false><<<nb, 128, stage_bytes<S>(32, 4, false), h->stream>>>(
                in, td, h->L.glob);
    } else {
        return LBM_EINVAL;
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

// select a tile shape: rebuild and upload the tile table
lbm_status set_shape(lbm_handle* h, int k) {
    std::vector<TileDesc> tiles = make_tiles(h->cfg.data(), (int)h->cfg.size(), SHAPES[k]);
    if (tiles.size() > h->L.tile_cap || tiles.empty()) return LBM_EINVAL;
    CK(cudaMemcpyAsync(h->L.d_tiles, tiles.data(), sizeof(TileDesc) * tiles.size(), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->L.ntiles = (int)tiles.size();
    h->shape = k;
    h->graph_dirty = true;
    return LBM_OK;
}

template <class S>
lbm_status launch_heights(lbm_handle* h, cudaStream_t st);

// Bead start of a step on stream st: clear the flag set, step-start kernel
// (cells, flags, reach bits, first kick-drift), neighbour list.  ahead = 1 starts
// the step after the one whose sub-steps have run (it overlaps that step's fused
// kernel); ahead = 0 starts the current step (the first one, or after the host
// changed the beads).
lbm_status launch_bead_start(lbm_handle* h, cudaStream_t st, int ahead) {
    const int n = (int)h->cfg.size();
    size_t maxclr = 0;
    for (auto& I : h->L.inst)
        maxclr = std::max(maxclr, (size_t)I.ntile + 1 + (size_t)I.cgx * I.cgy * I.cgz + (size_t)I.nword);
    k_bead_clear<<<dim3((unsigned)std::min<size_t>((maxclr + 255) / 256, 4 * 148), n), 256, 0, st>>>(
        h->L.d_inst, h->L.glob, ahead);
    const dim3 gw((h->max_nb * 32 + 255) / 256, n);  // one warp per bead
    k_bead_begin<<<gw, 256, 0, st>>>(h->L.d_inst, h->L.glob, ahead);
    k_bead_nlist<<<gw, 256, 0, st>>>(h->L.d_inst);
    CK(cudaGetLastError());
    return LBM_OK;
}

// One step with beads.  Main stream: coupling fields, the sub-steps, the fused
// kernel.  Side stream: column heights (from the start of the step), then, once
// the sub-steps are done, the start of the next step beside the fused kernel;
// the step ends when both streams have.  Events, if given, bracket the fused launch.
template <class S>
lbm_status launch_bead_step(lbm_handle* h, cudaEvent_t before, cudaEvent_t after) {
    using T = typename S::T;
    const int n = (int)h->cfg.size();
    CK(cudaEventRecord(h->ev_start, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->ev_start, 0));
    lbm_status st = launch_heights<S>(h, h->side);
    if (st != LBM_OK) return st;
    CK(cudaEventRecord(h->ev_side, h->side));
    int maxt = 0;
    for (auto& I : h->L.inst) maxt = std::max(maxt, I.ntile);
    const dim3 fgrid(std::min(maxt, 3 * 148), n);  // every resident block of k_bead_field
    if (h->inplace)
        k_bead_field<S, true><<<fgrid, 512, 0, h->stream>>>(h->L.d_inst, h->L.glob);
    else
        k_bead_field<S, false><<<fgrid, 512, 0, h->stream>>>(h->L.d_inst, h->L.glob);
    const int S_ = h->cfg[0].substeps;
    // blocks of 64 threads, so that the FP64 integration and the stencils of a few
    // hundred beads spread over many SMs; sixteen lanes per bead up to 2048 beads in
    // the whole batch (measured faster at 800), four beyond (more beads per warp share
    // the per-bead FP64 steps, which the narrow FP64 pipe makes the limit at 16,000
    // beads in one lattice and at 18,000 over 64)
    int total_nb = 0;
    for (auto& I : h->L.inst) total_nb += I.nb;
    if (total_nb <= 2048) {
        const dim3 g((h->max_nb * 16 + 63) / 64, n);
        for (int s = 1; s <= S_; ++s) k_bead_force<T, 16><<<g, 64, 0, h->stream>>>(h->L.d_inst, h->L.glob, s);
    } else {
        const dim3 g((h->max_nb * 4 + 63) / 64, n);
        for (int s = 1; s <= S_; ++s) k_bead_force<T, 4><<<g, 64, 0, h->stream>>>(h->L.d_inst, h->L.glob, s);
    }
    CK(cudaGetLastError());
    CK(cudaStreamWaitEvent(h->stream, h->ev_side, 0));  // column heights before the fused kernel
    CK(cudaEventRecord(h->ev_forced, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->ev_forced, 0));
    st = launch_bead_start(h, h->side, 1);
    if (st != LBM_OK) return st;
    CK(cudaEventRecord(h->ev_next, h->side));
    if (before) CK(cudaEventRecord(before, h->stream));
    st = launch_fused<S>(h);
    if (st != LBM_OK) return st;
    if (after) CK(cudaEventRecord(after, h->stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_next, 0));
    return LBM_OK;
}

template <class S>
lbm_status launch_heights(lbm_handle* h, cudaStream_t st) {
    using T = typename S::T;
    int maxc = 0;
    bool any = false;
    for (size_t k = 0; k < h->cfg.size(); ++k) {
        maxc = std::max(maxc, h->cfg[k].nx * h->cfg[k].ny);
        any |= h->cfg[k].J0 > 0 && h->cfg[k].evap_start >= 0;
    }
    if (!any) return LBM_OK;
    k_column_height<T><<<dim3((maxc + HCOL_X - 1) / HCOL_X, (unsigned)h->cfg.size()), dim3(HCOL_X, HCOL_Z), 0,
                         st>>>(h->L.d_inst, h->L.glob);
    CK(cudaGetLastError());
    return LBM_OK;
}

// one step: with beads the pipelined bead step; else column heights, fused kernel
// (events, if given, bracket the fused launch on the handle's stream)
template <class S>
lbm_status enqueue_step(lbm_handle* h, cudaEvent_t before = nullptr, cudaEvent_t after = nullptr) {
    if (h->max_nb > 0) return launch_bead_step<S>(h, before, after);
    lbm_status st = launch_heights<S>(h, h->stream);
    if (st != LBM_OK) return st;
    if (before) CK(cudaEventRecord(before, h->stream));
    st = launch_fused<S>(h);
    if (st != LBM_OK) return st;
    if (after) CK(cudaEventRecord(after, h->stream));
    return LBM_OK;
}

// the bead start of the current step, once after creation or a host change of the beads
lbm_status ensure_bead_start(lbm_handle* h) {
    if (h->max_nb == 0 || h->beads_ready) return LBM_OK;
    lbm_status st = launch_bead_start(h, h->stream, 0);
    if (st == LBM_OK) h->beads_ready = true;
    return st;
}

lbm_status enqueue_step_any(lbm_handle* h) {
    switch (h->prec) {
        case LBM_FP64: return enqueue_step<StoreF64>(h);
        case LBM_FP32: return enqueue_step<StoreF32>(h);
        case LBM_FP16_SHIFTED: return enqueue_step<StoreF16>(h);
        default: return enqueue_step<StoreB16>(h);
    }
}

template <class S>
lbm_status run_moments(lbm_handle* h, int k) {
    const InstDev& I = h->L.inst[k];
    const int bt = 256;
    k_moments<S><<<(unsigned)((I.N + bt - 1) / bt), bt, 0, h->stream>>>(I, h->step, 0, I.N, nullptr);
    CK(cudaGetLastError());
    return LBM_OK;
}

lbm_status run_moments_any(lbm_handle* h, int k) {
    switch (h->prec) {
        case LBM_FP64: return run_moments<StoreF64>(h, k);
        case LBM_FP32: return run_moments<StoreF32>(h, k);
        case LBM_FP16_SHIFTED: return run_moments<StoreF16>(h, k);
        default: return run_moments<StoreB16>(h, k);
    }
}

lbm_status upload_tables(lbm_handle* h) {
    CK(cudaMemcpyAsync(h->L.d_inst, h->L.inst.data(), sizeof(InstDev) * h->L.inst.size(),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->graph_dirty = true;
    return LBM_OK;
}

lbm_status latched(lbm_handle* h) {
    int worst = 0;
    for (auto& I : h->L.inst) {
        int e = 0;
        CK(cudaMemcpyAsync(&e, I.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        worst |= e;
    }
    if (worst & ERR_NAN) return LBM_ENAN;
    if (worst & ERR_FENE) return LBM_EFENE;
    if (worst & ERR_BEAD) return LBM_EBEAD_OOB;
    if (worst & ERR_TIMEOUT) return LBM_ETIMEOUT;
    if (worst & ERR_CAP) return LBM_ECAPACITY;
    return LBM_OK;
}

template <class S>
lbm_status init_instance(lbm_handle* h, int k) {
    const lbm_config& c = h->cfg[k];
    const InstDev& I = h->L.inst[k];
    const int bt = 256;
    k_init_droplet<S><<<(unsigned)((I.N + bt - 1) / bt), bt, 0, h->stream>>>(I, c.shape, c.cx, c.cy, c.cz, c.a,
                                                                              c.b, c.c, c.width);
    CK(cudaGetLastError());
    return run_moments<S>(h, k);
}

lbm_status init_any(lbm_handle* h, int k) {
    switch (h->prec) {
        case LBM_FP64: return init_instance<StoreF64>(h, k);
        case LBM_FP32: return init_instance<StoreF32>(h, k);
        case LBM_FP16_SHIFTED: return init_instance<StoreF16>(h, k);
        default: return init_instance<StoreB16>(h, k);
    }
}


// populations <-> host FP64 [2][19][N], chunked through the staging buffer
template <class S>
lbm_status pop_transfer(lbm_handle* h, int k, double* host, bool to_host) {
    const InstDev& I = h->L.inst[k];
    const long long total = 19 * I.N;
    const long long chunk = (long long)(h->L.stage_bytes / (2 * sizeof(double)));
    const int bt = 256;
    for (long long t0 = 0; t0 < total; t0 += chunk) {
        const long long len = std::min(chunk, total - t0);
        const unsigned nb = (unsigned)((len + bt - 1) / bt);
        if (to_host) {
            k_pop_to_f64<S><<<nb, bt, 0, h->stream>>>(I, h->step, t0, len, h->L.stage);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(host + t0, h->L.stage, len * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaMemcpyAsync(host + total + t0, h->L.stage + len, len * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
        } else {
            CK(cudaMemcpyAsync(h->L.stage, host + t0, len * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(h->L.stage + len, host + total + t0, len * sizeof(double),
                               cudaMemcpyHostToDevice, h->stream));
            k_pop_from_f64<S><<<nb, bt, 0, h->stream>>>(I, h->step, t0, len, h->L.stage);
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

// node fields (moments / colour / fext) -> host FP64, chunked
template <class S>
lbm_status node_field(lbm_handle* h, int k, unsigned field, double* host) {
    using T = typename S::T;
    const InstDev& I = h->L.inst[k];
    const int per = field == LBM_FIELD_MOMENTS ? 5 : (field == LBM_FIELD_FEXT ? 3 : 1);
    const long long chunk = (long long)(h->L.stage_bytes / (per * sizeof(double)));
    const int bt = 256;
    for (long long n0 = 0; n0 < I.N; n0 += chunk) {
        const long long len = std::min(chunk, I.N - n0);
        const unsigned nb = (unsigned)((per * len + bt - 1) / bt);
        if (field == LBM_FIELD_MOMENTS)
            k_moments<S><<<nb, bt, 0, h->stream>>>(I, h->step, n0, len, h->L.stage);
        else if (field == LBM_FIELD_COLOUR)
            k_colour<T><<<nb, bt, 0, h->stream>>>(I, h->step, n0, len, h->L.stage);
        else
            // the flag set of the last fused launch (step - 1)
            k_fext<T><<<nb, bt, 0, h->stream>>>(I, (int)((h->step + 1) & 1), n0, len, h->L.stage);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(host + per * n0, h->L.stage, per * len * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

template <class S>
lbm_status mass_of(lbm_handle* h, int k, double* out2) {
    const InstDev& I = h->L.inst[k];
    CK(cudaMemsetAsync(h->L.stage, 0, 2 * sizeof(double), h->stream));
    k_mass<S><<<4 * 148, 256, 0, h->stream>>>(I, h->step, h->L.stage);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out2, h->L.stage, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

#define DISPATCH(fn, ...)                                          \
    switch (h->prec) {                                             \
        case LBM_FP64: return fn<StoreF64>(__VA_ARGS__);           \
        case LBM_FP32: return fn<StoreF32>(__VA_ARGS__);           \
        case LBM_FP16_SHIFTED: return fn<StoreF16>(__VA_ARGS__);   \
        default: return fn<StoreB16>(__VA_ARGS__);                 \
    }

lbm_status pop_transfer_any(lbm_handle* h, int k, double* host, bool to_host) {
    DISPATCH(pop_transfer, h, k, host, to_host)
}
lbm_status node_field_any(lbm_handle* h, int k, unsigned f, double* host) { DISPATCH(node_field, h, k, f, host) }
lbm_status mass_any(lbm_handle* h, int k, double* out2) { DISPATCH(mass_of, h, k, out2) }

lbm_status h0_any(lbm_handle* h, int k) {
    const InstDev& I = h->L.inst[k];
    CK(cudaMemsetAsync(I.acc + 1, 0, sizeof(double), h->stream));
    const int ncol = I.nx * I.ny, bt = 256;
    if (h->prec == LBM_FP64)
        k_h0<double><<<(ncol + bt - 1) / bt, bt, 0, h->stream>>>(I, h->step);
    else
        k_h0<float><<<(ncol + bt - 1) / bt, bt, 0, h->stream>>>(I, h->step);
    CK(cudaGetLastError());
    return LBM_OK;
}

// capture one time step into a graph (all step dependence lives on the device)
lbm_status build_graph(lbm_handle* h) {
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    h->stream = cap;
    lbm_status st = LBM_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = LBM_ECUDA;
    if (st == LBM_OK) st = enqueue_step_any(h);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess) st = LBM_ECUDA;
    h->stream = saved;
    cudaStreamDestroy(cap);
    if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return st;
    }
    h->graph = g;
    CK(cudaGraphInstantiate(&h->gexec, g, 0));
    h->graph_dirty = false;
    return LBM_OK;
}

bool valid_inst(lbm_handle* h, int inst) { return h && inst >= 0 && inst < (int)h->cfg.size(); }

// random straight filaments inside the liquid (C > 0.9), non-overlapping
lbm_status place_random(lbm_handle* h, int k, int nw, int nbf, double spacing, uint64_t seed,
                        std::vector<double>& X) {
    const lbm_config& c = h->cfg[k];
    const InstDev& I = h->L.inst[k];
    std::vector<double> C(I.N);
    lbm_status st = node_field_any(h, k, LBM_FIELD_COLOUR, C.data());
    if (st != LBM_OK) return st;
    std::vector<double> have(3 * (size_t)I.nb);
    if (I.nb) {
        CK(cudaMemcpy(have.data(), I.bx, sizeof(double) * 3 * I.nb, cudaMemcpyDeviceToHost));
    }
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::normal_distribution<double> G(0.0, 1.0);
    // bounding box of the liquid
    int lo[3] = {c.nx, c.ny, c.nz}, hi[3] = {-1, -1, -1};
    for (long long n = 0; n < I.N; ++n)
        if (C[n] > 0.9) {
            const int p[3] = {(int)(n % c.nx), (int)((n / c.nx) % c.ny), (int)(n / ((long long)c.nx * c.ny))};
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], p[d]);
                hi[d] = std::max(hi[d], p[d]);
            }
        }
    if (hi[0] < 0) return LBM_EINVAL;
    auto colour_at = [&](const double* P) {
        // nearest-node colour (placement only needs "well inside the liquid")
        const int x = wrapi((int)lround(P[0]), c.nx), y = wrapi((int)lround(P[1]), c.ny);
        const int z = (int)lround(P[2]);
        if (z < 0 || z >= c.nz) return -1.0;
        return C[((long long)z * c.ny + y) * c.nx + x];
    };
    // beads already placed, hashed on a grid of cell size d0 for the overlap test
    const double cell = c.d0;
    const int gx = std::max(1, (int)floor(c.nx / cell)), gy = std::max(1, (int)floor(c.ny / cell)),
              gz = std::max(1, (int)ceil((c.nz + 1.0) / cell));
    std::vector<std::vector<int>> grid((size_t)gx * gy * gz);
    std::vector<double> placed = have;
    auto cell_of = [&](const double* P, int& ix, int& iy, int& iz) {
        ix = std::min(gx - 1, std::max(0, (int)floor(P[0] / cell)));
        iy = std::min(gy - 1, std::max(0, (int)floor(P[1] / cell)));
        iz = std::min(gz - 1, std::max(0, (int)floor((P[2] + 1.0) / cell)));
    };
    auto add = [&](int q) {
        int ix, iy, iz;
        cell_of(&placed[3 * q], ix, iy, iz);
        grid[((size_t)iz * gy + iy) * gx + ix].push_back(q);
    };
    for (size_t q = 0; q < placed.size() / 3; ++q) add((int)q);
    auto clash = [&](const double* P) {
        int ix, iy, iz;
        cell_of(P, ix, iy, iz);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int zz = iz + dz;
                    if (zz < 0 || zz >= gz) continue;
                    const int xx = ((ix + dx) % gx + gx) % gx, yy = ((iy + dy) % gy + gy) % gy;
                    for (int q : grid[((size_t)zz * gy + yy) * gx + xx]) {
                        double dd = 0;
                        for (int d = 0; d < 3; ++d) {
                            double e = P[d] - placed[3 * q + d];
                            if (d == 0) e -= c.nx * floor(e / c.nx + 0.5);
                            if (d == 1) e -= c.ny * floor(e / c.ny + 0.5);
                            dd += e * e;
                        }
                        if (dd <= c.d0 * c.d0) return true;
                    }
                }
        return false;
    };
    const long long max_tries = 200000LL + 2000LL * nw;
    long long tries = 0;
    int got = 0;
    while (got < nw && tries < max_tries) {
        ++tries;
        double cen[3], dir[3];
        for (int d = 0; d < 3; ++d) cen[d] = lo[d] + U(rng) * (hi[d] - lo[d] + 1);
        double nrm = 0;
        for (int d = 0; d < 3; ++d) {
            dir[d] = G(rng);
            nrm += dir[d] * dir[d];
        }
        nrm = sqrt(nrm);
        if (nrm == 0) continue;
        for (int d = 0; d < 3; ++d) dir[d] /= nrm;
        std::vector<double> cand(3 * nbf);
        bool ok = true;
        for (int b = 0; b < nbf && ok; ++b) {
            for (int d = 0; d < 3; ++d) cand[3 * b + d] = cen[d] + (b - (nbf - 1) / 2.0) * spacing * dir[d];
            cand[3 * b] -= c.nx * floor(cand[3 * b] / c.nx);
            cand[3 * b + 1] -= c.ny * floor(cand[3 * b + 1] / c.ny);
            if (cand[3 * b + 2] < 1.0 || cand[3 * b + 2] > c.nz - 2.0) ok = false;
            if (ok && colour_at(&cand[3 * b]) <= 0.9) ok = false;
            if (ok && clash(&cand[3 * b])) ok = false;
        }
        if (!ok) continue;
        for (int b = 0; b < nbf; ++b) {
            placed.insert(placed.end(), &cand[3 * b], &cand[3 * b] + 3);
            add((int)(placed.size() / 3 - 1));
        }
        X.insert(X.end(), cand.begin(), cand.end());
        ++got;
    }
    return got == nw ? LBM_OK : LBM_EINVAL;
}

template <class S>
lbm_status droplet_shape(lbm_handle* h, int inst, double* res) {
    using T = typename S::T;
    const InstDev& I = h->L.inst[inst];
    const size_t ncol = (size_t)I.nx * I.ny;
    if ((ncol + 16) * sizeof(double) > h->L.stage_bytes) return LBM_ENOMEM_WS;
    double* out = h->L.stage;  // [4] sums, then h(x,y)
    double* dres = out + 4;
    double* hbuf = out + 16;
    CK(cudaMemsetAsync(out, 0, 16 * sizeof(double), h->stream));
    k_shape_columns<T><<<(unsigned)((ncol + 255) / 256), 256, 0, h->stream>>>(I, h->step, hbuf, out);
    k_shape_finish<S><<<1, 32, 0, h->stream>>>(I, h->step, out, dres);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(res, dres, 10 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // namespace

// ===========================================================================
// Public C ABI
// ===========================================================================
extern "C" {

size_t lbm_workspace_bytes(const lbm_config* cfgs, int n) {
    if (!cfgs || n < 1) return 0;
    Carver cv{nullptr};
    Layout L;
    carve(cfgs, n, cv, L);
    return align_up(cv.off, 256);
}

lbm_status lbm_create(const lbm_config* cfgs, int n, void* dev_ws, size_t ws_bytes, void* stream,
                      lbm_handle** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!cfgs || n < 1 || !dev_ws) return LBM_EINVAL;
    if (((uintptr_t)dev_ws) & 15) return LBM_EINVAL;
    for (int k = 0; k < n; ++k) {
        lbm_status st = check_config(cfgs[k]);
        if (st != LBM_OK) return st;
        if (cfgs[k].prec != cfgs[0].prec || cfgs[k].inplace != cfgs[0].inplace) return LBM_EINVAL;
        if (cfgs[k].max_beads > 0 && cfgs[0].max_beads > 0 && cfgs[k].substeps != cfgs[0].substeps)
            return LBM_EINVAL;
    }
    if (ws_bytes < lbm_workspace_bytes(cfgs, n)) return LBM_ENOMEM_WS;
    lbm_handle* h = new lbm_handle();
    h->cfg.assign(cfgs, cfgs + n);
    h->stream = (cudaStream_t)stream;
    h->prec = cfgs[0].prec;
    h->inplace = cfgs[0].inplace != 0;
    h->bulk = h->prec != LBM_FP64 && !h->inplace;
    for (int k = 0; k < n; ++k) h->bulk = h->bulk && cfgs[k].nx % 4 == 0;
    Carver cv{(char*)dev_ws};
    carve(cfgs, n, cv, h->L);
    // substeps must match across instances with beads: use the first with beads
    for (int k = 0; k < n; ++k)
        if (cfgs[k].max_beads > 0) {
            for (auto& c : h->cfg) c.substeps = cfgs[k].substeps;
            break;
        }
    lbm_status st = LBM_OK;
    auto fail = [&](lbm_status s) {
        delete h;
        return s;
    };
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_begun, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_forced, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_next, cudaEventDisableTiming) != cudaSuccess)
        return fail(LBM_ECUDA);
    if (cudaMemsetAsync(h->L.glob, 0, sizeof(StepGlobals), h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    if (set_shape(h, 0) != LBM_OK) return fail(LBM_ECUDA);
    for (int k = 0; k < n; ++k) {
        const lbm_config& c = h->cfg[k];
        InstDev& I = h->L.inst[k];
        I.tau_R = c.tau_R;
        I.tau_B = c.tau_B;
        I.beta = c.beta;
        I.sigma = c.sigma;
        I.rho0 = c.rho0;
        I.J0 = c.J0;
        I.K = c.K;
        for (int d = 0; d < 3; ++d) I.body[d] = c.body[d];
        I.evap_start = c.evap_start;
        I.substeps = c.substeps;
        I.ks = c.ks;
        I.Rm = c.Rm;
        I.d0 = c.d0;
        I.eps_wca = c.eps_wca;
        I.kb = c.kb;
        I.eps_coh = c.eps_coh;
        I.eps_s = c.eps_s;
        I.rc = c.rc;
        I.gamma = c.gamma;
        I.xi = c.xi;
        I.mu = c.mu;
        I.gamma_t = c.gamma_t;
        I.mass = c.bead_mass;
        I.dt_sub = 1.0 / c.substeps;
        I.hk_sub = 0.5 * I.dt_sub / c.bead_mass;
        I.f_ks = (float)I.ks;
        I.f_Rm2 = (float)(I.Rm * I.Rm);
        I.f_d0 = (float)I.d0;
        I.f_eps_wca = (float)I.eps_wca;
        I.f_kb = (float)I.kb;
        I.f_eps_coh = (float)I.eps_coh;
        I.f_eps_s = (float)I.eps_s;
        I.f_rc = (float)I.rc;
        I.f_gamma = (float)I.gamma;
        I.f_xi = (float)I.xi;
        I.f_mu = (float)I.mu;
        I.f_gamma_t = (float)I.gamma_t;
        I.f_dt_sub = (float)I.dt_sub;
        I.rlist = rlist_of(c);
        I.rcon = c.rcon;
        I.x_src = c.x_src;
        I.x_snk = c.x_snk;
        I.nb = 0;
        std::vector<double> cot((size_t)c.nx * c.ny, cot_deg(c.theta_deg));
        if (cudaMemcpyAsync(I.cot, cot.data(), sizeof(double) * cot.size(), cudaMemcpyHostToDevice, h->stream) !=
                cudaSuccess ||
            cudaMemsetAsync(I.acc, 0, sizeof(double) * 8, h->stream) != cudaSuccess ||
            cudaMemsetAsync(I.err, 0, sizeof(int), h->stream) != cudaSuccess)
            return fail(LBM_ECUDA);
        if (I.fext) {
            const size_t cb = comp_bytes(c.prec);
            if (cudaMemsetAsync(I.fext, 0, 3 * I.N * cb, h->stream) != cudaSuccess ||
                cudaMemsetAsync(I.ust, 0, 3 * I.N * cb, h->stream) != cudaSuccess ||
                cudaMemsetAsync(I.gcol, 0, 3 * I.N * cb, h->stream) != cudaSuccess ||
                cudaMemsetAsync(I.tflag, 0, sizeof(unsigned) * 2 * ((size_t)I.ntile + 1), h->stream) != cudaSuccess ||
                cudaMemsetAsync(I.bF, 0, sizeof(double) * 3 * c.max_beads, h->stream) != cudaSuccess)
                return fail(LBM_ECUDA);
        }
        // cot is needed by cudaMemcpyAsync until the copy ends
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    }
    st = upload_tables(h);
    if (st != LBM_OK) return fail(st);
    switch (h->prec) {
        case LBM_FP64: st = prepare_fused<StoreF64>(); break;
        case LBM_FP32: st = prepare_fused<StoreF32>(); break;
        case LBM_FP16_SHIFTED: st = prepare_fused<StoreF16>(); break;
        default: st = prepare_fused<StoreB16>(); break;
    }
    if (st != LBM_OK) return fail(st);
    for (int k = 0; k < n; ++k) {
        st = init_any(h, k);
        if (st != LBM_OK) return fail(st);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LBM_ECUDA);
    *out = h;
    return LBM_OK;
}

lbm_status lbm_set_substrate_pattern(lbm_handle* h, int inst, const double* theta) {
    if (!valid_inst(h, inst) || !theta) return LBM_EINVAL;
    const lbm_config& c = h->cfg[inst];
    std::vector<double> cot((size_t)c.nx * c.ny);
    for (size_t a = 0; a < cot.size(); ++a) {
        if (!(theta[a] > 0.0 && theta[a] < 180.0)) return LBM_EINVAL;
        cot[a] = cot_deg(theta[a]);
    }
    CK(cudaMemcpyAsync(h->L.inst[inst].cot, cot.data(), sizeof(double) * cot.size(), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_add_nanowires(lbm_handle* h, int inst, int n_wires, double length, const double* centers,
                             const double* dirs, uint64_t seed) {
    if (!valid_inst(h, inst) || n_wires < 0 || !(length > 0)) return LBM_EINVAL;
    if ((centers == nullptr) != (dirs == nullptr)) return LBM_EINVAL;
    const lbm_config& c = h->cfg[inst];
    InstDev& I = h->L.inst[inst];
    if (c.max_beads == 0) return LBM_ECAPACITY;
    const int nbf = std::max(1, (int)lround(length / c.d0));
    if ((long long)I.nb + (long long)n_wires * nbf > c.max_beads) return LBM_ECAPACITY;
    if (n_wires == 0) return LBM_OK;
    CK(cudaStreamSynchronize(h->stream));
    std::vector<double> X;
    if (centers) {
        for (int w = 0; w < n_wires; ++w) {
            double d[3] = {dirs[3 * w], dirs[3 * w + 1], dirs[3 * w + 2]};
            const double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (!(nn > 0)) return LBM_EINVAL;
            for (int b = 0; b < nbf; ++b) {
                double P[3];
                for (int k = 0; k < 3; ++k) P[k] = centers[3 * w + k] + (b - (nbf - 1) / 2.0) * c.d0 * d[k] / nn;
                P[0] -= c.nx * floor(P[0] / c.nx);
                P[1] -= c.ny * floor(P[1] / c.ny);
                if (!(P[2] > -0.5 && P[2] < c.nz - 0.5)) return LBM_EINVAL;
                X.insert(X.end(), P, P + 3);
            }
        }
    } else {
        lbm_status st = place_random(h, inst, n_wires, nbf, c.d0, seed ? seed : c.seed, X);
        if (st != LBM_OK) return st;
    }
    // filament ids continue after the existing ones
    int fil0 = 0;
    if (I.nb > 0) {
        int lastfil = 0;
        CK(cudaMemcpy(&lastfil, I.bfil + I.nb - 1, sizeof(int), cudaMemcpyDeviceToHost));
        fil0 = lastfil + 1;
    }
    const int nadd = n_wires * nbf;
    std::vector<int> fil(nadd), pos(nadd);
    for (int w = 0; w < n_wires; ++w)
        for (int b = 0; b < nbf; ++b) {
            fil[w * nbf + b] = fil0 + w;
            pos[w * nbf + b] = b;
        }
    std::vector<double> zero(3 * (size_t)nadd, 0.0);
    CK(cudaMemcpy(I.bx + 3 * I.nb, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(I.bv + 3 * I.nb, zero.data(), sizeof(double) * zero.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(I.bF + 3 * I.nb, zero.data(), sizeof(double) * zero.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(I.bfil + I.nb, fil.data(), sizeof(int) * nadd, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(I.bpos + I.nb, pos.data(), sizeof(int) * nadd, cudaMemcpyHostToDevice));
    I.nb += nadd;
    h->max_nb = 0;
    for (auto& J : h->L.inst) h->max_nb = std::max(h->max_nb, J.nb);
    h->beads_ready = false;
    return upload_tables(h);
}

lbm_status lbm_step(lbm_handle* h, int n_steps) {
    if (!h || n_steps < 0) return LBM_EINVAL;
    const int n = (int)h->cfg.size();
    if (n_steps > 0) {
        lbm_status st = ensure_bead_start(h);
        if (st != LBM_OK) return st;
    }
    for (int s = 0; s < n_steps; ++s) {
        // h0 is taken from the moments of the first evaporating step
        for (int k = 0; k < n; ++k) {
            const lbm_config& c = h->cfg[k];
            if (c.J0 > 0 && c.evap_start >= 0 && h->step == c.evap_start) {
                lbm_status st = h0_any(h, k);
                if (st != LBM_OK) return st;
            }
        }
        if (n_steps - s >= 2 || h->gexec) {
            if (h->graph_dirty) {
                lbm_status st = build_graph(h);
                if (st != LBM_OK) return st;
            }
            CK(cudaGraphLaunch(h->gexec, h->stream));
        } else {
            lbm_status st = enqueue_step_any(h);
            if (st != LBM_OK) return st;
        }
        ++h->step;
    }
    return LBM_OK;
}

lbm_status lbm_profile_steps(lbm_handle* h, int n_steps, double* ms_fluid, double* ms_step) {
    if (!h || n_steps < 1 || !ms_fluid || !ms_step) return LBM_EINVAL;
    const int n = (int)h->cfg.size();
    std::vector<cudaEvent_t> ev(3 * (size_t)n_steps + 1, nullptr);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto& f : ev)
                if (f) cudaEventDestroy(f);
            return LBM_ECUDA;
        }
    lbm_status st = ensure_bead_start(h);
    for (int s = 0; s < n_steps && st == LBM_OK; ++s) {
        cudaEventRecord(ev[3 * s], h->stream);
        for (int k = 0; k < n && st == LBM_OK; ++k) {
            const lbm_config& c = h->cfg[k];
            if (c.J0 > 0 && c.evap_start >= 0 && h->step == c.evap_start) st = h0_any(h, k);
        }
        if (st != LBM_OK) break;
        switch (h->prec) {
            case LBM_FP64: st = enqueue_step<StoreF64>(h, ev[3 * s + 1], ev[3 * s + 2]); break;
            case LBM_FP32: st = enqueue_step<StoreF32>(h, ev[3 * s + 1], ev[3 * s + 2]); break;
            case LBM_FP16_SHIFTED: st = enqueue_step<StoreF16>(h, ev[3 * s + 1], ev[3 * s + 2]); break;
            default: st = enqueue_step<StoreB16>(h, ev[3 * s + 1], ev[3 * s + 2]); break;
        }
        ++h->step;
    }
    cudaEventRecord(ev[3 * (size_t)n_steps], h->stream);
    double tf = 0.0, ts = 0.0;
    if (st == LBM_OK && cudaStreamSynchronize(h->stream) == cudaSuccess) {
        for (int s = 0; s < n_steps; ++s) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[3 * s + 1], ev[3 * s + 2]);
            cudaEventElapsedTime(&b, ev[3 * s], ev[3 * s + 3 <= 3 * n_steps ? 3 * s + 3 : 3 * n_steps]);
            tf += a;
            ts += b;
        }
        *ms_fluid = tf / n_steps;
        *ms_step = ts / n_steps;
    } else if (st == LBM_OK) {
        st = LBM_ECUDA;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    (void)cudaGetLastError();
    return st;
}

lbm_status lbm_autotune(lbm_handle* h, int steps_per_candidate, int* chosen, double* best_ms) {
    if (!h || steps_per_candidate < 1) return LBM_EINVAL;
    int best = -1;
    double bt = 1e300;
    // tile-edge nodes of the next moment buffer are zeroed by the shape that
    // wrote the previous one; after a change of shape the moments are rebuilt
    // from the populations so that the new edges start from zero
    auto reshape = [&](int k) {
        lbm_status st = set_shape(h, k);
        for (int i = 0; st == LBM_OK && i < (int)h->cfg.size(); ++i) st = run_moments_any(h, i);
        return st;
    };
    for (int k = 0; k < NSHAPES; ++k) {
        lbm_status st = reshape(k);
        if (st != LBM_OK) return st;
        double f = 0, s = 0;
        st = lbm_profile_steps(h, 1, &f, &s);  // first launch of this shape: untimed
        if (st == LBM_OK) st = lbm_profile_steps(h, steps_per_candidate, &f, &s);
        if (st != LBM_OK) return st;
        if (f < bt) {
            bt = f;
            best = k;
        }
    }
    lbm_status st = reshape(best);
    if (st != LBM_OK) return st;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = bt;
    return LBM_OK;
}

int lbm_tiling_count(void) { return NSHAPES; }

lbm_status lbm_set_tiling(lbm_handle* h, int index) {
    if (!h || index < 0 || index >= NSHAPES) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    lbm_status st = set_shape(h, index);
    for (int i = 0; st == LBM_OK && i < (int)h->cfg.size(); ++i) st = run_moments_any(h, i);
    if (st == LBM_OK) CK(cudaStreamSynchronize(h->stream));
    return st;
}

lbm_status lbm_tiling_table(const lbm_config* cfgs, int n, int index, int* out, int cap, int* n_blocks) {
    if (!cfgs || n < 1 || index < 0 || index >= NSHAPES || cap < 0 || !n_blocks || (cap > 0 && !out))
        return LBM_EINVAL;
    for (int k = 0; k < n; ++k) {
        lbm_status st = check_config(cfgs[k]);
        if (st != LBM_OK) return st;
    }
    const Shape& sh = SHAPES[index];
    const std::vector<TileDesc> t = make_tiles(cfgs, n, sh);
    *n_blocks = (int)t.size();
    if ((size_t)cap < t.size()) return LBM_ENOMEM_WS;
    for (size_t i = 0; i < t.size(); ++i) {
        const lbm_config& c = cfgs[t[i].inst];
        const int v[7] = {t[i].inst, t[i].x0, t[i].y0, t[i].z0, t[i].z1, std::min(sh.tx, c.nx - t[i].x0),
                          std::min(sh.ty, c.ny - t[i].y0)};
        for (int j = 0; j < 7; ++j) out[7 * i + j] = v[j];
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_handle* h) {
    if (!h) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    return latched(h);
}

lbm_status lbm_clear_error(lbm_handle* h) {
    if (!h) return LBM_EINVAL;
    for (auto& I : h->L.inst) CK(cudaMemsetAsync(I.err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

static size_t field_bytes(const lbm_config& c, int nb, unsigned f) {
    const size_t N = (size_t)c.nx * c.ny * c.nz;
    switch (f) {
        case LBM_FIELD_POPULATIONS: return 2 * 19 * N * 8;
        case LBM_FIELD_MOMENTS: return 5 * N * 8;
        case LBM_FIELD_COLOUR: return N * 8;
        case LBM_FIELD_BEAD_X:
        case LBM_FIELD_BEAD_V:
        case LBM_FIELD_BEAD_F: return 3 * (size_t)nb * 8;
        case LBM_FIELD_BEAD_TOPO: return 2 * (size_t)nb * 4;
        case LBM_FIELD_ACCUM: return 6 * 8;
        case LBM_FIELD_FEXT: return 3 * N * 8;
        case LBM_FIELD_THETA_COT: return (size_t)c.nx * c.ny * 8;
        case LBM_FIELD_BEAD_POTENTIAL:
        case LBM_FIELD_BEAD_CURRENT: return (size_t)nb * 8;
        default: return 0;
    }
}

lbm_status lbm_read_accum_async(lbm_handle* h, int inst, double* dst) {
    if (!valid_inst(h, inst) || !dst) return LBM_EINVAL;
    const InstDev& I = h->L.inst[inst];
    dst[0] = (double)h->step;
    dst[5] = (double)I.nb;
    CK(cudaMemcpyAsync(dst + 1, I.acc + 1, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return LBM_OK;
}

lbm_status lbm_read_fields(lbm_handle* h, int inst, unsigned field, void* dst, size_t bytes) {
    if (!valid_inst(h, inst) || !dst) return LBM_EINVAL;
    const lbm_config& c = h->cfg[inst];
    const InstDev& I = h->L.inst[inst];
    const size_t need = field_bytes(c, I.nb, field);
    if (need == 0 || bytes != need) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    lbm_status st = LBM_OK;
    switch (field) {
        case LBM_FIELD_POPULATIONS: st = pop_transfer_any(h, inst, (double*)dst, true); break;
        case LBM_FIELD_MOMENTS:
        case LBM_FIELD_COLOUR: st = node_field_any(h, inst, field, (double*)dst); break;
        case LBM_FIELD_FEXT:
            if (!I.fext) {
                memset(dst, 0, bytes);
                break;
            }
            st = node_field_any(h, inst, field, (double*)dst);
            break;
        case LBM_FIELD_BEAD_X:
        case LBM_FIELD_BEAD_V:
        case LBM_FIELD_BEAD_F: {
            if (I.nb == 0) break;
            const double* p = field == LBM_FIELD_BEAD_X ? I.bx : (field == LBM_FIELD_BEAD_V ? I.bv : I.bF);
            CK(cudaMemcpy(dst, p, bytes, cudaMemcpyDeviceToHost));
            break;
        }
        case LBM_FIELD_BEAD_TOPO: {
            if (I.nb == 0) break;
            std::vector<int> f(I.nb), p(I.nb);
            CK(cudaMemcpy(f.data(), I.bfil, sizeof(int) * I.nb, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(p.data(), I.bpos, sizeof(int) * I.nb, cudaMemcpyDeviceToHost));
            int* o = (int*)dst;
            for (int a = 0; a < I.nb; ++a) {
                o[2 * a] = f[a];
                o[2 * a + 1] = p[a];
            }
            break;
        }
        case LBM_FIELD_ACCUM: {
            double a[8];
            CK(cudaMemcpy(a, I.acc, sizeof(a), cudaMemcpyDeviceToHost));
            double* o = (double*)dst;
            o[0] = (double)h->step;
            o[1] = a[1];
            o[2] = a[2];
            o[3] = a[3];
            o[4] = a[4];
            o[5] = (double)I.nb;
            break;
        }
        case LBM_FIELD_THETA_COT: CK(cudaMemcpy(dst, I.cot, bytes, cudaMemcpyDeviceToHost)); break;
        case LBM_FIELD_BEAD_POTENTIAL:
        case LBM_FIELD_BEAD_CURRENT: {
            const double* p = field == LBM_FIELD_BEAD_POTENTIAL ? I.net : I.net + 5 * (size_t)I.nb_max;
            CK(cudaMemcpy(dst, p, bytes, cudaMemcpyDeviceToHost));
            break;
        }
    }
    if (st != LBM_OK) return st;
    return latched(h);
}

lbm_status lbm_write_fields(lbm_handle* h, int inst, unsigned field, const void* src, size_t bytes) {
    if (!valid_inst(h, inst) || !src) return LBM_EINVAL;
    const lbm_config& c = h->cfg[inst];
    InstDev& I = h->L.inst[inst];
    const size_t need = field_bytes(c, I.nb, field);
    if (need == 0 || bytes != need) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    switch (field) {
        case LBM_FIELD_POPULATIONS: {
            lbm_status st = pop_transfer_any(h, inst, (double*)src, false);
            if (st != LBM_OK) return st;
            st = run_moments_any(h, inst);
            if (st != LBM_OK) return st;
            CK(cudaStreamSynchronize(h->stream));
            return LBM_OK;
        }
        case LBM_FIELD_BEAD_X:
        case LBM_FIELD_BEAD_V:
        case LBM_FIELD_BEAD_F: {
            if (I.nb == 0) return LBM_OK;
            double* p = field == LBM_FIELD_BEAD_X ? I.bx : (field == LBM_FIELD_BEAD_V ? I.bv : I.bF);
            CK(cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice));
            h->beads_ready = false;  // the next step starts the beads again
            return LBM_OK;
        }
        case LBM_FIELD_ACCUM: {
            const double* a = (const double*)src;
            if (a[0] < 0 || a[0] != floor(a[0])) return LBM_EINVAL;
            // the step counter is shared by all instances of the handle
            h->step = (long long)a[0];
            StepGlobals g{h->step, 0u, 0, h->step};
            CK(cudaMemcpy(h->L.glob, &g, sizeof(g), cudaMemcpyHostToDevice));
            h->beads_ready = false;  // the flag set follows the step's parity
            double v[8] = {a[0], a[1], a[2], a[3], a[4], 0, 0, 0};
            CK(cudaMemcpy(I.acc, v, sizeof(v), cudaMemcpyHostToDevice));
            return LBM_OK;
        }
        default: return LBM_EINVAL;
    }
}

lbm_status lbm_deposit_descriptors(lbm_handle* h, int inst, lbm_descriptors* out) {
    if (!valid_inst(h, inst) || !out) return LBM_EINVAL;
    const InstDev& I = h->L.inst[inst];
    memset(out, 0, sizeof(*out));
    CK(cudaStreamSynchronize(h->stream));
    if (I.nb > 0) {
        CK(cudaMemsetAsync(I.nedges, 0, sizeof(int), h->stream));
        k_desc_edges<<<(I.nb + 127) / 128, 128, 0, h->stream>>>(h->L.d_inst, inst);
        k_desc_solve<<<1, 1024, 0, h->stream>>>(h->L.d_inst, inst);
        CK(cudaGetLastError());
        double d[8];
        CK(cudaMemcpyAsync(d, I.desc, sizeof(d), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        out->S_x = d[0];
        out->n_clusters = (int)d[1];
        out->percolates = (int)d[2];
        out->n_bonds = (int)d[3];
    }
    out->n_beads = I.nb;
    double m[2];
    lbm_status st = mass_any(h, inst, m);
    if (st != LBM_OK) return st;
    out->mass_R = m[0];
    out->mass_B = m[1];
    double a[8];
    CK(cudaMemcpy(a, I.acc, sizeof(a), cudaMemcpyDeviceToHost));
    out->h0 = a[1];
    out->evaporated = a[2];
    out->top_in = a[3];
    out->top_out = a[4];
    out->step = h->step;
    return latched(h);
}

lbm_status lbm_deposit_conductivity(lbm_handle* h, int inst, double tol, int max_iter,
                                    lbm_conductivity* out) {
    if (!valid_inst(h, inst) || !out || !(tol > 0.0) || max_iter < 1) return LBM_EINVAL;
    const lbm_config& c = h->cfg[inst];
    if (!(c.x_snk > c.x_src)) return LBM_EINVAL;
    const InstDev& I = h->L.inst[inst];
    memset(out, 0, sizeof(*out));
    out->I_ref = 1.0 / (c.x_snk - c.x_src);
    CK(cudaStreamSynchronize(h->stream));
    if (I.nb_max == 0) return latched(h);
    CK(cudaMemsetAsync(I.nedges, 0, sizeof(int), h->stream));
    if (I.nb > 0) k_desc_edges<<<(I.nb + 127) / 128, 128, 0, h->stream>>>(h->L.d_inst, inst);
    // the search direction in shared memory when it fits (up to 25,600 beads)
    const size_t p_bytes = sizeof(double) * (size_t)I.nb_max;
    const int p_smem = p_bytes <= (size_t)200 * 1024 ? 1 : 0;
    if (p_smem)
        CK(cudaFuncSetAttribute(k_net_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_bytes));
    k_net_solve<<<1, NET_THREADS, p_smem ? p_bytes : 0, h->stream>>>(h->L.d_inst, inst, tol, max_iter, p_smem);
    CK(cudaGetLastError());
    double o[10];
    CK(cudaMemcpyAsync(o, I.netout, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->kappa = o[0];
    out->I_tot = o[1];
    out->I_sink = o[2];
    out->I_ref = o[3];
    out->residual = o[4];
    out->iterations = (int)o[5];
    out->n_src = (int)o[6];
    out->n_snk = (int)o[7];
    out->n_edges = (int)o[8];
    const lbm_status st = latched(h);
    if (st != LBM_OK) return st;
    return o[9] != 0.0 ? LBM_OK : LBM_ETIMEOUT;
}

lbm_status lbm_deposit_profiles(lbm_handle* h, int inst, int axis, double lo, double hi, int nbins,
                                double centre, double half_width, double* S_x, double* g, int* n_bonds,
                                int* n_beads) {
    if (!valid_inst(h, inst) || !S_x || !g || (axis != 0 && axis != 1) || nbins < 1 ||
        nbins > PROFILE_MAX_BINS || !(hi > lo) || !(half_width >= 0.0) || !std::isfinite(centre))
        return LBM_EINVAL;
    const InstDev& I = h->L.inst[inst];
    CK(cudaStreamSynchronize(h->stream));
    if (I.nb_max == 0) {
        for (int k = 0; k < nbins; ++k) {
            S_x[k] = g[k] = 0.0;
            if (n_bonds) n_bonds[k] = 0;
            if (n_beads) n_beads[k] = 0;
        }
        return latched(h);
    }
    double* Sd = h->L.stage;
    double* gd = Sd + nbins;
    int* bd = (int*)(gd + nbins);
    int* nd = bd + nbins;
    k_net_profiles<<<1, NET_THREADS, 0, h->stream>>>(h->L.d_inst, inst, axis, lo, hi, nbins, centre, half_width,
                                                      Sd, gd, bd, nd);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(S_x, Sd, sizeof(double) * nbins, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(g, gd, sizeof(double) * nbins, cudaMemcpyDeviceToHost, h->stream));
    if (n_bonds) CK(cudaMemcpyAsync(n_bonds, bd, sizeof(int) * nbins, cudaMemcpyDeviceToHost, h->stream));
    if (n_beads) CK(cudaMemcpyAsync(n_beads, nd, sizeof(int) * nbins, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return latched(h);
}

lbm_status lbm_droplet_shape(lbm_handle* h, int inst, lbm_shape* out) {
    if (!valid_inst(h, inst) || !out) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    double r[10];
    lbm_status st;
    switch (h->prec) {
        case LBM_FP64: st = droplet_shape<StoreF64>(h, inst, r); break;
        case LBM_FP32: st = droplet_shape<StoreF32>(h, inst, r); break;
        case LBM_FP16_SHIFTED: st = droplet_shape<StoreF16>(h, inst, r); break;
        default: st = droplet_shape<StoreB16>(h, inst, r); break;
    }
    if (st != LBM_OK) return st;
    out->volume = r[0];
    out->height = r[1];
    out->xc = r[2];
    out->yc = r[3];
    out->r_x = r[4];
    out->r_y = r[5];
    out->theta_x = r[6];
    out->theta_y = r[7];
    out->v_x = r[8];
    out->v_y = r[9];
    return latched(h);
}

lbm_status lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_EINVAL;
    cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    delete h;
    return LBM_OK;
}

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument or configuration";
        case LBM_ENOMEM_WS: return "workspace too small";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_ENAN: return "non-finite or non-positive density";
        case LBM_EFENE: return "FENE bond reached its maximum extension";
        case LBM_EBEAD_OOB: return "bead left the fluid or moved too far in one step";
        case LBM_ETIMEOUT: return "device-side wait gave up";
        case LBM_ESTATE: return "call not valid in the current state";
        case LBM_ECAPACITY: return "capacity exceeded";
        default: return "unknown status";
    }
}

}  // extern "C"

// ===========================================================================
// Descriptors without any allocation: the same contact-graph kernels, with
// their scratch (instance table, labels, flags, edge list, counters) in one
// file-scope device array instead of a caller-provided workspace.
// ===========================================================================
namespace {

constexpr int NOALLOC_MAX_BEADS = LBM_NOALLOC_MAX_BEADS;
constexpr int NOALLOC_MAX_EDGES = 8 * NOALLOC_MAX_BEADS + 64;
constexpr size_t NA_INST = 0;                                   // InstDev copy
constexpr size_t NA_LAB = 1024;                                 // 3 x max int labels/flags
constexpr size_t NA_EDGES = NA_LAB + sizeof(int) * 3 * (size_t)NOALLOC_MAX_BEADS;
constexpr size_t NA_COUNT = NA_EDGES + sizeof(int2) * (size_t)NOALLOC_MAX_EDGES;  // edge counter
constexpr size_t NA_ERR = NA_COUNT + 256;                                         // error bits
constexpr size_t NA_BYTES = NA_ERR + 256;
static_assert(sizeof(InstDev) <= NA_LAB, "instance table must fit its slot");

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the array per device, found once with that device current.
unsigned char* g_noalloc_ptr[256] = {nullptr};
std::mutex g_noalloc_mu;

__global__ void k_noalloc_finish(const int* __restrict__ err, double* __restrict__ out) { out[4] = (double)*err; }

}  // namespace

extern "C" lbm_status lbm_deposit_descriptors_noalloc(const double* bead_x, const int* bead_fil,
                                                      const int* bead_pos, int n_beads, int nx, int ny,
                                                      double rcon, double x_src, double x_snk, double* out,
                                                      void* stream) {
    if (!bead_x || !bead_fil || !bead_pos || !out || n_beads < 1 || nx < 1 || ny < 1 || !(rcon > 0.0))
        return LBM_EINVAL;
    if (n_beads > NOALLOC_MAX_BEADS) return LBM_ECAPACITY;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return LBM_EINVAL;
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_ptr[dev] = (unsigned char*)p;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    InstDev J{};
    J.nx = nx;
    J.ny = ny;
    J.nb = n_beads;
    J.nb_max = NOALLOC_MAX_BEADS;
    J.bx = const_cast<double*>(bead_x);
    J.bfil = const_cast<int*>(bead_fil);
    J.bpos = const_cast<int*>(bead_pos);
    J.rcon = rcon;
    J.x_src = x_src;
    J.x_snk = x_snk;
    J.lab = (int*)(base + NA_LAB);
    J.edges = (int2*)(base + NA_EDGES);
    J.nedges = (int*)(base + NA_COUNT);
    J.max_edges = NOALLOC_MAX_EDGES;
    J.err = (int*)(base + NA_ERR);
    J.desc = out;
    InstDev* slot = (InstDev*)(base + NA_INST);
    // pageable source: the copy has read J before the call returns
    CK(cudaMemcpyAsync(slot, &J, sizeof(J), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(J.nedges, 0, sizeof(int), st));
    CK(cudaMemsetAsync(J.err, 0, sizeof(int), st));
    k_desc_edges<<<(n_beads + 127) / 128, 128, 0, st>>>(slot, 0);
    k_desc_solve<<<1, 1024, 0, st>>>(slot, 0);
    k_noalloc_finish<<<1, 1, 0, st>>>(J.err, out);
    CK(cudaGetLastError());
    return LBM_OK;
}
