// Deposit analysis kernels (Sec. II.B): the Kirchhoff network of Eqs. (15)-(18)
// and the per-bin morphology profiles of Eqs. (13)-(14).
//
// Both run as one block per instance: the deposit of one lattice holds at most
// a few 10^4 beads, and one block keeps every global reduction in a fixed
// order without any wait on another block.
#pragma once

#include "kernels_beads.cuh"

namespace lbm {

constexpr int NET_THREADS = 1024;

// deterministic block sum of one value per thread (fixed shuffle and shared trees);
// every thread gets the result
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // `red` may still be read by the previous call
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// deterministic block sums of two values per thread
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        red[w] = a;
        red[32 + w] = b;
    }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        sa += red[k];
        sb += red[32 + k];
    }
    a = sa;
    b = sb;
}

// conductance and end points of edge e (bond or contact) with its nearest-image length
__device__ __forceinline__ double edge_conductance(const InstDev& I, int a, int b) {
    const double dx = min_image(I.bx[3 * b] - I.bx[3 * a], I.nx),
                 dy = min_image(I.bx[3 * b + 1] - I.bx[3 * a + 1], I.ny),
                 dz = I.bx[3 * b + 2] - I.bx[3 * a + 2];
    return 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
}

// Kirchhoff network of one instance (edges from k_desc_edges):
//   1. CSR of the symmetric conductance matrix (rows sorted by column, so that
//      every later sum runs in a fixed order);
//   2. Jacobi-preconditioned CG on the free nodes,
//        sum_j G_ij (V_i - V_j) = 0,  V = 1 on x < x_src, V = 0 on x > x_snk;
//   3. node currents I_i = 1/2 sum_j G_ij |V_i - V_j| (Eq. (15)), the currents
//      leaving the source and entering the sink, kappa* (Eq. (18)).
// Output I.netout: kappa, I_tot, I_sink, I_ref, residual, iterations, n_src,
// n_snk, n_edges, converged.
// dynamic shared memory: the search direction p when the instance's beads fit (p_smem)
__global__ void __launch_bounds__(NET_THREADS) k_net_solve(const InstDev* __restrict__ insts, int only,
                                                           double tol, int max_iter, int p_smem) {
    const InstDev I = insts[only];
    const int n = I.nb, nbm = I.nb_max;
    const int ne = min(*I.nedges, I.max_edges);
    const int tid = threadIdx.x, NTH = blockDim.x;
    double* V = I.net;
    double* r = V + nbm;
    extern __shared__ double p_sh[];
    double* q = r + 2 * (size_t)nbm;
    double* dinv = q + nbm;
    double* cur = dinv + nbm;
    double* p = p_smem ? p_sh : r + nbm;  // zero on the fixed nodes throughout
    double* diag = cur;                   // sum_j G_ij during the solve; the node currents after it
    int* row = I.csr_row;   // [nbm + 1]
    int* cnt = I.csr_cnt;   // [nbm]
    int* cls = cnt + nbm;   // [nbm]: 1 source, 2 sink, 0 free
    int* col = I.csr_col;   // [2 max_edges]
    double* val = I.csr_val;
    __shared__ double red[64];
    __shared__ int scan[NET_THREADS];

    for (int a = tid; a < n; a += NTH) {
        cnt[a] = 0;
        const double x = I.bx[3 * a];
        cls[a] = x < I.x_src ? 1 : (x > I.x_snk ? 2 : 0);
    }
    __syncthreads();
    for (int e = tid; e < ne; e += NTH) {
        const int2 ed = I.edges[e];
        atomicAdd(cnt + ed.x, 1);
        atomicAdd(cnt + ed.y, 1);
    }
    __syncthreads();
    // exclusive scan of the degrees: contiguous chunks per thread, then across threads
    const int chunk = (n + NTH - 1) / NTH;
    const int a0 = min(n, tid * chunk), a1 = min(n, a0 + chunk);
    int local = 0;
    for (int a = a0; a < a1; ++a) local += cnt[a];
    scan[tid] = local;
    __syncthreads();
    for (int o = 1; o < NTH; o <<= 1) {
        const int v = tid >= o ? scan[tid - o] : 0;
        __syncthreads();
        scan[tid] += v;
        __syncthreads();
    }
    int run = scan[tid] - local;
    for (int a = a0; a < a1; ++a) {
        row[a] = run;
        run += cnt[a];
    }
    if (tid == NTH - 1) row[n] = scan[NTH - 1];
    __syncthreads();
    for (int a = tid; a < n; a += NTH) cnt[a] = 0;
    __syncthreads();
    for (int e = tid; e < ne; e += NTH) {
        const int2 ed = I.edges[e];
        const double g = edge_conductance(I, ed.x, ed.y);
        const int sa = row[ed.x] + atomicAdd(cnt + ed.x, 1);
        const int sb = row[ed.y] + atomicAdd(cnt + ed.y, 1);
        col[sa] = ed.y;
        val[sa] = g;
        col[sb] = ed.x;
        val[sb] = g;
    }
    __syncthreads();
    // sort each row by column; diagonal, preconditioner, right-hand side, start vectors
    double bb = 0.0, rz = 0.0, rr = 0.0;
    for (int a = tid; a < n; a += NTH) {
        const int s0 = row[a], s1 = row[a + 1];
        for (int s = s0 + 1; s < s1; ++s) {
            const int c = col[s];
            const double v = val[s];
            int t = s - 1;
            while (t >= s0 && col[t] > c) {
                col[t + 1] = col[t];
                val[t + 1] = val[t];
                --t;
            }
            col[t + 1] = c;
            val[t + 1] = v;
        }
        double d = 0.0, b = 0.0;
        for (int s = s0; s < s1; ++s) {
            d += val[s];
            if (cls[col[s]] == 1) b += val[s];
        }
        const bool fr = cls[a] == 0;
        V[a] = cls[a] == 1 ? 1.0 : 0.0;
        diag[a] = d;
        dinv[a] = (fr && d > 0.0) ? 1.0 / d : 0.0;
        r[a] = fr ? b : 0.0;  // start from V = 0 on the free nodes
        p[a] = dinv[a] * r[a];
        bb += r[a] * r[a];
        rz += r[a] * p[a];
    }
    bb = block_sum(bb, red);
    rz = block_sum(rz, red);
    rr = bb;
    int it = 0;
    const double stop = tol * tol * bb;
    while (it < max_iter && rr > stop && rz > 0.0) {
        // q = A p on the free rows: A_ii = sum_j G_ij, A_ij = -G_ij (j free)
        // (p vanishes on the fixed nodes, so their columns drop out by themselves)
        double pq = 0.0;
        for (int a = tid; a < n; a += NTH) {
            double v = 0.0;
            if (cls[a] == 0) {
                double off = 0.0;
                const int s1 = row[a + 1];
                for (int s = row[a]; s < s1; ++s) off += val[s] * p[col[s]];
                v = diag[a] * p[a] - off;
            }
            q[a] = v;
            pq += p[a] * v;
        }
        pq = block_sum(pq, red);
        if (!(pq > 0.0)) break;
        const double alpha = rz / pq;
        double rz1 = 0.0, rr1 = 0.0;
        for (int a = tid; a < n; a += NTH) {
            if (cls[a] == 0) {
                V[a] += alpha * p[a];
                r[a] -= alpha * q[a];
            }
            rz1 += r[a] * dinv[a] * r[a];
            rr1 += r[a] * r[a];
        }
        block_sum2(rz1, rr1, red);
        const double beta = rz1 / rz;
        rz = rz1;
        rr = rr1;
        for (int a = tid; a < n; a += NTH) p[a] = dinv[a] * r[a] + beta * p[a];
        __syncthreads();
        ++it;
    }
    // currents
    double isrc = 0.0, isnk = 0.0;
    const double iref = 1.0 / (I.x_snk - I.x_src);
    double nsrc = 0.0, nsnk = 0.0;
    for (int a = tid; a < n; a += NTH) {
        double c = 0.0;
        for (int s = row[a]; s < row[a + 1]; ++s) {
            const int j = col[s];
            const double iij = val[s] * (V[a] - V[j]);
            c += fabs(iij);
            if (cls[a] == 1 && cls[j] != 1) isrc += iij;
            if (cls[a] == 2 && cls[j] != 2) isnk -= iij;
        }
        cur[a] = 0.5 * c / iref;
        nsrc += cls[a] == 1;
        nsnk += cls[a] == 2;
    }
    isrc = block_sum(isrc, red);
    isnk = block_sum(isnk, red);
    nsrc = block_sum(nsrc, red);
    nsnk = block_sum(nsnk, red);
    if (tid == 0) {
        double* o = I.netout;
        o[0] = isrc / iref;
        o[1] = isrc;
        o[2] = isnk;
        o[3] = iref;
        o[4] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        o[5] = it;
        o[6] = nsrc;
        o[7] = nsnk;
        o[8] = ne;
        o[9] = (rr <= stop || rz <= 0.0) ? 1.0 : 0.0;
    }
}

// Per-bin profiles (Eqs. (13)-(14)) into caller scratch:
// sums[nbins] (sum of 2 cos^2 - 1), nbond[nbins], nbead[nbins], then S and g.
__global__ void __launch_bounds__(NET_THREADS) k_net_profiles(const InstDev* __restrict__ insts, int only, int axis,
                                                              double lo, double hi, int nbins, double centre,
                                                              double half_width, double* __restrict__ S,
                                                              double* __restrict__ g, int* __restrict__ nbond,
                                                              int* __restrict__ nbead) {
    const InstDev I = insts[only];
    const int n = I.nb, tid = threadIdx.x, NTH = blockDim.x;
    const int other = 1 - axis;
    const double w = (hi - lo) / nbins;
    __shared__ double red[32];
    for (int k = tid; k < nbins; k += NTH) {
        S[k] = 0.0;
        nbond[k] = 0;
        nbead[k] = 0;
    }
    __syncthreads();
    for (int a = tid; a < n; a += NTH) {
        const double* X = I.bx + 3 * a;
        if (fabs(X[other] - centre) <= half_width) {
            const double f = floor((X[axis] - lo) / w);
            if (f >= 0.0 && f < nbins) atomicAdd(nbead + (int)f, 1);
        }
        if (a + 1 < n && I.bfil[a + 1] == I.bfil[a] && I.bpos[a + 1] == I.bpos[a] + 1) {
            const double d[3] = {min_image(I.bx[3 * (a + 1)] - X[0], I.nx),
                                 min_image(I.bx[3 * (a + 1) + 1] - X[1], I.ny), I.bx[3 * (a + 1) + 2] - X[2]};
            const double m[2] = {X[0] + 0.5 * d[0], X[1] + 0.5 * d[1]};
            if (fabs(m[other] - centre) <= half_width) {
                const double f = floor((m[axis] - lo) / w);
                if (f >= 0.0 && f < nbins) {
                    atomicAdd(S + (int)f, 2.0 * d[0] * d[0] / (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - 1.0);
                    atomicAdd(nbond + (int)f, 1);
                }
            }
        }
    }
    __syncthreads();
    double tot = 0.0;
    for (int k = tid; k < nbins; k += NTH) tot += nbead[k];
    tot = block_sum(tot, red);
    const double mean = tot / nbins;
    for (int k = tid; k < nbins; k += NTH) {
        S[k] = nbond[k] > 0 ? S[k] / nbond[k] : 0.0;
        g[k] = mean > 0.0 ? nbead[k] / mean : 0.0;
    }
}

}  // namespace lbm
