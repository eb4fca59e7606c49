// Droplet-shape observables of the drying runs (Sec. III.A, Fig. 2): height,
// volume, centre, footprint radii, contact angles and mean flow at half the
// footprint radius, from the moments of the current step.  Readings: the
// liquid column height is h(x,y) = sum_z (1 + C)/2; the footprint radii are
// half the positive runs of C on the first fluid layer through the centre,
// ends at the linearly interpolated C = 0 crossings; the contact angles follow
// the spherical-cap relation tan(theta/2) = H / r in each principal section;
// the flow is the mean of j/rho over the liquid nodes of one column.
#pragma once

#include "kernels_fluid.cuh"

namespace lbm {

// out[0..3] = sum h, sum x h, sum y h, max h (as bits); h into hbuf[ny][nx]
template <typename T>
__global__ void k_shape_columns(InstDev I, long long step, double* __restrict__ hbuf, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncol = I.nx * I.ny;
    double h = 0.0;
    if (c < ncol) {
        const T* rho = (const T*)I.rho[step % 3];
        for (int z = 0; z < I.nz; ++z) h += (1.0 + (double)colour_of(rho, I.N, (long long)z * ncol + c)) / 2.0;
        hbuf[c] = h;
    }
    const double x = c < ncol ? (double)(c % I.nx) : 0.0, y = c < ncol ? (double)(c / I.nx) : 0.0;
    double v[3] = {h, x * h, y * h};
    double m = h;
    for (int o = 16; o > 0; o >>= 1) {
        for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) atomicAdd(out + k, v[k]);
        atomicMax((unsigned long long*)(out + 3), (unsigned long long)__double_as_longlong(m));
    }
}

// C = 0 crossings of the positive run through index i0 of a profile p(i), i in [0, n)
template <class F>
__device__ void crossing_run(int n, int i0, F p, double& left, double& right) {
    left = right = i0;
    if (i0 < 0 || i0 >= n || !(p(i0) > 0.0)) return;
    int lo = i0, hi = i0;
    while (lo - 1 >= 0 && p(lo - 1) > 0.0) --lo;
    while (hi + 1 < n && p(hi + 1) > 0.0) ++hi;
    left = lo > 0 ? lo - p(lo) / (p(lo) - p(lo - 1)) : (double)lo;
    right = hi + 1 < n ? hi + p(hi) / (p(hi) - p(hi + 1)) : (double)hi;
}

// one thread: out[0..3] from k_shape_columns; writes res[10] = volume, height,
// xc, yc, r_x, r_y, theta_x, theta_y, v_x, v_y
template <class S>
__global__ void k_shape_finish(InstDev I, long long step, const double* __restrict__ out, double* __restrict__ res) {
    using T = typename S::T;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nx = I.nx, ny = I.ny;
    const long long N = I.N;
    const T* rho = (const T*)I.rho[step % 3];
    const double V = out[0], H = __longlong_as_double((long long)((const unsigned long long*)out)[3]);
    const double xc = V > 0.0 ? out[1] / V : 0.0, yc = V > 0.0 ? out[2] / V : 0.0;
    const int ix = (int)floor(xc + 0.5), iy = (int)floor(yc + 0.5);
    auto C0 = [&](int x, int y) { return (double)colour_of(rho, N, (long long)y * nx + x); };
    double lx, rx, ly, ry;
    crossing_run(nx, ix, [&](int x) { return C0(x, min(max(iy, 0), ny - 1)); }, lx, rx);
    crossing_run(ny, iy, [&](int y) { return C0(min(max(ix, 0), nx - 1), y); }, ly, ry);
    const double r_x = (rx - lx) / 2.0, r_y = (ry - ly) / 2.0;
    const double rad = 180.0 / 3.14159265358979323846;
    auto column_mean = [&](double xf, double yf, int d) {
        const int x = wrapi((int)floor(xf + 0.5), nx), y = wrapi((int)floor(yf + 0.5), ny);
        double s = 0.0;
        int cnt = 0;
        for (int z = 0; z < I.nz; ++z) {
            const long long n = ((long long)z * ny + y) * nx + x;
            if (!(colour_of(rho, N, n) > T(0))) continue;
            T m[5];
            stream_moments<S>(I, step, n, m);
            s += (double)m[2 + d] / ((double)m[0] + (double)m[1]);
            ++cnt;
        }
        return cnt ? s / cnt : 0.0;
    };
    res[0] = V;
    res[1] = H;
    res[2] = xc;
    res[3] = yc;
    res[4] = r_x;
    res[5] = r_y;
    res[6] = 2.0 * atan2(H, r_x) * rad;
    res[7] = 2.0 * atan2(H, r_y) * rad;
    res[8] = column_mean(xc + r_x / 2.0, yc, 0);
    res[9] = column_mean(xc, yc + r_y / 2.0, 1);
}

}  // namespace lbm
