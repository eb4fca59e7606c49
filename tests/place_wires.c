/*
 * Seeded random placement of straight wires inside an ellipsoidal droplet: the
 * input generator behind tests/inputs.py:wires_in_droplet.  Geometry only (no
 * arithmetic of the simulated method); it serves the oracle and GPU sides alike.
 *
 * Candidates: centre uniform in the box `lo`..`hi`, direction isotropic (three
 * normal deviates, normalised), beads at centre + (k - (n_beads-1)/2) spacing dir.
 * A candidate is taken when every bead has lo_z <= z <= hi_z, ellipsoidal radius
 * q < q_max about `c` with semi-axes `ax` (minimum image in x and y), and lies
 * further than min_dist from every bead taken before (minimum image).  Random
 * numbers: splitmix64 (Steele, Lea, Flood 2014) -> uniform doubles (53 bits),
 * normals by Box-Muller.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t sm64(uint64_t* s) {
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static double unif(uint64_t* s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
static double gauss(uint64_t* s) {
    double u = unif(s), v = unif(s);
    if (u < 1e-300) u = 1e-300;
    return sqrt(-2.0 * log(u)) * cos(6.283185307179586 * v);
}
static double wrapd(double e, double L) { return e - L * floor(e / L + 0.5); }

/* returns the number of wires placed (<= n_wires); cen, dir: [n_wires][3] */
int place_wires(uint64_t seed, int n_wires, int n_beads, double spacing, int nx, int ny, int nz,
                const double* c, const double* ax, double q_max, double min_dist, double zlo,
                double zhi, long long max_tries, double* cen, double* dir) {
    double lo[3] = {c[0] - ax[0], c[1] - ax[1], c[2] - ax[2] > zlo ? c[2] - ax[2] : zlo};
    double hi[3] = {c[0] + ax[0], c[1] + ax[1], c[2] + ax[2] < zhi ? c[2] + ax[2] : zhi};
    const double cell = min_dist;
    int gx = (int)(nx / cell), gy = (int)(ny / cell), gz = (int)((nz + 2) / cell) + 2;
    if (gx < 1) gx = 1;
    if (gy < 1) gy = 1;
    const int cap = 16;
    long long ncell = (long long)gx * gy * gz;
    int* cells = malloc(sizeof(int) * ncell * cap);
    int* cnt = calloc(ncell, sizeof(int));
    double* pts = malloc(sizeof(double) * 3 * ((size_t)n_wires * n_beads + 1));
    double* X = malloc(sizeof(double) * 3 * n_beads);
    int npts = 0, got = 0;
    uint64_t s = seed;
    for (long long t = 0; t < max_tries && got < n_wires; ++t) {
        double C[3], D[3], nd = 0.0;
        for (int k = 0; k < 3; ++k) C[k] = lo[k] + unif(&s) * (hi[k] - lo[k]);
        for (int k = 0; k < 3; ++k) {
            D[k] = gauss(&s);
            nd += D[k] * D[k];
        }
        nd = sqrt(nd);
        if (!(nd > 0.0)) continue;
        for (int k = 0; k < 3; ++k) D[k] /= nd;
        int ok = 1;
        for (int b = 0; b < n_beads && ok; ++b) {
            double* P = X + 3 * b;
            double q = 0.0;
            for (int k = 0; k < 3; ++k) P[k] = C[k] + (b - (n_beads - 1) / 2.0) * spacing * D[k];
            if (P[2] < zlo || P[2] > zhi) ok = 0;
            double e[3] = {wrapd(P[0] - c[0], nx), wrapd(P[1] - c[1], ny), P[2] - c[2]};
            for (int k = 0; k < 3; ++k) q += (e[k] / ax[k]) * (e[k] / ax[k]);
            if (sqrt(q) >= q_max) ok = 0;
            P[0] -= nx * floor(P[0] / nx);
            P[1] -= ny * floor(P[1] / ny);
        }
        for (int b = 0; b < n_beads && ok; ++b) {
            const double* P = X + 3 * b;
            int ix = (int)(P[0] / cell), iy = (int)(P[1] / cell), iz = (int)((P[2] + 1.0) / cell) + 1;
            if (ix >= gx) ix = gx - 1;
            if (iy >= gy) iy = gy - 1;
            for (int dz = -1; dz <= 1 && ok; ++dz)
                for (int dy = -1; dy <= 1 && ok; ++dy)
                    for (int dx = -1; dx <= 1 && ok; ++dx) {
                        int zz = iz + dz;
                        if (zz < 0 || zz >= gz) continue;
                        int xx = ((ix + dx) % gx + gx) % gx, yy = ((iy + dy) % gy + gy) % gy;
                        long long cc = ((long long)zz * gy + yy) * gx + xx;
                        for (int m = 0; m < cnt[cc] && ok; ++m) {
                            const double* Q = pts + 3 * (size_t)cells[cc * cap + m];
                            double v0 = wrapd(P[0] - Q[0], nx), v1 = wrapd(P[1] - Q[1], ny), v2 = P[2] - Q[2];
                            if (v0 * v0 + v1 * v1 + v2 * v2 <= min_dist * min_dist) ok = 0;
                        }
                    }
        }
        if (!ok) continue;
        for (int b = 0; b < n_beads; ++b) {
            const double* P = X + 3 * b;
            int ix = (int)(P[0] / cell), iy = (int)(P[1] / cell), iz = (int)((P[2] + 1.0) / cell) + 1;
            if (ix >= gx) ix = gx - 1;
            if (iy >= gy) iy = gy - 1;
            if (iz < 0) iz = 0;
            if (iz >= gz) iz = gz - 1;
            long long cc = ((long long)iz * gy + iy) * gx + ix;
            if (cnt[cc] >= cap) { got = -1; goto done; }
            cells[cc * cap + cnt[cc]++] = npts;
            for (int k = 0; k < 3; ++k) pts[3 * (size_t)npts + k] = P[k];
            ++npts;
        }
        for (int k = 0; k < 3; ++k) {
            cen[3 * got + k] = C[k];
            dir[3 * got + k] = D[k];
        }
        ++got;
    }
done:
    free(cells);
    free(cnt);
    free(pts);
    free(X);
    return got;
}
