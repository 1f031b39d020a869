/*
 * Random sequential addition (RSA) of polydisperse hard spheres in a cube.
 *
 * Input generator only: it produces the DEM-shaped particle positions that
 * stand in for the charged-sphere packings of the paper's examples (Sec. 3.1,
 * spheres with elastic walls).  It holds none of the multipole method's
 * arithmetic and is shared, as a pure input source, by the CPU oracle and the
 * GPU library.
 *
 * Recipe: radii r ~ U[rmin, rmax] are drawn, sorted in descending order and
 * inserted one by one at uniform random centres in [r, L - r]^3 (hard walls).
 * A candidate is rejected if it overlaps (|c_i - c_j| < r_i + r_j) a sphere
 * already placed; after max_attempts rejections for one sphere the insertion
 * stalls, L grows by 1 % and the whole packing restarts from the same seed.
 * A cell grid with cells no smaller than 2 rmax bounds each overlap test to
 * the 27 surrounding cells.
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), top 53 bits -> [0, 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double sm64_unit(uint64_t *s) {
    return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}

static int cmp_desc(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/*
 * Returns the number of restarts used (>= 0), or -1 on allocation failure.
 * xyz: [n,3] centres (out), rad: [n] radii (out, descending), side: cube side
 * actually used (out).
 */
int rsa_pack(int64_t n, uint64_t seed, double phi, double rmin, double rmax,
             int64_t max_attempts, int max_restarts, double *xyz, double *rad,
             double *side_out) {
    uint64_t s = seed;
    double vol = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        rad[i] = rmin + (rmax - rmin) * sm64_unit(&s);
        vol += (4.0 / 3.0) * M_PI * rad[i] * rad[i] * rad[i];
    }
    qsort(rad, (size_t)n, sizeof(double), cmp_desc);
    double L = cbrt(vol / phi);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!next) return -1;
    for (int restart = 0; restart <= max_restarts; ++restart) {
        double cs_min = 2.0 * rmax;
        int64_t nc = (int64_t)floor(L / cs_min);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        double cs = L / (double)nc;
        int64_t ncell = nc * nc * nc;
        int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        if (!head) { free(next); return -1; }
        for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
        uint64_t st = seed ^ 0xD1B54A32D192ED03ULL;
        int stalled = 0;
        for (int64_t i = 0; i < n && !stalled; ++i) {
            double r = rad[i];
            int placed = 0;
            for (int64_t a = 0; a < max_attempts; ++a) {
                double c[3];
                for (int d = 0; d < 3; ++d) c[d] = r + (L - 2.0 * r) * sm64_unit(&st);
                int64_t ci[3];
                for (int d = 0; d < 3; ++d) {
                    ci[d] = (int64_t)floor(c[d] / cs);
                    if (ci[d] >= nc) ci[d] = nc - 1;
                }
                int ok = 1;
                for (int64_t dx = -1; dx <= 1 && ok; ++dx)
                    for (int64_t dy = -1; dy <= 1 && ok; ++dy)
                        for (int64_t dz = -1; dz <= 1 && ok; ++dz) {
                            int64_t x = ci[0] + dx, y = ci[1] + dy, z = ci[2] + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= nc || y >= nc || z >= nc) continue;
                            for (int64_t j = head[(x * nc + y) * nc + z]; j >= 0; j = next[j]) {
                                double ex = c[0] - xyz[3 * j], ey = c[1] - xyz[3 * j + 1],
                                       ez = c[2] - xyz[3 * j + 2];
                                double rr = r + rad[j];
                                if (ex * ex + ey * ey + ez * ez < rr * rr) { ok = 0; break; }
                            }
                        }
                if (ok) {
                    for (int d = 0; d < 3; ++d) xyz[3 * i + d] = c[d];
                    int64_t cell = (ci[0] * nc + ci[1]) * nc + ci[2];
                    next[i] = head[cell];
                    head[cell] = i;
                    placed = 1;
                    break;
                }
            }
            if (!placed) stalled = 1;
        }
        free(head);
        if (!stalled) {
            free(next);
            *side_out = L;
            return restart;
        }
        L *= 1.01;
    }
    free(next);
    return -2;
}
