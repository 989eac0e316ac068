/*
 * Seeded synthetic lattice inputs, shared by the oracle side and the CUDA side.
 *
 * This file holds no arithmetic of the method being tested (no site products,
 * sums, adjoints or expression evaluation).  It only draws random fields:
 *
 *   - a counter-based stream: every value is a pure function of
 *     (seed, field id, element index), so any slice of a field can be
 *     regenerated on its own and the result does not depend on thread count;
 *     the bit mixer is SplitMix64 (Steele, Lea and Flood, "Fast splittable
 *     pseudorandom number generators", OOPSLA 2014);
 *   - uniforms u in (0,1) from the top 53 bits;
 *   - standard normals by the Box-Muller transform (one pair per two uniforms);
 *   - SU(3) matrices: 9 complex Gaussian entries, modified Gram-Schmidt over the
 *     rows (two sweeps), then the phase of the determinant divided out with the principal
 *     cube root, so that det = 1 up to rounding.
 *
 * Output layout is the canonical host layout of a lattice field:
 *   double[n][3][3][2] (matrix), double[n][3][2] (vector), double[n] (real),
 * with n = volume * links and the matrix index m = site * links + mu.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Base of the stream for one (seed, field) pair. */
static uint64_t stream_base(uint64_t seed, uint32_t field) {
    return mix64(seed + GAMMA * ((uint64_t)field + 1ULL));
}

/* k-th raw 64-bit draw of a stream. */
static uint64_t draw(uint64_t base, uint64_t k) { return mix64(base + GAMMA * (k + 1ULL)); }

/* Uniform in the open interval (0,1). */
static double unif(uint64_t base, uint64_t k) {
    return ((double)(draw(base, k) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Normals 2j and 2j+1 of a stream (Box-Muller on uniforms 2j, 2j+1). */
static void normal_pair(uint64_t base, uint64_t j, double* n0, double* n1) {
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = unif(base, 2 * j), u2 = unif(base, 2 * j + 1);
    double r = sqrt(-2.0 * log(u1));
    *n0 = r * cos(two_pi * u2);
    *n1 = r * sin(two_pi * u2);
}

/* 2*npairs normals for element idx (each element owns a block of 32 uniforms). */
static void normals(uint64_t base, int64_t idx, int npairs, double* out) {
    for (int p = 0; p < npairs; ++p)
        normal_pair(base, (uint64_t)idx * 16ULL + (uint64_t)p, &out[2 * p], &out[2 * p + 1]);
}

/* ---- SU(3) projection of a Gaussian matrix (input generation only) ---- */
typedef struct { double re, im; } cpx;

static void su3_from_gauss(const double* g, double* out) {
    cpx r[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { r[i][j].re = g[2 * (3 * i + j)]; r[i][j].im = g[2 * (3 * i + j) + 1]; }
    for (int i = 0; i < 3; ++i) {
        /* two projection sweeps ("twice is enough") keep the rows orthonormal to
         * rounding even when the Gaussian rows are nearly dependent */
        for (int sweep = 0; sweep < 2 * i; ++sweep) {
        int p = sweep % i;
        {                                       /* r_i -= <r_p, r_i> r_p */
            double cr = 0.0, ci = 0.0;
            for (int j = 0; j < 3; ++j) {       /* conj(r_p[j]) * r_i[j] */
                cr += r[p][j].re * r[i][j].re + r[p][j].im * r[i][j].im;
                ci += r[p][j].re * r[i][j].im - r[p][j].im * r[i][j].re;
            }
            for (int j = 0; j < 3; ++j) {
                double xr = cr * r[p][j].re - ci * r[p][j].im;
                double xi = cr * r[p][j].im + ci * r[p][j].re;
                r[i][j].re -= xr; r[i][j].im -= xi;
            }
        }
        }
        double nn = 0.0;
        for (int j = 0; j < 3; ++j) nn += r[i][j].re * r[i][j].re + r[i][j].im * r[i][j].im;
        double inv = 1.0 / sqrt(nn);
        for (int j = 0; j < 3; ++j) { r[i][j].re *= inv; r[i][j].im *= inv; }
    }
    /* det by cofactor expansion along row 0 */
    cpx c0, c1, c2, d;
    c0.re = r[1][1].re * r[2][2].re - r[1][1].im * r[2][2].im - (r[1][2].re * r[2][1].re - r[1][2].im * r[2][1].im);
    c0.im = r[1][1].re * r[2][2].im + r[1][1].im * r[2][2].re - (r[1][2].re * r[2][1].im + r[1][2].im * r[2][1].re);
    c1.re = r[1][2].re * r[2][0].re - r[1][2].im * r[2][0].im - (r[1][0].re * r[2][2].re - r[1][0].im * r[2][2].im);
    c1.im = r[1][2].re * r[2][0].im + r[1][2].im * r[2][0].re - (r[1][0].re * r[2][2].im + r[1][0].im * r[2][2].re);
    c2.re = r[1][0].re * r[2][1].re - r[1][0].im * r[2][1].im - (r[1][1].re * r[2][0].re - r[1][1].im * r[2][0].im);
    c2.im = r[1][0].re * r[2][1].im + r[1][0].im * r[2][1].re - (r[1][1].re * r[2][0].im + r[1][1].im * r[2][0].re);
    d.re = r[0][0].re * c0.re - r[0][0].im * c0.im + r[0][1].re * c1.re - r[0][1].im * c1.im + r[0][2].re * c2.re - r[0][2].im * c2.im;
    d.im = r[0][0].re * c0.im + r[0][0].im * c0.re + r[0][1].re * c1.im + r[0][1].im * c1.re + r[0][2].re * c2.im + r[0][2].im * c2.re;
    double phi = atan2(d.im, d.re);
    double pr = cos(-phi / 3.0), pi = sin(-phi / 3.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            out[2 * (3 * i + j)]     = pr * r[i][j].re - pi * r[i][j].im;
            out[2 * (3 * i + j) + 1] = pr * r[i][j].im + pi * r[i][j].re;
        }
}

/* kind: 0 = SU(3) matrix (18 doubles), 1 = Gaussian matrix (18), 2 = Gaussian vector (6),
 *       3 = uniform(-1,1) real (1) */
static int kind_width(int kind) { return kind == 0 || kind == 1 ? 18 : kind == 2 ? 6 : 1; }

static void gen_range(int kind, uint64_t base, int64_t first, int64_t count, double* out) {
    int w = kind_width(kind);
    double g[18];
    for (int64_t e = 0; e < count; ++e) {
        int64_t idx = first + e;
        double* o = out + e * w;
        switch (kind) {
        case 0: normals(base, idx, 9, g); su3_from_gauss(g, o); break;
        case 1: normals(base, idx, 9, o); break;
        case 2: normals(base, idx, 3, o); break;
        default: o[0] = 2.0 * unif(base, (uint64_t)idx * 32ULL) - 1.0; break;
        }
    }
}

typedef struct { int kind; uint64_t base; int64_t first, count; double* out; } job_t;
static void* job_run(void* p) {
    job_t* j = (job_t*)p;
    gen_range(j->kind, j->base, j->first, j->count, j->out);
    return NULL;
}

/* Fill out[count * width] with elements first..first+count-1 of field `field`.
 * Returns 0 on success, -1 on bad arguments. nthreads <= 0 means 1. */
int synth_fill(int kind, uint64_t seed, uint32_t field, int64_t first, int64_t count,
               double* out, int nthreads) {
    if (kind < 0 || kind > 3 || first < 0 || count < 0 || (count > 0 && !out)) return -1;
    uint64_t base = stream_base(seed, field);
    int w = kind_width(kind);
    if (nthreads <= 1 || count < 4096) { gen_range(kind, base, first, count, out); return 0; }
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256]; job_t jobs[256]; int live[256];
    int64_t chunk = (count + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        int64_t lo = (int64_t)t * chunk, hi = lo + chunk > count ? count : lo + chunk;
        if (lo >= hi) break;
        jobs[t].kind = kind; jobs[t].base = base; jobs[t].first = first + lo;
        jobs[t].count = hi - lo; jobs[t].out = out + lo * w;
        live[t] = pthread_create(&th[t], NULL, job_run, &jobs[t]) == 0;
        if (!live[t]) job_run(&jobs[t]);
        started = t + 1;
    }
    for (int t = 0; t < started; ++t) if (live[t]) pthread_join(th[t], NULL);
    return 0;
}
