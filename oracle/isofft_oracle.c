/*
 * isofft_oracle.c -- plain FP64 CPU oracle for the isolated-system Poisson
 * solve of Budiardja & Cardall (PSPFFT).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, tables or helpers with the GPU library.
 *
 * What it computes (paper Sec. 2.1):
 *   - the anisotropic free-space Green's function, Eq. 6,
 *   - its doubled-mesh table with mirrored inactive regions and the
 *     regularised origin value, Eq. 9,
 *   - the potential as the discrete aperiodic convolution of that Green's
 *     function with the source (Eq. 8 on the mesh), two ways:
 *       route 1: direct summation over all source cells,
 *       route 2: the paper's route -- zero-pad the source to the doubled mesh,
 *                forward 3-D DFT (x, then y, then z as in Sec. 2.2.2),
 *                multiply by the transform of the Green's table (Eq. 5),
 *                inverse DFT (z, y, x), divide by Mx*My*Mz, keep the active
 *                region.
 *   - its own recursive mixed-radix FFT (smallest-prime-factor split,
 *     direct O(p^2) DFT on prime lengths); no FFT library is used.
 *
 * Layout: every 3-D array is C order [z][y][x], x contiguous, the mesh
 * indices (i, j, k) of Sec. 2.1 map to (x, y, z).
 *
 * Readings of the paper used here:
 *   - Eq. 9 writes the table for 0 <= p <= n with mirror images 2n - p; on a
 *     doubled mesh of any even length M >= 2N-1 this is G at offset
 *     min(i, M - i) per axis (entries between N and M - N never reach the
 *     active region).
 *   - the normalisation "due to the multiple transforms" (Sec. 2.2.2) is the
 *     usual 1/(Mx My Mz) of an unnormalised forward/backward DFT pair.
 *   - Newton's constant is 1: the caller passes S = 4*pi*rho.
 *
 * Compiled with -ffp-contract=off so that no fused multiply-add changes the
 * rounding of what is written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double re, im;
} cx;

/* ------------------------------------------------------------------ */
/* Green's function, Sec. 2.1                                          */
/* ------------------------------------------------------------------ */

/* Eq. 6 at integer offset (dx, dy, dz); Eq. 9 fixes the origin value to the
 * largest off-origin magnitude, -hx hy hz / (4 pi min(h)). */
double oracle_green(long dx, long dy, long dz, const double h[3])
{
    double hx = h[0], hy = h[1], hz = h[2];
    if (dx == 0 && dy == 0 && dz == 0) {
        double hmin = hx;
        if (hy < hmin) hmin = hy;
        if (hz < hmin) hmin = hz;
        return -hx * hy * hz / (4.0 * M_PI * hmin);
    }
    double X = hx * (double)dx, Y = hy * (double)dy, Z = hz * (double)dz;
    double dist = sqrt(X * X + Y * Y + Z * Z);
    return -hx * hy * hz / (4.0 * M_PI * dist);
}

/* Eq. 9 on a doubled mesh of M = (Mx, My, Mz) points: the value at index i
 * per axis is the Green's function at offset min(i, M - i). Output is a real
 * [Mz][My][Mx] array. */
void oracle_green_table(const int64_t M[3], const double h[3], double *G)
{
    int64_t Mx = M[0], My = M[1], Mz = M[2];
    for (int64_t k = 0; k < Mz; ++k) {
        long dz = (long)(k <= Mz - k ? k : Mz - k);
        for (int64_t j = 0; j < My; ++j) {
            long dy = (long)(j <= My - j ? j : My - j);
            for (int64_t i = 0; i < Mx; ++i) {
                long dx = (long)(i <= Mx - i ? i : Mx - i);
                G[(k * My + j) * Mx + i] = oracle_green(dx, dy, dz, h);
            }
        }
    }
}

/* Eq. 6 (Eq. 9 at the origin) on the block of offsets d = lo + [0, n) per
 * axis: the potential of a unit source at a corner, read at the cells of a
 * box, without the doubled table.  Output is a real [n2][n1][n0] array. */
void oracle_green_block(const int64_t lo[3], const int64_t n[3], const double h[3], double *out)
{
    for (int64_t k = 0; k < n[2]; ++k)
        for (int64_t j = 0; j < n[1]; ++j)
            for (int64_t i = 0; i < n[0]; ++i)
                out[(k * n[1] + j) * n[0] + i] =
                    oracle_green((long)(lo[0] + i), (long)(lo[1] + j), (long)(lo[2] + k), h);
}

/* ------------------------------------------------------------------ */
/* Recursive mixed-radix FFT                                            */
/* ------------------------------------------------------------------ */

static int64_t smallest_factor(int64_t n)
{
    if (n % 2 == 0) return 2;
    for (int64_t p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

/* e^{sign 2 pi i r / n} for 0 <= r < n */
static cx unit_root(int64_t r, int64_t n, int sign)
{
    double a = 2.0 * M_PI * (double)r / (double)n;
    cx w = {cos(a), (double)sign * sin(a)};
    return w;
}

static cx cmul(cx a, cx b)
{
    cx c = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return c;
}

/* A transform of top length n0 keeps one table w[e] = e^{sign 2 pi i e/n0};
 * the root e^{sign 2 pi i e/m} of a sub-length m | n0 is w[e * (n0/m)]. */
typedef struct {
    int64_t n0;
    const cx *w;
} roots_t;

static cx root_of(const roots_t *R, int64_t e, int64_t m)
{
    int64_t idx = (e % m) * (R->n0 / m);
    return R->w[idx];
}

/* out[k] = sum_{j<n} in[j*stride] e^{sign 2 pi i j k / n}, 0 <= k < n.
 * Decimation in time on the smallest prime factor p of n: with m = n/p and
 * F_q the length-m transform of the subsequence x[q + p j],
 *     X[k + m s] = sum_{q<p} e^{sign 2 pi i q (k + m s)/n} F_q[k].
 * A prime length is summed directly. `scratch` holds n entries and is only
 * used after the sub-transforms return, so one buffer serves every level. */
static void fft_rec(const cx *in, int64_t stride, cx *out, int64_t n,
                    const roots_t *R, cx *scratch)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int64_t p = smallest_factor(n);
    if (p == n) {
        for (int64_t k = 0; k < n; ++k) {
            cx acc = {0.0, 0.0};
            for (int64_t j = 0; j < n; ++j) {
                cx t = cmul(in[j * stride], root_of(R, j * k, n));
                acc.re += t.re;
                acc.im += t.im;
            }
            out[k] = acc;
        }
        return;
    }
    int64_t m = n / p;
    for (int64_t q = 0; q < p; ++q)
        fft_rec(in + q * stride, stride * p, out + q * m, m, R, scratch);
    memcpy(scratch, out, (size_t)n * sizeof(cx));
    for (int64_t s = 0; s < p; ++s) {
        for (int64_t k = 0; k < m; ++k) {
            cx acc = {0.0, 0.0};
            for (int64_t q = 0; q < p; ++q) {
                cx t = cmul(scratch[q * m + k], root_of(R, q * (k + m * s), n));
                acc.re += t.re;
                acc.im += t.im;
            }
            out[k + m * s] = acc;
        }
    }
}

static cx *make_roots(int64_t n, int sign)
{
    cx *w = (cx *)malloc((size_t)n * sizeof(cx));
    if (!w) return NULL;
    for (int64_t e = 0; e < n; ++e) w[e] = unit_root(e, n, sign);
    return w;
}

/* 1-D transform of n complex values (interleaved re, im), in place.
 * sign = -1: forward e^{-2 pi i jk/n}; sign = +1: unnormalised inverse. */
int oracle_fft1d(double *data, int64_t n, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return 1;
    cx *w = make_roots(n, sign);
    cx *in = (cx *)malloc((size_t)n * sizeof(cx));
    cx *scr = (cx *)malloc((size_t)n * sizeof(cx));
    if (!w || !in || !scr) {
        free(w); free(in); free(scr);
        return 2;
    }
    roots_t R = {n, w};
    memcpy(in, data, (size_t)n * sizeof(cx));
    fft_rec(in, 1, (cx *)data, n, &R, scr);
    free(w); free(in); free(scr);
    return 0;
}

/* Transform every line of a complex [Mz][My][Mx] grid along one axis
 * (0 = x, 1 = y, 2 = z).  Lines are independent, so they are spread over
 * OpenMP threads when the oracle is built with OpenMP. */
static int fft_axis(cx *g, const int64_t M[3], int axis, int sign)
{
    int64_t n = M[axis];
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? M[0] : M[0] * M[1]);
    int64_t nlines = (M[0] * M[1] * M[2]) / n;
    cx *w = make_roots(n, sign);
    if (!w) return 2;
    roots_t R = {n, w};
    int fail = 0;
#pragma omp parallel
    {
        cx *line = (cx *)malloc((size_t)n * sizeof(cx));
        cx *out = (cx *)malloc((size_t)n * sizeof(cx));
        cx *scr = (cx *)malloc((size_t)n * sizeof(cx));
        if (!line || !out || !scr) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t L = 0; L < nlines; ++L) {
                /* base address of line L: enumerate the two other axes */
                int64_t base;
                if (axis == 0) {
                    base = L * M[0];
                } else if (axis == 1) {
                    int64_t z = L / M[0], x = L % M[0];
                    base = z * M[0] * M[1] + x;
                } else {
                    base = L; /* L = y*Mx + x */
                }
                for (int64_t j = 0; j < n; ++j) line[j] = g[base + j * stride];
                fft_rec(line, 1, out, n, &R, scr);
                for (int64_t j = 0; j < n; ++j) g[base + j * stride] = out[j];
            }
        }
        free(line); free(out); free(scr);
    }
    free(w);
    return fail ? 2 : 0;
}

/* Forward (sign -1) or unnormalised inverse (sign +1) 3-D DFT of a complex
 * [Mz][My][Mx] grid, in place.  Forward runs x, y, z; inverse runs z, y, x,
 * the order of Sec. 2.2.2. */
int oracle_fft3d(double *grid, const int64_t M[3], int sign)
{
    cx *g = (cx *)grid;
    int rc = 0;
    if (sign == -1) {
        for (int a = 0; a < 3 && !rc; ++a) rc = fft_axis(g, M, a, -1);
    } else if (sign == 1) {
        for (int a = 2; a >= 0 && !rc; --a) rc = fft_axis(g, M, a, 1);
    } else {
        rc = 1;
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Route 2: the mesh-doubling solve, Sec. 2.1 and Sec. 2.2.2             */
/* ------------------------------------------------------------------ */

/* Transform of the Eq. 9 table on the doubled mesh M, computed once per
 * (M, h) as the paper does at initialisation, and divided by Mx My Mz so
 * that a forward/inverse pair needs no further scaling.  Output: complex
 * [Mz][My][Mx] (interleaved re, im). */
int oracle_green_spectrum(const int64_t M[3], const double h[3], double *Gt)
{
    int64_t tot = M[0] * M[1] * M[2];
    double *G = (double *)malloc((size_t)tot * sizeof(double));
    if (!G) return 2;
    oracle_green_table(M, h, G);
    cx *g = (cx *)Gt;
    for (int64_t i = 0; i < tot; ++i) {
        g[i].re = G[i];
        g[i].im = 0.0;
    }
    free(G);
    int rc = oracle_fft3d(Gt, M, -1);
    if (rc) return rc;
    double scale = 1.0 / (double)tot;
    for (int64_t i = 0; i < tot; ++i) {
        g[i].re *= scale;
        g[i].im *= scale;
    }
    return 0;
}

/* Solve with a precomputed spectrum (from oracle_green_spectrum):
 * zero-pad src [Nz][Ny][Nx] into the doubled mesh, forward 3-D DFT, multiply
 * by the spectrum, inverse 3-D DFT, keep the active region in phi. */
int oracle_solve_with_spectrum(const double *src, const int64_t N[3],
                               const int64_t M[3], const double *Gt, double *phi)
{
    int64_t Nx = N[0], Ny = N[1], Nz = N[2];
    int64_t Mx = M[0], My = M[1];
    int64_t tot = M[0] * M[1] * M[2];
    if (M[0] < 2 * N[0] - 1 || M[1] < 2 * N[1] - 1 || M[2] < 2 * N[2] - 1) return 1;
    cx *g = (cx *)calloc((size_t)tot, sizeof(cx));
    if (!g) return 2;
    for (int64_t k = 0; k < Nz; ++k)
        for (int64_t j = 0; j < Ny; ++j)
            for (int64_t i = 0; i < Nx; ++i)
                g[(k * My + j) * Mx + i].re = src[(k * Ny + j) * Nx + i];
    int rc = oracle_fft3d((double *)g, M, -1);
    if (!rc) {
        const cx *gt = (const cx *)Gt;
        for (int64_t i = 0; i < tot; ++i) g[i] = cmul(g[i], gt[i]);
        rc = oracle_fft3d((double *)g, M, 1);
    }
    if (!rc) {
        for (int64_t k = 0; k < Nz; ++k)
            for (int64_t j = 0; j < Ny; ++j)
                for (int64_t i = 0; i < Nx; ++i)
                    phi[(k * Ny + j) * Nx + i] = g[(k * My + j) * Mx + i].re;
    }
    free(g);
    return rc;
}

/* The whole route: spectrum, then solve.  M may be any mesh with
 * M >= 2N - 1 per axis; the paper's choice is M = 2N. */
int oracle_solve(const double *src, const int64_t N[3], const int64_t M[3],
                 const double h[3], double *phi)
{
    int64_t tot = M[0] * M[1] * M[2];
    double *Gt = (double *)malloc((size_t)tot * 2 * sizeof(double));
    if (!Gt) return 2;
    int rc = oracle_green_spectrum(M, h, Gt);
    if (!rc) rc = oracle_solve_with_spectrum(src, N, M, Gt, phi);
    free(Gt);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Route 1: direct summation, the definition of the discrete result      */
/* ------------------------------------------------------------------ */

/* phi(i,j,k) = sum over source cells of G(i-i', j-j', k-k') S(i',j',k'),
 * with G from Eq. 6 / Eq. 9.  Summed with Neumaier's compensation so the
 * sum itself adds no error comparable to the methods it checks. */
double oracle_direct_point(const double *src, const int64_t N[3], const double h[3],
                           int64_t i, int64_t j, int64_t k)
{
    int64_t Nx = N[0], Ny = N[1], Nz = N[2];
    double sum = 0.0, comp = 0.0;
    for (int64_t kk = 0; kk < Nz; ++kk)
        for (int64_t jj = 0; jj < Ny; ++jj)
            for (int64_t ii = 0; ii < Nx; ++ii) {
                double s = src[(kk * Ny + jj) * Nx + ii];
                if (s == 0.0) continue;
                double t = oracle_green((long)(i - ii), (long)(j - jj), (long)(k - kk), h) * s;
                double u = sum + t;
                if (fabs(sum) >= fabs(t))
                    comp += (sum - u) + t;
                else
                    comp += (t - u) + sum;
                sum = u;
            }
    return sum + comp;
}

void oracle_direct_sum(const double *src, const int64_t N[3], const double h[3], double *phi)
{
    int64_t Nx = N[0], Ny = N[1], Nz = N[2];
    int64_t tot = Nx * Ny * Nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < tot; ++c) {
        int64_t i = c % Nx, j = (c / Nx) % Ny, k = c / (Nx * Ny);
        phi[c] = oracle_direct_point(src, N, h, i, j, k);
    }
}

/* Potential at a list of cells (flat indices), for sampled checks at sizes
 * where the full direct sum is out of reach. */
void oracle_direct_points(const double *src, const int64_t N[3], const double h[3],
                          const int64_t *cells, int64_t count, double *out)
{
    int64_t Nx = N[0], Ny = N[1];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < count; ++c) {
        int64_t f = cells[c];
        int64_t i = f % Nx, j = (f / Nx) % Ny, k = f / (Nx * Ny);
        out[c] = oracle_direct_point(src, N, h, i, j, k);
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
