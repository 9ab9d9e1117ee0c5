// greens.cu -- the transform of the doubled-mesh Green's function (Eq. 9),
// built once per (doubled mesh, width ratios) in FP64 on the device.
//
// The Eq. 9 table is real and even in every axis (its inactive regions are
// mirror images), so its DFT is real and even too and equals a separable
// cosine sum over the even octant 0 <= p <= Mx/2, 0 <= q <= My/2,
// 0 <= r <= Mz/2:
//   Gt(kx,ky,kz) = sum w_p w_q w_r G(p,q,r) cos(2 pi kx p/Mx) cos(2 pi ky q/My)
//                  cos(2 pi kz r/Mz),   w = 1 at 0 and M/2, 2 otherwise.
// Three dense passes (one per axis) compute it; the cost is a one-off per
// cached spectrum, and FP64 is what sets the accuracy floor of the solve.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "launch.h"

namespace isofft {

static __global__ void k_green_octant(double *__restrict__ g, int X, int Y, int Z, double hx, double hy,
                                      double hz)
{
    const int64_t n = (int64_t)X * Y * Z;
    const double num = -hx * hy * hz / (4.0 * 3.14159265358979323846);
    const double hmin = fmin(hx, fmin(hy, hz));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % X, y = (i / X) % Y, z = i / ((int64_t)X * Y);
        double v;
        if (x == 0 && y == 0 && z == 0) {
            v = num / hmin;  // Eq. 9: the largest off-origin magnitude
        } else {
            const double dx = hx * (double)x, dy = hy * (double)y, dz = hz * (double)z;
            v = num / sqrt(dx * dx + dy * dy + dz * dz);  // Eq. 6
        }
        g[i] = v;
    }
}

// out[a][k][c] = sum_p CT[p][k] in[a][p][c], a < A, k < n, c < Cc.
static __global__ void k_cos_axis(const double *__restrict__ in, double *__restrict__ out,
                                  const double *__restrict__ CT, int64_t A, int n, int64_t Cc)
{
    const int64_t tot = A * n * Cc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i % Cc;
        const int k = (int)((i / Cc) % n);
        const int64_t a = i / (Cc * n);
        const double *src = in + a * n * Cc + c;
        double acc = 0.0;
        for (int p = 0; p < n; ++p) acc = fma(CT[(int64_t)p * n + k], src[(int64_t)p * Cc], acc);
        out[i] = acc;
    }
}

// oct [Z][Y][X] (X = Mx/2 + 1) -> G in the z pass's tiled layout
// [Y][ntx][blk] with block element kz * tx + c (kx = xt * tx + c, zero past
// Kx = Mx/2, zero in the padding past Z * tx) and Gs [Y][Z], of type T;
// column kx = 0 packs the kx = 0 and kx = Mx/2 planes.
template <typename T>
static __global__ void k_pack(const double *__restrict__ oct, T *__restrict__ G, T *__restrict__ Gs, int X,
                              int Y, int Z, int tx, int ntx, int blk, double scale)
{
    const int Kx = X - 1;
    const int64_t tot = (int64_t)Y * ntx * blk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % blk);
        if (j >= Z * tx) {
            G[i] = (T)0;
            continue;
        }
        const int c = j % tx;
        const int64_t kz = j / tx;
        const int xt = (int)((i / blk) % ntx);
        const int64_t ky = i / ((int64_t)blk * ntx);
        const int kx = xt * tx + c;
        const double *o = oct + (kz * Y + ky) * X;
        if (kx >= Kx) {
            G[i] = (T)0;
        } else if (kx == 0) {
            const double g0 = o[0], gn = o[Kx];
            G[i] = (T)(0.5 * (g0 + gn) * scale);
            Gs[ky * Z + kz] = (T)(0.5 * (g0 - gn) * scale);
        } else {
            G[i] = (T)(o[kx] * scale);
        }
    }
}

template <typename T>
size_t spectrum_elems(const int64_t M[3])
{
    const int tx = z_tile_for<T>((int)M[2]);
    const size_t Y = M[1] / 2 + 1, Z = M[2] / 2 + 1, Kx = M[0] / 2;
    const size_t ntx = (Kx + tx - 1) / tx;
    return Y * ntx * (size_t)z_spec_block(tx, (int)Z, (int)sizeof(T)) + Y * Z;
}
template size_t spectrum_elems<float>(const int64_t *);
template size_t spectrum_elems<double>(const int64_t *);
template size_t spectrum_elems<df64>(const int64_t *);

void host_roots(int64_t n, int64_t count, double *re, double *im)
{
    // e^{-2 pi i k/n}: reduce k to [0, n/8] by the exact symmetries of the
    // circle (n is a multiple of 8 for every length used here; other n fall
    // back to the direct angle).
    for (int64_t k = 0; k < count; ++k) {
        int64_t r = ((k % n) + n) % n;
        double c, s;  // cos and sin of 2 pi r / n
        if (n % 8 == 0) {
            const int64_t q = n / 8;
            bool neg_s = false;
            if (r > 4 * q) {  // lower half: sin negative
                r = n - r;
                neg_s = true;
            }
            // r in [0, n/2]
            bool neg_c = false;
            if (r > 2 * q) {  // second quadrant: cos(pi - a) = -cos a, sin same
                r = 4 * q - r;
                neg_c = true;
            }
            // r in [0, n/4]
            double cc, ss;
            if (r > q) {  // (q, 2q]: swap cos and sin of the complement
                const double a = 2.0 * M_PI * (double)(2 * q - r) / (double)n;
                cc = sin(a);
                ss = cos(a);
            } else {
                const double a = 2.0 * M_PI * (double)r / (double)n;
                cc = cos(a);
                ss = sin(a);
            }
            c = neg_c ? -cc : cc;
            s = neg_s ? -ss : ss;
        } else {
            const double a = 2.0 * M_PI * (double)r / (double)n;
            c = cos(a);
            s = sin(a);
        }
        re[k] = c;
        im[k] = -s;
    }
}

size_t green_build_scratch_bytes(const int64_t M[3])
{
    const size_t X = M[0] / 2 + 1, Y = M[1] / 2 + 1, Z = M[2] / 2 + 1;
    return 2 * X * Y * Z * sizeof(double) + (X * X + Y * Y + Z * Z) * sizeof(double);
}

static int grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t build_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, cudaStream_t st)
{
    const int X = (int)(M[0] / 2 + 1), Y = (int)(M[1] / 2 + 1), Z = (int)(M[2] / 2 + 1);
    const int64_t n = (int64_t)X * Y * Z;
    // cosine tables CT[p][k] = w_p cos(2 pi k p / M) per axis
    std::vector<double> hostCT;
    int64_t off[3], len[3] = {X, Y, Z};
    int64_t tot = 0;
    for (int a = 0; a < 3; ++a) {
        off[a] = tot;
        tot += len[a] * len[a];
    }
    hostCT.resize(tot);
    for (int a = 0; a < 3; ++a) {
        const int64_t m = M[a], nn = len[a];
        std::vector<double> re(m), im(m);
        host_roots(m, m, re.data(), im.data());
        for (int64_t p = 0; p < nn; ++p) {
            const double w = (p == 0 || 2 * p == m) ? 1.0 : 2.0;
            for (int64_t k = 0; k < nn; ++k) hostCT[off[a] + p * nn + k] = w * re[(k * p) % m];
        }
    }
    double *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (2 * n + tot) * sizeof(double));
    if (e != cudaSuccess) return e;
    double *o0 = buf, *o1 = buf + n, *ct = buf + 2 * n;
    e = cudaMemcpyAsync(ct, hostCT.data(), tot * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_green_octant<<<grid_for(n), 256, 0, st>>>(o0, X, Y, Z, hn[0], hn[1], hn[2]);
        count_launch();
        k_cos_axis<<<grid_for(n), 256, 0, st>>>(o0, o1, ct + off[0], (int64_t)Z * Y, X, 1);
        count_launch();
        k_cos_axis<<<grid_for(n), 256, 0, st>>>(o1, o0, ct + off[1], Z, Y, X);
        count_launch();
        k_cos_axis<<<grid_for(n), 256, 0, st>>>(o0, o1, ct + off[2], 1, Z, (int64_t)Y * X);
        count_launch();
        const double scale = 1.0 / (2.0 * (double)M[0] * (double)M[1] * (double)M[2]);
        const int tx = z_tile_for<T>((int)M[2]);
        const int ntx = (int)((M[0] / 2 + tx - 1) / tx);
        const int blk = z_spec_block(tx, Z, (int)sizeof(T));
        k_pack<T><<<grid_for((int64_t)Y * ntx * blk), 256, 0, st>>>(o1, G, Gs, X, Y, Z, tx, ntx, blk, scale);
        count_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    cudaFree(buf);
    return e;
}

// Same spectrum as build_green_spectrum, enqueued on `st` without allocating
// or synchronising: the FP64 octants live in the caller's `oct` scratch
// (green_octant_elems(M) doubles each, two of them), the cosine tables in
// `ct` (green_cos_elems(M) doubles, filled on the device by k_cos_tables).
static __global__ void k_cos_tables(double *__restrict__ ct, int mx, int my, int mz)
{
    const int X = mx / 2 + 1, Y = my / 2 + 1, Z = mz / 2 + 1;
    const int64_t tot = (int64_t)X * X + (int64_t)Y * Y + (int64_t)Z * Z;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = i;
        int n, m;
        if (j < (int64_t)X * X) {
            n = X, m = mx;
        } else if ((j -= (int64_t)X * X) < (int64_t)Y * Y) {
            n = Y, m = my;
        } else {
            j -= (int64_t)Y * Y;
            n = Z, m = mz;
        }
        const int64_t p = j / n, k = j % n;
        const double w = (p == 0 || 2 * p == m) ? 1.0 : 2.0;
        ct[i] = w * cospi(2.0 * (double)((k * p) % m) / (double)m);
    }
}

int64_t green_octant_elems(const int64_t M[3])
{
    return (M[0] / 2 + 1) * (M[1] / 2 + 1) * (M[2] / 2 + 1);
}
int64_t green_cos_elems(const int64_t M[3])
{
    int64_t t = 0;
    for (int a = 0; a < 3; ++a) t += (M[a] / 2 + 1) * (M[a] / 2 + 1);
    return t;
}

template <typename T>
cudaError_t enqueue_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, double *oct,
                                   double *ct, cudaStream_t st)
{
    const int X = (int)(M[0] / 2 + 1), Y = (int)(M[1] / 2 + 1), Z = (int)(M[2] / 2 + 1);
    const int64_t n = (int64_t)X * Y * Z;
    double *o0 = oct, *o1 = oct + n;
    double *ctx = ct, *cty = ct + (int64_t)X * X, *ctz = cty + (int64_t)Y * Y;
    k_cos_tables<<<grid_for(green_cos_elems(M)), 256, 0, st>>>(ct, (int)M[0], (int)M[1], (int)M[2]);
    count_launch();
    k_green_octant<<<grid_for(n), 256, 0, st>>>(o0, X, Y, Z, hn[0], hn[1], hn[2]);
    count_launch();
    k_cos_axis<<<grid_for(n), 256, 0, st>>>(o0, o1, ctx, (int64_t)Z * Y, X, 1);
    count_launch();
    k_cos_axis<<<grid_for(n), 256, 0, st>>>(o1, o0, cty, Z, Y, X);
    count_launch();
    k_cos_axis<<<grid_for(n), 256, 0, st>>>(o0, o1, ctz, 1, Z, (int64_t)Y * X);
    count_launch();
    const double scale = 1.0 / (2.0 * (double)M[0] * (double)M[1] * (double)M[2]);
    const int tx = z_tile_for<T>((int)M[2]);
    const int ntx = (int)((M[0] / 2 + tx - 1) / tx);
    const int blk = z_spec_block(tx, Z, (int)sizeof(T));
    k_pack<T><<<grid_for((int64_t)Y * ntx * blk), 256, 0, st>>>(o1, G, Gs, X, Y, Z, tx, ntx, blk, scale);
    count_launch();
    return cudaGetLastError();
}
template cudaError_t enqueue_green_spectrum<float>(const int64_t *, const double *, float *, float *, double *,
                                                   double *, cudaStream_t);
template cudaError_t enqueue_green_spectrum<double>(const int64_t *, const double *, double *, double *,
                                                    double *, double *, cudaStream_t);

template cudaError_t build_green_spectrum<float>(const int64_t *, const double *, float *, float *,
                                                 cudaStream_t);
template cudaError_t build_green_spectrum<double>(const int64_t *, const double *, double *, double *,
                                                  cudaStream_t);
template cudaError_t build_green_spectrum<df64>(const int64_t *, const double *, df64 *, df64 *, cudaStream_t);

}  // namespace isofft
