// greens.cu -- the transform of the doubled-mesh Green's function (Eq. 9),
// built once per (doubled mesh, width ratios) in FP64 on the device.
//
// The Eq. 9 table is real and even in every axis (its inactive regions are
// mirror images), so its DFT is real and even too and is separable over the
// even octant 0 <= p <= Mx/2, 0 <= q <= My/2, 0 <= r <= Mz/2:
//   Gt(kx,ky,kz) = sum w_p w_q w_r G(p,q,r) cos(2 pi kx p/Mx) cos(2 pi ky q/My)
//                  cos(2 pi kz r/Mz),   w = 1 at 0 and M/2, 2 otherwise.
// Each axis's cosine sum is the M-point DFT of the octant line mirrored to
// its full length (c[p] = G[min(p, M - p)]), whose bins 0..M/2 are real.
// One pass per axis transforms every octant line that way in place, with
// the FFT engine of the solve passes in FP64 (O(M^3 log M) in all); FP64 is
// what sets the accuracy floor of the solve.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "launch.h"
#include "passes.cuh"

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

// One axis of the octant transform, in place: line (a, c) of the octant,
// elements base[q Cc] (q <= L/2, base = oct + a (L/2 + 1) Cc + c), is
// mirrored to L points, transformed, and bins 0..L/2 (real) are written back.
// Lines are grouped NL per CTA (one row buffer each, as the x passes use).
template <int L>
struct DctCfg {
    using SH = Shape<double, L>;
    static constexpr int E = SH::E, NT = L / E;
    static constexpr int NL = NT >= 128 ? 1 : 128 / NT;
    static constexpr int THREADS = NL * NT;
    static constexpr size_t SMEM = (size_t)NL * RowPad<double, L>::LP * sizeof(Cx<double>);
};

template <int L>
static __global__ void __launch_bounds__(DctCfg<L>::THREADS)
k_cos_lines(double *__restrict__ oct, const Cx<double> *__restrict__ tw, int64_t A, int64_t Cc)
{
    using C = DctCfg<L>;
    constexpr int E = C::E, NT = C::NT, n = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char dct_smem[];
    Cx<double> *row = reinterpret_cast<Cx<double> *>(dct_smem) + (threadIdx.x / NT) * RowPad<double, L>::LP;
    const int l = threadIdx.x / NT, t = threadIdx.x % NT;
    const int64_t lines = A * Cc;
    for (int64_t l0 = (int64_t)blockIdx.x * C::NL; l0 < lines; l0 += (int64_t)gridDim.x * C::NL) {
        const int64_t line = l0 + l;
        const bool active = line < lines;
        const int64_t a = active ? line / Cc : 0, c = active ? line % Cc : 0;
        double *base = oct + a * n * Cc + c;
        Cx<double> v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int p = t + m * NT;
            const int q = p <= L / 2 ? p : L - p;
            v[m] = {active ? base[(int64_t)q * Cc] : 0.0, 0.0};
        }
        // every thread has read its line before the first exchange's barrier,
        // and writes after the last one
        RowXch<double, L, E> xch{row};
        run_stages<double, L, E, false>(v, t, tw, xch, typename C::SH::Rad{});
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + m * NT;
            if (active && k <= L / 2) base[(int64_t)k * Cc] = v[m].x;
        }
    }
}

#define ISOFFT_DCT_LENGTHS(X) \
    X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2304)

template <int L>
static cudaError_t run_cos_lines(double *oct, const Cx<double> *tw, int64_t A, int64_t Cc, cudaStream_t st)
{
    using C = DctCfg<L>;
    const int64_t groups = (A * Cc + C::NL - 1) / C::NL;
    const int grid = (int)(groups < 152 * 8 ? groups : 152 * 8);
    if (C::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_cos_lines<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
    }
    k_cos_lines<L><<<grid, C::THREADS, C::SMEM, st>>>(oct, tw, A, Cc);
    count_launch();
    return cudaGetLastError();
}

// Cosine transform of every octant line along one axis of length M (one of
// the supported doubled lengths); tw = W_M^k, k < M.
static cudaError_t cos_axis(int M, double *oct, const Cx<double> *tw, int64_t A, int64_t Cc, cudaStream_t st)
{
    switch (M) {
#define X_(n) \
    case n: return run_cos_lines<n>(oct, tw, A, Cc, st);
        ISOFFT_DCT_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}

// The three axis passes of the octant transform, in place on oct [Z][Y][X];
// tws[a] = W_{M_a}^k.
static cudaError_t cos_transform(const int64_t M[3], double *oct, const Cx<double> *const tws[3], cudaStream_t st)
{
    const int64_t X = M[0] / 2 + 1, Y = M[1] / 2 + 1, Z = M[2] / 2 + 1;
    cudaError_t e = cos_axis((int)M[0], oct, tws[0], Z * Y, 1, st);
    if (e == cudaSuccess) e = cos_axis((int)M[1], oct, tws[1], Z, X, st);
    if (e == cudaSuccess) e = cos_axis((int)M[2], oct, tws[2], 1, X * Y, st);
    return e;
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

// Root tables of the three axes, W_{M_a}^k for k < M_a, one after another.
int64_t green_cos_elems(const int64_t M[3]) { return 2 * (M[0] + M[1] + M[2]); }
// The FP64 octant; its element count rounded up to even, so that root
// tables placed after it start on a 16-byte boundary (complex doubles).
int64_t green_octant_elems(const int64_t M[3])
{
    const int64_t n = (M[0] / 2 + 1) * (M[1] / 2 + 1) * (M[2] / 2 + 1);
    return (n + 1) & ~(int64_t)1;
}

size_t green_build_scratch_bytes(const int64_t M[3])
{
    return (size_t)(green_octant_elems(M) + green_cos_elems(M)) * sizeof(double);
}

static int grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

// G from the transformed octant, in the z pass's layout and dtype.
template <typename T>
static cudaError_t pack_spectrum(const int64_t M[3], const double *oct, T *G, T *Gs, cudaStream_t st)
{
    const int X = (int)(M[0] / 2 + 1), Y = (int)(M[1] / 2 + 1), Z = (int)(M[2] / 2 + 1);
    const double scale = 1.0 / (2.0 * (double)M[0] * (double)M[1] * (double)M[2]);
    const int tx = z_tile_for<T>((int)M[2]);
    const int ntx = (int)((M[0] / 2 + tx - 1) / tx);
    const int blk = z_spec_block(tx, Z, (int)sizeof(T));
    k_pack<T><<<grid_for((int64_t)Y * ntx * blk), 256, 0, st>>>(oct, G, Gs, X, Y, Z, tx, ntx, blk, scale);
    count_launch();
    return cudaGetLastError();
}

// The octant of Eq. 9 (FP64), its three axis transforms in place, the pack.
// tws: the root tables of the three axes (green_cos_elems doubles).
template <typename T>
static cudaError_t spectrum_steps(const int64_t M[3], const double hn[3], T *G, T *Gs, double *oct,
                                  const double *tws, cudaStream_t st)
{
    const int X = (int)(M[0] / 2 + 1), Y = (int)(M[1] / 2 + 1), Z = (int)(M[2] / 2 + 1);
    const int64_t n = (int64_t)X * Y * Z;
    if ((reinterpret_cast<uintptr_t>(tws) & 15) || (reinterpret_cast<uintptr_t>(oct) & 7))
        return cudaErrorMisalignedAddress;  // complex-double tables need 16-byte alignment
    k_green_octant<<<grid_for(n), 256, 0, st>>>(oct, X, Y, Z, hn[0], hn[1], hn[2]);
    count_launch();
    const Cx<double> *tw[3] = {reinterpret_cast<const Cx<double> *>(tws),
                               reinterpret_cast<const Cx<double> *>(tws) + M[0],
                               reinterpret_cast<const Cx<double> *>(tws) + M[0] + M[1]};
    cudaError_t e = cos_transform(M, oct, tw, st);
    if (e == cudaSuccess) e = pack_spectrum<T>(M, oct, G, Gs, st);
    return e;
}

template <typename T>
cudaError_t build_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, cudaStream_t st)
{
    const int64_t n = green_octant_elems(M), nt = green_cos_elems(M);
    // roots W_M^k per axis, by exact reduction to the first octant (host)
    std::vector<double> host(nt);
    int64_t off = 0;
    for (int a = 0; a < 3; ++a) {
        std::vector<double> re(M[a]), im(M[a]);
        host_roots(M[a], M[a], re.data(), im.data());
        for (int64_t k = 0; k < M[a]; ++k) {
            host[off + 2 * k] = re[k];
            host[off + 2 * k + 1] = im[k];
        }
        off += 2 * M[a];
    }
    double *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (size_t)(n + nt) * sizeof(double));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(buf + n, host.data(), nt * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = spectrum_steps<T>(M, hn, G, Gs, buf, buf + n, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    cudaFree(buf);
    return e;
}

// Same spectrum as build_green_spectrum, enqueued on `st` without allocating
// or synchronising: the FP64 octant lives in the caller's `oct` scratch
// (green_octant_elems(M) doubles), the root tables in `ct`
// (green_cos_elems(M) doubles, computed on the device by k_axis_roots).
static __global__ void k_axis_roots(double *__restrict__ ct, int mx, int my, int mz)
{
    const int tot = mx + my + mz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        int k = i, m = mx;
        if (k >= mx) {
            k -= mx;
            m = my;
            if (k >= my) {
                k -= my;
                m = mz;
            }
        }
        double sn, cs;
        sincospi(2.0 * (double)k / (double)m, &sn, &cs);
        ct[2 * i] = cs;
        ct[2 * i + 1] = -sn;
    }
}

template <typename T>
cudaError_t enqueue_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, double *oct,
                                   double *ct, cudaStream_t st)
{
    k_axis_roots<<<grid_for(M[0] + M[1] + M[2]), 256, 0, st>>>(ct, (int)M[0], (int)M[1], (int)M[2]);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = spectrum_steps<T>(M, hn, G, Gs, oct, ct, st);
    return e;
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
