// passes.cuh -- the five passes of one isolated-system solve (Sec. 2.2.2),
// re-expressed for one GPU: no pillars, no transposes, each pass one HBM
// round trip over its data.
//
// Buffers (C order, x fastest):
//   src, phi : real [Nz][Ny][Nx]
//   W        : complex [Nz][My][Kx], Kx = Mx / 2, the plan's workspace.  The
//              z padding is never stored: the z pass reads z < Nz, treats the
//              rest of its line as zero, and writes back only z < Nz.
//   G        : real [My/2 + 1][Mz/2 + 1][Kx], the transform of the Eq. 9
//              table on the even octant (it is real and even in every axis),
//              pre-divided by 2 Mx My Mz (the factor 2 undoes the packed x
//              spectra, which carry 2X); column kx = 0 holds (G0 + GN) / 2,
//   Gs       : real [My/2 + 1][Mz/2 + 1], (G0 - GN) / 2, where G0 and GN are
//              the spectrum at kx = 0 and kx = Mx/2.
//
// x spectra are packed: a row of Mx real points has a Hermitian spectrum with
// real bins 0 and Mx/2, stored as P[0] = 2X[0] + i 2X[Mx/2] and
// P[k] = 2X[k] for 0 < k < Mx/2, so every line of the y and z passes is a
// plain complex line of power-of-two-friendly length.  The packed column is a
// sum of two real fields, so its spectrum multiply combines bins k and -k,
// which the z pass has at hand by processing ky and My - ky in one CTA.
//
//   K1 x forward : real rows y < Ny, z < Nz  -> W rows y < Ny   (input pruned)
//   K2 y forward : W rows y < Ny -> W all My rows               (input pruned)
//   K3 z         : W z < Nz -> FFT_z, x spectrum, inverse FFT_z -> W z < Nz
//   K4 y inverse : W all rows -> W rows y < Ny                  (output pruned)
//   K5 x inverse : W rows y < Ny -> real rows, x < Nx           (output pruned)
#pragma once
#include "fft_engine.cuh"

namespace isofft {

// Shared-memory exchange for column passes: lines are the COLS columns of a
// tile, stored [position][column] so a warp touches whole 128-byte rows.
template <typename T, int L, int E, int COLS>
struct ColXch {
    Cx<T> *s;
    int c;
    template <int NS, int R>
    __device__ __forceinline__ void exchange(Cx<T> (&v)[E], int t)
    {
        using G = StageGeom<L, E, NS, R>;
#pragma unroll
        for (int q = 0; q < G::B; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) s[G::out_pos(t, q, r) * COLS + c] = v[q + r * G::B];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[(t + m * G::NT) * COLS + c];
        __syncthreads();
    }
};

// Shared-memory exchange for row passes: one padded line per row; one pad
// slot every 16 points spreads the strided first-stage writes over banks.
template <int L>
struct RowPad {
    static constexpr int LP = L + L / 16;
    static __device__ __forceinline__ int at(int p) { return p + (p >> 4); }
};

template <typename T, int L, int E>
struct RowXch {
    Cx<T> *s;  // this row's line
    template <int NS, int R>
    __device__ __forceinline__ void exchange(Cx<T> (&v)[E], int t)
    {
        using G = StageGeom<L, E, NS, R>;
#pragma unroll
        for (int q = 0; q < G::B; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) s[RowPad<L>::at(G::out_pos(t, q, r))] = v[q + r * G::B];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[RowPad<L>::at(t + m * G::NT)];
        __syncthreads();
    }
};

template <typename T, int L>
struct RowCfg {
    static constexpr int E = Shape<T, L>::E;
    static constexpr int NT = L / E;
    static constexpr int NL = NT >= 256 ? 1 : 256 / NT;  // rows per CTA
    static constexpr int THREADS = NL * NT;
    static constexpr size_t SMEM = (size_t)NL * RowPad<L>::LP * sizeof(Cx<T>);
};

// Column tile width: 128 bytes of complex per row (16 FP32 or 8 FP64 lines).
template <typename T, int L>
struct ColCfg {
    static constexpr int E = Shape<T, L>::E;
    static constexpr int NT = L / E;
    static constexpr int TX = 128 / (int)sizeof(Cx<T>);
    static constexpr int THREADS = TX * NT;
    static constexpr size_t SMEM = (size_t)L * TX * sizeof(Cx<T>);
    static_assert(THREADS <= 1024, "column tile too large");
};

// The z pass processes two lines groups (ky and My - ky) per tile.
template <typename T, int L>
struct ZCfg {
    static constexpr int E = Shape<T, L>::E;
    static constexpr int NT = L / E;
    static constexpr int TX0 = 128 / (int)sizeof(Cx<T>);
    static constexpr int TX = (2 * TX0 * NT <= 1024 && (size_t)L * 2 * TX0 * sizeof(Cx<T>) <= 200 * 1024)
                                  ? TX0
                                  : TX0 / 2;
    static constexpr int COLS = 2 * TX;
    static constexpr int THREADS = COLS * NT;
    static constexpr size_t SMEM = (size_t)L * COLS * sizeof(Cx<T>);
    static_assert(THREADS <= 1024, "z tile too large");
};

// ---------------------------------------------------------------------
// K1: x forward, real rows -> packed half spectra.
// tw: W_L^k (k < L), rtw: W_{2L}^k (k < L), L = Mx / 2.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(RowCfg<T, L>::THREADS)
k_x_forward(const T *__restrict__ src, Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw,
            const Cx<T> *__restrict__ rtw, int Nx, int Ny, int My, int64_t nrows)
{
    using C = RowCfg<T, L>;
    constexpr int E = C::E, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x % NT, l = threadIdx.x / NT;
    Cx<T> *line = reinterpret_cast<Cx<T> *>(smem_raw) + l * RowPad<L>::LP;
    const int64_t row = (int64_t)blockIdx.x * C::NL + l;  // row = z * Ny + y
    const bool active = row < nrows;
    const int64_t rr = active ? row : 0;
    const T *in = src + rr * Nx;

    // pairs (x[2p], x[2p+1]) as one complex point; p >= L/2 is padding
    Cx<T> v[E];
    const bool vec = (Nx & 1) == 0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        v[m] = {(T)0, (T)0};
        if (m < E / 2 && active) {
            const int p = t + m * NT;
            if (vec && 2 * p + 1 < Nx) {
                v[m] = reinterpret_cast<const Cx<T> *>(in)[p];
            } else {
                if (2 * p < Nx) v[m].x = in[2 * p];
                if (2 * p + 1 < Nx) v[m].y = in[2 * p + 1];
            }
        }
    }
    RowXch<T, L, E> xch{line};
    run_stages<T, L, E, true>(v, t, tw, xch, typename Shape<T, L>::Rad{});

    // split the half-length transform Z into the real row's spectrum:
    //   2X[k] = (Z[k] + conj Z[L-k]) + W_2L^k (-i)(Z[k] - conj Z[L-k]),
    //   2X[0] = 2(Re Z0 + Im Z0), 2X[L] = 2(Re Z0 - Im Z0).
#pragma unroll
    for (int m = 0; m < E; ++m) line[RowPad<L>::at(t + m * NT)] = v[m];
    __syncthreads();
    const int y = (int)(rr % Ny);
    const int64_t z = rr / Ny;
    Cx<T> *out = W + ((size_t)z * My + y) * L;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        const Cx<T> zk = v[m];
        const Cx<T> zr = cconj(line[RowPad<L>::at(k == 0 ? 0 : L - k)]);
        const Cx<T> a = cadd(zk, zr);
        const Cx<T> b = cmul_mi(csub(zk, zr));
        Cx<T> p = cadd(a, cmul(b, rtw[k]));
        if (k == 0) p = {(T)2 * (zk.x + zk.y), (T)2 * (zk.x - zk.y)};
        if (active) out[k] = p;
    }
}

// ---------------------------------------------------------------------
// K5: x inverse, packed half spectra -> real rows, cropped to x < Nx.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(RowCfg<T, L>::THREADS)
k_x_inverse(const Cx<T> *__restrict__ W, T *__restrict__ phi, const Cx<T> *__restrict__ tw,
            const Cx<T> *__restrict__ rtw, int Nx, int Ny, int My, int64_t nrows)
{
    using C = RowCfg<T, L>;
    constexpr int E = C::E, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x % NT, l = threadIdx.x / NT;
    Cx<T> *line = reinterpret_cast<Cx<T> *>(smem_raw) + l * RowPad<L>::LP;
    const int64_t row = (int64_t)blockIdx.x * C::NL + l;
    const bool active = row < nrows;
    const int64_t rr = active ? row : 0;
    const int y = (int)(rr % Ny);
    const int64_t z = rr / Ny;
    const Cx<T> *in = W + ((size_t)z * My + y) * L;

#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        line[RowPad<L>::at(k)] = active ? in[k] : Cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    // rebuild the half-length spectrum of z[m] = y[2m] + i y[2m+1]:
    //   Z[k] = A + i B,  A = X[k] + conj X[L-k],  B = (X[k] - conj X[L-k]) W_2L^{-k}
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        const Cx<T> xk = line[RowPad<L>::at(k)];
        Cx<T> a, b;
        if (k == 0) {
            a = {xk.x + xk.y, (T)0};
            b = {xk.x - xk.y, (T)0};
        } else {
            const Cx<T> xr = cconj(line[RowPad<L>::at(L - k)]);
            a = cadd(xk, xr);
            b = cmul(csub(xk, xr), cconj(rtw[k]));
        }
        v[m] = {a.x - b.y, a.y + b.x};
    }
    __syncthreads();
    // inverse transform = swap o forward o swap
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cswap(v[m]);
    RowXch<T, L, E> xch{line};
    run_stages<T, L, E, false>(v, t, tw, xch, typename Shape<T, L>::Rad{});
    T *out = phi + rr * Nx;
    const bool vec = (Nx & 1) == 0;
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
        const int p = t + m * NT;
        const Cx<T> o = cswap(v[m]);
        if (!active) continue;
        if (vec && 2 * p + 1 < Nx) {
            reinterpret_cast<Cx<T> *>(out)[p] = o;
        } else {
            if (2 * p < Nx) out[2 * p] = o.x;
            if (2 * p + 1 < Nx) out[2 * p + 1] = o.y;
        }
    }
}

// ---------------------------------------------------------------------
// K2: y forward on columns; grid (ceil(Kx / TX), Nz).  Rows y >= Ny are zero
// padding and are not read.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(ColCfg<T, L>::THREADS)
k_y_forward(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx)
{
    using C = ColCfg<T, L>;
    constexpr int E = C::E, NT = C::NT, TX = C::TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, t = threadIdx.x / TX;
    const int kx = blockIdx.x * TX + c;
    const bool active = kx < Kx;
    Cx<T> *base = W + (size_t)blockIdx.y * L * Kx + (active ? kx : 0);
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int y = t + m * NT;
        v[m] = (m < E / 2 && active && y < Ny) ? base[(size_t)y * Kx] : Cx<T>{(T)0, (T)0};
    }
    ColXch<T, L, E, TX> xch{reinterpret_cast<Cx<T> *>(smem_raw), c};
    run_stages<T, L, E, true>(v, t, tw, xch, typename Shape<T, L>::Rad{});
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[(size_t)(t + m * NT) * Kx] = v[m];
    }
}

// ---------------------------------------------------------------------
// K4: y inverse on columns, keeping rows y < Ny.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(ColCfg<T, L>::THREADS)
k_y_inverse(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx)
{
    using C = ColCfg<T, L>;
    constexpr int E = C::E, NT = C::NT, TX = C::TX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = threadIdx.x % TX, t = threadIdx.x / TX;
    const int kx = blockIdx.x * TX + c;
    const bool active = kx < Kx;
    Cx<T> *base = W + (size_t)blockIdx.y * L * Kx + (active ? kx : 0);
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = active ? cswap(base[(size_t)(t + m * NT) * Kx]) : Cx<T>{(T)0, (T)0};
    ColXch<T, L, E, TX> xch{reinterpret_cast<Cx<T> *>(smem_raw), c};
    run_stages<T, L, E, false>(v, t, tw, xch, typename Shape<T, L>::Rad{});
    if (active) {
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
            const int y = t + m * NT;
            if (y < Ny) base[(size_t)y * Kx] = cswap(v[m]);
        }
    }
}

// ---------------------------------------------------------------------
// K3: z forward, multiply by the Green's spectrum, z inverse.
// grid (ceil(Kx / TX), My / 2); CTA y index p handles the line pair
// (ky, My - ky) = (p, My - p) for p > 0 and (0, My/2) for p = 0.
// gscale multiplies the cached spectrum (the cache stores it for widths
// divided by min(h); G scales as h^2).
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(ZCfg<T, L>::THREADS)
k_z_convolve(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, const T *__restrict__ G,
             const T *__restrict__ Gs, T gscale, int Nz, int My, int Kx)
{
    using C = ZCfg<T, L>;
    constexpr int E = C::E, NT = C::NT, TX = C::TX, COLS = C::COLS;
    constexpr int Lh = L / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T> *sm = reinterpret_cast<Cx<T> *>(smem_raw);
    const int c = threadIdx.x % TX;
    const int rest = threadIdx.x / TX;
    const int t = rest % NT, g = rest / NT;
    const int pr = blockIdx.y;
    const int ky = g == 0 ? pr : (pr == 0 ? My / 2 : My - pr);
    const int kyp = ky <= My - ky ? ky : My - ky;
    const int kx = blockIdx.x * TX + c;
    const bool active = kx < Kx;
    const int col = g * TX + c;
    const size_t zstride = (size_t)My * Kx;
    Cx<T> *base = W + (size_t)ky * Kx + (active ? kx : 0);

    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int z = t + m * NT;
        v[m] = (m < E / 2 && active && z < Nz) ? base[(size_t)z * zstride] : Cx<T>{(T)0, (T)0};
    }
    ColXch<T, L, E, COLS> xch{sm, col};
    run_stages<T, L, E, true>(v, t, tw, xch, typename Shape<T, L>::Rad{});

    const T *grow = G + (size_t)kyp * (Lh + 1) * Kx;
    const bool packed = blockIdx.x == 0 && c == 0;  // the kx = 0 / Mx/2 column
    if (blockIdx.x == 0) {
        // the packed column needs the partner bin (-ky, -kz)
        if (c == 0) {
#pragma unroll
            for (int m = 0; m < E; ++m) sm[(t + m * NT) * COLS + col] = v[m];
        }
        __syncthreads();
        if (c == 0) {
            const int gp = pr == 0 ? g : 1 - g;
            const T *gsrow = Gs + (size_t)kyp * (Lh + 1);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kz = t + m * NT;
                const int kzp = kz <= L - kz ? kz : L - kz;
                const Cx<T> partner = cconj(sm[(kz == 0 ? 0 : L - kz) * COLS + gp * TX]);
                const T gp_ = grow[(size_t)kzp * Kx] * gscale;
                const T gm_ = gsrow[kzp] * gscale;
                v[m] = {v[m].x * gp_ + partner.x * gm_, v[m].y * gp_ + partner.y * gm_};
            }
        }
        __syncthreads();
    }
    if (!packed) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int kz = t + m * NT;
            const int kzp = kz <= L - kz ? kz : L - kz;
            const T gv = active ? grow[(size_t)kzp * Kx + kx] * gscale : (T)0;
            v[m] = cscale(v[m], gv);
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cswap(v[m]);
    run_stages<T, L, E, false>(v, t, tw, xch, typename Shape<T, L>::Rad{});
    if (active) {
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
            const int z = t + m * NT;
            if (z < Nz) base[(size_t)z * zstride] = cswap(v[m]);
        }
    }
}

}  // namespace isofft
