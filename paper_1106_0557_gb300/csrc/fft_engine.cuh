// fft_engine.cuh -- register-resident Stockham FFT building blocks for sm_103a.
//
// One line of L complex points is spread over NT = L / E threads, each thread
// holding E points in registers.  Thread t always holds the points at
// positions t + m * NT (m < E) before a stage; the stage multiplies by the
// Stockham twiddles, runs E / R radix-R butterflies in registers, and the
// outputs are exchanged through shared memory so that every thread again
// holds positions t + m * NT.  After the last stage thread t holds output
// bins t + m * NT in natural order, so global loads and stores of a line are
// coalesced along the line for row passes and along the tile for column
// passes, and the spectrum multiply of the z pass needs no exchange at all.
//
// The forward transform is X[k] = sum_j x[j] e^{-2 pi i jk/L} (unnormalised).
// The inverse is obtained as swap(FFT(swap(x))), swap exchanging real and
// imaginary parts, which costs nothing in registers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"

namespace isofft {

// Building blocks are host-callable too, so a host harness can run the
// exact stage code against a direct DFT.
#define ISOFFT_HD __host__ __device__ __forceinline__

template <typename T>
struct alignas(2 * sizeof(T)) Cx {
    T x, y;
};

// Sums inside the butterflies: plain for float and double; for float pairs
// without the closing renormalisation (df64_add_lazy), which every product
// below restores on its data operand first (crenorm; a no-op elsewhere).
template <typename T>
ISOFFT_HD T radd(T a, T b) { return a + b; }
template <typename T>
ISOFFT_HD T rsub(T a, T b) { return a - b; }
template <typename T>
ISOFFT_HD T rmul(T a, T b) { return a * b; }  // a product that only enters sums
ISOFFT_HD df64 radd(df64 a, df64 b) { return df64_add_lazy(a, b); }
ISOFFT_HD df64 rmul(df64 a, df64 b) { return df64_mul_lazy(a, b); }
ISOFFT_HD df64 rsub(df64 a, df64 b) { return df64_add_lazy(a, -b); }
template <typename T>
ISOFFT_HD Cx<T> crenorm(Cx<T> a) { return a; }
ISOFFT_HD Cx<df64> crenorm(Cx<df64> a) { return {df64_renorm(a.x), df64_renorm(a.y)}; }

template <typename T>
ISOFFT_HD Cx<T> cadd(Cx<T> a, Cx<T> b) { return {radd(a.x, b.x), radd(a.y, b.y)}; }
template <typename T>
ISOFFT_HD Cx<T> csub(Cx<T> a, Cx<T> b) { return {rsub(a.x, b.x), rsub(a.y, b.y)}; }
template <typename T>
ISOFFT_HD Cx<T> cmul(Cx<T> a, Cx<T> b)
{
    a = crenorm(a);
    return {rsub(rmul(a.x, b.x), rmul(a.y, b.y)), radd(rmul(a.x, b.y), rmul(a.y, b.x))};
}
template <typename T>
ISOFFT_HD Cx<T> cscale(Cx<T> a, T s)
{
    a = crenorm(a);
    return {a.x * s, a.y * s};
}
template <typename T>
ISOFFT_HD Cx<T> cconj(Cx<T> a) { return {a.x, -a.y}; }
// multiply by -i
template <typename T>
ISOFFT_HD Cx<T> cmul_mi(Cx<T> a) { return {a.y, -a.x}; }
// exchange real and imaginary parts
template <typename T>
ISOFFT_HD Cx<T> cswap(Cx<T> a) { return {a.y, a.x}; }

// cos(2 pi j / 48) for j in [0, 12] (first quadrant); other angles follow by
// exact symmetry so that W and its mirror images round identically.
__host__ __device__ constexpr double cos48_base(int j)
{
    constexpr double b[13] = {1.0, 0.9914448613738104, 0.9659258262890683, 0.9238795325112867,
                              0.8660254037844387, 0.7933533402912352, 0.7071067811865476,
                              0.6087614290087207, 0.5, 0.3826834323650898, 0.25881904510252074,
                              0.13052619222005157, 0.0};
    return b[j];
}
__host__ __device__ constexpr double cos48(int j)
{
    j %= 48;
    if (j < 0) j += 48;
    if (j > 24) j = 48 - j;
    return j > 12 ? -cos48_base(24 - j) : cos48_base(j);
}
__host__ __device__ constexpr double sin48(int j) { return cos48(12 - j); }

// cos(2 pi j / 96) for j in [0, 24], for the radices that 48 does not
// divide (32); even j are the 48-table's values.  The odd ones were summed
// from the Taylor series in 50-digit decimal arithmetic and rounded.
__host__ __device__ constexpr double cos96_base(int j)
{
    constexpr double odd[12] = {0.9978589232386035, 0.9807852804032304, 0.9469301294951057,
                                0.8968727415326883, 0.8314696123025452, 0.7518398074789774,
                                0.6593458151000688, 0.5555702330196022, 0.4422886902190013,
                                0.3214394653031616, 0.19509032201612828, 0.06540312923014306};
    return (j & 1) ? odd[j / 2] : cos48_base(j / 2);
}
__host__ __device__ constexpr double cos96(int j)
{
    j %= 96;
    if (j < 0) j += 96;
    if (j > 48) j = 96 - j;
    return j > 24 ? -cos96_base(48 - j) : cos96_base(j);
}
__host__ __device__ constexpr double sin96(int j) { return cos96(24 - j); }

// Multiply by the compile-time root W_R^e = e^{-2 pi i e / R} (96 % R == 0).
template <typename T, int R, int e>
ISOFFT_HD Cx<T> mul_root96(Cx<T> a)
{
    static_assert(96 % R == 0, "roots of unity of 96ths");
    constexpr int ee = ((e % R) + R) % R;
    constexpr int j = ee * (96 / R);  // angle in units of 2 pi / 96
    if constexpr (j != 0 && j % 24 != 0) a = crenorm(a);  // a product follows
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 24) {
        return cmul_mi(a);  // -i
    } else if constexpr (j == 48) {
        return {-a.x, -a.y};
    } else if constexpr (j == 72) {
        return {-a.y, a.x};  // +i
    } else if constexpr (j == 12 || j == 36 || j == 60 || j == 84) {
        constexpr T r = (T)0.7071067811865476;
        constexpr bool cp = cos96(j) > 0, sp = sin96(j) > 0;
        const T cx = cp ? a.x : -a.x, cy = cp ? a.y : -a.y;
        const T sx = sp ? a.x : -a.x, sy = sp ? a.y : -a.y;
        return {(cx + sy) * r, (cy - sx) * r};  // normalised sums: products follow
    } else {
        constexpr T c = (T)cos96(j);
        constexpr T s = (T)sin96(j);
        return {radd(rmul(a.x, c), rmul(a.y, s)), rsub(rmul(a.y, c), rmul(a.x, s))};
    }
}

template <typename T, int R, int e>
ISOFFT_HD Cx<T> mul_root(Cx<T> a)
{
    if constexpr (48 % R != 0) {
        return mul_root96<T, R, e>(a);
    } else {
        constexpr int ee = ((e % R) + R) % R;
        constexpr int j = ee * (48 / R);  // angle in units of 2 pi / 48
        if constexpr (j != 0 && j % 12 != 0) a = crenorm(a);  // a product follows
        if constexpr (j == 0) {
            return a;
        } else if constexpr (j == 12) {
            return cmul_mi(a);  // -i
        } else if constexpr (j == 24) {
            return {-a.x, -a.y};
        } else if constexpr (j == 36) {
            return {-a.y, a.x};  // +i
        } else if constexpr (j == 6 || j == 18 || j == 30 || j == 42) {
            // |cos| = |sin| = 1/sqrt(2): a * (c - i s) with only the signs differing
            constexpr T r = (T)0.7071067811865476;
            constexpr bool cp = cos48(j) > 0, sp = sin48(j) > 0;
            const T cx = cp ? a.x : -a.x, cy = cp ? a.y : -a.y;  // c a / |c|
            const T sx = sp ? a.x : -a.x, sy = sp ? a.y : -a.y;  // s a / |s|
            return {(cx + sy) * r, (cy - sx) * r};  // normalised sums: products follow
        } else {
            constexpr T c = (T)cos48(j);
            constexpr T s = (T)sin48(j);
            return {radd(rmul(a.x, c), rmul(a.y, s)), rsub(rmul(a.y, c), rmul(a.x, s))};
        }
    }
}

// ---------------------------------------------------------------------
// Small DFTs in registers: a[k] <- sum_r a[r] e^{-2 pi i r k / R}.
// ---------------------------------------------------------------------
template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
    static ISOFFT_HD void run(Cx<T> (&a)[2])
    {
        Cx<T> t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <typename T>
struct Dft<T, 3> {
    static ISOFFT_HD void run(Cx<T> (&a)[3])
    {
        constexpr T s3 = (T)0.8660254037844387;  // sin(2 pi / 3)
        Cx<T> sum = crenorm(cadd(a[1], a[2]));  // both enter products
        Cx<T> dif = crenorm(csub(a[1], a[2]));
        Cx<T> t = {a[0].x - (T)0.5 * sum.x, a[0].y - (T)0.5 * sum.y};
        Cx<T> u = {dif.y * s3, -dif.x * s3};  // -i s3 (a1 - a2)
        a[0] = cadd(a[0], sum);
        a[1] = cadd(t, u);
        a[2] = csub(t, u);
    }
};

template <typename T>
struct Dft<T, 4> {
    static ISOFFT_HD void run(Cx<T> (&a)[4])
    {
        Cx<T> s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        Cx<T> s13 = cadd(a[1], a[3]), d13 = cmul_mi(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, d13);
        a[3] = csub(d02, d13);
    }
};

template <typename T>
struct Dft<T, 5> {
    static ISOFFT_HD void run(Cx<T> (&a)[5])
    {
        constexpr T c1 = (T)0.30901699437494745, c2 = (T)-0.8090169943749473;
        constexpr T s1 = (T)0.9510565162951535, s2 = (T)0.5877852522924732;
        Cx<T> b1 = crenorm(cadd(a[1], a[4])), b2 = crenorm(cadd(a[2], a[3]));  // all enter products
        Cx<T> d1 = crenorm(csub(a[1], a[4])), d2 = crenorm(csub(a[2], a[3]));
        Cx<T> t1 = {a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y};
        Cx<T> t2 = {a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y};
        Cx<T> u1 = {s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y};
        Cx<T> u2 = {s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y};
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(t1, cmul_mi(u1));
        a[4] = csub(t1, cmul_mi(u1));
        a[2] = cadd(t2, cmul_mi(u2));
        a[3] = csub(t2, cmul_mi(u2));
    }
};

// Composite length R = R1 * R2 by one Cooley-Tukey step:
// X[k1 + R1 k2] = sum_n2 W_R2^{n2 k2} W_R^{n2 k1} sum_n1 a[R2 n1 + n2] W_R1^{n1 k1}.
template <typename T, int R1, int R2>
struct DftCT {
    static constexpr int R = R1 * R2;
    template <int n2, int k1>
    static ISOFFT_HD void twiddle(Cx<T> (&b)[R])
    {
        b[k1 * R2 + n2] = mul_root<T, R, n2 * k1>(b[k1 * R2 + n2]);
        if constexpr (k1 + 1 < R1) twiddle<n2, k1 + 1>(b);
    }
    template <int n2>
    static ISOFFT_HD void inner(const Cx<T> (&a)[R], Cx<T> (&b)[R])
    {
        Cx<T> t[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) t[n1] = a[R2 * n1 + n2];
        Dft<T, R1>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) b[k1 * R2 + n2] = t[k1];
        twiddle<n2, 0>(b);
        if constexpr (n2 + 1 < R2) inner<n2 + 1>(a, b);
    }
    static ISOFFT_HD void run(Cx<T> (&a)[R])
    {
        Cx<T> b[R];
        inner<0>(a, b);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            Cx<T> t[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) t[n2] = b[k1 * R2 + n2];
            Dft<T, R2>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = t[k2];
        }
    }
};

// Radix 8 as 2 x 4 (the DftCT order: even bins from the sums, odd bins from
// the differences twiddled by W_8^n), with the two 1/sqrt(2) roots of the odd
// half factored out: W_8 m1 + W_8^3 m3 = r (c1 + c3) with r = 1/sqrt(2) and
// c1, c3 sums and differences of the components, so that r multiplies
// inside the last level's additions (one fused multiply-add each) instead of
// four separate products.  Odd bins: the 4-point DFT of
// (m0, W_8 m1, -i m2, W_8^3 m3).
template <typename T>
ISOFFT_HD void dft4_w8_odd(Cx<T> m0, Cx<T> m1, Cx<T> m2, Cx<T> m3, Cx<T> &o0, Cx<T> &o1, Cx<T> &o2, Cx<T> &o3)
{
    constexpr T r = (T)0.7071067811865476;
    const Cx<T> c1 = {radd(m1.x, m1.y), rsub(m1.y, m1.x)};    // W_8 m1 / r
    const Cx<T> c3 = {rsub(m3.y, m3.x), -radd(m3.x, m3.y)};  // W_8^3 m3 / r
    const Cx<T> S = crenorm(cadd(c1, c3)), D = crenorm(csub(c1, c3));  // enter the products
    const Cx<T> s02 = {radd(m0.x, m2.y), rsub(m0.y, m2.x)}, d02 = {rsub(m0.x, m2.y), radd(m0.y, m2.x)};
    o0 = {radd(s02.x, rmul(r, S.x)), radd(s02.y, rmul(r, S.y))};
    o2 = {rsub(s02.x, rmul(r, S.x)), rsub(s02.y, rmul(r, S.y))};
    o1 = {radd(d02.x, rmul(r, D.y)), rsub(d02.y, rmul(r, D.x))};  // d02 - i r D
    o3 = {rsub(d02.x, rmul(r, D.y)), radd(d02.y, rmul(r, D.x))};
}

template <typename T>
struct Dft<T, 8> {
    static ISOFFT_HD void run(Cx<T> (&a)[8])
    {
        Cx<T> p[4], m[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            p[n] = cadd(a[n], a[n + 4]);
            m[n] = csub(a[n], a[n + 4]);
        }
        Dft<T, 4>::run(p);
        a[0] = p[0];
        a[2] = p[1];
        a[4] = p[2];
        a[6] = p[3];
        dft4_w8_odd(m[0], m[1], m[2], m[3], a[1], a[3], a[5], a[7]);
    }
};
template <typename T>
struct Dft<T, 6> {
    static ISOFFT_HD void run(Cx<T> (&a)[6]) { DftCT<T, 2, 3>::run(a); }
};
template <typename T>
struct Dft<T, 12> {
    static ISOFFT_HD void run(Cx<T> (&a)[12]) { DftCT<T, 4, 3>::run(a); }
};
template <typename T>
struct Dft<T, 16> {
    static ISOFFT_HD void run(Cx<T> (&a)[16]) { DftCT<T, 4, 4>::run(a); }
};
template <typename T>
struct Dft<T, 32> {
    static ISOFFT_HD void run(Cx<T> (&a)[32]) { DftCT<T, 4, 8>::run(a); }
};
template <typename T>
struct Dft<T, 24> {
    static ISOFFT_HD void run(Cx<T> (&a)[24]) { DftCT<T, 8, 3>::run(a); }
};
template <typename T>
struct Dft<T, 48> {
    static ISOFFT_HD void run(Cx<T> (&a)[48]) { DftCT<T, 16, 3>::run(a); }
};

// DFT of R inputs whose upper half a[R/2..R) is zero (first stage of a line
// that is half zero padding): even bins are the length-R/2 DFT of a, odd bins
// the length-R/2 DFT of a[r] W_R^r.
template <typename T, int R>
struct DftHalf {
    template <int r>
    static ISOFFT_HD void tw(Cx<T> (&o)[R / 2])
    {
        o[r] = mul_root<T, R, r>(o[r]);
        if constexpr (r + 1 < R / 2) tw<r + 1>(o);
    }
    static ISOFFT_HD void run(Cx<T> (&a)[R])
    {
        Cx<T> e[R / 2], o[R / 2];
#pragma unroll
        for (int r = 0; r < R / 2; ++r) e[r] = o[r] = a[r];
        tw<1>(o);
        Dft<T, R / 2>::run(e);
        Dft<T, R / 2>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            a[2 * k] = e[k];
            a[2 * k + 1] = o[k];
        }
    }
};
// Radix 8 with a[4..8) zero: even bins the 4-point DFT of a[0..4), odd
// bins as in Dft<T, 8> with m = a.
template <typename T>
struct DftHalf<T, 8> {
    static ISOFFT_HD void run(Cx<T> (&a)[8])
    {
        Cx<T> e[4] = {a[0], a[1], a[2], a[3]};
        dft4_w8_odd(a[0], a[1], a[2], a[3], a[1], a[3], a[5], a[7]);
        Dft<T, 4>::run(e);
        a[0] = e[0];
        a[2] = e[1];
        a[4] = e[2];
        a[6] = e[3];
    }
};
template <typename T>
struct DftHalf<T, 2> {
    static ISOFFT_HD void run(Cx<T> (&a)[2]) { a[1] = a[0]; }
};

// ---------------------------------------------------------------------
// Radix plans and stages
// ---------------------------------------------------------------------
template <int... Rs>
struct Radices {};
template <typename Rad>
struct RadixCount;
template <int... Rs>
struct RadixCount<Radices<Rs...>> {
    static constexpr int value = sizeof...(Rs);  // stages of the transform
};

template <int L, int E, int NS, int R>
struct StageGeom {
    static constexpr int NT = L / E;  // threads per line
    static constexpr int B = E / R;   // butterflies per thread
    static_assert(E % R == 0, "radix must divide the points per thread");
    static_assert(L % (NS * R) == 0, "radices must multiply to L");
    // Stockham output position of butterfly q, output r, for thread t
    static ISOFFT_HD int out_pos(int t, int q, int r)
    {
        const int j = t + q * NT;
        return (j / NS) * NS * R + (j % NS) + r * NS;
    }
};

// One Stockham stage in registers.  HALF: the stage's inputs at positions
// >= L/2 are known zero (only legal as the first stage, NS == 1).
template <typename T, int L, int E, int NS, int R, bool HALF>
ISOFFT_HD void stage(Cx<T> (&v)[E], int t, const Cx<T> *__restrict__ tw)
{
    using G = StageGeom<L, E, NS, R>;
#pragma unroll
    for (int q = 0; q < G::B; ++q) {
        Cx<T> a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[q + r * G::B];
        if constexpr (NS > 1) {
            const int k = (t + q * G::NT) % NS;
            constexpr int step = L / (NS * R);
#pragma unroll
            for (int r = 1; r < R; ++r) a[r] = cmul(a[r], tw[r * k * step]);
        }
        if constexpr (HALF) {
            static_assert(NS == 1, "pruned butterflies only in the first stage");
            DftHalf<T, R>::run(a);
        } else {
            Dft<T, R>::run(a);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) v[q + r * G::B] = a[r];
    }
}

// Runs the stages of a Radices<...> plan.  Xch is an exchanger providing
//   template <int NS, int R> void exchange(Cx<T>(&)[E], int t)
// that writes register (q, r) to StageGeom::out_pos(t, q, r) and reads back
// positions t + m * NT.
template <typename T, int L, int E, int NS, bool HALF, typename Xch, int R, int... Rest>
ISOFFT_HD void run_stages_impl(Cx<T> (&v)[E], int t, const Cx<T> *__restrict__ tw,
                                                Xch &xch)
{
    stage<T, L, E, NS, R, HALF>(v, t, tw);
    if constexpr (sizeof...(Rest) > 0) {
        xch.template exchange<NS, R>(v, t);
        run_stages_impl<T, L, E, NS * R, false, Xch, Rest...>(v, t, tw, xch);
    }
}

template <typename T, int L, int E, bool HALF, typename Xch, int... Rs>
ISOFFT_HD void run_stages(Cx<T> (&v)[E], int t, const Cx<T> *__restrict__ tw, Xch &xch,
                                           Radices<Rs...>)
{
    run_stages_impl<T, L, E, 1, HALF, Xch, Rs...>(v, t, tw, xch);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = crenorm(v[m]);  // the transform's results leave normalised
}

// ---------------------------------------------------------------------
// Register-resident twiddles.  A thread's twiddles depend only on its line
// position t, so a persistent kernel loads them once and reuses them for
// every tile.  Stage s keeps w[q][r-1] = W_L^{r k step} for its butterflies
// q; when every butterfly of the thread has the same k (NT a multiple of
// NS) only one set is kept.
// ---------------------------------------------------------------------
template <typename T, int L, int E, int NS, int... Rs>
struct TwRegs {
    ISOFFT_HD void load(const Cx<T> *__restrict__, int) {}
};
template <typename T, int L, int E, int NS, int R, int... Rest>
struct TwRegs<T, L, E, NS, R, Rest...> {
    static constexpr int NT = L / E, B = E / R;
    static constexpr bool SHARED = NS > 1 && NT % NS == 0;
    static constexpr int NQ = NS == 1 ? 1 : (SHARED ? 1 : B);
    Cx<T> w[NQ][R - 1];
    TwRegs<T, L, E, NS * R, Rest...> next;
    ISOFFT_HD void load(const Cx<T> *__restrict__ tw, int t)
    {
        if constexpr (NS > 1) {
            constexpr int step = L / (NS * R);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int k = (t + q * NT) % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) w[q][r - 1] = tw[r * k * step];
            }
        }
        next.load(tw, t);
    }
    ISOFFT_HD Cx<T> get(int q, int r) const { return w[SHARED ? 0 : q][r - 1]; }
};

// Stage with twiddles from registers (same arithmetic as `stage`).
template <typename T, int L, int E, int NS, int R, bool HALF, typename TWR>
ISOFFT_HD void stage_reg(Cx<T> (&v)[E], const TWR &twr)
{
    using G = StageGeom<L, E, NS, R>;
#pragma unroll
    for (int q = 0; q < G::B; ++q) {
        Cx<T> a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[q + r * G::B];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) a[r] = cmul(a[r], twr.get(q, r));
        }
        if constexpr (HALF) {
            static_assert(NS == 1, "pruned butterflies only in the first stage");
            DftHalf<T, R>::run(a);
        } else {
            Dft<T, R>::run(a);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) v[q + r * G::B] = a[r];
    }
}

template <typename T, int L, int E, int NS, bool HALF, typename Xch, typename TWR, int R, int... Rest>
ISOFFT_HD void run_stages_reg_impl(Cx<T> (&v)[E], int t, const TWR &twr, Xch &xch)
{
    stage_reg<T, L, E, NS, R, HALF>(v, twr);
    if constexpr (sizeof...(Rest) > 0) {
        xch.template exchange<NS, R>(v, t);
        run_stages_reg_impl<T, L, E, NS * R, false, Xch, decltype(twr.next), Rest...>(v, t, twr.next, xch);
    }
}

template <typename T, int L, int E, int... Rs>
using TwRegsFor = TwRegs<T, L, E, 1, Rs...>;

template <typename T, int L, int E, bool HALF, typename Xch, typename TWR, int... Rs>
ISOFFT_HD void run_stages_reg(Cx<T> (&v)[E], int t, const TWR &twr, Xch &xch, Radices<Rs...>)
{
    run_stages_reg_impl<T, L, E, 1, HALF, Xch, TWR, Rs...>(v, t, twr, xch);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = crenorm(v[m]);  // the transform's results leave normalised
}

template <typename T, int L, int E, typename Rad>
struct TwRegsOf;
template <typename T, int L, int E, int... Rs>
struct TwRegsOf<T, L, E, Radices<Rs...>> {
    using type = TwRegs<T, L, E, 1, Rs...>;
};

// Per-length configuration: points per thread E and the radix sequence.
// Eight (or twelve for lengths with a factor 3) points per thread keep the
// register footprint small enough for a next-tile prefetch; 1024-point
// lines take sixteen so a line needs no more than 64 threads.
template <int L>
struct Shape32;
template <int L>
struct Shape64 : Shape32<L> {};
#define ISOFFT_SHAPE(S, L_, E_, ...)                       \
    template <>                                           \
    struct S<L_> {                                        \
        static constexpr int E = E_;                      \
        using Rad = Radices<__VA_ARGS__>;                 \
    };
ISOFFT_SHAPE(Shape32, 16, 8, 8, 2)
ISOFFT_SHAPE(Shape32, 24, 12, 12, 2)
ISOFFT_SHAPE(Shape32, 32, 8, 8, 4)
ISOFFT_SHAPE(Shape32, 48, 12, 12, 4)
ISOFFT_SHAPE(Shape32, 64, 8, 8, 8)
ISOFFT_SHAPE(Shape32, 96, 12, 12, 4, 2)
ISOFFT_SHAPE(Shape32, 128, 8, 8, 8, 2)
ISOFFT_SHAPE(Shape32, 192, 12, 12, 4, 4)
ISOFFT_SHAPE(Shape32, 256, 8, 8, 8, 4)
ISOFFT_SHAPE(Shape32, 384, 12, 12, 4, 4, 2)
ISOFFT_SHAPE(Shape32, 512, 8, 8, 8, 8)
ISOFFT_SHAPE(Shape32, 768, 12, 12, 4, 4, 4)
ISOFFT_SHAPE(Shape32, 1024, 16, 16, 8, 8)
ISOFFT_SHAPE(Shape32, 1152, 12, 12, 12, 4, 2)
ISOFFT_SHAPE(Shape32, 1536, 12, 12, 4, 4, 4, 2)
ISOFFT_SHAPE(Shape32, 2304, 12, 12, 12, 4, 4)
ISOFFT_SHAPE(Shape64, 1024, 8, 8, 8, 8, 2)
#undef ISOFFT_SHAPE

template <typename T, int L>
struct Shape;
template <int L>
struct Shape<float, L> : Shape32<L> {};
template <int L>
struct Shape<double, L> : Shape64<L> {};
template <int L>
struct Shape<df64, L> : Shape64<L> {};  // float pairs: register footprint of FP64

// The y passes' line shapes: Shape<T, L>, except FP32 lines where fewer,
// wider stages measured faster (one or two exchanges fewer per transform, at
// 170-255 registers and half the warps):
//   512 points: 16 32 (at 256^3: K2 81.1 -> 78.3 us, K4 74.1 -> 68.5 us);
//   1024: 32 32 (at 512^3: K2 0.739 -> 0.620 ms, K4 0.595 -> 0.550 ms);
//   384: 48 8 (at 192^3: K2 41.1 -> 37.4 us, K4 36.8 -> 36.1 us);
//   256: 16 16 (at 128^3: K2 14.5 -> 12.9 us, K4 14.3 -> 12.6 us);
//   192: 24 8 (at 96^3: K2 10.3 -> 9.4 us; 16 8 at 128 points no faster);
//   768 and 1536: 24 8 4 and 24 8 8 (5-28 %; 48 16 at 768 was 10 % slower);
//   2304: 48 48 (at 1152^3: K2 13.4 -> 10.6 ms, K4 10.1 -> 9.5 ms).
template <typename T, int L>
struct YShape : Shape<T, L> {};
template <>
struct YShape<float, 512> {
    static constexpr int E = 32;
    using Rad = Radices<16, 32>;
};
template <>
struct YShape<float, 1024> {
    static constexpr int E = 32;
    using Rad = Radices<32, 32>;
};
template <>
struct YShape<float, 384> {
    static constexpr int E = 48;
    using Rad = Radices<48, 8>;
};
template <>
struct YShape<float, 256> {
    static constexpr int E = 16;
    using Rad = Radices<16, 16>;
};
template <>
struct YShape<float, 192> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8>;
};
template <>
struct YShape<float, 2304> {
    static constexpr int E = 48;
    using Rad = Radices<48, 48>;
};
template <>
struct YShape<float, 1536> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8, 8>;
};
template <>
struct YShape<float, 768> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8, 4>;
};

// The z pass holds two lines groups per tile and stages its prefetches in
// shared memory.  512-point FP32 lines run 32 points per thread in two
// stages (16 32): one exchange per transform instead of two with 8 8 8 (16
// points), on 256 threads at 254 registers (8 warps per SM instead of 16):
// 221.2 -> 198.7 us at 256^3, the shared-memory traffic and a twiddle
// stage halved.
// TW_REGS: the pass keeps its twiddles in registers across tiles (else it
// reads them from the table, through L1).
template <typename T, int L>
struct ZShape : Shape<T, L> {
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 512> {
    static constexpr int E = 32;
    using Rad = Radices<16, 32>;
    static constexpr bool TW_REGS = true;
};
// The other FP32 lengths likewise run two or three stages of 16 to 32
// points a thread instead of three to five of 8 or 12: one or two exchanges
// fewer per transform, at half the warps per SM (170-255 registers).
// Measured, z pass alone: 128 points (16 8) 22.1 -> 20.4 us at 128^2 x 64;
// 192 (24 8) 32.7 -> 26.7 us at 128^2 x 96; 256 (16 16) 38.9 -> 32.7 us at
// 128^3; 384 (24 4 4) and 768 (24 8 4) 14-16 % (384^3: 1.124 -> 0.960 ms);
// 1024 (32 32) 2.90 -> 2.79 ms at 512^3.
template <>
struct ZShape<float, 128> {
    static constexpr int E = 16;
    using Rad = Radices<16, 8>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 192> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 256> {
    static constexpr int E = 16;
    using Rad = Radices<16, 16>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 1024> {
    static constexpr int E = 32;
    using Rad = Radices<32, 32>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 384> {
    static constexpr int E = 24;
    using Rad = Radices<24, 4, 4>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<float, 768> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8, 4>;
    static constexpr bool TW_REGS = true;
};
// 16-byte points on 768-point lines (one-column tiles of 128 threads): the
// radix 12 goes last, where a thread's stage twiddles are shared by all its
// butterflies (the thread count is a multiple of every stage's stride): 17
// twiddles a thread instead of 27, and no spills under the 168-register cap
// (df64 z pass 10.43 -> 9.14 ms at 384^3; the same order at 384 points
// measured 8 % slower).
struct ZShape16B768 {
    static constexpr int E = 12;
    using Rad = Radices<4, 4, 4, 12>;
    static constexpr bool TW_REGS = true;
};
template <>
struct ZShape<double, 768> : ZShape16B768 {};
template <>
struct ZShape<df64, 768> : ZShape16B768 {};
// 2304-point lines read their twiddles from the table (a thread's share
// would not fit in registers next to its points).  FP32 takes 24 points per
// thread and three stages, so that a tile of two columns (16 bytes, the
// narrowest tensor-copy row) fits 384 threads; 16-byte FP64-class points
// keep 12 per thread on one-column tiles.  (48 points a thread in two
// stages, as the y passes take, measured 11 % slower here: 192 threads, 6
// warps per SM.)
template <typename T>
struct ZShape<T, 2304> : Shape<T, 2304> {
    static constexpr bool TW_REGS = false;
};
template <>
struct ZShape<float, 2304> {
    static constexpr int E = 24;
    using Rad = Radices<24, 24, 4>;
    static constexpr bool TW_REGS = false;
};

// The x passes hold one row per (half) warp; a 256-point FP32 row runs 16
// points per thread and two radix-16 stages, so it takes one exchange
// instead of two and fewer twiddle loads (the x passes are bound by the
// L1/shared pipe).
template <typename T, int L>
struct XShape : Shape<T, L> {};
template <>
struct XShape<float, 256> {
    static constexpr int E = 16;
    using Rad = Radices<16, 16>;
};
// K1's rows: FP32 rows of 768 and 1152 points run 24 points per thread in
// three stages (two exchanges instead of three); measured 42 % and 22 %
// faster than 12 points per thread, while K5 on the same rows was slower
// (48 24 at 1152 points: 18 % slower again).  512-point rows run 32 points
// in two stages (32 16) instead of 8 in three: K1 0.477 -> 0.402 ms at
// 512^3.
template <typename T, int L>
struct XShapeF : XShape<T, L> {};
template <>
struct XShapeF<float, 768> {
    static constexpr int E = 24;
    using Rad = Radices<24, 8, 4>;
};
template <>
struct XShapeF<float, 512> {
    static constexpr int E = 32;
    using Rad = Radices<32, 16>;
};
template <>
struct XShapeF<float, 1152> {
    static constexpr int E = 24;
    using Rad = Radices<24, 12, 4>;
};

}  // namespace isofft
