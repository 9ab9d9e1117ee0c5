// pf2.cuh -- a pair of FP32 values operated on by the packed FP32x2
// instructions of sm_100+ (one add, multiply or fused multiply-add issues
// for both halves).
//
// The z pass uses it to transform two lines in one thread: a point held is
// Cx<pf2> = {(re_A, re_B), (im_A, im_B)}, so every butterfly and twiddle
// operation applies to both lines at the cost of one issue slot.  The FP32
// pipe does the same lane work either way; what halves is the instruction
// issue the FP32 arithmetic takes, which bounds the z pass.
//
// Each half is rounded exactly as the scalar FP32 operation would round it
// (IEEE round-to-nearest; fma rounds once).  Subtraction is a fused
// multiply-add by -1, which is exact rounding of a - b.  Host code (the CPU
// check of the engine) runs the same operations on each half.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace isofft {

struct pf2 {
    float2 v;
    pf2() = default;
    __host__ __device__ constexpr pf2(float2 p) : v(p) {}
    __host__ __device__ constexpr pf2(float a, float b) : v{a, b} {}
    // a constant in both halves
    __host__ __device__ constexpr pf2(double d) : v{(float)d, (float)d} {}
    __host__ __device__ constexpr explicit pf2(int i) : v{(float)i, (float)i} {}
};

__host__ __device__ __forceinline__ pf2 pf2_fma(pf2 a, pf2 b, pf2 c)
{
#ifdef __CUDA_ARCH__
    return pf2(__ffma2_rn(a.v, b.v, c.v));
#else
    return pf2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y));
#endif
}
__host__ __device__ __forceinline__ pf2 operator+(pf2 a, pf2 b)
{
#ifdef __CUDA_ARCH__
    return pf2(__fadd2_rn(a.v, b.v));
#else
    return pf2(a.v.x + b.v.x, a.v.y + b.v.y);
#endif
}
__host__ __device__ __forceinline__ pf2 operator*(pf2 a, pf2 b)
{
#ifdef __CUDA_ARCH__
    return pf2(__fmul2_rn(a.v, b.v));
#else
    return pf2(a.v.x * b.v.x, a.v.y * b.v.y);
#endif
}
// a - b as fma(b, -1, a): one packed instruction, rounded as a - b
__host__ __device__ __forceinline__ pf2 operator-(pf2 a, pf2 b) { return pf2_fma(b, pf2(-1.0), a); }
__host__ __device__ __forceinline__ pf2 operator-(pf2 a) { return a * pf2(-1.0); }

}  // namespace isofft

#include "fft_engine.cuh"

namespace isofft {

// A point of two lines: x = (re_A, re_B), y = (im_A, im_B).  Multiplying by
// -i or +i exchanges the halves of a point and flips a sign, which the
// butterflies below fold into the choice of add or subtract: no operation
// here negates a value on its own.
using PCx = Cx<pf2>;

// twiddle of both lines (the same root for both)
struct PTw {
    pf2 x, y;
};
__host__ __device__ __forceinline__ PTw ptw(Cx<float> w) { return {pf2((double)w.x), pf2((double)w.y)}; }
// a * w: re = a.x w.x - a.y w.y, im = a.x w.y + a.y w.x
__host__ __device__ __forceinline__ PCx pcmul(PCx a, PTw w)
{
    return {pf2_fma(a.y * w.y, pf2(-1.0), a.x * w.x), pf2_fma(a.x, w.y, a.y * w.x)};
}

// Forward 4-point DFT of c[0..3] (the engine's Dft<T, 4> arithmetic).
__host__ __device__ __forceinline__ void pdft4(PCx &c0, PCx &c1, PCx &c2, PCx &c3)
{
    const PCx s02 = {c0.x + c2.x, c0.y + c2.y}, d02 = {c0.x - c2.x, c0.y - c2.y};
    const PCx s13 = {c1.x + c3.x, c1.y + c3.y}, e = {c1.x - c3.x, c1.y - c3.y};
    c0 = {s02.x + s13.x, s02.y + s13.y};
    c2 = {s02.x - s13.x, s02.y - s13.y};
    c1 = {d02.x + e.y, d02.y - e.x};  // d02 - i e
    c3 = {d02.x - e.y, d02.y + e.x};  // d02 + i e
}

// The odd-output half of an 8-point DFT (X[1], X[3], X[5], X[7]) from the
// differences b = x[n] - x[n + 4] (n < 4): a 4-point DFT of b[n] W_8^n with
// the roots W_8 and W_8^3 = r (1 - i), r (-1 - i) (r = 1/sqrt 2) applied
// through fused multiply-adds.
__host__ __device__ __forceinline__ void pdft8_odd(PCx b0, PCx b1, PCx b2, PCx b3, PCx &X1, PCx &X3, PCx &X5,
                                                   PCx &X7)
{
    const pf2 r(0.7071067811865476), nr(-0.7071067811865476);
    // W_8 b1 + W_8^3 b3 = r S, W_8 b1 - W_8^3 b3 = r D
    const PCx P = {b1.x + b3.x, b1.y + b3.y}, Q = {b1.x - b3.x, b1.y - b3.y};
    const PCx S = {Q.x + P.y, Q.y - P.x}, D = {P.x + Q.y, P.y - Q.x};
    // W_8^2 b2 = -i b2
    const PCx s02 = {b0.x + b2.y, b0.y - b2.x}, d02 = {b0.x - b2.y, b0.y + b2.x};
    X1 = {pf2_fma(r, S.x, s02.x), pf2_fma(r, S.y, s02.y)};
    X5 = {pf2_fma(nr, S.x, s02.x), pf2_fma(nr, S.y, s02.y)};
    X3 = {pf2_fma(r, D.y, d02.x), pf2_fma(nr, D.x, d02.y)};  // d02 - i r D
    X7 = {pf2_fma(nr, D.y, d02.x), pf2_fma(r, D.x, d02.y)};  // d02 + i r D
}

// Forward 8-point DFT in place, a[k] <- sum_n a[n] W_8^{nk} (2 x 4
// Cooley-Tukey, as Dft<T, 8>).
__host__ __device__ __forceinline__ void pdft8(PCx (&a)[8])
{
    PCx s[4], d[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        s[n] = {a[n].x + a[n + 4].x, a[n].y + a[n + 4].y};
        d[n] = {a[n].x - a[n + 4].x, a[n].y - a[n + 4].y};
    }
    pdft4(s[0], s[1], s[2], s[3]);
    pdft8_odd(d[0], d[1], d[2], d[3], a[1], a[3], a[5], a[7]);
    a[0] = s[0];
    a[2] = s[1];
    a[4] = s[2];
    a[6] = s[3];
}

// The same with a[4..7] zero (the first stage of a half-zero line): sums
// and differences are the inputs themselves.
__host__ __device__ __forceinline__ void pdft8_half(PCx (&a)[8])
{
    PCx s0 = a[0], s1 = a[1], s2 = a[2], s3 = a[3];
    pdft4(s0, s1, s2, s3);
    pdft8_odd(a[0], a[1], a[2], a[3], a[1], a[3], a[5], a[7]);
    a[0] = s0;
    a[2] = s1;
    a[4] = s2;
    a[6] = s3;
}

}  // namespace isofft
