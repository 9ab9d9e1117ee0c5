// Read-pattern probe behind the z-blocked workspace of the 2304-point z
// lines.  The workspace of a 1152^3 solve, as 8-byte pairs, is [Z][Y][X]
// with X = 1152 (one Kx row, 9 KB), Y = 2304 rows per plane; here Z = 576
// planes (12.2 GB).  Planes are grouped in blocks of zb:
// [Z/zb][Y][zb][X].  The "z" pattern reads 32-byte chunks of one (x, y) over
// all z (the z pass's line groups); the "y" pattern reads 32-byte chunks of
// one (x, z) over all y (the y passes' columns).  Consecutive CTAs take
// adjacent chunks, as the passes' persistent grids do.  Prints one line per
// (zb, pattern): "zb pattern GB/s".
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ long row_of(long z, long y, long Y, long zb)
{
    return ((z / zb) * Y + y) * zb + z % zb;
}

// which = 0: chunk (xc, y) over all z; which = 1: chunk (xc, z) over all y
__global__ void read_pattern(const uint4 *__restrict__ a, long X16, long Y, long Z, long zb, long units, int which,
                             float *out)
{
    float acc = 0.f;
    const long xch = X16 / 2;
    for (long u = blockIdx.x; u < units; u += gridDim.x) {
        const long xc = u % xch, o = u / xch;
        const long n = which == 0 ? Z : Y;
#pragma unroll 4
        for (long i = threadIdx.x >> 1; i < n; i += 128) {
            const long r = which == 0 ? row_of(i, o, Y, zb) : row_of(o, i, Y, zb);
            const uint4 v = __ldg(a + r * X16 + xc * 2 + (threadIdx.x & 1));
            acc += __int_as_float(v.x) + __int_as_float(v.w);
        }
    }
    if (acc == 1.2345f) out[0] = acc;  // keeps the loads
}

int main()
{
    const long X = 9216, Y = 2304, Z = 576;  // Z divisible by every zb below
    const long bytes = X * Y * Z;
    uint4 *a = nullptr;
    float *o = nullptr;
    if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&o, 4) != cudaSuccess) return 1;
    if (cudaMemset(a, 0, bytes) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    for (long zb : {1L, 4L, 16L}) {
        for (int which = 0; which < 2; ++which) {
            const long units = (X / 32) * (which == 0 ? Y : Z);
            auto run = [&]() { read_pattern<<<sms * 16, 256>>>(a, X / 16, Y, Z, zb, units, which, o); };
            run();
            run();
            cudaEventRecord(e0);
            run();
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            printf("%ld %s %.1f\n", zb, which == 0 ? "z" : "y", (double)bytes / ms / 1e6);
        }
    }
    cudaFree(a);
    cudaFree(o);
    return cudaGetLastError() != cudaSuccess;
}
