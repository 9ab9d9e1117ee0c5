// noalloc.cu -- ipf_solve_noalloc: one solve that allocates no memory.
//
// Some callers cannot call cudaMalloc: a simulation that hands its whole
// device memory to its own pool allocator, code that runs while a stream is
// being captured into a CUDA graph, or a time-step loop that must not pay the
// device-wide synchronisation cudaMalloc/cudaFree may imply.  For them this
// entry point solves small meshes with every intermediate -- twiddle tables,
// the Green's spectrum and the transform workspace -- carved out of one
// file-scope device array that the library owns for the life of the process.
// Nothing is cached between calls: each call rebuilds its tables and spectrum
// (cheap at the sizes the array admits) and then runs the same five passes
// as ipf_solve.
#include <math.h>

#include <mutex>

#include "../../include/isofft.h"
#include "launch.h"
#include "fft_engine.cuh"

namespace isofft {

// The scratch every ipf_solve_noalloc call shares; every device that loads
// the library holds it until the process exits.
constexpr size_t kNoallocScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

template <typename T>
static __global__ void k_roots(Cx<T> *__restrict__ out, int n, int count)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)n, &s, &c);
        out[k] = {(T)c, (T)-s};
    }
}

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

int64_t noalloc_mesh(int64_t n)
{
    for (int m : kSupportedM)
        if (m >= 2 * n) return m;
    return -1;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Host-side address of this device's copy of the array (set up on the first
// call on each device, with that device current).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

struct Carve {
    size_t tw_x, rtw, tw_y, tw_z, spec, work, total;
};

template <typename T>
Carve carve(const int64_t N[3], const int64_t M[3])
{
    const size_t cs = 2 * sizeof(T);
    const int64_t Lx = M[0] / 2;
    Carve c;
    size_t off = align256(sizeof(unsigned));  // the status word comes first
    c.tw_x = off;
    off += align256(Lx * cs);
    c.rtw = off;
    off += align256(Lx * cs);
    c.tw_y = off;
    off += align256(M[1] * cs);
    c.tw_z = off;
    off += align256(M[2] * cs);
    c.spec = off;
    off += align256(spectrum_elems<T>(M) * sizeof(T));
    // the workspace and the FP64 spectrum-build scratch are never live at once
    const size_t work = (size_t)N[2] * M[1] * Lx * cs;
    const size_t build = (green_octant_elems(M) + green_cos_elems(M)) * sizeof(double);
    c.work = off;
    off += align256(work > build ? work : build);
    c.total = off;
    return c;
}

template <typename T>
int solve_noalloc(const int64_t N[3], const int64_t M[3], const double hn[3], double gscale, const void *src,
                  void *phi, cudaStream_t st)
{
    const Carve cv = carve<T>(N, M);
    if (cv.total > kNoallocScratchBytes) return IPF_BUDGET_EXCEEDED;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return IPF_CUDA_ERROR;
    unsigned char *b = (unsigned char *)base;
    Cx<T> *tw_x = (Cx<T> *)(b + cv.tw_x), *rtw = (Cx<T> *)(b + cv.rtw);
    Cx<T> *tw_y = (Cx<T> *)(b + cv.tw_y), *tw_z = (Cx<T> *)(b + cv.tw_z);
    T *G = (T *)(b + cv.spec);
    T *Gs = G + spectrum_elems<T>(M) - (M[1] / 2 + 1) * (M[2] / 2 + 1);
    void *W = b + cv.work;
    const int Nx = (int)N[0], Ny = (int)N[1], Nz = (int)N[2];
    const int Lx = (int)(M[0] / 2), My = (int)M[1], Mz = (int)M[2];

    // tables: W_Lx^k, W_Mx^k (k < Lx), W_My^k, W_Mz^k
    k_roots<T><<<(Lx + 255) / 256, 256, 0, st>>>(tw_x, Lx, Lx);
    count_launch();
    k_roots<T><<<(Lx + 255) / 256, 256, 0, st>>>(rtw, 2 * Lx, Lx);
    count_launch();
    k_roots<T><<<(My + 255) / 256, 256, 0, st>>>(tw_y, My, My);
    count_launch();
    k_roots<T><<<(Mz + 255) / 256, 256, 0, st>>>(tw_z, Mz, Mz);
    count_launch();
    // the spectrum, built in the workspace region before the workspace is used
    double *oct = (double *)W;
    double *ct = oct + green_octant_elems(M);
    e = enqueue_green_spectrum<T>(M, hn, G, Gs, oct, ct, st);
    if (e == cudaSuccess)
        e = launch_x_forward<T>(Lx, (const T *)src, W, tw_x, rtw, Nx, Ny, My, (int64_t)Ny * Nz, 0, st);
    if (e == cudaSuccess) e = launch_y_forward<T>(My, W, tw_y, Ny, Lx, Nz, 0, (unsigned *)b, y_default_variant(My, sizeof(T)), st);
    if (e == cudaSuccess) e = launch_z_convolve<T>(Mz, W, tw_z, G, Gs, (T)gscale, Nz, My, Lx, 0, (unsigned *)b, 0u, st);
    if (e == cudaSuccess) e = launch_y_inverse<T>(My, W, tw_y, Ny, Lx, Nz, 0, (unsigned *)b, y_default_variant(My, sizeof(T)), st);
    if (e == cudaSuccess) e = launch_x_inverse<T>(Lx, W, (T *)phi, tw_x, rtw, Nx, Ny, My, (int64_t)Ny * Nz, 0, st);
    return e == cudaSuccess ? IPF_OK : IPF_CUDA_ERROR;
}

}  // namespace
}  // namespace isofft

using namespace isofft;

extern "C" int ipf_noalloc_check(void *stream)
{
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return IPF_CUDA_ERROR;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, base, sizeof(w), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return IPF_CUDA_ERROR;
    if (w == 0) return IPF_OK;
    e = cudaMemsetAsync(base, 0, sizeof(w), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return IPF_CUDA_ERROR;
    return (w & 1u) ? IPF_TIMEOUT : IPF_CUDA_ERROR;
}

extern "C" int ipf_solve_noalloc(const int64_t n[3], const double h[3], int dtype, const void *d_src, void *d_phi,
                                 void *stream)
{
    if (!n || !h || !d_src || !d_phi) return IPF_INVALID_ARG;
    if (dtype != IPF_F32 && dtype != IPF_F64) return IPF_INVALID_ARG;
    if ((((uintptr_t)d_src) & 15u) || (((uintptr_t)d_phi) & 15u)) return IPF_INVALID_ARG;
    int64_t M[3];
    double hmin = h[0];
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || !(h[a] > 0.0) || !isfinite(h[a])) return IPF_INVALID_ARG;
        M[a] = noalloc_mesh(n[a]);
        if (M[a] < 0) return IPF_UNSUPPORTED_SIZE;
        if (h[a] < hmin) hmin = h[a];
    }
    // widths over their minimum, rounded as the spectrum cache rounds them
    double hn[3];
    const double q = 17592186044416.0;  // 2^44
    for (int a = 0; a < 3; ++a) hn[a] = nearbyint(h[a] / hmin * q) / q;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == IPF_F32 ? solve_noalloc<float>(n, M, hn, hmin * hmin, d_src, d_phi, st)
                            : solve_noalloc<double>(n, M, hn, hmin * hmin, d_src, d_phi, st);
}
