// launch.h -- host-side launchers of the device passes (internal to the
// library; the public surface is include/isofft.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "df64.cuh"

namespace isofft {

// Doubled-mesh lengths the kernels are instantiated for (any M >= 2N - 1
// gives the same cropped result, so a plan rounds 2N up to the next one).
constexpr int kSupportedM[] = {32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2304};
constexpr int kMaxM = 2304;

// Counts every kernel launch the library makes (ipf_launch_count).
void count_launch();

// All pointers are device pointers of the current device; complex buffers
// are interleaved (re, im) of the arithmetic type T; source and potential
// arrays hold IoReal<T>::type (double for df64).
// `zsh`: the workspace's z planes are grouped in blocks of 2^zsh (w_row in
// passes.cuh; 0 = plain [Nz][My][Kx]).  Every launch must cover whole blocks
// (cudaErrorInvalidValue otherwise); plans block the workspace only where the
// z lines have 2304 points (the paired z pass).
// Planes per z block of a blocked workspace, as a shift: 16.  The z pass
// then reads each line group in runs of 16 rows one Kx row (9 KB at 1152^3)
// apart instead of rows a whole plane (21 MB) apart: 32-byte strided reads
// measured 3.5 TB/s against 1.5 TB/s, while the y passes' rows move from Kx
// to 16 Kx apart (4.7 -> 3.2 TB/s on the same read test, on passes that are
// bound elsewhere).
constexpr int kZBlockShift = 4;
template <typename T>
cudaError_t launch_x_forward(int L, const typename IoReal<T>::type *src, void *W, const void *tw, const void *rtw,
                             int Nx, int Ny, int My, int64_t nrows, int zsh, cudaStream_t st);
template <typename T>
cudaError_t launch_x_inverse(int L, const void *W, typename IoReal<T>::type *phi, const void *tw, const void *rtw,
                             int Nx, int Ny, int My, int64_t nrows, int zsh, cudaStream_t st);
// The y passes come in three forms with bitwise the same arithmetic:
//   kYTile        one CTA per column tile (plain loads; many CTAs per SM),
//   kYStream      persistent CTAs fed by tensor-map copies (see passes.cuh),
//   kYTileNarrow  the tile form on tiles of half the width.
// Plans pick one per pass by timing all three (y_default_variant without).
enum { kYTile = 0, kYStream = 1, kYTileNarrow = 2 };
constexpr int kYForms = 3;
template <typename T>
cudaError_t launch_y_forward(int L, void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status,
                             int variant, cudaStream_t st);
template <typename T>
cudaError_t launch_y_inverse(int L, void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status,
                             int variant, cudaStream_t st);
// The form used without timing: streamed for 8-byte points on lines of 512
// to 1024 points (where it measured faster), tiles elsewhere.
inline int y_default_variant(int L, size_t real_bytes)
{
    return real_bytes == 4 && L >= 512 && L <= 1024 ? kYStream : kYTile;
}
// `status` (device word, may be null) gets bit 0 set when one of the pass's
// bounded waits for its tile copies gave up (ipf_plan_check reads it); the
// y passes and the z pass share it.  `test_extra_tx` (normally 0) is the
// run-out test hook: bytes each CTA's first tile expects beyond its copies.
template <typename T>
cudaError_t launch_z_convolve(int L, void *W, const void *tw, const T *G, const T *Gs, T gscale, int Nz,
                              int My, int Kx, int zsh, unsigned *status, unsigned test_extra_tx, cudaStream_t st);

// Width (kx columns per tile) of the z pass for line length L; the cached
// Green's spectrum is stored in tiles of this width (0: unsupported L).
template <typename T>
int z_tile_for(int L);

// Elements of one (k_y', kx tile) block of the cached spectrum: nkz x tx
// values, padded so that every block starts on a 16-byte boundary (the z pass
// copies a block with one bulk copy).
constexpr int z_spec_block(int tx, int nkz, int elem_bytes)
{
    return (nkz * tx + 16 / elem_bytes - 1) / (16 / elem_bytes) * (16 / elem_bytes);
}

// Device bytes of the cached Green's spectrum of a doubled mesh M.
template <typename T>
size_t spectrum_elems(const int64_t M[3]);

// Green's spectrum (FP64 build).  M = doubled mesh, hn = widths divided by
// their minimum.  Writes G [My/2+1][Mz/2+1][Mx/2] and Gs [My/2+1][Mz/2+1] of
// type T in the z pass's tiled layout, pre-divided by 2 Mx My Mz (see
// passes.cuh).  Allocates and frees its FP64 scratch; synchronises `st`
// before returning.
template <typename T>
cudaError_t build_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, cudaStream_t st);

// The same spectrum enqueued without allocating or synchronising, in caller
// scratch: `oct` holds green_octant_elems(M) doubles (the FP64 octant,
// transformed in place), `ct` holds green_cos_elems(M) doubles (the root
// tables of the three axes, computed on the device).
template <typename T>
cudaError_t enqueue_green_spectrum(const int64_t M[3], const double hn[3], T *G, T *Gs, double *oct,
                                   double *ct, cudaStream_t st);
int64_t green_octant_elems(const int64_t M[3]);
int64_t green_cos_elems(const int64_t M[3]);

// Device bytes of the FP64 scratch build_green_spectrum needs for mesh M.
size_t green_build_scratch_bytes(const int64_t M[3]);

// One grid of a batch run in one launch per pass (batch.cu): the plan's
// buffers and sizes.
struct BatchGridDesc {
    const void *src;
    void *phi;
    void *W;
    const void *tw_x, *rtw, *tw_y, *tw_z;
    const void *G, *Gs;
    double gscale;
    int Nx, Ny, Nz, Mx, My, Mz;
    int runout;  // test hook (IPF_FLAG_TEST_WAIT_RUNOUT): in one launch, the z items' wait runs out
};
// Whether a grid of this dtype and doubled mesh can join a batched launch
// (FP32, every doubled length at most 256).
bool batch_fits(int dtype_is_f32, const int64_t M[3]);
// The five passes of `count` such grids on `st`: mode 1, one launch per
// pass; mode 2, one persistent launch for all five (per-(grid, pass)
// completion counters; a wait that runs out sets bit 0 of *status, which
// may be null).  The first call for a given set of grids builds and uploads
// its work tables (synchronously); later calls only launch.
cudaError_t batch_enqueue(const BatchGridDesc *grids, int count, int mode, unsigned *status, cudaStream_t st);

// e^{-2 pi i k / n} for 0 <= k < count, by exact reduction to the first
// octant (host, libm in double).
void host_roots(int64_t n, int64_t count, double *re, double *im);

}  // namespace isofft
