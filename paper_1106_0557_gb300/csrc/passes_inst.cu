// passes_inst.cu -- instantiates and launches the pass kernels for one real
// type and one group of passes.  The build compiles this file several times:
//   -DISOFFT_REAL=float|double|isofft::df64   the arithmetic type
//   -DISOFFT_GROUP=1|2|3         1: x passes (K1, K5), 2: y passes (K2, K4),
//                                3: z pass (K3)
// so that the instantiations compile in parallel.
#include <atomic>

#include "launch.h"
#include "passes.cuh"

#ifndef ISOFFT_REAL
#error "define ISOFFT_REAL"
#endif
#ifndef ISOFFT_GROUP
#error "define ISOFFT_GROUP"
#endif

namespace isofft {

using Real = ISOFFT_REAL;

// Raise a kernel's dynamic shared memory limit once per device.
template <typename F>
static cudaError_t ensure_smem(F *func, size_t bytes, std::atomic<uint64_t> &done)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

#define ISOFFT_ROW_LENGTHS(X) \
    X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1152)
#define ISOFFT_COL_LENGTHS(X) \
    X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2304)

// Resident CTAs per SM of a kernel on the current device (queried once).
template <typename F>
static int resident_ctas(F *func, int threads, size_t smem, std::atomic<int> &cache)
{
    int v = cache.load(std::memory_order_acquire);
    if (v > 0) return v;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, func, threads, smem) != cudaSuccess) return 0;
    v = sms * (per > 0 ? per : 1);
    cache.store(v, std::memory_order_release);
    return v;
}

// cuTensorMapEncodeTiled, resolved once through the runtime (no link
// dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static std::atomic<EncodeTiledFn> fn{nullptr};
    EncodeTiledFn f = fn.load(std::memory_order_acquire);
    if (f) return f;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return nullptr;
    f = reinterpret_cast<EncodeTiledFn>(p);
    fn.store(f, std::memory_order_release);
    return f;
}


#if ISOFFT_GROUP == 1
// Row grid: one CTA per group of nl rows, at most `resident` when that is
// set (persistent CTAs).
static unsigned row_grid(int64_t nrows, int nl, int resident)
{
    const int64_t groups = (nrows + nl - 1) / nl;
    return (unsigned)(resident > 0 && groups > resident ? resident : groups);
}
template <typename T, int L>
static cudaError_t run_x_forward(const In<T> *src, void *W, const void *tw, const void *rtw, int Nx, int Ny,
                                 int My, int64_t nrows, int zsh, cudaStream_t st)
{
    using C = RowCfg<T, L, XShapeF<T, L>>;
    static std::atomic<uint64_t> done{0};
    static std::atomic<int> resident{0};
    if (Ny <= 0 || nrows % Ny || !w_blocks_ok(nrows / Ny, zsh)) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem(k_x_forward<T, L>, C::SMEM, done);
    if (e != cudaSuccess) return e;
    const unsigned grid =
        row_grid(nrows, C::NL, C::TWR_F ? resident_ctas(k_x_forward<T, L>, C::THREADS, C::SMEM, resident) : 0);
    k_x_forward<T, L><<<grid, C::THREADS, C::SMEM, st>>>(src, (Cx<T> *)W, (const Cx<T> *)tw,
                                                        (const Cx<T> *)rtw, Nx, Ny, My, nrows, zsh);
    count_launch();
    return cudaGetLastError();
}
template <typename T, int L>
static cudaError_t run_x_inverse(const void *W, In<T> *phi, const void *tw, const void *rtw, int Nx, int Ny,
                                 int My, int64_t nrows, int zsh, cudaStream_t st)
{
    using C = RowCfg<T, L>;
    static std::atomic<uint64_t> done{0};
    static std::atomic<int> resident{0};
    if (Ny <= 0 || nrows % Ny || !w_blocks_ok(nrows / Ny, zsh)) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem(k_x_inverse<T, L>, C::SMEM, done);
    if (e != cudaSuccess) return e;
    const unsigned grid =
        row_grid(nrows, C::NL, C::TWR_I ? resident_ctas(k_x_inverse<T, L>, C::THREADS, C::SMEM, resident) : 0);
    k_x_inverse<T, L><<<grid, C::THREADS, C::SMEM, st>>>((const Cx<T> *)W, phi, (const Cx<T> *)tw,
                                                        (const Cx<T> *)rtw, Nx, Ny, My, nrows, zsh);
    count_launch();
    return cudaGetLastError();
}

template <typename R_>
cudaError_t launch_x_forward(int L, const In<R_> *src, void *W, const void *tw, const void *rtw, int Nx,
                                 int Ny, int My, int64_t nrows, int zsh, cudaStream_t st)
{
    switch (L) {
#define X_(n) \
    case n: return run_x_forward<R_, n>(src, W, tw, rtw, Nx, Ny, My, nrows, zsh, st);
        ISOFFT_ROW_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}
template <typename R_>
cudaError_t launch_x_inverse(int L, const void *W, In<R_> *phi, const void *tw, const void *rtw, int Nx,
                                 int Ny, int My, int64_t nrows, int zsh, cudaStream_t st)
{
    switch (L) {
#define X_(n) \
    case n: return run_x_inverse<R_, n>(W, phi, tw, rtw, Nx, Ny, My, nrows, zsh, st);
        ISOFFT_ROW_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_x_forward<Real>(int, const In<Real> *, void *, const void *, const void *, int, int,
                                            int, int64_t, int, cudaStream_t);
template cudaError_t launch_x_inverse<Real>(int, const void *, In<Real> *, const void *, const void *, int, int,
                                            int, int64_t, int, cudaStream_t);
#endif

#if ISOFFT_GROUP == 2
template <typename T, int L, bool FWD, bool NARROW>
static cudaError_t run_y_tile(void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, cudaStream_t st)
{
    using C = ColCfg<T, L, NARROW>;
    static std::atomic<uint64_t> done0{0}, doneb{0};
    // plain and z-blocked workspace instances
    auto *k = zsh ? (FWD ? k_y_forward<T, L, NARROW, true> : k_y_inverse<T, L, NARROW, true>)
                  : (FWD ? k_y_forward<T, L, NARROW, false> : k_y_inverse<T, L, NARROW, false>);
    if (!w_blocks_ok(Nz, zsh)) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem(k, C::SMEM, zsh ? doneb : done0);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((Kx + C::TX - 1) / C::TX), (unsigned)Nz);
    k<<<grid, C::THREADS, C::SMEM, st>>>((Cx<T> *)W, (const Cx<T> *)tw, Ny, Kx, zsh);
    count_launch();
    return cudaGetLastError();
}
template <typename T, int L, bool FWD>
static cudaError_t run_y_stream(void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status,
                                cudaStream_t st)
{
    using C = YCfg<T, L>;
    constexpr size_t SMEM = FWD ? C::SMEM_F : C::SMEM_I;
    static std::atomic<uint64_t> done0{0}, doneb{0};
    static std::atomic<int> slots0{0}, slotsb{0};
    if ((uintptr_t)W & 15) return cudaErrorMisalignedAddress;
    // plain and z-blocked workspace instances
    auto *k = zsh ? k_y_pass<T, L, FWD, true> : k_y_pass<T, L, FWD, false>;
    cudaError_t e = ensure_smem(k, SMEM, zsh ? doneb : done0);
    if (e != cudaSuccess) return e;
    const int ntx = (Kx + C::TX - 1) / C::TX;
    const int ntiles = ntx * Nz;
    int grid = resident_ctas(k, C::THREADS, SMEM, zsh ? slotsb : slots0);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (grid > ntiles) grid = ntiles;
    // W as 8-byte elements [Nz][My][Kx * EPC] (z-blocked: [Nz >> zsh][My][2^zsh][Kx * EPC], mapped as
    // {Kx EPC, 2^zsh, rows, Nz >> zsh}); K2 sees only rows y < Ny
    EncodeTiledFn encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    if (!w_blocks_ok(Nz, zsh)) return cudaErrorInvalidValue;
    CUtensorMap map;
    const cuuint64_t rows = (cuuint64_t)(FWD ? Ny : L), cb = sizeof(Cx<T>);
    const cuuint64_t dims3[3] = {(cuuint64_t)Kx * C::EPC, rows, (cuuint64_t)Nz};
    const cuuint64_t strides3[2] = {(cuuint64_t)Kx * cb, (cuuint64_t)L * Kx * cb};
    const cuuint32_t box3[3] = {(cuuint32_t)(C::TX * C::EPC), (cuuint32_t)(FWD ? C::BOX_F : C::BOX_I), 1u};
    const cuuint64_t dims4[4] = {(cuuint64_t)Kx * C::EPC, (cuuint64_t)1 << zsh, rows, (cuuint64_t)(Nz >> zsh)};
    const cuuint64_t strides4[3] = {(cuuint64_t)Kx * cb, ((cuuint64_t)Kx * cb) << zsh,
                                    ((cuuint64_t)L * Kx * cb) << zsh};
    const cuuint32_t box4[4] = {(cuuint32_t)(C::TX * C::EPC), 1u, (cuuint32_t)(FWD ? C::BOX_F : C::BOX_I), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, zsh ? 4 : 3, W, zsh ? dims4 : dims3, zsh ? strides4 : strides3,
               zsh ? box4 : box3, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // K2's output map on the plain workspace (every row y < My), for the
    // kernels that write their tiles by tensor stores; elsewhere unused
    CUtensorMap omap = map;
    if (FWD && !zsh) {
        const cuuint64_t odims[3] = {(cuuint64_t)Kx * C::EPC, (cuuint64_t)L, (cuuint64_t)Nz};
        const cuuint32_t obox[3] = {(cuuint32_t)(C::TX * C::EPC), (cuuint32_t)C::BOX_I, 1u};
        if (encode(&omap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, W, odims, strides3, obox, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    k<<<grid, C::THREADS, SMEM, st>>>(map, omap, (Cx<T> *)W, (const Cx<T> *)tw, Ny, Kx, ntiles, status, zsh);
    count_launch();
    return cudaGetLastError();
}
template <typename T, int L, bool FWD>
static cudaError_t run_y(void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status, int variant,
                         cudaStream_t st)
{
    if (variant == kYStream) return run_y_stream<T, L, FWD>(W, tw, Ny, Kx, Nz, zsh, status, st);
    if (variant == kYTileNarrow) return run_y_tile<T, L, FWD, true>(W, tw, Ny, Kx, Nz, zsh, st);
    return run_y_tile<T, L, FWD, false>(W, tw, Ny, Kx, Nz, zsh, st);
}
template <typename R_>
cudaError_t launch_y_forward(int L, void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status,
                             int variant, cudaStream_t st)
{
    switch (L) {
#define X_(n) \
    case n: return run_y<R_, n, true>(W, tw, Ny, Kx, Nz, zsh, status, variant, st);
        ISOFFT_COL_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}
template <typename R_>
cudaError_t launch_y_inverse(int L, void *W, const void *tw, int Ny, int Kx, int Nz, int zsh, unsigned *status,
                             int variant, cudaStream_t st)
{
    switch (L) {
#define X_(n) \
    case n: return run_y<R_, n, false>(W, tw, Ny, Kx, Nz, zsh, status, variant, st);
        ISOFFT_COL_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_y_forward<Real>(int, void *, const void *, int, int, int, int, unsigned *, int,
                                            cudaStream_t);
template cudaError_t launch_y_inverse<Real>(int, void *, const void *, int, int, int, int, unsigned *, int,
                                            cudaStream_t);
#endif

#if ISOFFT_GROUP == 3
// The z pass: k_z_convolve on tiles of TX columns, or k_z_convolve_pairs on
// pairs of adjacent tiles (one box of 2 TX columns) where the line leaves no
// room for two exchange buffers.
template <typename T, int L>
static cudaError_t run_z(void *W, const void *tw, const T *G, const T *Gs, T gscale, int Nz, int My, int Kx,
                         int zsh, unsigned *status, unsigned test_extra_tx, cudaStream_t st)
{
    using C = ZCfg<T, L>;
    // the paired form comes in a plain and a z-blocked instance
    constexpr auto kernel0 = []() {
        if constexpr (C::DBX)
            return k_z_convolve<T, L>;
        else
            return k_z_convolve_pairs<T, L, 0>;
    }();
    constexpr auto kernelb = []() {
        if constexpr (C::DBX)
            return k_z_convolve<T, L>;
        else
            return k_z_convolve_pairs<T, L, kZBlockShift>;
    }();
    static std::atomic<uint64_t> done0{0}, doneb{0};
    static std::atomic<int> slots0{0}, slotsb{0};
    if (((uintptr_t)W & 15) || ((uintptr_t)G & 15)) return cudaErrorMisalignedAddress;
    // the z-blocked workspace is read by the paired form only, in boxes of
    // whole blocks
    if (!w_blocks_ok(Nz, zsh) || (zsh && (C::DBX || zsh != kZBlockShift || C::BOXZ % (1 << zsh))))
        return cudaErrorInvalidValue;
    const auto kernel = zsh ? kernelb : kernel0;
    cudaError_t e = ensure_smem(kernel, C::SMEM, zsh ? doneb : done0);
    if (e != cudaSuccess) return e;
    const int ntx = (Kx + C::TX - 1) / C::TX;
    // work units: tiles, or tile pairs
    const int units = (C::DBX ? ntx : (ntx + 1) / 2) * (My / 2);
    int grid = resident_ctas(kernel, C::THREADS, C::SMEM, zsh ? slotsb : slots0);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (grid > units) grid = units;
    // W as 8-byte elements [Nz][My][Kx * EPC]; one box = TX (pairs: 2 TX)
    // columns of one line for BOXZ planes.  z-blocked: [Nz >> zsh][My][2^zsh][Kx * EPC],
    // mapped as {Kx EPC, 2^zsh, My, Nz >> zsh}; one box = BOXZ >> zsh blocks
    EncodeTiledFn encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t cb = sizeof(Cx<T>);
    const cuuint32_t bx = (cuuint32_t)((C::DBX ? C::TX : C::PTX) * C::EPC);
    const cuuint64_t dims3[3] = {(cuuint64_t)Kx * C::EPC, (cuuint64_t)My, (cuuint64_t)Nz};
    const cuuint64_t strides3[2] = {(cuuint64_t)Kx * cb, (cuuint64_t)My * Kx * cb};
    const cuuint32_t box3[3] = {bx, 1u, (cuuint32_t)C::BOXZ};
    const cuuint64_t dims4[4] = {(cuuint64_t)Kx * C::EPC, (cuuint64_t)1 << zsh, (cuuint64_t)My,
                                 (cuuint64_t)(Nz >> zsh)};
    const cuuint64_t strides4[3] = {(cuuint64_t)Kx * cb, ((cuuint64_t)Kx * cb) << zsh,
                                    ((cuuint64_t)My * Kx * cb) << zsh};
    const cuuint32_t box4[4] = {bx, 1u << zsh, 1u, (cuuint32_t)(C::BOXZ >> zsh)};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, zsh ? 4 : 3, W, zsh ? dims4 : dims3, zsh ? strides4 : strides3,
               zsh ? box4 : box3, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    kernel<<<grid, C::THREADS, C::SMEM, st>>>(map, (Cx<T> *)W, (const Cx<T> *)tw, G, Gs, gscale, Nz, My, Kx, units,
                                             status, test_extra_tx);
    count_launch();
    return cudaGetLastError();
}
template <typename R_>
cudaError_t launch_z_convolve(int L, void *W, const void *tw, const R_ *G, const R_ *Gs, R_ gscale,
                                  int Nz, int My, int Kx, int zsh, unsigned *status, unsigned test_extra_tx,
                                  cudaStream_t st)
{
    switch (L) {
#define X_(n) \
    case n: return run_z<R_, n>(W, tw, G, Gs, gscale, Nz, My, Kx, zsh, status, test_extra_tx, st);
        ISOFFT_COL_LENGTHS(X_)
#undef X_
    default: return cudaErrorInvalidValue;
    }
}
template <typename R_>
int z_tile_for(int L)
{
    switch (L) {
#define X_(n) \
    case n: return ZCfg<R_, n>::TX;
        ISOFFT_COL_LENGTHS(X_)
#undef X_
    default: return 0;
    }
}
template cudaError_t launch_z_convolve<Real>(int, void *, const void *, const Real *, const Real *, Real, int,
                                             int, int, int, unsigned *, unsigned, cudaStream_t);
template int z_tile_for<Real>(int);
#endif

}  // namespace isofft
