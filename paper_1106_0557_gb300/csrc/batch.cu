// batch.cu -- many small solves in one launch per pass (ipf_submit_batch).
//
// A batch of independent solves of different mesh shapes runs the five
// passes of Sec. 2.2.2 as five launches, each over a table of work items
// drawn from every grid of the batch: K1 row groups, K2 column tiles, K3
// z tiles, K4 column tiles, K5 row groups.  An item names its grid and its
// line-length class; the CTA branches (uniformly) to that class's pass body
// -- the same device functions the single-solve kernels run, so a batched
// result is bitwise the single solve's.  Where a class's body needs fewer
// threads than the launch has, the CTA runs several of its items side by
// side (sub-groups with their own shared memory).  Each pass waits for the
// previous one by stream order, so a batch costs five launches whatever its
// size, instead of five per grid.  k_batch_all (below) runs all five passes
// in one persistent launch instead.
//
// Classes: FP32 grids whose doubled mesh is at most 256 on every axis
// (row lengths Mx/2 of 16 to 128, column lengths 32 to 256).  Other grids
// of a batch are solved by the per-grid path.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "launch.h"
#include "passes.cuh"

namespace isofft {

// One grid of a batch, as the batched kernels read it.
struct BatchGrid {
    const float *src;
    float *phi;
    Cx<float> *W;
    const Cx<float> *tw_x, *rtw, *tw_y, *tw_z;
    const float *G, *Gs;
    float gscale;
    int Nx, Ny, Nz, Kx, My, Mz;
};

// A work item: grid (16 bits), class (8 bits), and the item's index within
// the grid's items of that pass (one CTA per item).
struct BatchItem {
    uint32_t grid_cls;
    uint32_t idx;
};

// The line-length classes of the batched passes: row lengths (x passes,
// Mx / 2) and column lengths (y and z passes).
constexpr int kBatchRows[] = {16, 24, 32, 48, 64, 96, 128};
constexpr int kBatchCols[] = {32, 48, 64, 96, 128, 192, 256};
constexpr int kBatchClasses = 7;
constexpr int kBatchXThreads = 256;
constexpr int kBatchColThreads = 512;

int batch_row_class(int L)
{
    for (int i = 0; i < kBatchClasses; ++i)
        if (kBatchRows[i] == L) return i;
    return -1;
}
int batch_col_class(int L)
{
    for (int i = 0; i < kBatchClasses; ++i)
        if (kBatchCols[i] == L) return i;
    return -1;
}

// ---------------------------------------------------------------------
// K1 / K5 on a batch: the row groups of RowCfg (256 threads for every
// class here).
// ---------------------------------------------------------------------
template <int L>
struct BRow {
    using C = RowCfg<float, L>;
    static_assert(C::THREADS == kBatchXThreads, "batched row classes run 256 threads");
    static constexpr size_t SMEM = (size_t)C::NL * RowPad<float, L>::LP * sizeof(Cx<float>);
    __host__ __device__ static int64_t items(const BatchGrid &g) { return ((int64_t)g.Ny * g.Nz + C::NL - 1) / C::NL; }
};

template <int L, bool FWD>
__device__ __forceinline__ void batch_row(const BatchGrid &g, uint32_t idx, unsigned char *smem)
{
    using C = RowCfg<float, L>;
    const int t = threadIdx.x % C::NT, l = threadIdx.x / C::NT;
    Cx<float> *line = reinterpret_cast<Cx<float> *>(smem) + l * RowPad<float, L>::LP;
    const int64_t nrows = (int64_t)g.Ny * g.Nz;
    const int64_t row = (int64_t)idx * C::NL + l;
    const bool active = row < nrows;
    if constexpr (FWD)
        x_forward_row<float, L>(g.src, g.W, g.tw_x, g.rtw, g.Nx, g.Ny, g.My, active ? row : 0, active, line, t, 0);
    else
        x_inverse_row<float, L>(g.W, g.phi, g.tw_x, g.rtw, g.Nx, g.Ny, g.My, active ? row : 0, active, line, t, 0);
}

template <bool FWD>
__global__ void __launch_bounds__(kBatchXThreads)
k_batch_x(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    const BatchItem it = items[blockIdx.x];
    const BatchGrid &g = grids[it.grid_cls >> 8];
    switch (it.grid_cls & 255) {
#define X_(i) \
    case i: batch_row<kBatchRows[i], FWD>(g, it.idx, bsm); break;
        X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    default: break;
    }
}

// ---------------------------------------------------------------------
// K2 / K4 on a batch: column tiles of ColCfg (TX columns of one z plane);
// a CTA of 512 threads runs 512 / THREADS tiles side by side.
// ---------------------------------------------------------------------
template <int L>
struct BCol {
    using C = ColCfg<float, L>;
    static constexpr int SUB = kBatchColThreads / C::THREADS;  // tiles per CTA
    static_assert(SUB >= 1 && SUB * C::THREADS == kBatchColThreads, "batched column tiles fill the CTA");
    static constexpr size_t SMEM = (size_t)SUB * C::SMEM;
    __host__ __device__ static int64_t tiles(const BatchGrid &g) { return (int64_t)((g.Kx + C::TX - 1) / C::TX) * g.Nz; }
    __host__ __device__ static int64_t items(const BatchGrid &g) { return (tiles(g) + SUB - 1) / SUB; }
};

template <int L, bool FWD>
__device__ __forceinline__ void batch_col(const BatchGrid &g, uint32_t idx, unsigned char *smem)
{
    using B = BCol<L>;
    using C = typename B::C;
    const int s = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
    const int ntx = (g.Kx + C::TX - 1) / C::TX;
    const int64_t tile = (int64_t)idx * B::SUB + s;
    const bool live = tile < B::tiles(g);
    // a sub-group without a tile runs one with no columns (Kx = 0: nothing
    // is read or written) so that it meets every barrier of the others
    const int z = live ? (int)(tile / ntx) : 0, xt = live ? (int)(tile % ntx) : 0;
    const int Kx = live ? g.Kx : 0;
    Cx<float> *sm = reinterpret_cast<Cx<float> *>(smem + (size_t)s * C::SMEM);
    if constexpr (FWD)
        y_forward_tile<float, L, C::TX>(g.W, g.tw_y, g.Ny, Kx, z, xt * C::TX, sm, lt % C::TX, lt / C::TX);
    else
        y_inverse_tile<float, L, C::TX>(g.W, g.tw_y, g.Ny, Kx, z, xt * C::TX, sm, lt % C::TX, lt / C::TX);
}

// y_forward_tile and y_inverse_tile address W with the grid's Kx as row
// pitch; a tile-less sub-group passes Kx = 0, so that pitch is 0 too and no
// access happens (every access is guarded by kx < Kx).
template <bool FWD>
__global__ void __launch_bounds__(kBatchColThreads)
k_batch_y(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    const BatchItem it = items[blockIdx.x];
    const BatchGrid &g = grids[it.grid_cls >> 8];
    switch (it.grid_cls & 255) {
#define X_(i) \
    case i: batch_col<kBatchCols[i], FWD>(g, it.idx, bsm); break;
        X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    default: break;
    }
}

// ---------------------------------------------------------------------
// K3 on a batch: z tiles of ZCfg (TX columns of the line pair ky, My - ky).
// The kernel is persistent over its items; each item's tiles and spectrum
// blocks are staged into shared memory by cp.async one item ahead (two
// staging sets), so the copies of the next item overlap the transforms of
// this one.  (The single-solve kernel's tensor copies would need one tensor
// map per grid.)
// ---------------------------------------------------------------------
// The batched z pass keeps the 8- and 12-point shapes (three or four stages)
// on every class: its CTAs of 512 threads run several tiles side by side
// within 128 registers a thread, where the single-solve kernel's 16- and
// 24-point shapes (lines of 128 to 256 points) would spill.
template <int L>
struct BZShape : Shape<float, L> {
    static constexpr bool TW_REGS = true;
};
template <int L>
struct BZ {
    using SH = BZShape<L>;
    using C = ZCfg<float, L, SH>;
    static constexpr int SUB = kBatchColThreads / C::THREADS;
    static_assert(SUB >= 1 && SUB * C::THREADS == kBatchColThreads, "batched z tiles fill the CTA");
    static_assert(C::TX % 2 == 0, "16-byte copies of tile rows");
    static constexpr size_t XCH2 = 2 * C::XCH;  // two exchange buffers per tile
    static constexpr size_t STAGE = C::IN_SET + C::G_SET;  // one tile's input and spectrum blocks
    static constexpr size_t SMEM_X = (size_t)SUB * XCH2, SMEM_S = (size_t)SUB * STAGE;
    static_assert(C::XCH % 16 == 0 && C::IN_SET % 16 == 0 && C::G_SET % 16 == 0, "16-byte aligned regions");
    __host__ __device__ static int64_t tiles(const BatchGrid &g) { return (int64_t)((g.Kx + C::TX - 1) / C::TX) * (g.My / 2); }
    __host__ __device__ static int64_t items(const BatchGrid &g) { return (tiles(g) + SUB - 1) / SUB; }
};

// Issue the copies of one item's tiles into staging set `S` (this thread's
// share; every thread then commits one group).  Rows of planes z >= Nz
// arrive as zeros; the batched classes have Kx a multiple of TX, so no
// tile column lies past Kx.
template <int L>
__device__ __forceinline__ void batch_z_stage(const BatchGrid &g, uint32_t idx, unsigned char *S)
{
    using B = BZ<L>;
    using C = typename B::C;
    constexpr int TX = C::TX, Lh = L / 2, CH = TX / 2;  // 16-byte chunks per row
    const int s = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
    const int ntx = g.Kx / TX;
    const int64_t tile = (int64_t)idx * B::SUB + s;
    const bool live = tile < B::tiles(g);
    const int pr = live ? (int)(tile / ntx) : 0, xt = live ? (int)(tile % ntx) : 0;
    const int ky1 = pr == 0 ? g.My / 2 : g.My - pr;
    unsigned char *base = S + (size_t)s * B::STAGE;
    Cx<float> *s_in = reinterpret_cast<Cx<float> *>(base);
    float *s_g = reinterpret_cast<float *>(base + C::IN_SET);
    for (int i = lt; i < 2 * Lh * CH; i += C::THREADS) {
        const int gi = i / (Lh * CH), r = i % (Lh * CH), z = r / CH, q = r % CH;
        const bool ok = live && z < g.Nz;
        const Cx<float> *src = ok ? g.W + ((size_t)z * g.My + (gi == 0 ? pr : ky1)) * g.Kx + xt * TX + 2 * q : g.W;
        // line group 1 one row later (ZCfg::SHIFT: opposite bank halves)
        cp_async<16>(s_in + (size_t)(gi * (Lh + (C::SHIFT ? 1 : 0)) + z) * TX + 2 * q, src, ok);
    }
    const ZSpecLayout lay{TX, ntx, Lh + 1, C::GBLK};
    for (int i = lt; i < 2 * C::GBLK / 4; i += C::THREADS) {
        const int b = i / (C::GBLK / 4), j = i % (C::GBLK / 4);
        const bool ok = live && (b == 0 || pr == 0);
        const float *src = ok ? g.G + lay.block(b == 0 ? pr : g.My / 2, xt) + 4 * j : g.G;
        cp_async<16>(s_g + (size_t)b * C::GBLK + 4 * j, src, ok);
    }
}

// The transforms of one staged item (its SUB tiles side by side).
template <int L>
__device__ __forceinline__ void batch_z_compute(const BatchGrid &g, uint32_t idx, const unsigned char *S,
                                                unsigned char *X)
{
    using B = BZ<L>;
    using C = typename B::C;
    constexpr int TX = C::TX, COLS = C::COLS, Lh = L / 2, E = C::E;
    using Rad = typename B::SH::Rad;
    const int s = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
    const int c = lt % TX, grp = (lt / TX) & 1, t = lt / COLS;
    const int ntx = g.Kx / TX;
    const int64_t tile = (int64_t)idx * B::SUB + s;
    const bool live = tile < B::tiles(g);
    const int pr = live ? (int)(tile / ntx) : 0, xt = live ? (int)(tile % ntx) : 0;
    const int Kx = live ? g.Kx : 0;  // a tile-less sub-group stores nothing
    const unsigned char *base = S + (size_t)s * B::STAGE;
    const Cx<float> *s_in = reinterpret_cast<const Cx<float> *>(base);
    const float *s_g = reinterpret_cast<const float *>(base + C::IN_SET);
    typename ZTwiddles<C::TWR, float, L, E, Rad>::type twr;
    twr.load(g.tw_z, t);
    auto hook = [](int) {};
    ZXch<float, L, E, COLS, C::SWZ, true, decltype(hook)> xch{
        reinterpret_cast<Cx<float> *>(X + (size_t)s * B::XCH2), grp * TX + c, hook};
    const float *sg = s_g + (pr == 0 ? grp : 0) * C::GBLK;
    // every sub-group meets the packed column's barriers (the sub-groups'
    // tiles differ in xt)
    z_tile<float, L, TX, true, typename B::SH>(s_in + grp * (Lh + (C::SHIFT ? 1 : 0)) * TX, sg, pr, xt, g.W, g.Gs, g.gscale, g.Nz,
                               g.My, Kx, 0, c, grp, t,
                               twr, g.tw_z, xch, [] { return true; });
}

template <int... I>
struct BZMax;
template <>
struct BZMax<> {
    static constexpr size_t X = 0, S = 0;
};
template <int I, int... R>
struct BZMax<I, R...> {
    static constexpr size_t X = BZ<kBatchCols[I]>::SMEM_X > BZMax<R...>::X ? BZ<kBatchCols[I]>::SMEM_X : BZMax<R...>::X;
    static constexpr size_t S = BZ<kBatchCols[I]>::SMEM_S > BZMax<R...>::S ? BZ<kBatchCols[I]>::SMEM_S : BZMax<R...>::S;
};
using BZAll = BZMax<0, 1, 2, 3, 4, 5, 6>;
constexpr size_t kBatchZSmem = BZAll::X + 2 * BZAll::S;

__global__ void __launch_bounds__(kBatchColThreads)
k_batch_z(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items, int nitems)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    unsigned char *X = bsm, *S[2] = {bsm + BZAll::X, bsm + BZAll::X + BZAll::S};
    auto stage = [&](int i, unsigned char *dst) {
        const BatchItem it = items[i];
        const BatchGrid &g = grids[it.grid_cls >> 8];
        switch (it.grid_cls & 255) {
#define X_(k) \
    case k: batch_z_stage<kBatchCols[k]>(g, it.idx, dst); break;
            X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
        default: break;
        }
    };
    int i = blockIdx.x, buf = 0;
    if (i < nitems) stage(i, S[0]);
    cp_async_commit();
    for (; i < nitems; i += gridDim.x, buf ^= 1) {
        const int next = i + gridDim.x;
        if (next < nitems) stage(next, S[buf ^ 1]);  // the other set was last read before the loop's barrier
        cp_async_commit();
        cp_async_wait<1>();  // this item's copies (this thread's) have landed
        __syncthreads();     // ... and every thread's
        const BatchItem it = items[i];
        const BatchGrid &g = grids[it.grid_cls >> 8];
        switch (it.grid_cls & 255) {
#define X_(k) \
    case k: batch_z_compute<kBatchCols[k]>(g, it.idx, S[buf], X); break;
            X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
        default: break;
        }
        __syncthreads();  // the set is refilled by the next iteration's prefetch
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------
// The whole batch in one launch (k_batch_all): a persistent kernel walks one
// table holding every grid's items of all five passes.  An item of pass p
// of grid g may start only when every item of pass p - 1 of g has finished:
// per (grid, pass) completion counters, raised by each item's CTA after its
// stores (thread 0: barrier, device-scope fence, atomic add) and awaited by
// thread 0 of a dependent item (acquire load, bounded wait, fence, barrier).
// Items are taken in table order from one atomic queue head, so an item
// only ever waits for items taken before it by running CTAs: no deadlock,
// whatever the number of resident CTAs.  The table is ordered along
// diagonals of (grid, pass): (0,K1), (0,K2), (1,K1), (0,K3), (1,K2), (2,K1),
// ..., so each grid's passes follow each other closely and only about five
// grids' workspaces are live at a time (L2-sized for these grids), while a
// wait for the tail of one pass overlaps other grids' items.
//
// A wait that runs out (2 s) sets bit 0 of the status word and an abort
// flag that every CTA checks, so the launch ends promptly with the error.
// Loads of data written in the launch bypass L1 (L2-only loads, cp.async.cg).
// ---------------------------------------------------------------------
constexpr int kMegaThreads = kBatchColThreads;
// Grids per window of the table order.  Measured on the 64-grid batch:
// 2.53 ms per batch with windows of 1 grid, 2.57-2.67 ms with 4 to 64 (64:
// plain pass order); the waits are not what costs.  What does is occupancy:
// the z body's 128 registers at 512 threads leave one CTA per SM, where the
// x and y bodies run 3-4 CTAs per SM in their own launches (five launches:
// 1.40 ms; per-grid passes on the library's streams: 0.94 ms).
constexpr int kMegaWindow = 1;
constexpr uint32_t kPassShift = 28;  // BatchItem::grid_cls bits 28..30: the pass

// x items cover two row groups (512 threads)
template <int L>
__host__ __device__ int64_t mega_row_items(const BatchGrid &g)
{
    return (BRow<L>::items(g) + 1) / 2;
}

template <int L, bool FWD>
__device__ __forceinline__ void mega_row(const BatchGrid &g, uint32_t idx, unsigned char *smem)
{
    using C = RowCfg<float, L>;
    const int t = threadIdx.x % C::NT, l = threadIdx.x / C::NT;  // l < 2 NL
    Cx<float> *line = reinterpret_cast<Cx<float> *>(smem) + l * RowPad<float, L>::LP;
    const int64_t nrows = (int64_t)g.Ny * g.Nz;
    const int64_t row = (int64_t)idx * 2 * C::NL + l;
    const bool active = row < nrows;
    if constexpr (FWD)
        x_forward_row<float, L>(g.src, g.W, g.tw_x, g.rtw, g.Nx, g.Ny, g.My, active ? row : 0, active, line, t, 0);
    else
        x_inverse_row<float, L, true>(g.W, g.phi, g.tw_x, g.rtw, g.Nx, g.Ny, g.My, active ? row : 0, active, line,
                                      t, 0);
}

template <int L, bool FWD>
__device__ __forceinline__ void mega_col(const BatchGrid &g, uint32_t idx, unsigned char *smem)
{
    using B = BCol<L>;
    using C = typename B::C;
    const int s = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
    const int ntx = (g.Kx + C::TX - 1) / C::TX;
    const int64_t tile = (int64_t)idx * B::SUB + s;
    const bool live = tile < B::tiles(g);
    const int z = live ? (int)(tile / ntx) : 0, xt = live ? (int)(tile % ntx) : 0;
    const int Kx = live ? g.Kx : 0;
    Cx<float> *sm = reinterpret_cast<Cx<float> *>(smem + (size_t)s * C::SMEM);
    if constexpr (FWD)
        y_forward_tile<float, L, C::TX, true>(g.W, g.tw_y, g.Ny, Kx, z, xt * C::TX, sm, lt % C::TX, lt / C::TX);
    else
        y_inverse_tile<float, L, C::TX, false, true>(g.W, g.tw_y, g.Ny, Kx, z, xt * C::TX, sm, lt % C::TX,
                                                     lt / C::TX);
}

template <int L>
__device__ __forceinline__ void mega_z(const BatchGrid &g, uint32_t idx, unsigned char *smem)
{
    unsigned char *X = smem, *S = smem + BZAll::X;
    batch_z_stage<L>(g, idx, S);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    batch_z_compute<L>(g, idx, S, X);
}

constexpr size_t kMegaSmem = BZAll::X + BZAll::S;

// Thread 0: wait until *cnt reaches `need` (acquire), giving up after the
// copy-wait limit or when another CTA has aborted.
__device__ __forceinline__ bool mega_wait(const uint32_t *cnt, uint32_t need, const uint32_t *abort_flag)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(cnt) : "memory");
    if (v >= need) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < (1u << 26); ++i) {
        __nanosleep(64);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(cnt) : "memory");
        if (v >= need) return true;
        if ((i & 31) == 0) {
            uint32_t a;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(a) : "l"(abort_flag) : "memory");
            if (a || global_ns() - t0 > kCopyWaitNs) return false;
        }
    }
    return false;
}

// state: [0] queue head, [1] abort flag, [2 + 5 g + p] items of pass p of
// grid g finished; need[5 g + p]: items of pass p of grid g.
__global__ void __launch_bounds__(kMegaThreads)
k_batch_all(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items, int nitems,
            const uint32_t *__restrict__ need, uint32_t *state, unsigned *status)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_item, s_ok;
    uint32_t *done = state + 2;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&state[0], 1u);
        __syncthreads();
        const int i = s_item;
        if (i >= nitems) break;
        const BatchItem it = items[i];
        const int pass = (int)(it.grid_cls >> kPassShift), grid = (int)((it.grid_cls >> 8) & 0xFFFFFu);
        const int cls = (int)(it.grid_cls & 255u);
        if (threadIdx.x == 0) {
            uint32_t aborted;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(aborted) : "l"(&state[1]) : "memory");
            bool ok = !aborted;
            if (ok && pass > 0) {
                ok = mega_wait(&done[5 * grid + pass - 1], need[5 * grid + pass - 1], &state[1]);
                if (!ok) {  // ran out (or another CTA did): flag it, stop every CTA
                    if (status) atomicOr(status, 1u);
                    atomicExch(&state[1], 1u);
                }
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        const BatchGrid &g = grids[grid];
        switch (pass * 8 + cls) {
#define X_(c)                                                            \
    case 0 * 8 + c: mega_row<kBatchRows[c], true>(g, it.idx, bsm); break;  \
    case 1 * 8 + c: mega_col<kBatchCols[c], true>(g, it.idx, bsm); break;  \
    case 2 * 8 + c: mega_z<kBatchCols[c]>(g, it.idx, bsm); break;          \
    case 3 * 8 + c: mega_col<kBatchCols[c], false>(g, it.idx, bsm); break; \
    case 4 * 8 + c: mega_row<kBatchRows[c], false>(g, it.idx, bsm); break;
            X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
        default: break;
        }
        __syncthreads();  // every store of the item precedes the release
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[5 * grid + pass], 1u);
        }
    }
}

// ---------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------
static int64_t row_items(int cls, const BatchGrid &g)
{
    switch (cls) {
#define X_(i) \
    case i: return BRow<kBatchRows[i]>::items(g);
        X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    default: return 0;
    }
}
static int64_t col_items(int cls, const BatchGrid &g)
{
    switch (cls) {
#define X_(i) \
    case i: return BCol<kBatchCols[i]>::items(g);
        X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    default: return 0;
    }
}
static int64_t z_items(int cls, const BatchGrid &g)
{
    switch (cls) {
#define X_(i) \
    case i: return BZ<kBatchCols[i]>::items(g);
        X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    default: return 0;
    }
}

static size_t row_smem()
{
    size_t m = 0;
#define X_(i) m = std::max(m, BRow<kBatchRows[i]>::SMEM);
    X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    return m;
}
static size_t col_smem()
{
    size_t m = 0;
#define X_(i) m = std::max(m, BCol<kBatchCols[i]>::SMEM);
    X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
    return m;
}
static size_t z_smem_max() { return kBatchZSmem; }
static size_t mega_smem() { return std::max(std::max(2 * row_smem(), col_smem()), kMegaSmem); }
static int64_t mega_items(int pass, const BatchGrid &g)
{
    if (pass == 0 || pass == 4) {
        switch (batch_row_class(g.Kx)) {
#define X_(i) \
    case i: return mega_row_items<kBatchRows[i]>(g);
            X_(0) X_(1) X_(2) X_(3) X_(4) X_(5) X_(6)
#undef X_
        default: return 0;
        }
    }
    if (pass == 2) return z_items(batch_col_class(g.Mz), g);
    return col_items(batch_col_class(g.My), g);
}

// The device tables of one batch: grids, the five passes' items, and for
// the one-launch form its item table, the items per (grid, pass) and its
// counters (zeroed before every launch).
struct BatchTables {
    void *dev = nullptr;
    size_t bytes = 0;
    const BatchGrid *grids = nullptr;
    const BatchItem *items[5] = {};
    int count[5] = {};
    const BatchItem *all = nullptr;
    int nall = 0;
    const uint32_t *need = nullptr;
    uint32_t *state = nullptr;
    size_t state_bytes = 0;
};

namespace {
std::mutex g_batch_mu;
// tables by (device, the batch's grid descriptors), at most kBatchCache of
// them; the least recently used is freed first
constexpr size_t kBatchCache = 64;
struct BatchCacheEntry {
    BatchTables tables;
    uint64_t last_use = 0;
};
std::map<std::pair<int, std::vector<unsigned char>>, BatchCacheEntry> g_batch_tables;
uint64_t g_batch_clock = 0;
std::atomic<uint64_t> g_batch_attr{0};
}  // namespace

bool batch_fits(int dtype_is_f32, const int64_t M[3])
{
    return dtype_is_f32 && batch_row_class((int)(M[0] / 2)) >= 0 && batch_col_class((int)M[1]) >= 0 &&
           batch_col_class((int)M[2]) >= 0;
}

cudaError_t batch_enqueue(const BatchGridDesc *descs, int count, int mode, unsigned *status, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(g_batch_attr.load() & bit)) {
        e = cudaFuncSetAttribute(k_batch_x<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_x<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_y<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_y<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)z_smem_max());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mega_smem());
        if (e != cudaSuccess) return e;
        g_batch_attr.fetch_or(bit);
    }
    std::pair<int, std::vector<unsigned char>> key{dev, {}};
    key.second.resize((size_t)count * sizeof(BatchGridDesc));
    memcpy(key.second.data(), descs, key.second.size());
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch_tables.find(key);
    if (it == g_batch_tables.end()) {
        if (g_batch_tables.size() >= kBatchCache) {
            auto victim = g_batch_tables.begin();
            for (auto v = g_batch_tables.begin(); v != g_batch_tables.end(); ++v)
                if (v->second.last_use < victim->second.last_use) victim = v;
            cudaFree(victim->second.tables.dev);  // waits for the device
            g_batch_tables.erase(victim);
        }
        // build the grids and the items of every pass (items of one class
        // adjacent, longest classes first)
        std::vector<BatchGrid> grids(count);
        std::vector<BatchItem> items[5];
        for (int i = 0; i < count; ++i) {
            const BatchGridDesc &d = descs[i];
            BatchGrid &g = grids[i];
            g = {(const float *)d.src, (float *)d.phi, (Cx<float> *)d.W, (const Cx<float> *)d.tw_x,
                 (const Cx<float> *)d.rtw, (const Cx<float> *)d.tw_y, (const Cx<float> *)d.tw_z,
                 (const float *)d.G, (const float *)d.Gs, (float)d.gscale, d.Nx, d.Ny, d.Nz, d.Mx / 2, d.My, d.Mz};
        }
        for (int pass = 0; pass < 5; ++pass) {
            for (int cls = kBatchClasses - 1; cls >= 0; --cls) {
                for (int i = 0; i < count; ++i) {
                    const BatchGrid &g = grids[i];
                    int gc;
                    int64_t n;
                    if (pass == 0 || pass == 4) {
                        gc = batch_row_class(g.Kx);
                        n = gc == cls ? row_items(cls, g) : 0;
                    } else if (pass == 2) {
                        gc = batch_col_class(g.Mz);
                        n = gc == cls ? z_items(cls, g) : 0;
                    } else {
                        gc = batch_col_class(g.My);
                        n = gc == cls ? col_items(cls, g) : 0;
                    }
                    for (int64_t k = 0; k < n; ++k)
                        items[pass].push_back({(uint32_t)(i << 8) | (uint32_t)cls, (uint32_t)k});
                }
            }
        }
        // the one-launch table: windows of kMegaWindow grids; (window, pass)
        // pairs along the diagonals window + pass = d, later passes (older
        // windows) first on a diagonal
        std::vector<BatchItem> all;
        std::vector<uint32_t> need((size_t)count * 5, 0);
        const int win = kMegaWindow;
        const int nwin = (count + win - 1) / win;
        for (int d = 0; d < nwin + 4; ++d) {
            for (int pass = 4; pass >= 0; --pass) {
                const int w = d - pass;
                if (w < 0 || w >= nwin) continue;
                for (int i = w * win; i < count && i < (w + 1) * win; ++i) {
                    const BatchGrid &g = grids[i];
                    const int cls = pass == 0 || pass == 4 ? batch_row_class(g.Kx)
                                                           : batch_col_class(pass == 2 ? g.Mz : g.My);
                    const int64_t n = mega_items(pass, g);
                    // test hook: one more y-forward item than exist, so the
                    // grid's z items wait for it until the wait runs out
                    need[(size_t)5 * i + pass] = (uint32_t)n + (pass == 1 && descs[i].runout ? 1u : 0u);
                    for (int64_t k = 0; k < n; ++k)
                        all.push_back(
                            {((uint32_t)pass << kPassShift) | ((uint32_t)i << 8) | (uint32_t)cls, (uint32_t)k});
                }
            }
        }
        BatchTables tb;
        tb.bytes = count * sizeof(BatchGrid);
        size_t off[5];
        for (int p = 0; p < 5; ++p) {
            off[p] = tb.bytes;
            tb.bytes += items[p].size() * sizeof(BatchItem);
            tb.count[p] = (int)items[p].size();
        }
        const size_t off_all = tb.bytes;
        tb.bytes += all.size() * sizeof(BatchItem);
        tb.nall = (int)all.size();
        const size_t off_need = tb.bytes;
        tb.bytes += need.size() * sizeof(uint32_t);
        const size_t off_state = (tb.bytes + 15) / 16 * 16;
        tb.state_bytes = (2 + need.size()) * sizeof(uint32_t);
        tb.bytes = off_state + tb.state_bytes;
        std::vector<unsigned char> host(off_state, 0);
        memcpy(host.data(), grids.data(), count * sizeof(BatchGrid));
        for (int p = 0; p < 5; ++p) memcpy(host.data() + off[p], items[p].data(), items[p].size() * sizeof(BatchItem));
        memcpy(host.data() + off_all, all.data(), all.size() * sizeof(BatchItem));
        memcpy(host.data() + off_need, need.data(), need.size() * sizeof(uint32_t));
        e = cudaMalloc(&tb.dev, tb.bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(tb.dev, host.data(), off_state, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(tb.dev);
            return e;
        }
        tb.grids = (const BatchGrid *)tb.dev;
        for (int p = 0; p < 5; ++p) tb.items[p] = (const BatchItem *)((unsigned char *)tb.dev + off[p]);
        tb.all = (const BatchItem *)((unsigned char *)tb.dev + off_all);
        tb.need = (const uint32_t *)((unsigned char *)tb.dev + off_need);
        tb.state = (uint32_t *)((unsigned char *)tb.dev + off_state);
        it = g_batch_tables.emplace(key, BatchCacheEntry{tb, 0}).first;
    }
    it->second.last_use = ++g_batch_clock;
    const BatchTables &tb = it->second.tables;
    if (mode == 2) {
        // one persistent launch: as many CTAs as are resident
        static std::atomic<int> mgrid{0};
        int grid = mgrid.load();
        if (grid == 0) {
            int sms = 0, per = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_all, kMegaThreads, mega_smem());
            if (e != cudaSuccess) return e;
            grid = sms * (per > 0 ? per : 1);
            mgrid.store(grid);
        }
        if (grid > tb.nall) grid = tb.nall;
        e = cudaMemsetAsync(tb.state, 0, tb.state_bytes, st);
        if (e != cudaSuccess) return e;
        if (tb.nall) {
            k_batch_all<<<grid, kMegaThreads, mega_smem(), st>>>(tb.grids, tb.all, tb.nall, tb.need, tb.state,
                                                                  status);
            count_launch();
        }
        return cudaGetLastError();
    }
    if (tb.count[0]) {
        k_batch_x<true><<<tb.count[0], kBatchXThreads, row_smem(), st>>>(tb.grids, tb.items[0]);
        count_launch();
    }
    if (tb.count[1]) {
        k_batch_y<true><<<tb.count[1], kBatchColThreads, col_smem(), st>>>(tb.grids, tb.items[1]);
        count_launch();
    }
    if (tb.count[2]) {
        // persistent: as many CTAs as are resident (one per SM at this size)
        static std::atomic<int> zgrid{0};
        int grid = zgrid.load();
        if (grid == 0) {
            int sms = 0, per = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_z, kBatchColThreads, z_smem_max());
            if (e != cudaSuccess) return e;
            grid = sms * (per > 0 ? per : 1);
            zgrid.store(grid);
        }
        if (grid > tb.count[2]) grid = tb.count[2];
        k_batch_z<<<grid, kBatchColThreads, z_smem_max(), st>>>(tb.grids, tb.items[2], tb.count[2]);
        count_launch();
    }
    if (tb.count[3]) {
        k_batch_y<false><<<tb.count[3], kBatchColThreads, col_smem(), st>>>(tb.grids, tb.items[3]);
        count_launch();
    }
    if (tb.count[4]) {
        k_batch_x<false><<<tb.count[4], kBatchXThreads, row_smem(), st>>>(tb.grids, tb.items[4]);
        count_launch();
    }
    return cudaGetLastError();
}


}  // namespace isofft
