// passes.cuh -- the five passes of one isolated-system solve (Sec. 2.2.2),
// re-expressed for one GPU: no pillars, no transposes, each pass one HBM
// round trip over its data.
//
// Buffers (C order, x fastest):
//   src, phi : real [Nz][Ny][Nx]
//   W        : complex [Nz][My][Kx], Kx = Mx / 2, the plan's workspace (on
//              2304-point z lines in blocks of 16 planes, w_row below).  The
//              z padding is never stored: the z pass reads z < Nz, treats the
//              rest of its line as zero, and writes back only z < Nz.
//   G        : real, the transform of the Eq. 9 table on the even octant (it
//              is real and even in every axis) in the tiled order of
//              ZSpecLayout, [My/2 + 1][kx tiles][Mz/2 + 1][tile width] (each
//              tile block padded to 16 bytes), pre-divided by 2 Mx My Mz (the
//              factor 2 undoes the packed x spectra, which carry 2X); column
//              kx = 0 holds (G0 + GN) / 2,
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
//
// K3 and the streamed form of K2/K4 are persistent and receive their tiles
// through the tensor memory accelerator (tma.cuh); K1, K5 and the tile form
// of K2/K4 load with plain coalesced accesses, many CTAs per SM (K1 and K5
// run a persistent grid on the lengths that keep their twiddles in
// registers).
#pragma once
#include "fft_engine.cuh"
#include "launch.h"
#include "tma.cuh"

namespace isofft {

// Row (z, y) of the workspace W, in complex elements / Kx.  With zsh > 0 the
// planes are grouped in blocks of 2^zsh: [z >> zsh][My][z & (2^zsh - 1)][Kx],
// so that the z lines of one (kx, ky) lie 2^zsh rows apart within a block
// (the z pass reads them in long runs of nearby rows); zsh = 0 is the plain
// [Nz][My][Kx].  Every pass addresses W through this map.
__host__ __device__ __forceinline__ size_t w_row(int64_t z, int64_t y, int64_t My, int zsh)
{
    if (zsh == 0) return (size_t)(z * My + y);  // (a uniform branch: the plain layout's arithmetic)
    return (size_t)((((z >> zsh) * My + y) << zsh) + (z & ((int64_t(1) << zsh) - 1)));
}
// A launch on nz planes of a z-blocked workspace covers whole blocks only
// (the map above leaves the allocation otherwise).
inline bool w_blocks_ok(int64_t nz, int zsh) { return zsh >= 0 && zsh <= 6 && (nz & ((int64_t(1) << zsh) - 1)) == 0; }

// Asynchronous global -> shared copies (cp.async): BYTES = 4, 8 or 16;
// when `valid` is false nothing is read and the slot is zero-filled.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = valid ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gsrc), "n"(BYTES), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory exchange for column passes: lines are the COLS columns of a
// tile, stored [position][column].  A warp's accesses cover 32 / COLS
// positions; when a position row is narrower than a 128-byte bank row,
// several positions share one, and the strided first-stage writes (position
// stride 8, 12, 16 or 24) would land on the same banks.  Rows are therefore
// swizzled by position bits:
//   64-byte rows:        p ^ (bit 3 ^ bit 4 of p)
//   32- and 16-byte rows: p ^ (bits 3-4 of p)
// which makes every exchange pattern of the column shapes conflict-free or
// nearly so (counted per pattern, per half- or quarter-warp).  The z pass
// swizzles only the 32-byte rows of its 2304-point lines, where 42 % of its
// shared wavefronts were conflict replays: on 64-byte rows the per-access
// address arithmetic cost it more (measured at 768 points) than the
// conflicts it removes, and the register-twiddle shapes would spill.
template <typename T, int L, int E, int COLS, bool SWIZZLE = true>
struct ColXch {
    static constexpr int ROW_BYTES = COLS * (int)sizeof(Cx<T>);
    static constexpr int MODE = !SWIZZLE || ROW_BYTES >= 128 ? 0 : (ROW_BYTES == 64 ? 1 : 2);
    Cx<T> *s;
    int c;
    static __device__ __forceinline__ int row(int p)
    {
        if constexpr (MODE == 1)
            return p ^ (((p >> 3) ^ (p >> 4)) & 1);
        else if constexpr (MODE == 2)
            return p ^ ((p >> 3) & 3);
        else
            return p;
    }
    template <int NS, int R>
    __device__ __forceinline__ void exchange(Cx<T> (&v)[E], int t)
    {
        using G = StageGeom<L, E, NS, R>;
#pragma unroll
        for (int q = 0; q < G::B; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) s[row(G::out_pos(t, q, r)) * COLS + c] = v[q + r * G::B];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[row(t + m * G::NT) * COLS + c];
        __syncthreads();
    }
};

// Shared-memory exchange for row passes: one line per row.  A warp's 8-byte
// accesses are served per half-warp (16-byte ones per quarter-warp), which
// is conflict-free when those lanes hit distinct bank pairs (quads).
// * Positions are XOR-swizzled within blocks of 16: p ^ ((p >> 4) & 15), or
//   for 8-byte points of 8- and 12-point shapes from 128 points up
//   p ^ ((p >> 4) & 7) ^ (bit 6 of p moved to bit 3), which also separates
//   the blocked writes of the second stage (positions 64 a + b + 8 r).
// * Rows shorter than 128 points are several to a half-warp, so the row
//   stride is padded (by 2, 4 or 8 points) to spread the rows over the
//   banks.
// The choice per length comes from counting wavefronts of every exchange
// pattern of the row shapes.
template <typename T, int L>
struct RowPad {
    static constexpr bool WIDE = sizeof(Cx<T>) == 16;
    static constexpr int PAD = L <= 24 ? 2 : (L <= 48 ? 4 : (L <= 96 && !WIDE ? 8 : 0));
    static constexpr int LP = ((L + 15) & ~15) + PAD;
    static constexpr bool ALT = !WIDE && L >= 128 && XShape<T, L>::E != 16;
    static __device__ __forceinline__ int at(int p)
    {
        if constexpr (ALT)
            return p ^ ((p >> 4) & 7) ^ (((p >> 6) & 1) << 3);
        else
            return p ^ ((p >> 4) & 15);
    }
};

// A row held by at most one warp needs only a warp barrier between the
// writes and reads of its line.
template <int NT>
__device__ __forceinline__ void row_sync()
{
    if constexpr (NT <= 32 && 32 % NT == 0)
        __syncwarp();
    else
        __syncthreads();
}

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
            for (int r = 0; r < R; ++r) s[RowPad<T, L>::at(G::out_pos(t, q, r))] = v[q + r * G::B];
        row_sync<G::NT>();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[RowPad<T, L>::at(t + m * G::NT)];
        row_sync<G::NT>();
    }
};

template <typename T, int L, typename SH = XShape<T, L>>
struct RowCfg {
    static constexpr int E = SH::E;
    static constexpr int NT = L / E;
    static constexpr int NL = NT >= 256 ? 1 : 256 / NT;  // rows per CTA
    static constexpr int THREADS = NL * NT;
    static constexpr size_t SMEM = (size_t)NL * RowPad<T, L>::LP * sizeof(Cx<T>);
    // Stage twiddles held in registers across the rows of a persistent CTA
    // (K1: TWR_F, K5: TWR_I) where that measured faster than reading the
    // table in every stage: FP32 forward rows of 192 and 384 points, inverse
    // rows of 128, 384, 768 and 1152.  Elsewhere the extra registers cost
    // more occupancy than the table reads do.
    static constexpr bool TWR_F = sizeof(T) == 4 && (L == 192 || L == 384);
    static constexpr bool TWR_I = sizeof(T) == 4 && (L == 128 || L == 384 || L == 768 || L == 1152);
};

// Column tiles of the y passes: up to 128 bytes of complex per row and at
// most 512 threads, so two or three tiles are resident per SM and one tile's
// global loads overlap the others' butterflies; rows of at least 32 bytes
// (one sector) even where that takes more threads (FP32 2304-point lines).
// NARROW: tiles of half that width (at least one column), the third y-pass
// form the plan's timing chooses from (half the threads and shared memory
// per CTA, twice the CTAs).
template <typename T, int L, bool NARROW = false>
struct ColCfg {
    static constexpr int E = YShape<T, L>::E;
    static constexpr int NT = L / E;
    static constexpr int TX0 = 128 / (int)sizeof(Cx<T>);
    static constexpr int TXS = 32 / (int)sizeof(Cx<T>);  // one 32-byte sector
    static constexpr int pow2_floor(int v) { return v >= 2 ? 2 * pow2_floor(v / 2) : 1; }
    static constexpr int TXT = TX0 * NT <= 512 ? TX0 : pow2_floor(512 / NT >= 1 ? 512 / NT : 1);
    static constexpr int TXW = TXT >= TXS || TXS * NT > 1024 ? TXT : TXS;
    static constexpr int TX = NARROW ? (TXW > 1 ? TXW / 2 : 1) : TXW;
    static constexpr int THREADS = TX * NT;
    static constexpr size_t SMEM = (size_t)L * TX * sizeof(Cx<T>);
    // FP32 forward: registers low enough for 3 resident CTAs per SM with 8
    // points per thread, 2 with 12 (the inverse, which holds every point of
    // its lines, and the 16-point shape would spill under such caps)
    static constexpr int MIN_BLOCKS_FWD = sizeof(T) == 4 && THREADS <= 512 ? (E <= 8 ? 3 : (E <= 12 ? 2 : 1)) : 1;
    static_assert(THREADS <= 1024, "column tile too large");
    static_assert(SMEM <= 227 * 1024, "column tile exceeds shared memory");
};

// z pass tiles: TX columns of the two lines ky and My - ky (2 TX lines),
// processed by a persistent CTA.  While it transforms one tile, the tensor
// memory accelerator copies the next tile's non-zero half (z < Mz/2, one box
// per line group and 256 planes) and its Green's spectrum block into shared
// memory (k_z_convolve describes the two staging schemes).  FP64 tiles are
// narrower: FP64 arithmetic, not memory, bounds that path.  The tile width
// is chosen on the layout with one exchange buffer and two input sets:
constexpr size_t z_smem(int tx, int L, int rb)
{
    return (size_t)L * 2 * tx * 2 * rb                                  // exchange buffer
           + 2 * (size_t)2 * (L / 2) * tx * 2 * rb                      // input, two sets
           + 2 * 2 * (size_t)z_spec_block(tx, L / 2 + 1, rb) * rb  // spectrum blocks, two sets
           + 16;                                                      // mbarriers
}
constexpr int z_tile_width(int rb, int nt, int L, int e)
{
    // 16-byte points on 12-point lines of 384 and 768: tiles of 128 threads,
    // three CTAs per SM (measured 23 % faster than one CTA of 256 threads at
    // 255 registers, despite some spills under the 168-register cap)
    if (rb == 8 && e == 12 && nt >= 32 && nt <= 64) return 64 / nt;
    int tx = rb == 4 ? 8 : 4;
    while (tx > 1 && (2 * tx * nt > (e > 8 ? 512 : 1024) || z_smem(tx, L, rb) > 200 * 1024)) tx /= 2;
    return tx;
}

// SH: the line's shape (points per thread, radices, where the twiddles
// live); the batched z pass takes its own (tiles that fit its CTAs).
template <typename T, int L, typename SH = ZShape<T, L>>
struct ZCfg {
    static constexpr int E = SH::E;
    static constexpr int NT = L / E;
    static constexpr int LH = L / 2;
    static constexpr int TX = z_tile_width((int)sizeof(T), NT, L, E);
    static constexpr int COLS = 2 * TX;
    static constexpr int THREADS = COLS * NT;
    // FP32 tiles of 8 columns (64-byte rows): a half-warp reads one position
    // row of both line groups, whose staging regions lie a multiple of 128
    // bytes apart, so both land on the same half of the banks (a 2-way
    // conflict on every input read).  Line group 1 is therefore staged from
    // plane -1 (zeros), one row later, which puts it on the other half.
    static constexpr bool SHIFT = sizeof(T) == 4 && TX * (int)sizeof(Cx<T>) == 64;
    static constexpr int ZROWS = LH + (SHIFT ? 1 : 0);  // rows staged per line group
    // tensor boxes: NZB equal boxes of at most 256 planes per line group
    // (exactly LH planes, or with SHIFT at least LH + 1 in boxes of an even
    // number of rows, so that every box starts 128-byte aligned)
    static constexpr int boxes()
    {
        int n = 1;
        if (SHIFT) {
            while ((ZROWS + n - 1) / n > 256) ++n;
        } else {
            while (LH % n != 0 || LH / n > 256) ++n;
        }
        return n;
    }
    static constexpr int NZB = boxes();
    static constexpr int BOXZ = SHIFT ? ((ZROWS + NZB - 1) / NZB + 1) / 2 * 2 : LH / NZB;
    static constexpr int EPC = (int)sizeof(Cx<T>) / 8;  // 8-byte tensor elements per complex
    static constexpr int GBLK = z_spec_block(TX, LH + 1, (int)sizeof(T));
    static constexpr size_t XCH = (size_t)L * COLS * sizeof(Cx<T>);
    static constexpr size_t IN_GROUP = (size_t)NZB * BOXZ * TX * sizeof(Cx<T>);  // one line group
    static constexpr size_t IN_SET = 2 * IN_GROUP;
    static constexpr size_t G_BLK = (size_t)GBLK * sizeof(T);
    static constexpr size_t G_SET = 2 * G_BLK;  // the blocks of k_y' = pr and of My/2 (pr = 0 only)
    // without register twiddles the CTA keeps the line's twiddle table in
    // shared memory (read by every stage, loaded once per CTA)
    static constexpr bool TWR = SH::TW_REGS;
    static constexpr size_t TWS = TWR ? 0 : (size_t)L * sizeof(Cx<T>);
    static constexpr int MIN_BLOCKS = sizeof(T) == 8 && E == 12 && NT >= 32 && NT <= 64 ? 3 : 1;
    // Two exchange buffers used in turn need one CTA barrier per exchange
    // instead of two; the input is then staged once per tile (the next
    // tile's copies start after the first exchange's barrier, when every
    // thread has read its input).  Taken wherever the extra buffer fits the
    // CTAs per SM (k_z_convolve; every length but 2304) and the tiles are
    // wider than one 16-byte column.  Otherwise one exchange buffer and an
    // input set twice as wide (k_z_convolve_pairs: 2304-point lines, and the
    // 768-point lines of 16-byte points, 6.93 -> 6.62 ms for a df64 384^3
    // solve's z pass).
    static constexpr size_t SMEM_DBX = 2 * XCH + IN_SET + 2 * G_SET + 16 + TWS;
    // 16-byte points on 1-column tiles copy 16-byte rows; two tiles per box
    // (the paired form) make them 32 bytes
    static constexpr bool PAIR_NARROW = sizeof(Cx<T>) == 16 && TX == 1;
    static constexpr bool DBX =
        !PAIR_NARROW && SMEM_DBX <= 227 * 1024 && MIN_BLOCKS * (SMEM_DBX + 1024) <= 228 * 1024;
    static constexpr int NXB = DBX ? 2 : 1;  // exchange buffers
    static constexpr int NIN = DBX ? 1 : 2;  // input sets of one tile's width
    static constexpr size_t OFF_IN = NXB * XCH, OFF_G = OFF_IN + NIN * IN_SET, OFF_BAR = OFF_G + 2 * G_SET,
                            OFF_TW = OFF_BAR + 16;
    static constexpr size_t SMEM = OFF_TW + TWS;
    // without DBX, two adjacent tiles share each box (k_z_convolve_pairs):
    // the input set holds 2 TX columns, the spectrum sets both tiles' blocks
    static constexpr int PTX = 2 * TX;
    static constexpr size_t PIN_GROUP = (size_t)LH * PTX * sizeof(Cx<T>), PIN_SET = 2 * PIN_GROUP;
    static_assert(DBX || (PIN_SET == NIN * IN_SET && PIN_GROUP % 128 == 0 &&
                          ((size_t)BOXZ * PTX * sizeof(Cx<T>)) % 128 == 0),
                  "paired z tiles: layout and 128-byte aligned copy destinations");
    // rows of 32 bytes or less put several positions on one bank row: the
    // lines that keep their twiddles in shared memory swizzle them (the
    // register-twiddle shapes would spill under the extra address registers;
    // wider rows go without, see ColXch)
    static constexpr bool SWZ = !TWR && COLS * sizeof(Cx<T>) <= 32;
    static_assert(DBX || SMEM == z_smem(TX, L, (int)sizeof(T)) + TWS, "z pass shared-memory layout");
    static_assert(MIN_BLOCKS * SMEM <= 227 * 1024, "z pass CTAs per SM exceed shared memory");
    static_assert(THREADS <= 1024, "z tile too large");
    static_assert(SMEM <= 227 * 1024, "z tile exceeds shared memory");
    static_assert((SHIFT ? BOXZ * NZB >= ZROWS : BOXZ * NZB == LH) && BOXZ <= 256,
                  "tensor boxes must cover the half line");
    static_assert(TX * sizeof(Cx<T>) % 16 == 0, "tensor box rows must be multiples of 16 bytes");
    static_assert(XCH % 128 == 0 && IN_GROUP % 128 == 0 && ((size_t)BOXZ * TX * sizeof(Cx<T>)) % 128 == 0,
                  "tensor copy destinations must stay 128-byte aligned");
    static_assert(G_BLK % 16 == 0, "bulk copies move multiples of 16 bytes");
    static_assert(E % 2 == 0, "the z pass splits a thread's points at L/2");
};

// Layout of the Green's spectrum read by the z pass: [ky'][kx tile][kz'][TX]
// with ky' <= My/2, kz' <= Mz/2 and kx = tile * TX + c (padded with zeros
// past Mx/2); the (Mz/2 + 1) x TX block of one tile is contiguous and padded
// to blk elements (a multiple of 16 bytes).
struct ZSpecLayout {
    int tx, ntx, nkz, blk;  // tile width, kx tiles, Mz/2 + 1, block stride
    __host__ __device__ size_t block(int kyp, int xt) const { return ((size_t)kyp * ntx + xt) * blk; }
    __host__ __device__ size_t at(int kyp, int xt, int kzp, int c) const
    {
        return block(kyp, xt) + (size_t)kzp * tx + c;
    }
};

// ---------------------------------------------------------------------
// Pass bodies.  Each works on one row (x passes) or one column tile (y
// passes) and contains CTA-wide barriers, so every thread of the CTA calls it
// the same number of times.  CG selects L2-only global loads (FP32 and FP64
// points), for data that other CTAs of the same launch wrote moments earlier.
// ---------------------------------------------------------------------
template <bool CG, typename T>
__device__ __forceinline__ Cx<T> ld_cx(const Cx<T> *p)
{
    if constexpr (CG) {
        if constexpr (sizeof(T) == 4) {
            const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
            return {v.x, v.y};
        } else {
            const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
            return {v.x, v.y};
        }
    } else {
        return *p;
    }
}

// Lane shuffle of one complex point within segments of `width` lanes.
__device__ __forceinline__ float shfl_real(float v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
__device__ __forceinline__ double shfl_real(double v, int src, int width)
{
    return __shfl_sync(0xffffffffu, v, src, width);
}
__device__ __forceinline__ df64 shfl_real(df64 v, int src, int width)
{
    return {__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width)};
}
template <typename T>
__device__ __forceinline__ Cx<T> shfl_cx(Cx<T> v, int src, int width)
{
    return {shfl_real(v.x, src, width), shfl_real(v.y, src, width)};
}

// For a row held by NT <= 32 lanes at positions k = t + m NT: the point at
// L - k (L = E NT), which lane NT - t holds as its point E - 1 - m (lane 0
// holds its own at (E - m) mod E).  Every lane of the warp must call it.
template <typename T, int E, int NT>
__device__ __forceinline__ Cx<T> mirror_partner(const Cx<T> (&v)[E], int m, int t)
{
    const Cx<T> other = shfl_cx(v[E - 1 - m], (NT - t) & (NT - 1), NT);
    return t == 0 ? v[(E - m) % E] : other;
}

// K1 body: row rr = z * Ny + y of the source, real -> packed half spectrum.
// tw: W_L^k (k < L), rtw: W_{2L}^k (k < L), L = Mx / 2.
template <typename T>
using In = typename IoReal<T>::type;  // real type of the source / potential arrays

// Twiddles of the persistent passes: held in registers across lines, or
// (TWR false) read from the table by each stage.
template <bool TWR, typename T, int L, int E, typename Rad>
struct ZTwiddles {
    using type = typename TwRegsOf<T, L, E, Rad>::type;
};
template <typename T, int L, int E, typename Rad>
struct ZTwiddles<false, T, L, E, Rad> {
    using type = TwRegs<T, L, E, 1>;  // holds nothing
};
template <bool TWR, bool HALF, typename T, int L, int E, typename TW, typename Xch, typename Rad>
__device__ __forceinline__ void z_fft(Cx<T> (&v)[E], int t, const TW &twr, const Cx<T> *__restrict__ tw, Xch &xch,
                                      Rad)
{
    if constexpr (TWR)
        run_stages_reg<T, L, E, HALF>(v, t, twr, xch, Rad{});
    else
        run_stages<T, L, E, HALF>(v, t, tw, xch, Rad{});
}
template <bool TWR, typename T, int L, typename SH = XShape<T, L>>
using RowTwiddles = typename ZTwiddles<TWR, T, L, SH::E, typename SH::Rad>::type;

// K1 body: real row -> packed half spectrum (row shape SH).
template <typename T, int L, bool TWR = false, typename SH = XShape<T, L>>
__device__ __forceinline__ void x_forward_row_at(const In<T> *in, Cx<T> *__restrict__ out,
                                                 const Cx<T> *__restrict__ tw, const Cx<T> *__restrict__ rtw, int Nx,
                                                 bool active, Cx<T> *line, int t,
                                                 const RowTwiddles<TWR, T, L, SH> &twr = {})
{
    constexpr int E = SH::E, NT = L / E;
    using IO = IoReal<T>;

    // pairs (x[2p], x[2p+1]) as one complex point; p >= L/2 is padding
    Cx<T> v[E];
    const bool vec = (Nx & 1) == 0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        v[m] = {(T)0, (T)0};
        if (m < E / 2 && active) {
            const int p = t + m * NT;
            if (vec && 2 * p + 1 < Nx) {
                const Cx<In<T>> pr = reinterpret_cast<const Cx<In<T>> *>(in)[p];
                v[m] = {IO::in(pr.x), IO::in(pr.y)};
            } else {
                if (2 * p < Nx) v[m].x = IO::in(in[2 * p]);
                if (2 * p + 1 < Nx) v[m].y = IO::in(in[2 * p + 1]);
            }
        }
    }
    RowXch<T, L, E> xch{line};
    z_fft<TWR, true, T, L, E>(v, t, twr, tw, xch, typename SH::Rad{});

    // split the half-length transform Z into the real row's spectrum:
    //   2X[k] = (Z[k] + conj Z[L-k]) + W_2L^k (-i)(Z[k] - conj Z[L-k]),
    //   2X[0] = 2(Re Z0 + Im Z0), 2X[L] = 2(Re Z0 - Im Z0).
    // Z[L-k] comes from the mirror lane by a shuffle when the row lies within
    // a warp, else through shared memory.
    constexpr bool SHFL = NT <= 32 && 32 % NT == 0;
    if constexpr (!SHFL) {
#pragma unroll
        for (int m = 0; m < E; ++m) line[RowPad<T, L>::at(t + m * NT)] = v[m];
        row_sync<NT>();
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        const Cx<T> zk = v[m];
        Cx<T> zm;
        if constexpr (SHFL)
            zm = mirror_partner<T, E, NT>(v, m, t);
        else
            zm = line[RowPad<T, L>::at(k == 0 ? 0 : L - k)];
        const Cx<T> zr = cconj(zm);
        const Cx<T> a = cadd(zk, zr);
        const Cx<T> b = cmul_mi(csub(zk, zr));
        Cx<T> p = cadd(a, cmul(b, rtw[k]));
        if (k == 0) p = {(T)2 * (zk.x + zk.y), (T)2 * (zk.x - zk.y)};
        if (active) out[k] = p;
    }
}

template <typename T, int L, bool TWR = false, typename SH = XShape<T, L>>
__device__ __forceinline__ void x_forward_row(const In<T> *__restrict__ src, Cx<T> *__restrict__ W,
                                              const Cx<T> *__restrict__ tw, const Cx<T> *__restrict__ rtw, int Nx,
                                              int Ny, int My, int64_t rr, bool active, Cx<T> *line, int t,
                                              int zsh, const RowTwiddles<TWR, T, L, SH> &twr = {})
{
    const int y = (int)(rr % Ny);
    const int64_t z = rr / Ny;
    x_forward_row_at<T, L, TWR, SH>(src + rr * Nx, W + w_row(z, y, My, zsh) * L, tw, rtw, Nx, active, line, t,
                                    twr);
}

// K5 body: packed half spectrum of row rr -> real row, cropped to x < Nx.
template <typename T, int L, bool CG = false, bool TWR = false>
__device__ __forceinline__ void x_inverse_row_at(const Cx<T> *in, In<T> *__restrict__ out, const Cx<T> *__restrict__ tw,
                                                 const Cx<T> *__restrict__ rtw, int Nx, bool active, Cx<T> *line,
                                                 int t, const RowTwiddles<TWR, T, L> &twr = {})
{
    constexpr int E = XShape<T, L>::E, NT = L / E;
    // (The mirror point X[L-k] goes through shared memory here: a shuffle
    // from the loaded registers, as in K1, measured slower, since every
    // shuffle then waits on the row's global loads.)
    // The row is staged for the mirror reads X[L - k].  For 256-point FP32
    // rows (16 points a thread, 16 lanes a row) it is staged unswizzled: a
    // half-warp's mirror reads then fall in one 16-element group (offsets
    // 1..15) plus thread 0's read at offset 0 of the next group, 16 distinct
    // bank pairs; the exchange swizzle would put thread 0's read on a bank
    // pair another lane uses.  The FFT below swizzles its own exchanges.
    constexpr bool PLAIN = sizeof(T) == 4 && L == 256 && E == 16;
    auto at0 = [](int p) { return PLAIN ? p : RowPad<T, L>::at(p); };
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        line[at0(k)] = active ? ld_cx<CG>(in + k) : Cx<T>{(T)0, (T)0};
    }
    row_sync<NT>();
    // rebuild the half-length spectrum of z[m] = y[2m] + i y[2m+1]:
    //   Z[k] = A + i B,  A = X[k] + conj X[L-k],  B = (X[k] - conj X[L-k]) W_2L^{-k}
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k = t + m * NT;
        const Cx<T> xk = line[at0(k)];
        Cx<T> a, b;
        if (k == 0) {
            a = {xk.x + xk.y, (T)0};
            b = {xk.x - xk.y, (T)0};
        } else {
            const Cx<T> xm = line[at0(L - k)];
            const Cx<T> xr = cconj(xm);
            a = cadd(xk, xr);
            b = cmul(csub(xk, xr), cconj(rtw[k]));
        }
        v[m] = {a.x - b.y, a.y + b.x};
    }
    row_sync<NT>();
    // inverse transform = swap o forward o swap
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cswap(v[m]);
    RowXch<T, L, E> xch{line};
    z_fft<TWR, false, T, L, E>(v, t, twr, tw, xch, typename XShape<T, L>::Rad{});
    const bool vec = (Nx & 1) == 0;
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
        const int p = t + m * NT;
        const Cx<T> o = cswap(v[m]);
        if (!active) continue;
        using IO = IoReal<T>;
        if (vec && 2 * p + 1 < Nx) {
            reinterpret_cast<Cx<In<T>> *>(out)[p] = {IO::out(o.x), IO::out(o.y)};
        } else {
            if (2 * p < Nx) out[2 * p] = IO::out(o.x);
            if (2 * p + 1 < Nx) out[2 * p + 1] = IO::out(o.y);
        }
    }
}

template <typename T, int L, bool CG = false, bool TWR = false>
__device__ __forceinline__ void x_inverse_row(const Cx<T> *__restrict__ W, In<T> *__restrict__ phi,
                                              const Cx<T> *__restrict__ tw, const Cx<T> *__restrict__ rtw, int Nx,
                                              int Ny, int My, int64_t rr, bool active, Cx<T> *line, int t,
                                              int zsh, const RowTwiddles<TWR, T, L> &twr = {})
{
    const int y = (int)(rr % Ny);
    const int64_t z = rr / Ny;
    x_inverse_row_at<T, L, CG, TWR>(W + w_row(z, y, My, zsh) * L, phi + rr * Nx, tw, rtw, Nx, active, line, t,
                                    twr);
}

// K2 body: y forward of columns kx0 .. kx0 + TX - 1 of plane z.  Rows
// y >= Ny are zero padding and are not read.
// BLK: the workspace is z-blocked (w_row with shift zsh); otherwise plain
// and zsh is ignored.
template <typename T, int L, int TX, bool CG = false, bool BLK = false>
__device__ __forceinline__ void y_forward_tile(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx,
                                               int z, int kx0, Cx<T> *smem, int c, int t,
                                               const Cx<T> *staged = nullptr, int zsh = 0)
{
    constexpr int E = YShape<T, L>::E, NT = L / E;
    const int kx = kx0 + c;
    const bool active = kx < Kx;
    Cx<T> *base = W + (BLK ? w_row(z, 0, L, zsh) : (size_t)z * L) * Kx + (active ? kx : 0);
    const int ys = BLK ? Kx << zsh : Kx;  // row stride
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int y = t + m * NT;
        const bool ok = m < E / 2 && active && y < Ny;
        if (staged)
            v[m] = ok ? staged[y * TX + c] : Cx<T>{(T)0, (T)0};
        else
            v[m] = ok ? ld_cx<CG>(base + (size_t)y * ys) : Cx<T>{(T)0, (T)0};
    }
    ColXch<T, L, E, TX> xch{smem, c};
    run_stages<T, L, E, true>(v, t, tw, xch, typename YShape<T, L>::Rad{});
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[(size_t)(t + m * NT) * ys] = v[m];
    }
}

// K4 body: y inverse of a column tile of plane z, keeping rows y < Ny.
template <typename T, int L, int TX, bool BLK = false, bool CG = false>
__device__ __forceinline__ void y_inverse_tile(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx,
                                               int z, int kx0, Cx<T> *smem, int c, int t,
                                               const Cx<T> *staged = nullptr, int zsh = 0)
{
    constexpr int E = YShape<T, L>::E, NT = L / E;
    const int kx = kx0 + c;
    const bool active = kx < Kx;
    Cx<T> *base = W + (BLK ? w_row(z, 0, L, zsh) : (size_t)z * L) * Kx + (active ? kx : 0);
    const int ys = BLK ? Kx << zsh : Kx;  // row stride
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int y = t + m * NT;
        if (staged)
            v[m] = active ? cswap(staged[y * TX + c]) : Cx<T>{(T)0, (T)0};
        else
            v[m] = active ? cswap(ld_cx<CG>(base + (size_t)y * ys)) : Cx<T>{(T)0, (T)0};
    }
    ColXch<T, L, E, TX> xch{smem, c};
    run_stages<T, L, E, false>(v, t, tw, xch, typename YShape<T, L>::Rad{});
    if (active) {
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
            const int y = t + m * NT;
            if (y < Ny) base[(size_t)y * ys] = cswap(v[m]);
        }
    }
}

// ---------------------------------------------------------------------
// K1 / K5: x passes, RowCfg::NL rows per CTA and round.  With register
// twiddles the grid is persistent (as many CTAs as are resident) and each
// CTA walks groups of NL rows, loading its threads' twiddles once; otherwise
// every CTA takes one group.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(RowCfg<T, L, XShapeF<T, L>>::THREADS)
k_x_forward(const In<T> *__restrict__ src, Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw,
            const Cx<T> *__restrict__ rtw, int Nx, int Ny, int My, int64_t nrows, int zsh)
{
    using SH = XShapeF<T, L>;
    using C = RowCfg<T, L, SH>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x % C::NT, l = threadIdx.x / C::NT;
    Cx<T> *line = reinterpret_cast<Cx<T> *>(smem_raw) + l * RowPad<T, L>::LP;
    if constexpr (C::TWR_F) {
        RowTwiddles<true, T, L, SH> twr;
        twr.load(tw, t);
        for (int64_t r0 = (int64_t)blockIdx.x * C::NL; r0 < nrows; r0 += (int64_t)gridDim.x * C::NL) {
            const int64_t row = r0 + l;  // row = z * Ny + y
            const bool active = row < nrows;
            x_forward_row<T, L, true, SH>(src, W, tw, rtw, Nx, Ny, My, active ? row : 0, active, line, t, zsh, twr);
            // rows wider than a warp read their mirror points from `line`
            // last: the next row's first exchange must wait for those reads
            if constexpr (!(C::NT <= 32 && 32 % C::NT == 0)) {
                if (r0 + (int64_t)gridDim.x * C::NL < nrows) __syncthreads();
            }
        }
    } else {
        const int64_t row = (int64_t)blockIdx.x * C::NL + l;
        const bool active = row < nrows;
        x_forward_row<T, L, false, SH>(src, W, tw, rtw, Nx, Ny, My, active ? row : 0, active, line, t, zsh);
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(RowCfg<T, L>::THREADS)
k_x_inverse(const Cx<T> *__restrict__ W, In<T> *__restrict__ phi, const Cx<T> *__restrict__ tw,
            const Cx<T> *__restrict__ rtw, int Nx, int Ny, int My, int64_t nrows, int zsh)
{
    using C = RowCfg<T, L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x % C::NT, l = threadIdx.x / C::NT;
    Cx<T> *line = reinterpret_cast<Cx<T> *>(smem_raw) + l * RowPad<T, L>::LP;
    if constexpr (C::TWR_I) {
        RowTwiddles<true, T, L> twr;
        twr.load(tw, t);
        for (int64_t r0 = (int64_t)blockIdx.x * C::NL; r0 < nrows; r0 += (int64_t)gridDim.x * C::NL) {
            const int64_t row = r0 + l;
            const bool active = row < nrows;
            x_inverse_row<T, L, false, true>(W, phi, tw, rtw, Nx, Ny, My, active ? row : 0, active, line, t, zsh,
                                             twr);
        }
    } else {
        const int64_t row = (int64_t)blockIdx.x * C::NL + l;
        const bool active = row < nrows;
        x_inverse_row<T, L>(W, phi, tw, rtw, Nx, Ny, My, active ? row : 0, active, line, t, zsh);
    }
}

// ---------------------------------------------------------------------
// K2 / K4, tile form: one CTA per column tile; grid (ceil(Kx / TX), Nz).
// Each CTA loads its columns with plain coalesced loads, so many CTAs per SM
// keep the loads in flight; best where the persistent form (below) would
// hold fewer warps per SM (small lines, 16-byte points).
// ---------------------------------------------------------------------
template <typename T, int L, bool NARROW = false, bool BLK = false>
__global__ void __launch_bounds__(ColCfg<T, L, NARROW>::THREADS, ColCfg<T, L, NARROW>::MIN_BLOCKS_FWD)
k_y_forward(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx, int zsh)
{
    using C = ColCfg<T, L, NARROW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    y_forward_tile<T, L, C::TX, false, BLK>(W, tw, Ny, Kx, blockIdx.y, blockIdx.x * C::TX,
                                            reinterpret_cast<Cx<T> *>(smem_raw), threadIdx.x % C::TX,
                                            threadIdx.x / C::TX, nullptr, zsh);
}

template <typename T, int L, bool NARROW = false, bool BLK = false>
__global__ void __launch_bounds__(ColCfg<T, L, NARROW>::THREADS)
k_y_inverse(Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw, int Ny, int Kx, int zsh)
{
    using C = ColCfg<T, L, NARROW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    y_inverse_tile<T, L, C::TX, BLK>(W, tw, Ny, Kx, blockIdx.y, blockIdx.x * C::TX,
                                     reinterpret_cast<Cx<T> *>(smem_raw), threadIdx.x % C::TX, threadIdx.x / C::TX,
                                     nullptr, zsh);
}

// z-pass exchanger.  With DB (two buffers, used in turn) an exchange needs a
// single CTA barrier: a buffer is next written two exchanges later, after
// the barrier of the exchange in between, which follows every read of its
// previous use.  `hook(k)` runs after the (first) barrier of the tile's
// exchange k, when every thread has finished what preceded that exchange;
// `free_buf()` is a buffer that no thread still reads.  PREWAIT: thread 0
// first waits, before that barrier, until its tensor stores have read their
// shared-memory source (an output staging area the threads write again
// after the barrier).
template <typename T, int L, int E, int COLS, bool SWZ, bool DB, typename Hook, bool PREWAIT = false>
struct ZXch {
    using Rows = ColXch<T, L, E, COLS, SWZ>;
    Cx<T> *a;  // DB: the second buffer follows at a + L COLS
    int c;
    Hook &hook;
    int k = 0;  // exchanges done in this tile
    __device__ __forceinline__ Cx<T> *buf(int i) const { return DB && (i & 1) ? a + (size_t)L * COLS : a; }
    __device__ __forceinline__ Cx<T> *free_buf() const { return buf(k); }
    template <int NS, int R>
    __device__ __forceinline__ void exchange(Cx<T> (&v)[E], int t)
    {
        using G = StageGeom<L, E, NS, R>;
        Cx<T> *s = buf(k);
#pragma unroll
        for (int q = 0; q < G::B; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) s[Rows::row(G::out_pos(t, q, r)) * COLS + c] = v[q + r * G::B];
        if constexpr (PREWAIT) {
            if (threadIdx.x == 0) bulk_wait_read_all();
        }
        __syncthreads();
        hook(k);
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = s[Rows::row(t + m * G::NT) * COLS + c];
        if constexpr (!DB) __syncthreads();
        ++k;
    }
};


// ---------------------------------------------------------------------
// K2 / K4, streamed form: persistent over column tiles (z, kx tile).  Thread 0
// issues the next tile's rows by tensor-map boxes (8-byte elements; K2:
// dims {Kx EPC, Ny, Nz}, so rows y >= Ny arrive as zeros; K4: {Kx EPC, My,
// Nz}) into the other of two staging sets while the CTA transforms the
// current tile; completion and bounded waits as in the z pass.  Twiddles
// stay in registers across tiles (lines up to 1024 points), and the
// exchanges alternate between two buffers where both fit (ZXch).  K2 on the
// plain workspace with one exchange per transform stages its output tile in
// the second exchange buffer, which that exchange leaves unused, and thread
// 0 writes it by tensor stores (tmO: dims {Kx EPC, My, Nz}) after the next
// tile's first barrier, when every thread has staged its points: the
// threads issue shared-memory stores instead of global ones (K2 writes
// twice what it reads).
// ---------------------------------------------------------------------
template <typename T, int L>
struct YCfg {
    static constexpr int E = YShape<T, L>::E;
    static constexpr int NT = L / E;
    static constexpr int CB = (int)sizeof(Cx<T>);
    static constexpr size_t smem_i(int tx) { return (size_t)3 * L * tx * CB + 16; }
    // the column tile's width, halved while its exchange buffer and two
    // input sets exceed shared memory (which keeps the 2304-point lines at
    // 32-byte rows: 221 KB)
    static constexpr int width()
    {
        int tx = ColCfg<T, L>::TX;
        while (tx > 1 && smem_i(tx) > 226 * 1024) tx /= 2;
        return tx;
    }
    static constexpr int TX = width();
    static constexpr int THREADS = TX * NT;
    static constexpr int EPC = CB / 8;
    static constexpr int boxes(int rows)
    {
        int n = 1;
        while (rows % n != 0 || rows / n > 256) ++n;
        return n;
    }
    static constexpr int NB_F = boxes(L / 2), BOX_F = L / 2 / NB_F;  // K2 reads y < L/2
    static constexpr int NB_I = boxes(L), BOX_I = L / NB_I;          // K4 reads every row
    static constexpr size_t XCH = (size_t)L * TX * CB;
    static constexpr size_t IN_F = (size_t)(L / 2) * TX * CB, IN_I = (size_t)L * TX * CB;
    static constexpr int MIN_BLOCKS = THREADS <= 512 && smem_i(TX) <= 110 * 1024 ? 2 : 1;
    // a second exchange buffer (one CTA barrier per exchange, see ZXch)
    // where it still fits the resident CTAs
    static constexpr bool fits(size_t bytes) { return bytes <= 227 * 1024 && MIN_BLOCKS * (bytes + 1024) <= 228 * 1024; }
    static constexpr bool DBX_F = fits(2 * XCH + 2 * IN_F + 16), DBX_I = fits(2 * XCH + 2 * IN_I + 16);
    static constexpr size_t SMEM_F = (DBX_F ? 2 : 1) * XCH + 2 * IN_F + 16,
                            SMEM_I = (DBX_I ? 2 : 1) * XCH + 2 * IN_I + 16;
    // twiddles in registers across tiles, except for the long lines, whose
    // per-thread share (29 points for 2304) would spill
    static constexpr bool TW_REGS = L <= 1024;
    static_assert(smem_i(TX) == XCH + 2 * IN_I + 16 && SMEM_I <= 227 * 1024 && SMEM_F <= 227 * 1024,
                  "y pass shared memory");
    static_assert(TX * CB % 16 == 0, "tensor box rows must be multiples of 16 bytes");
    static_assert(XCH % 128 == 0 && IN_F % 128 == 0 && ((size_t)BOX_F * TX * CB) % 128 == 0 &&
                      ((size_t)BOX_I * TX * CB) % 128 == 0,
                  "tensor copy destinations must stay 128-byte aligned");
};

template <typename T, int L, bool FWD, bool BLK = false>
__global__ void __launch_bounds__(YCfg<T, L>::THREADS, YCfg<T, L>::MIN_BLOCKS)
k_y_pass(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmO, Cx<T> *__restrict__ W,
         const Cx<T> *__restrict__ tw, int Ny, int Kx, int ntiles, unsigned *__restrict__ status, int zsh)
{
    using C = YCfg<T, L>;
    using Rad = typename YShape<T, L>::Rad;
    constexpr int E = C::E, NT = C::NT, TX = C::TX;
    constexpr int NB = FWD ? C::NB_F : C::NB_I, BOX = FWD ? C::BOX_F : C::BOX_I;
    constexpr size_t IN = FWD ? C::IN_F : C::IN_I;
    constexpr bool DBX = FWD ? C::DBX_F : C::DBX_I;
    constexpr bool TSTORE = FWD && !BLK && DBX && RadixCount<Rad>::value == 2;
    extern __shared__ __align__(128) unsigned char ysmem[];
    Cx<T> *xs = reinterpret_cast<Cx<T> *>(ysmem);            // exchange buffer(s)
    unsigned char *s_in = ysmem + (DBX ? 2 : 1) * C::XCH;  // [set][row][TX]
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_in + 2 * IN);
    const int tid = threadIdx.x;
    const int c = tid % TX, t = tid / TX;
    const int ntx = (Kx + TX - 1) / TX;
    if (smem_addr(ysmem) & 127u) {
        if (tid == 0 && status) atomicOr(status, 2u);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int tile, int set) {  // thread 0
        const int z = tile / ntx, xt = tile - z * ntx;
        mbar_arrive_expect_tx(&bar[set], (uint32_t)IN);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            void *dst = s_in + set * IN + (size_t)b * BOX * TX * sizeof(Cx<T>);
            if constexpr (!BLK)
                tma_load_3d(dst, &tmW, xt * TX * C::EPC, b * BOX, z, &bar[set]);
            else  // tmW dims {Kx EPC, 2^zsh, rows, Nz >> zsh}
                tma_load_4d(dst, &tmW, xt * TX * C::EPC, z & ((1 << zsh) - 1), b * BOX, z >> zsh, &bar[set]);
        }
    };
    auto no_hook = [](int) {};
    typename ZTwiddles<C::TW_REGS, T, L, E, Rad>::type twr;
    twr.load(tw, t);
    Cx<T> *so = xs + (size_t)L * TX;  // TSTORE: output staging [row][TX], 128-byte aligned
    int prev = -1;                     // TSTORE: the tile whose staged output awaits its stores
    auto store_prev = [&]() {          // thread 0
        const int z = prev / ntx, xt = prev - z * ntx;
#pragma unroll
        for (int b = 0; b < C::NB_I; ++b)
            tma_store_3d(&tmO, so + (size_t)b * C::BOX_I * TX, xt * TX * C::EPC, b * C::BOX_I, z);
        bulk_commit();
    };
    int tile = blockIdx.x, it = 0;
    bool ok = true;
    if (tid == 0 && tile < ntiles) issue(tile, 0);
    for (; tile < ntiles; tile += gridDim.x, ++it) {
        const int next = tile + gridDim.x;
        const int set = it & 1;
        if (tid == 0 && next < ntiles) issue(next, set ^ 1);
        const bool landed = mbar_wait_bounded(&bar[set], (uint32_t)(it >> 1) & 1u, kCopyWaitNs);
        if (!__syncthreads_and(landed)) {
            ok = false;
            break;
        }
        if constexpr (TSTORE) {
            if (tid == 0 && prev >= 0) store_prev();
        }
        const int z = tile / ntx, xt = tile - z * ntx;
        const int kx = xt * TX + c;
        const Cx<T> *sin = reinterpret_cast<const Cx<T> *>(s_in + set * IN) + t * TX + c;
        ZXch<T, L, E, TX, true, DBX, decltype(no_hook), TSTORE> xch{xs, c, no_hook};
        Cx<T> v[E];
        if constexpr (FWD) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = m < E / 2 ? sin[m * NT * TX] : Cx<T>{(T)0, (T)0};
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = cswap(sin[m * NT * TX]);
        }
        z_fft<C::TW_REGS, FWD, T, L, E>(v, t, twr, tw, xch, Rad{});
        if constexpr (TSTORE) {
            // the exchange's barrier followed thread 0's wait for the previous
            // tile's stores to read this area
#pragma unroll
            for (int m = 0; m < E; ++m) so[(size_t)(t + m * NT) * TX + c] = v[m];
            fence_async_smem();
            prev = tile;
        } else if (kx < Kx) {
            Cx<T> *base = W + (BLK ? w_row(z, 0, L, zsh) : (size_t)z * L) * Kx + kx;
            const int ys = BLK ? Kx << zsh : Kx;  // row stride
            if constexpr (FWD) {
#pragma unroll
                for (int m = 0; m < E; ++m) base[(size_t)(t + m * NT) * ys] = v[m];
            } else {
#pragma unroll
                for (int m = 0; m < E / 2; ++m) {
                    const int y = t + m * NT;
                    if (y < Ny) base[(size_t)y * ys] = cswap(v[m]);
                }
            }
        }
    }
    if constexpr (TSTORE) {
        __syncthreads();  // every thread has staged the last tile (the exit is uniform)
        if (tid == 0) {
            if (prev >= 0) store_prev();
            bulk_wait_all();  // the stores have read the staging area before the CTA ends
        }
    }
    if (!ok && tid == 0) {
        // a wait gave up: flag it and let the copies in flight land (bounded)
        if (status) atomicOr(status, 1u);
        mbar_wait_bounded(&bar[it & 1], (uint32_t)(it >> 1) & 1u, kCopyWaitNs);
        if (tile + (int)gridDim.x < ntiles)
            mbar_wait_bounded(&bar[(it + 1) & 1], (uint32_t)((it + 1) >> 1) & 1u, kCopyWaitNs);
    }
}

// One tile of the z pass on staged data: the forward transforms of the
// thread's line, the multiply by the Green's spectrum, the inverse
// transforms and the store of z < Nz.  `sin`: the thread's line group as
// staged, [z < L/2][IS] (IS = TX, or 2 TX where a box holds two tiles),
// offset to the tile's first column; `sg`: the spectrum block of the
// thread's line, [kz'][TX].  `before_g` runs before the spectrum is read and
// returns false (the same on every thread) to abandon the tile.
template <typename T, int L, int IS, bool SYNC_ALL = false, typename SH = ZShape<T, L>, typename TWR, typename Xch,
          typename BeforeG>
__device__ __forceinline__ bool z_tile(const Cx<T> *sin, const T *sg, int pr, int xt, Cx<T> *__restrict__ W,
                                       const T *__restrict__ Gs, T gscale, int Nz, int My, int Kx, int zsh, int c,
                                       int g, int t, const TWR &twr, const Cx<T> *twz, Xch &xch, BeforeG before_g)
{
    using C = ZCfg<T, L, SH>;
    using Rad = typename SH::Rad;
    constexpr int E = C::E, NT = C::NT, TX = C::TX, COLS = C::COLS, Lh = L / 2;
    const int col = g * TX + c;
    const int ky = g == 0 ? pr : (pr == 0 ? My / 2 : My - pr);
    const int kx = xt * TX + c;
    const bool active = kx < Kx;
    const int kyp = ky <= My - ky ? ky : My - ky;

    // z < Lh from the staged boxes (zeros past Nz), the upper half is zero
    sin += t * IS + c;
    Cx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = m < E / 2 ? sin[m * NT * IS] : Cx<T>{(T)0, (T)0};

    z_fft<C::TWR, true, T, L, E>(v, t, twr, twz, xch, Rad{});
    if (!before_g()) return false;

    // spectrum at kz = t + m NT: kz' = kz below Lh, L - kz from Lh on
    const T *g_lo = sg + t * TX + c;
    const T *g_hi = sg + (L - t) * TX + c;
    auto gval = [&](int m) -> T { return m < E / 2 ? g_lo[m * NT * TX] : g_hi[-m * NT * TX]; };
    const bool packed = xt == 0 && c == 0;  // the kx = 0 / Mx/2 column
    // SYNC_ALL: every thread of the CTA meets these barriers, whatever its
    // tile (CTAs that run several tiles side by side)
    if (SYNC_ALL || xt == 0) {
        // the packed column needs the partner bin (-ky, -kz)
        Cx<T> *sp = xch.free_buf();
        if (packed) {
#pragma unroll
            for (int m = 0; m < E; ++m) sp[(t + m * NT) * COLS + col] = v[m];
        }
        __syncthreads();
        if (packed) {
            const int gp = pr == 0 ? g : 1 - g;
            const T *gsrow = Gs + (size_t)kyp * (Lh + 1);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kz = t + m * NT;
                const int kzp = kz <= L - kz ? kz : L - kz;
                const Cx<T> partner = cconj(sp[(kz == 0 ? 0 : L - kz) * COLS + gp * TX]);
                const T gp_ = gval(m) * gscale;
                const T gm_ = gsrow[kzp] * gscale;
                v[m] = {v[m].x * gp_ + partner.x * gm_, v[m].y * gp_ + partner.y * gm_};
            }
        }
        __syncthreads();
    }
    if (!packed) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cscale(v[m], gval(m) * gscale);
    }

#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = cswap(v[m]);
    z_fft<C::TWR, false, T, L, E>(v, t, twr, twz, xch, Rad{});
    if (active && zsh == 0) {
        Cx<T> *base = W + (size_t)ky * Kx + kx;
        const size_t zstride = (size_t)My * Kx;
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
            const int z = t + m * NT;
            if (z < Nz) base[(size_t)z * zstride] = cswap(v[m]);
        }
    } else if (active) {
        Cx<T> *base = W + ((size_t)ky << zsh) * Kx + kx;
#pragma unroll
        for (int m = 0; m < E / 2; ++m) {
            const int z = t + m * NT;
            // w_row(z, ky) - w_row(0, ky): (z >> zsh) blocks, row z & (2^zsh - 1)
            const size_t zr = (((size_t)(z >> zsh) * My) << zsh) + (z & ((1 << zsh) - 1));
            if (z < Nz) base[zr * Kx] = cswap(v[m]);
        }
    }
    return true;
}

// ---------------------------------------------------------------------
// K3: z forward, multiply by the Green's spectrum, z inverse.
// Tiles: (pair p, kx tile xt), tile = p * ntx + xt; pair p holds the lines
// (ky, My - ky) = (p, My - p) for p > 0 and (0, My/2) for p = 0.  A
// persistent grid walks the tiles; each CTA keeps the next tile's copies in
// flight during the current tile's transforms.
// gscale multiplies the cached spectrum (the cache stores it for widths
// divided by min(h); G scales as h^2).
//
// Copies: thread 0 issues, per tile, one tensor-map box per line group and
// 256 planes of W (tmW: 8-byte elements, dims {Kx EPC, My, Nz}; planes
// z >= Nz and columns kx >= Kx read as zero) and a bulk copy of the tile's
// spectrum block (a second one for the pair p = 0, whose line My/2 has its
// own k_y').  The input has one staging set, the spectrum two (the tile's
// parity); both complete on one mbarrier, once per tile.  The next tile's
// copies are issued after the barrier of the tile's first exchange, which
// every thread reaches after reading its input; the other spectrum set was
// last read by the previous tile, before the barriers of its transforms.
// ---------------------------------------------------------------------
template <typename T, int L>
__global__ void __launch_bounds__(ZCfg<T, L>::THREADS, ZCfg<T, L>::MIN_BLOCKS)
k_z_convolve(const __grid_constant__ CUtensorMap tmW, Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw,
             const T *__restrict__ G, const T *__restrict__ Gs, T gscale, int Nz, int My, int Kx, int ntiles,
             unsigned *__restrict__ status, unsigned test_extra_tx)
{
    using C = ZCfg<T, L>;
    static_assert(C::DBX, "the paired lines take k_z_convolve_pairs");
    constexpr int E = C::E, TX = C::TX, COLS = C::COLS;
    constexpr int Lh = L / 2;
    extern __shared__ __align__(128) unsigned char zsmem[];
    Cx<T> *sm = reinterpret_cast<Cx<T> *>(zsmem);             // two exchange buffers
    unsigned char *s_in = zsmem + C::OFF_IN;                   // [g][z < Lh][TX]
    T *s_g = reinterpret_cast<T *>(zsmem + C::OFF_G);          // [set][2][GBLK]
    uint64_t *bar = reinterpret_cast<uint64_t *>(zsmem + C::OFF_BAR);
    // thread -> (column c, group g, position t): a warp holds both groups of
    // a few positions, so each position row of the exchange buffer is written
    // whole and the warp's shared-memory accesses are conflict-free
    const int tid = threadIdx.x;
    const int c = tid % TX;
    const int g = (tid / TX) & 1;
    const int t = tid / COLS;
    const int col = g * TX + c;
    const int ntx = (Kx + TX - 1) / TX;
    const ZSpecLayout lay{TX, ntx, Lh + 1, C::GBLK};

    // tensor copies need 128-byte aligned destinations (uniform per CTA)
    if (smem_addr(zsmem) & 127u) {
        if (tid == 0 && status) atomicOr(status, 2u);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init_fence();
    }
    const Cx<T> *twz = tw;  // the twiddle table the stages read
    if constexpr (!C::TWR) {
        Cx<T> *s_tw = reinterpret_cast<Cx<T> *>(zsmem + C::OFF_TW);
        for (int i = tid; i < L; i += C::THREADS) s_tw[i] = tw[i];
        twz = s_tw;
    }
    __syncthreads();

    // copies of a tile into the input set and spectrum set `set`, issued by
    // thread 0
    auto issue = [&](int tile, int set, uint32_t extra) {
        const int pr = tile / ntx, xt = tile - pr * ntx;
        const int ky1 = pr == 0 ? My / 2 : My - pr;
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(C::IN_SET + (pr == 0 ? 2 : 1) * C::G_BLK) + extra);
#pragma unroll
        for (int zb = 0; zb < C::NZB; ++zb) {
            const size_t off = (size_t)zb * C::BOXZ * TX * sizeof(Cx<T>);
            tma_load_3d(s_in + off, &tmW, xt * TX * C::EPC, pr, zb * C::BOXZ, &bar[0]);
            tma_load_3d(s_in + C::IN_GROUP + off, &tmW, xt * TX * C::EPC, ky1, zb * C::BOXZ - (C::SHIFT ? 1 : 0),
                        &bar[0]);
        }
        T *gdst = s_g + (size_t)set * 2 * C::GBLK;
        bulk_load(gdst, G + lay.block(pr, xt), (uint32_t)C::G_BLK, &bar[0]);
        if (pr == 0) bulk_load(gdst + C::GBLK, G + lay.block(My / 2, xt), (uint32_t)C::G_BLK, &bar[0]);
    };

    using Rad = typename ZShape<T, L>::Rad;
    typename ZTwiddles<C::TWR, T, L, E, Rad>::type twr;  // this thread's twiddles, for every tile (when TW_REGS)
    twr.load(tw, t);
    int tile = blockIdx.x, it = 0;
    bool ok = true;
    // test_extra_tx is a test hook: bytes the first tile's barrier expects
    // beyond what its copies deliver, so that its wait runs out (normally 0)
    if (tid == 0 && tile < ntiles) issue(tile, 0, test_extra_tx);
    for (; tile < ntiles; tile += gridDim.x, ++it) {
        const int next = tile + gridDim.x;
        const int set = it & 1;
        auto hook = [&](int k) {
            if (k == 0 && tid == 0 && next < ntiles) issue(next, set ^ 1, 0u);
        };
        ZXch<T, L, E, COLS, C::SWZ, true, decltype(hook)> xch{sm, col, hook};
        if (!__syncthreads_and(mbar_wait_bounded(&bar[0], (uint32_t)it & 1u, kCopyWaitNs))) {
            ok = false;
            break;
        }
        const int pr = tile / ntx, xt = tile - pr * ntx;
        // line group 1 staged one row later with SHIFT (its row 0 is plane -1)
        const Cx<T> *sin = reinterpret_cast<const Cx<T> *>(s_in + g * C::IN_GROUP) + (C::SHIFT && g ? TX : 0);
        const T *sg = s_g + ((size_t)set * 2 + (pr == 0 ? g : 0)) * C::GBLK;
        z_tile<T, L, TX>(sin, sg, pr, xt, W, Gs, gscale, Nz, My, Kx, 0, c, g, t, twr, twz, xch, [] { return true; });
    }
    if (!ok && tid == 0) {
        // a wait gave up: flag it, then let this tile's copies land (bounded
        // again) before the CTA's shared memory is freed
        if (status) atomicOr(status, 1u);
        mbar_wait_bounded(&bar[0], (uint32_t)it & 1u, kCopyWaitNs);
    }
}

// K3 for lines whose tile leaves no room for a second exchange buffer (2304
// points).  Their tiles are only 16 bytes wide per row, so the CTA takes
// two adjacent tiles at a time: one box of 2 TX columns (32-byte rows) per
// line group and 256 planes, and one bulk copy of both tiles' spectrum
// blocks (adjacent in the cache layout), then computes the tiles in turn on
// one exchange buffer.  Input and spectrum have one staging set each, on
// their own mbarrier (one phase per pair).  The next pair's input is issued
// after the barrier of the second tile's first exchange, its spectrum after
// the barrier of the second tile's first inverse exchange: by then every
// thread has read the current pair's input, and its spectrum, respectively.
// When ntx is odd the last pair of a line pair has one tile.
template <typename T, int L, int ZSH = 0>
__global__ void __launch_bounds__(ZCfg<T, L>::THREADS, ZCfg<T, L>::MIN_BLOCKS)
k_z_convolve_pairs(const __grid_constant__ CUtensorMap tmW, Cx<T> *__restrict__ W, const Cx<T> *__restrict__ tw,
                   const T *__restrict__ G, const T *__restrict__ Gs, T gscale, int Nz, int My, int Kx,
                   int npairs, unsigned *__restrict__ status, unsigned test_extra_tx)
{
    using C = ZCfg<T, L>;
    constexpr int zsh = ZSH;  // workspace z blocks of 2^ZSH planes (w_row)
    static_assert(!C::DBX, "lines with room for two exchange buffers take k_z_convolve");
    constexpr int E = C::E, TX = C::TX, COLS = C::COLS, PTX = C::PTX;
    constexpr int Lh = L / 2;
    using Rad = typename ZShape<T, L>::Rad;
    constexpr int NXF = RadixCount<Rad>::value - 1;  // exchanges of one transform
    extern __shared__ __align__(128) unsigned char zsmem[];
    Cx<T> *sm = reinterpret_cast<Cx<T> *>(zsmem);                 // exchange buffer
    unsigned char *s_in = zsmem + C::OFF_IN;                       // [g][z < Lh][2 TX]
    T *s_g = reinterpret_cast<T *>(zsmem + C::OFF_G);              // [line group j][tile s][GBLK]
    uint64_t *bar = reinterpret_cast<uint64_t *>(zsmem + C::OFF_BAR);  // input, spectrum
    const int tid = threadIdx.x;
    const int c = tid % TX;
    const int g = (tid / TX) & 1;
    const int t = tid / COLS;
    const int col = g * TX + c;
    const int ntx = (Kx + TX - 1) / TX;
    const int npx = (ntx + 1) / 2;  // tile pairs per line pair
    const ZSpecLayout lay{TX, ntx, Lh + 1, C::GBLK};

    if (smem_addr(zsmem) & 127u) {
        if (tid == 0 && status) atomicOr(status, 2u);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    const Cx<T> *twz = tw;
    if constexpr (!C::TWR) {
        Cx<T> *s_tw = reinterpret_cast<Cx<T> *>(zsmem + C::OFF_TW);
        for (int i = tid; i < L; i += C::THREADS) s_tw[i] = tw[i];
        twz = s_tw;
    }
    __syncthreads();

    // thread 0 issues; n_in / n_g count the phases issued on each barrier
    int n_in = 0, n_g = 0;
    auto issue_in = [&](int pair, uint32_t extra) {
        const int pr = pair / npx, xt0 = 2 * (pair - pr * npx);
        const int ky1 = pr == 0 ? My / 2 : My - pr;
        mbar_arrive_expect_tx(&bar[0], (uint32_t)C::PIN_SET + extra);
#pragma unroll
        for (int zb = 0; zb < C::NZB; ++zb) {
            const size_t off = (size_t)zb * C::BOXZ * PTX * sizeof(Cx<T>);
            if constexpr (zsh == 0) {
                tma_load_3d(s_in + off, &tmW, xt0 * TX * C::EPC, pr, zb * C::BOXZ, &bar[0]);
                tma_load_3d(s_in + C::PIN_GROUP + off, &tmW, xt0 * TX * C::EPC, ky1, zb * C::BOXZ, &bar[0]);
            } else {  // tmW dims {Kx EPC, 2^zsh, My, Nz >> zsh}, box {2 TX EPC, 2^zsh, 1, BOXZ >> zsh}
                tma_load_4d(s_in + off, &tmW, xt0 * TX * C::EPC, 0, pr, (zb * C::BOXZ) >> zsh, &bar[0]);
                tma_load_4d(s_in + C::PIN_GROUP + off, &tmW, xt0 * TX * C::EPC, 0, ky1, (zb * C::BOXZ) >> zsh,
                            &bar[0]);
            }
        }
        ++n_in;
    };
    auto issue_g = [&](int pair) {
        const int pr = pair / npx, xt0 = 2 * (pair - pr * npx);
        const uint32_t bytes = (uint32_t)((ntx - xt0 < 2 ? 1 : 2) * C::G_BLK);
        mbar_arrive_expect_tx(&bar[1], (pr == 0 ? 2u : 1u) * bytes);
        bulk_load(s_g, G + lay.block(pr, xt0), bytes, &bar[1]);
        if (pr == 0) bulk_load(s_g + 2 * C::GBLK, G + lay.block(My / 2, xt0), bytes, &bar[1]);
        ++n_g;
    };

    typename ZTwiddles<C::TWR, T, L, E, Rad>::type twr;
    twr.load(tw, t);
    int pair = blockIdx.x, it = 0;
    bool ok = true, in_done = false;
    if (tid == 0 && pair < npairs) {
        issue_in(pair, test_extra_tx);
        issue_g(pair);
    }
    for (; pair < npairs; pair += gridDim.x, ++it) {
        const int next = pair + gridDim.x;
        in_done = false;
        if (!__syncthreads_and(mbar_wait_bounded(&bar[0], (uint32_t)it & 1u, kCopyWaitNs))) {
            ok = false;
            break;
        }
        in_done = true;
        const int pr = pair / npx, xt0 = 2 * (pair - pr * npx);
        const int nsub = ntx - xt0 < 2 ? 1 : 2;
        for (int s = 0; s < nsub; ++s) {
            const bool last = s == nsub - 1;
            auto hook = [&](int k) {
                if (!last || tid != 0 || next >= npairs) return;
                if (k == 0) issue_in(next, 0u);
                if (k == NXF) issue_g(next);
            };
            ZXch<T, L, E, COLS, C::SWZ, false, decltype(hook)> xch{sm, col, hook};
            auto spectrum_landed = [&]() -> bool {
                return s != 0 || __syncthreads_and(mbar_wait_bounded(&bar[1], (uint32_t)it & 1u, kCopyWaitNs));
            };
            const Cx<T> *sin = reinterpret_cast<const Cx<T> *>(s_in + g * C::PIN_GROUP) + s * TX;
            const T *sg = s_g + ((size_t)(pr == 0 ? g : 0) * 2 + s) * C::GBLK;
            if (!z_tile<T, L, PTX>(sin, sg, pr, xt0 + s, W, Gs, gscale, Nz, My, Kx, zsh, c, g, t, twr, twz, xch,
                                   spectrum_landed)) {
                ok = false;
                break;
            }
        }
        if (!ok) break;
    }
    if (!ok && tid == 0) {
        // a wait gave up: flag it, then let the copies still in flight land
        // (bounded again): at most one phase per barrier is outstanding
        if (status) atomicOr(status, 1u);
        if (n_in > it + (in_done ? 1 : 0)) mbar_wait_bounded(&bar[0], (uint32_t)(n_in - 1) & 1u, kCopyWaitNs);
        if (n_g > it) mbar_wait_bounded(&bar[1], (uint32_t)(n_g - 1) & 1u, kCopyWaitNs);
    }
}

}  // namespace isofft
