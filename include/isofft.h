/*
 * isofft.h -- C ABI of the GB300 isolated-system Poisson solver.
 *
 * The library solves Poisson's equation  lap(Phi) = S  on a regular mesh of
 * N = (Nx, Ny, Nz) cells with widths h = (hx, hy, hz) and the boundary
 * condition Phi -> 0 at infinity (paper Sec. 2.1, Eq. 1), by Hockney's mesh
 * doubling: the source is zero-padded to a doubled mesh M >= 2N per axis, a
 * real-to-complex 3-D DFT is taken, the result is multiplied by the transform
 * of the doubled-mesh Green's function of Eq. 9 (built from Eq. 6), and the
 * inverse DFT is cropped back to the N active cells (Sec. 2.2.2).
 * The result is the discrete aperiodic convolution
 *     Phi[i,j,k] = sum_{i',j',k'} G(i-i', j-j', k-k') S[i',j',k']
 * with G(d) = -hx hy hz / (4 pi |(hx dx, hy dy, hz dz)|) for d != 0 and
 * G(0) = -hx hy hz / (4 pi min(h)); Phi <= 0 where S >= 0 (Eq. 2 sign).
 * For gravity with Newton's constant 1 pass S = 4 pi rho.
 *
 * Conventions shared by every entry point:
 *   - Arrays are C order [z][y][x], x contiguous (the paper's first Fortran
 *     index is x, Sec. 3.2), of `float` for IPF_F32 plans and `double` for
 *     IPF_F64 and IPF_DF64 plans.  Device buffers must be 16-byte aligned.
 *   - Device pointers are CUDA device (or managed) memory of the calling
 *     thread's current device; host pointers are ordinary host memory
 *     (pinned memory makes the copies faster but is not required).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued asynchronously on it unless stated otherwise.
 *   - Every call returns an int status (ipf_status below); nothing throws
 *     across the ABI.  ipf_status_string() names a status.
 *   - A plan is used by one stream at a time (it owns one workspace).
 *   - Plans may be created and destroyed from several host threads at once:
 *     the spectrum cache and the y-pass timing table are locked, and a
 *     spectrum that one thread is building is waited for, not built twice.
 *   - The caller owns its buffers.  A plan owns its workspace; the library
 *     owns the cache of Green's spectra, shared by plans of equal doubled
 *     mesh, width ratios and dtype.
 */
#ifndef ISOFFT_H
#define ISOFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipf_plan_s *ipf_plan_t;

/* Arithmetic type of a plan's butterflies (and of its buffers).
 *   IPF_F32   float buffers, FP32 arithmetic.
 *   IPF_F64   double buffers, FP64 arithmetic.
 *   IPF_DF64  double buffers, FP64-class arithmetic on the FP32 units: each
 *             value is a pair of floats (hi + lo, about 48 significant bits),
 *             added with Knuth's two-sum and multiplied with a fused
 *             multiply-add error term.  Not in the paper; it is a precision
 *             variant of the same path for GPUs whose FP64 rate is a small
 *             fraction of their FP32 rate.  The Green's spectrum is built in
 *             FP64 and split into float pairs. */
typedef enum { IPF_F32 = 0, IPF_F64 = 1, IPF_DF64 = 2 } ipf_dtype;

typedef enum {
    IPF_OK = 0,
    IPF_INVALID_ARG = 1,      /* null pointer, bad size/width/dtype/flag */
    IPF_UNSUPPORTED_SIZE = 2, /* a doubled mesh beyond the largest kernel */
    IPF_OUT_OF_MEMORY = 3,    /* a device or host allocation failed */
    IPF_CUDA_ERROR = 4,       /* a CUDA runtime call failed; see ipf_last_cuda_error */
    IPF_TIMEOUT = 5,          /* a bounded device wait gave up */
    IPF_BUDGET_EXCEEDED = 6,  /* the request does not fit the memory budget */
    IPF_NOT_READY = 7         /* asynchronous work has not finished */
} ipf_status;

/* Verbosity levels, in decreasing order of output (paper Sec. 3.2:
 * CONSOLE_INFO_2 > CONSOLE_INFO_1 > CONSOLE_WARNING > CONSOLE_ERROR, the
 * last being the default).  Messages go to stderr. */
enum { IPF_CONSOLE_ERROR = 0, IPF_CONSOLE_WARNING = 1, IPF_CONSOLE_INFO_1 = 2, IPF_CONSOLE_INFO_2 = 3 };

/* Plan flags. */
enum {
    IPF_FLAG_PASS_EVENTS = 1u << 0, /* record CUDA events around each pass so
                                       ipf_plan_pass_times can report them */
    IPF_FLAG_Y_TILES = 1u << 1,     /* run the y passes in their tile form  */
    IPF_FLAG_Y_STREAM = 1u << 2,    /* run the y passes in their streamed form
                                       (no y-form flag: the plan times the
                                       three forms and keeps the fastest, see
                                       ipf_plan_variants) */
    IPF_FLAG_TEST_WAIT_RUNOUT = 1u << 3, /* test hook: the z pass's first tile
                                       on each CTA expects 16 bytes more than
                                       its copies deliver, so its bounded wait
                                       runs out (about 4 s) and the solve
                                       reports IPF_TIMEOUT through
                                       ipf_plan_check; its potential is then
                                       unspecified.  In a batch run in one
                                       launch (ISOFFT_BATCH_FUSED=2) the
                                       wait of the plan's z items for its y
                                       pass runs out instead (2 s), and the
                                       batch's first plan reports it */
    IPF_FLAG_TEST_CANARY = 1u << 4, /* test hook: before every solve the
                                       plan's workspace is filled with NaN
                                       bytes, so a pass that read an element
                                       no earlier pass of that solve wrote
                                       would show in the potential */
    IPF_FLAG_Y_TILES_NARROW = 1u << 5 /* run the y passes in their tile form
                                       on tiles of half the width (at most one
                                       of the three y-form flags) */
};
/* Two more test hooks are read from the environment:
 *   ISOFFT_TEST_FAIL_ALLOC=workspace|tables|spectrum|staging  the device
 *       allocation of that buffer fails as if the device were out of memory
 *       (ipf_plan_create, or the first host-buffer solve for staging, then
 *       returns IPF_OUT_OF_MEMORY and frees what it had allocated);
 *   ISOFFT_NVTX=1  (read at plan creation) the plan's solves push one NVTX
 *       range per pass around its launches ("isofft K1 x forward", ...), so
 *       a profiler can select the kernels of one pass. */

/* Create a solver for an Nx x Ny x Nz mesh of widths h (paper Sec. 3.2,
 * `Create(PoissonSolver, CellWidth, nTotalCells, ...)`).
 *   out        receives the plan handle (NULL on failure).
 *   n          {Nx, Ny, Nz}, each >= 1 and at most 1152: the doubled mesh
 *              (2N rounded up to one of 32, 48, 64, 96, 128, 192, 256, 384,
 *              512, 768, 1024, 1536, 2304) must fit the largest supported
 *              length, else IPF_UNSUPPORTED_SIZE.  1152^3 cells in FP32 need
 *              about 37 GB of device memory: a 24.5 GB workspace and a 6 GB
 *              spectrum, plus 24.5 GB of FP64 scratch while the spectrum is
 *              built.
 *   h          {hx, hy, hz}, each finite and > 0.
 *   dtype      IPF_F32, IPF_F64 or IPF_DF64.  The Green's spectrum is always
 *              built in FP64 and rounded to the plan's dtype.
 *   flags      a bitwise OR of IPF_FLAG_*.
 *   verbosity  an IPF_CONSOLE_* level; the environment variable
 *              ISOFFT_VERBOSITY (0-3), if set, overrides it.
 *   stream     stream used for the one-off set-up work (Green's spectrum
 *              build, table uploads); the call synchronises on it before
 *              returning.
 * Allocates the plan's workspace (complex Nz x My x Mx/2) on the current
 * device and, on a cache miss, the Green's spectrum. */
int ipf_plan_create(ipf_plan_t *out, const int64_t n[3], const double h[3], int dtype,
                    uint32_t flags, int verbosity, void *stream);

/* Release a plan, its workspace and its reference to the cached spectrum
 * (paper Sec. 3.2, `Destroy(PoissonSolver)`).  Waits for nothing: the caller must not destroy a plan with work still in
 * flight.  NULL is accepted and ignored. */
int ipf_plan_destroy(ipf_plan_t plan);

/* The doubled mesh M = {Mx, My, Mz} the plan transforms on (>= 2N, a
 * supported length; any M >= 2N - 1 gives the same cropped result). */
int ipf_plan_padded_shape(const ipf_plan_t plan, int64_t m[3]);

/* Device bytes the plan owns (its workspace), and the bytes of the cached
 * Green's spectrum it references, for admission against a memory budget.
 * Not in the paper (which has one solver per process and no admission); the
 * spectrum is the transform the paper computes once and keeps (Sec. 2.2.2). */
int ipf_plan_workspace_bytes(const ipf_plan_t plan, size_t *bytes);
int ipf_plan_spectrum_bytes(const ipf_plan_t plan, size_t *bytes);

/* Device bytes a plan of this shape and dtype would need (workspace plus the
 * spectrum if it is not cached yet), without creating it.  Not in the
 * paper: an admission aid for serving. */
int ipf_estimate_bytes(const int64_t n[3], const double h[3], int dtype, size_t *bytes);

/* One solve (paper Sec. 3.2, `Solve(PoissonSolver, SourceSolution)`):
 * d_src and d_phi are device arrays of Nz*Ny*Nx elements of the plan's
 * dtype; d_phi may equal d_src (the paper overwrites the source with the
 * potential).  Enqueues the five passes on `stream` and returns without
 * waiting. */
int ipf_solve(ipf_plan_t plan, const void *d_src, void *d_phi, void *stream);

/* One solve from and to HOST memory: ipf_solve_host_async followed by
 * ipf_plan_host_wait.  Returns what ipf_plan_check would return for the
 * solve (IPF_TIMEOUT if a device wait of a pass gave up). */
int ipf_solve_host(ipf_plan_t plan, const void *h_src, void *h_phi, void *stream);

/* Enqueue one solve from and to host memory and return without waiting.
 *   h_src, h_phi  host arrays of Nz*Ny*Nx elements of the plan's dtype (FP64
 *                 for IPF_DF64); pinned memory lets the copies run
 *                 asynchronously.  h_src is read, and h_phi written, after the
 *                 call returns: keep both valid, h_src unchanged and h_phi
 *                 unread until ipf_plan_host_wait.
 *   stream        the passes run on it, after the work already enqueued there;
 *                 the copies run on two streams of the plan.
 * The source is copied whole into one of three device staging buffers of the
 * plan (allocated on the first host solve), the passes start when it lands,
 * and the potential is copied back when they finish.  Consecutive host
 * solves on a plan take the buffers in turn, so one solve's copies overlap
 * the passes of the solves before and after it.  The copy of h_src does not
 * wait for earlier work on `stream`. */
int ipf_solve_host_async(ipf_plan_t plan, const void *h_src, void *h_phi, void *stream);

/* Wait until every host solve enqueued on the plan has written its potential
 * back; returns what ipf_plan_check returns for them. */
int ipf_plan_host_wait(ipf_plan_t plan);

/* Device-side status of the solves made on this plan since the previous
 * check.  The z pass (forward z transform x spectrum x inverse) receives its
 * tiles through the tensor memory accelerator and waits for each tile's
 * copies on a shared-memory barrier; every such wait is bounded (2 s).  When
 * one gives up, the pass lets its outstanding copies land (bounded again),
 * stops early and sets a flag in a device word of the plan; the potential
 * of that solve is then unspecified.  This call synchronises `stream`, reads
 * and clears that word: IPF_OK, IPF_TIMEOUT (a wait gave up) or
 * IPF_CUDA_ERROR (a pass refused to run because its shared memory was not
 * aligned as the tensor copies require). */
int ipf_plan_check(ipf_plan_t plan, void *stream);

/* One solve that allocates no memory, for callers that cannot call
 * cudaMalloc: a code that has given all device memory to its own pool, a
 * solve issued while a stream is being captured into a CUDA graph, or a
 * time-step loop that must not take the device-wide synchronisation an
 * allocation or free may imply.  The paper has no counterpart; it is a
 * deployment variant of ipf_solve.
 *   n, h, dtype  as for ipf_plan_create (no plan is needed; IPF_F32 or
 *                IPF_F64 only).
 *   d_src, d_phi device arrays as for ipf_solve (d_phi may equal d_src).
 * Twiddle tables, the Green's spectrum and the workspace are all carved out
 * of one static device array of 64 MiB that the library holds on every
 * device it is loaded on until the process exits; the spectrum is rebuilt on
 * every call.  A mesh whose tables, spectrum and workspace exceed 64 MiB is
 * rejected with IPF_BUDGET_EXCEEDED before any device work (FP32 fits up to
 * about 128^3 cells, FP64 up to about 96^3).  The array's first word is a
 * status word: it starts at zero (static initialisation), the passes' bounded
 * waits set bits in it, and only ipf_noalloc_check reads and clears it, so a
 * flag raised by one call stays set for later calls until that check runs.
 * Every other byte the solve uses is written before it is read on every
 * call.  Calls whose work overlaps on the GPU -- on different streams, or
 * from different threads -- race on the array and must be serialised by the
 * caller.  The first call on each device looks up
 * the array's device address and sets kernel attributes; make that first
 * call before any stream capture.  Asynchronous on `stream`. */
int ipf_solve_noalloc(const int64_t n[3], const double h[3], int dtype, const void *d_src, void *d_phi,
                      void *stream);

/* ipf_plan_check for the solves of ipf_solve_noalloc on the current device
 * (their status word lives in the same static array). */
int ipf_noalloc_check(void *stream);

/* Submit `count` independent solves, possibly of different shapes and
 * dtypes; plans[i] solves d_src[i] into d_phi[i].  Not in the paper, which
 * runs one solve at a time per communicator; each solve is the Sec. 2.2.2
 * sequence of ipf_solve.  With the environment variable ISOFFT_BATCH_FUSED=1
 * the FP32 solves whose doubled mesh is at most 256 on every axis run
 * together in one launch per pass (five launches for all of them, over a
 * table of their work items, built and uploaded synchronously the first
 * time a given set of plans and buffers is submitted -- do that before any
 * capture; the library keeps the tables of the last 64 such sets); with
 * ISOFFT_BATCH_FUSED=2 they run in one persistent launch for all five
 * passes, an item waiting (bounded, 2 s) until its grid's previous pass is
 * complete; a wait that runs out sets the status word of the first such
 * plan (ipf_plan_check reports IPF_TIMEOUT).  A plan may appear only
 * once per batch (each owns one workspace).  The solves are spread over up to
 * 8 internal streams of the library that fork from and join back into
 * `stream`: the batch starts after the work already enqueued on `stream`, and
 * work enqueued on `stream` afterwards starts after the whole batch.  The
 * first batch of two or more solves on a device creates those streams; make
 * it before capturing `stream` into a CUDA graph (a capture then records the
 * batch as parallel branches).  Results are bitwise those of ipf_solve,
 * except that the five- and one-launch forms (ISOFFT_BATCH_FUSED=1 or 2) run
 * z lines of 128 to 256 points in another radix order than ipf_solve: there
 * the two agree to FP32 rounding.  Asynchronous. */
int ipf_submit_batch(const ipf_plan_t *plans, int count, const void *const *d_src,
                     void *const *d_phi, void *stream);

/* With IPF_FLAG_PASS_EVENTS: mean device milliseconds of each of the five
 * passes (x forward, y forward, z forward x spectrum x z inverse, y inverse,
 * x inverse) over the solves made on this plan since the previous call, then
 * a reset.  Events are recorded on the solving stream between the passes;
 * the call waits for them.  IPF_NOT_READY if no solve was made since the
 * previous call; IPF_INVALID_ARG without the flag. */
int ipf_plan_pass_times(ipf_plan_t plan, float ms[5]);

/* The form each y pass of the plan runs in, v[0] for the forward and v[1]
 * for the inverse pass: 0 tiles (one CTA per column tile, plain loads), 1
 * streamed (persistent CTAs fed by tensor-map copies), 2 tiles of half the
 * width (twice the CTAs, half the threads and shared memory each).  All give
 * bitwise the same potential.  Unless a flag forces one, ipf_plan_create
 * times the three forms on the plan's own workspace (a few launches of each)
 * and keeps the fastest per pass; the choice is remembered per (dtype, mesh,
 * shape, device) for the process, and in the file named by the environment
 * variable ISOFFT_TUNE_FILE if set (read at the first plan, rewritten as
 * choices are made).  ISOFFT_TUNE=0 skips the timing and takes the built-in
 * rule (streamed for FP32 lines of 512 to 1024 points, tiles elsewhere).
 * Not in the paper: the tuning of this implementation's tile shapes. */
int ipf_plan_variants(const ipf_plan_t plan, int v[2]);

/* Bytes held by the library's cache of Green's spectra, and a trim of
 * unreferenced entries.  The paper computes the transform of the Green's
 * function once at initialisation and keeps it for every later solve
 * (Sec. 2.2.2); the cache keeps one such transform per doubled mesh, width
 * ratios and dtype, shared by the plans that need it.  Trim frees
 * unreferenced entries (least recently used first) until the cache holds
 * at most `budget` bytes.  With the environment variable ISOFFT_SPECTRUM_DIR
 * naming a directory, every spectrum the cache builds is also written there
 * (one file per mesh, width ratios and dtype, with a checksum and a digest
 * of the library code that builds and lays out the spectrum), and a plan
 * whose spectrum is not in memory reads a matching file instead of
 * rebuilding it: the restart of a job skips the spectrum build, the
 * solver's only state.  Files that do not match (another mesh, corrupted,
 * or written by a library whose spectrum code differs) are ignored and
 * rebuilt. */
int ipf_greens_cache_bytes(size_t *bytes);
int ipf_greens_cache_trim(size_t budget);

/* Number of kernel launches made by this process so far (all entry points),
 * for checking that the GPU path ran. */
int ipf_launch_count(uint64_t *count);

/* The last CUDA error code seen by the library on this thread (0 if none). */
int ipf_last_cuda_error(void);

/* Static description of a status code; never NULL.  Not in the paper (its
 * Fortran interface reports errors through the console). */
const char *ipf_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* ISOFFT_H */
