// api.cu -- the C ABI of include/isofft.h: plans, the Green's-spectrum
// cache, and the enqueueing of the five passes of a solve.
//
// Create / Solve / Destroy follow the paper's usage (Sec. 3.2).  The
// transform of the Green's function is computed once per (doubled mesh,
// width ratios, dtype) and kept on the device (Sec. 2.2.2, "computed only
// once ... stored permanently"); plans of equal doubled mesh and ratios share
// it, scaled by min(h)^2 (the Green's function of Eq. 6 scales as h^2).
#include <math.h>
#include <stdarg.h>
#include <unistd.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <condition_variable>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/isofft.h"
#include "launch.h"

namespace isofft {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local int g_last_cuda = 0;

static int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return IPF_OK;
    g_last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // allocation failures are not sticky; clear them
        return IPF_OUT_OF_MEMORY;
    }
    return IPF_CUDA_ERROR;
}

// Device allocation of a plan's buffers.  The test hook
// ISOFFT_TEST_FAIL_ALLOC names one kind ("workspace", "tables", "spectrum",
// "staging") whose allocation then fails as if the device were out of memory.
static cudaError_t dev_alloc(void **ptr, size_t bytes, const char *kind)
{
    const char *f = getenv("ISOFFT_TEST_FAIL_ALLOC");
    if (f && strcmp(f, kind) == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

// NVTX range around one pass's launches (plans created with ISOFFT_NVTX=1)
struct PassRange {
    bool on;
    PassRange(bool enabled, const char *name) : on(enabled)
    {
        if (on) nvtxRangePushA(name);
    }
    ~PassRange()
    {
        if (on) nvtxRangePop();
    }
};

static void logf(int level, int verbosity, const char *fmt, ...)
{
    if (level > verbosity) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[isofft] ");
    vfprintf(stderr, fmt, ap);
    fprintf(stderr, "\n");
    va_end(ap);
}

static int env_verbosity()
{
    const char *s = getenv("ISOFFT_VERBOSITY");
    if (!s) return -1;
    int v = atoi(s);
    return v < 0 ? 0 : (v > 3 ? 3 : v);
}

// ----------------------------------------------------------------------
// Green's spectrum cache
// ----------------------------------------------------------------------
struct SpecKey {
    int device, dtype;
    int64_t M[3];
    double hn[3];
    bool operator<(const SpecKey &o) const
    {
        return std::tie(device, dtype, M[0], M[1], M[2], hn[0], hn[1], hn[2]) <
               std::tie(o.device, o.dtype, o.M[0], o.M[1], o.M[2], o.hn[0], o.hn[1], o.hn[2]);
    }
};
struct SpecEntry {
    void *G = nullptr;   // [My/2+1][Mz/2+1][Mx/2]
    void *Gs = nullptr;  // [My/2+1][Mz/2+1]
    size_t bytes = 0;
    int refs = 0;
    uint64_t last_use = 0;
    bool ready = false;  // false while a thread builds it (the cache lock is not held then)
};

static std::mutex g_cache_mu;
static std::condition_variable g_cache_cv;  // an entry was published or dropped
static std::map<SpecKey, SpecEntry> g_cache;
static uint64_t g_clock = 0;

static size_t spectrum_bytes(const int64_t M[3], int dtype)
{
    if (dtype == IPF_F32) return 4 * spectrum_elems<float>(M);
    if (dtype == IPF_F64) return 8 * spectrum_elems<double>(M);
    return 8 * spectrum_elems<df64>(M);
}

static void free_entry(SpecEntry &e)
{
    if (e.G) cudaFree(e.G);
    e.G = e.Gs = nullptr;
}

}  // namespace isofft

using namespace isofft;

struct ipf_plan_s {
    int64_t N[3];
    int64_t M[3];
    double h[3];
    int dtype;
    uint32_t flags;
    int verbosity;
    int device;
    SpecKey key;
    SpecEntry *spec;  // owned by the cache, referenced
    double gscale;
    void *W = nullptr;
    size_t W_bytes = 0;
    bool nvtx = false;  // NVTX range per pass (ISOFFT_NVTX=1 at creation)
    void *tables = nullptr;  // tw_x | rtw | tw_y | tw_z
    const void *tw_x = nullptr, *rtw = nullptr, *tw_y = nullptr, *tw_z = nullptr;
    unsigned *status = nullptr;  // device word after the tables: bit 0 = a bounded wait gave up
    // host-buffer solves: three device staging sets used in turn, copies on
    // two streams of the plan (host to device, device to host) so that one
    // solve's copies overlap its neighbours' passes (with three sets a
    // solve's upload waits only on the download of the solve two before it);
    // per-chunk events
    static constexpr int kChunks = 8, kAsyncChunks = 1, kSets = 3;
    void *stage[kSets] = {};
    int stage_set = 0;
    cudaStream_t h2d_st = nullptr, d2h_st = nullptr;
    cudaEvent_t ev_free[kSets] = {}, ev_in[kSets][kChunks] = {}, ev_out[kSets][kChunks] = {};
    // IPF_FLAG_PASS_EVENTS: a ring of event sets, one per recent solve; a
    // slot is folded into the running sums before it is reused, so timing
    // many back-to-back solves never waits on the device.
    static constexpr int kSlots = 64;
    cudaEvent_t ev[kSlots][6] = {};
    bool have_events = false;
    int yvar[2] = {kYTile, kYTile};  // form of the y forward / inverse pass
    int zsh = 0;  // the workspace's z planes in blocks of 2^zsh (plan_zsh)
    uint64_t solves = 0, folded = 0;
    double pass_sum[5] = {0, 0, 0, 0, 0};
    uint64_t pass_n = 0;
};

namespace {

// z blocking of the workspace (w_row): on 2304-point z lines, blocks of
// 2^kZBlockShift planes, where the plane count allows.
int plan_zsh(int64_t Mz, int64_t Nz)
{
    return Mz == 2304 && Nz % (1 << kZBlockShift) == 0 ? kZBlockShift : 0;
}

int64_t choose_mesh(int64_t n)
{
    for (int m : kSupportedM)
        if (m >= 2 * n) return m;
    return -1;
}

// bytes of one real of the source / potential arrays (FP64 for df64 solves);
// a workspace complex is twice that for every dtype
size_t elem_size(int dtype) { return dtype == IPF_F32 ? 4 : 8; }

int validate(const int64_t n[3], const double h[3], int dtype)
{
    if (!n || !h) return IPF_INVALID_ARG;
    if (dtype != IPF_F32 && dtype != IPF_F64 && dtype != IPF_DF64) return IPF_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return IPF_INVALID_ARG;
        if (!(h[a] > 0.0) || !isfinite(h[a])) return IPF_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (choose_mesh(n[a]) < 0) return IPF_UNSUPPORTED_SIZE;
    return IPF_OK;
}

// Widths divided by their minimum, rounded to a multiple of 2^-44 so that
// width sets that differ only by a common factor (0.1, 0.2, 0.15 and 1, 2,
// 1.5) share one cached spectrum; the rounding moves a ratio by at most
// 3e-14 relative, far below the FP64 tolerance.
void normalized_widths(const double h[3], double hn[3], double *hmin)
{
    double m = h[0];
    if (h[1] < m) m = h[1];
    if (h[2] < m) m = h[2];
    const double q = 17592186044416.0;  // 2^44
    for (int a = 0; a < 3; ++a) hn[a] = nearbyint(h[a] / m * q) / q;
    *hmin = m;
}

// Upload e^{-2 pi i k / n} tables in the plan's dtype.
template <typename T>
void fill_roots(std::vector<T> &dst, size_t off, int64_t n, int64_t count)
{
    std::vector<double> re(count), im(count);
    host_roots(n, count, re.data(), im.data());
    for (int64_t k = 0; k < count; ++k) {
        dst[off + 2 * k] = (T)re[k];
        dst[off + 2 * k + 1] = (T)im[k];
    }
}

template <typename T>
int upload_tables(ipf_plan_s *p, cudaStream_t st)
{
    const int64_t Lx = p->M[0] / 2, My = p->M[1], Mz = p->M[2];
    // tw_x: W_Lx^k (k < Lx); rtw: W_Mx^k (k < Lx); tw_y: W_My^k; tw_z: W_Mz^k
    const size_t ox = 0, orr = 2 * Lx, oy = 4 * Lx, oz = 4 * Lx + 2 * My, tot = 4 * Lx + 2 * My + 2 * Mz;
    std::vector<T> h(tot);
    fill_roots<T>(h, ox, Lx, Lx);
    fill_roots<T>(h, orr, p->M[0], Lx);
    fill_roots<T>(h, oy, My, My);
    fill_roots<T>(h, oz, Mz, Mz);
    const size_t tbytes = (tot * sizeof(T) + 15) / 16 * 16;
    cudaError_t e = dev_alloc(&p->tables, tbytes + 16, "tables");
    if (e != cudaSuccess) return cuda_status(e);
    p->status = (unsigned *)((char *)p->tables + tbytes);
    e = cudaMemcpyAsync(p->tables, h.data(), tot * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, 16, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    T *b = (T *)p->tables;
    p->tw_x = b + ox;
    p->rtw = b + orr;
    p->tw_y = b + oy;
    p->tw_z = b + oz;
    return IPF_OK;
}

// IPF_FLAG_TEST_WAIT_RUNOUT: bytes the z pass's first tile on each CTA
// expects beyond its copies, so that its bounded wait runs out.
unsigned runout_bytes(const ipf_plan_s *p) { return (p->flags & IPF_FLAG_TEST_WAIT_RUNOUT) ? 16u : 0u; }

// Reads and clears the plan's device status word after the work queued on
// `st` so far: IPF_TIMEOUT when a pass's bounded wait for its copies gave up,
// IPF_CUDA_ERROR when a pass refused its shared-memory layout.
int read_status(ipf_plan_s *p, cudaStream_t st)
{
    unsigned w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, p->status, sizeof(w), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (w == 0) return IPF_OK;
    e = cudaMemsetAsync(p->status, 0, sizeof(w), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return (w & 1u) ? IPF_TIMEOUT : IPF_CUDA_ERROR;
}

// ---------------------------------------------------------------------
// y-pass form tuning: the three forms (tiles, streamed, half-width tiles)
// run a few times each on the plan's workspace and the fastest is kept per
// direction, per (dtype, My, Kx, Ny, Nz, device capability); the choices
// persist for the process and, with ISOFFT_TUNE_FILE, in a JSON file of
// entries [dtype, My, Kx, Ny, Nz, sm, forward, inverse].
// ---------------------------------------------------------------------
struct TuneKey {
    int v[6];
    bool operator<(const TuneKey &o) const { return std::lexicographical_compare(v, v + 6, o.v, o.v + 6); }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

void tune_file_load()
{
    g_tune_loaded = true;
    const char *path = getenv("ISOFFT_TUNE_FILE");
    if (!path || !path[0]) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    // the integers of the file in order, eight per entry
    std::vector<long> nums;
    long cur = 0;
    bool in = false, neg = false;
    for (int ch; (ch = fgetc(f)) != EOF;) {
        if (ch >= '0' && ch <= '9') {
            cur = cur * 10 + (ch - '0');
            in = true;
        } else {
            if (in) nums.push_back(neg ? -cur : cur);
            neg = ch == '-';
            cur = 0;
            in = false;
        }
    }
    if (in) nums.push_back(neg ? -cur : cur);
    fclose(f);
    for (size_t i = 0; i + 8 <= nums.size(); i += 8) {
        TuneKey k;
        for (int j = 0; j < 6; ++j) k.v[j] = (int)nums[i + j];
        const int a = (int)nums[i + 6], b = (int)nums[i + 7];
        if (a >= 0 && a < kYForms && b >= 0 && b < kYForms) g_tune[k] = {a, b};
    }
}

void tune_file_save()
{
    const char *path = getenv("ISOFFT_TUNE_FILE");
    if (!path || !path[0]) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\"y_pass_forms\": [\n");
    size_t i = 0;
    for (const auto &kv : g_tune) {
        const int *v = kv.first.v;
        fprintf(f, "  [%d, %d, %d, %d, %d, %d, %d, %d]%s\n", v[0], v[1], v[2], v[3], v[4], v[5], kv.second.first,
                kv.second.second, ++i < g_tune.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    fclose(f);
}

// Mean device milliseconds of three launches after one warm-up.
template <typename Launch>
float time_launches(Launch launch, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, cudaError_t *err)
{
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    *err = e;
    return ms;
}

template <typename T>
int tune_y(ipf_plan_s *p, cudaStream_t st)
{
    const int Ny = (int)p->N[1], Nz = (int)p->N[2], My = (int)p->M[1], Lx = (int)(p->M[0] / 2);
    if (p->flags & (IPF_FLAG_Y_TILES | IPF_FLAG_Y_STREAM | IPF_FLAG_Y_TILES_NARROW)) {
        p->yvar[0] = p->yvar[1] = (p->flags & IPF_FLAG_Y_STREAM)         ? kYStream
                                  : (p->flags & IPF_FLAG_Y_TILES_NARROW) ? kYTileNarrow
                                                                         : kYTile;
        return IPF_OK;
    }
    const char *env = getenv("ISOFFT_TUNE");
    if (env && env[0] == '0') {
        p->yvar[0] = p->yvar[1] = y_default_variant(My, sizeof(T));
        return IPF_OK;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p->device);
    const TuneKey key{{p->dtype, My, Lx, Ny, Nz, major * 10 + minor}};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!g_tune_loaded) tune_file_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            p->yvar[0] = it->second.first;
            p->yvar[1] = it->second.second;
            return IPF_OK;
        }
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->W, 0, p->W_bytes, st);
    float t[2][kYForms] = {};
    for (int v = 0; v < kYForms && e == cudaSuccess; ++v) {
        t[0][v] = time_launches(
            [&] { return launch_y_forward<T>(My, p->W, p->tw_y, Ny, Lx, Nz, p->zsh, p->status, v, st); }, st, a, b,
            &e);
        if (e == cudaSuccess)
            t[1][v] = time_launches(
                [&] { return launch_y_inverse<T>(My, p->W, p->tw_y, Ny, Lx, Nz, p->zsh, p->status, v, st); }, st,
                a, b, &e);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_status(e);
    for (int d = 0; d < 2; ++d) {
        int best = kYTile;
        for (int v = 1; v < kYForms; ++v)
            if (t[d][v] < t[d][best]) best = v;
        p->yvar[d] = best;
    }
    logf(IPF_CONSOLE_INFO_2, p->verbosity,
         "y forms for mesh %dx%d (tiles/streamed/narrow tiles): forward %.4f/%.4f/%.4f ms, inverse %.4f/%.4f/%.4f ms",
         My, Lx, t[0][0], t[0][1], t[0][2], t[1][0], t[1][1], t[1][2]);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {p->yvar[0], p->yvar[1]};
    tune_file_save();
    return IPF_OK;
}

// ---------------------------------------------------------------------------
// On-disk copies of the Green's spectrum (ISOFFT_SPECTRUM_DIR): the only
// state of a solver, kept so that a restarted job skips K0.  One file per
// cache key: a header naming the key, the layout (the z tile width the
// spectrum is tiled for) and an FNV-1a checksum of the payload, then the
// device buffer's bytes.  A file whose header or checksum does not match is
// ignored (and replaced after the rebuild).
// ---------------------------------------------------------------------------
struct SpecFileHeader {
    char magic[8];
    uint32_t version;
    int32_t dtype;
    int64_t M[3];
    double hn[3];
    int32_t tile;
    int32_t pad;
    uint64_t bytes;
    uint64_t checksum;
};

static const char kSpecMagic[8] = {'I', 'S', 'O', 'F', 'F', 'T', 'G', 'S'};
#ifndef ISOFFT_SPECTRUM_CODE
#error "the build passes ISOFFT_SPECTRUM_CODE (a digest of the spectrum code)"
#endif

static uint64_t fnv1a(const unsigned char *d, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= d[i];
        h *= 1099511628211ull;
    }
    return h;
}

static int spectrum_tile(const SpecKey &k)
{
    const int mz = (int)k.M[2];
    return k.dtype == IPF_F32 ? z_tile_for<float>(mz) : (k.dtype == IPF_F64 ? z_tile_for<double>(mz) : z_tile_for<df64>(mz));
}

static bool spectrum_path(const SpecKey &k, char *path, size_t n)
{
    const char *dir = getenv("ISOFFT_SPECTRUM_DIR");
    if (!dir || !dir[0]) return false;
    uint64_t hb[3];
    memcpy(hb, k.hn, sizeof hb);
    const int w = snprintf(path, n, "%s/isofft_spectrum_%d_%lldx%lldx%lld_%016llx%016llx%016llx.bin", dir, k.dtype,
                           (long long)k.M[0], (long long)k.M[1], (long long)k.M[2], (unsigned long long)hb[0],
                           (unsigned long long)hb[1], (unsigned long long)hb[2]);
    return w > 0 && (size_t)w < n;
}

static SpecFileHeader spectrum_header(const SpecKey &k, size_t bytes)
{
    SpecFileHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kSpecMagic, sizeof h.magic);
    h.version = ISOFFT_SPECTRUM_CODE;  // digest of the spectrum's build and layout code
    h.dtype = k.dtype;
    for (int a = 0; a < 3; ++a) {
        h.M[a] = k.M[a];
        h.hn[a] = k.hn[a];
    }
    h.tile = spectrum_tile(k);
    h.bytes = bytes;
    return h;
}

// Loads the key's file into the device buffer; false if there is none or it
// does not match.
static bool spectrum_load(const SpecKey &k, SpecEntry &e, cudaStream_t st)
{
    char path[4096];
    if (!spectrum_path(k, path, sizeof path)) return false;
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    SpecFileHeader h, want = spectrum_header(k, e.bytes);
    std::vector<unsigned char> buf;
    bool ok = fread(&h, sizeof h, 1, f) == 1;
    if (ok) {
        want.checksum = h.checksum;
        ok = memcmp(&h, &want, sizeof h) == 0;
    }
    if (ok) {
        buf.resize(e.bytes);
        ok = fread(buf.data(), 1, e.bytes, f) == e.bytes && fnv1a(buf.data(), e.bytes) == h.checksum;
    }
    fclose(f);
    if (ok) ok = cudaMemcpyAsync(e.G, buf.data(), e.bytes, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                 cudaStreamSynchronize(st) == cudaSuccess;
    return ok;
}

// Writes the device buffer to the key's file (through a temporary file, so
// a reader never sees a partial one).  Failures only cost the next restart
// a rebuild.
static void spectrum_save(const SpecKey &k, const SpecEntry &e, cudaStream_t st)
{
    char path[4096], tmp[4200];
    if (!spectrum_path(k, path, sizeof path)) return;
    std::vector<unsigned char> buf(e.bytes);
    if (cudaMemcpyAsync(buf.data(), e.G, e.bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return;
    SpecFileHeader h = spectrum_header(k, e.bytes);
    h.checksum = fnv1a(buf.data(), e.bytes);
    snprintf(tmp, sizeof tmp, "%s.%d.tmp", path, (int)getpid());
    FILE *f = fopen(tmp, "wb");
    if (!f) return;
    const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), 1, e.bytes, f) == e.bytes;
    if (fclose(f) != 0 || !ok || rename(tmp, path) != 0) remove(tmp);
}

// The cache lock is held only to look up, reserve and publish an entry: the
// allocation, the file read or the build, and the file write of a missing
// spectrum run outside it (other plans, cache queries and trims go on
// meanwhile); a plan that needs a spectrum another thread is building waits
// for it to be published.
int acquire_spectrum(ipf_plan_s *p, cudaStream_t st)
{
    std::unique_lock<std::mutex> lk(g_cache_mu);
    for (;;) {
        auto it = g_cache.find(p->key);
        if (it == g_cache.end()) break;
        if (it->second.ready) {
            it->second.refs += 1;
            it->second.last_use = ++g_clock;
            p->spec = &it->second;
            return IPF_OK;
        }
        g_cache_cv.wait(lk);  // being built by another thread
    }
    // reserve the entry (a reference keeps trims away from it)
    SpecEntry e;
    e.bytes = spectrum_bytes(p->M, p->dtype);
    e.refs = 1;
    auto it = g_cache.emplace(p->key, e).first;
    lk.unlock();

    void *G = nullptr;
    cudaError_t ce = dev_alloc(&G, e.bytes, "spectrum");
    if (ce == cudaSuccess) {
        e.G = G;
        const size_t es = elem_size(p->dtype);
        const size_t Y = p->M[1] / 2 + 1, Z = p->M[2] / 2 + 1;
        e.Gs = (char *)e.G + e.bytes - es * Y * Z;
        const char *dn = p->dtype == IPF_F32 ? "f32" : (p->dtype == IPF_F64 ? "f64" : "df64");
        if (spectrum_load(p->key, e, st)) {
            logf(IPF_CONSOLE_INFO_1, p->verbosity, "loaded Green's spectrum for mesh %lldx%lldx%lld (%s) from disk",
                 (long long)p->M[0], (long long)p->M[1], (long long)p->M[2], dn);
        } else {
            logf(IPF_CONSOLE_INFO_1, p->verbosity, "building Green's spectrum for mesh %lldx%lldx%lld (%s)",
                 (long long)p->M[0], (long long)p->M[1], (long long)p->M[2], dn);
            if (p->dtype == IPF_F32)
                ce = build_green_spectrum<float>(p->M, p->key.hn, (float *)e.G, (float *)e.Gs, st);
            else if (p->dtype == IPF_F64)
                ce = build_green_spectrum<double>(p->M, p->key.hn, (double *)e.G, (double *)e.Gs, st);
            else
                ce = build_green_spectrum<df64>(p->M, p->key.hn, (df64 *)e.G, (df64 *)e.Gs, st);
            if (ce == cudaSuccess) spectrum_save(p->key, e, st);
        }
    }

    lk.lock();
    if (ce != cudaSuccess) {
        free_entry(e);
        g_cache.erase(it);
        g_cache_cv.notify_all();
        return cuda_status(ce);
    }
    it->second.G = e.G;
    it->second.Gs = e.Gs;
    it->second.ready = true;
    it->second.last_use = ++g_clock;
    p->spec = &it->second;
    g_cache_cv.notify_all();
    return IPF_OK;
}

void release_spectrum(ipf_plan_s *p)
{
    if (!p->spec) return;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(p->key);
    if (it != g_cache.end()) it->second.refs -= 1;
    p->spec = nullptr;
}

// Fold the pass times of solve number `i` (its events have completed or are
// waited for) into the plan's running sums.
cudaError_t fold_slot(ipf_plan_s *p, uint64_t i)
{
    cudaEvent_t *e = p->ev[i % ipf_plan_s::kSlots];
    cudaError_t r = cudaEventSynchronize(e[5]);
    if (r != cudaSuccess) return r;
    for (int k = 0; k < 5; ++k) {
        float ms = 0.f;
        r = cudaEventElapsedTime(&ms, e[k], e[k + 1]);
        if (r != cudaSuccess) return r;
        p->pass_sum[k] += ms;
    }
    p->pass_n += 1;
    return cudaSuccess;
}

template <typename T>
cudaError_t enqueue_solve(ipf_plan_s *p, const void *src, void *phi, cudaStream_t st)
{
    using IoT = typename IoReal<T>::type;
    const int Nx = (int)p->N[0], Ny = (int)p->N[1], Nz = (int)p->N[2];
    const int Lx = (int)(p->M[0] / 2), My = (int)p->M[1], Mz = (int)p->M[2];
    const int64_t nrows = (int64_t)Ny * Nz;
    const bool ev_on = p->have_events;
    cudaEvent_t *ev = nullptr;
    cudaError_t e;
    if (ev_on) {
        if (p->solves - p->folded == (uint64_t)ipf_plan_s::kSlots) {
            e = fold_slot(p, p->folded);
            if (e != cudaSuccess) return e;
            p->folded += 1;
        }
        ev = p->ev[p->solves % ipf_plan_s::kSlots];
        p->solves += 1;
    }
    // test hook: NaN bytes in every workspace element before the passes
    if (p->flags & IPF_FLAG_TEST_CANARY) {
        e = cudaMemsetAsync(p->W, 0xff, p->W_bytes, st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[0], st);
    {
        PassRange r(p->nvtx, "isofft K1 x forward");
        e = launch_x_forward<T>(Lx, (const IoT *)src, p->W, p->tw_x, p->rtw, Nx, Ny, My, nrows, p->zsh, st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[1], st);
    {
        PassRange r(p->nvtx, "isofft K2 y forward");
        e = launch_y_forward<T>(My, p->W, p->tw_y, Ny, Lx, Nz, p->zsh, p->status, p->yvar[0], st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[2], st);
    {
        PassRange r(p->nvtx, "isofft K3 z convolve");
        e = launch_z_convolve<T>(Mz, p->W, p->tw_z, (const T *)p->spec->G, (const T *)p->spec->Gs,
                                 (T)p->gscale, Nz, My, Lx, p->zsh, p->status, runout_bytes(p), st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[3], st);
    {
        PassRange r(p->nvtx, "isofft K4 y inverse");
        e = launch_y_inverse<T>(My, p->W, p->tw_y, Ny, Lx, Nz, p->zsh, p->status, p->yvar[1], st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[4], st);
    {
        PassRange r(p->nvtx, "isofft K5 x inverse");
        e = launch_x_inverse<T>(Lx, p->W, (IoT *)phi, p->tw_x, p->rtw, Nx, Ny, My, nrows, p->zsh, st);
        if (e != cudaSuccess) return e;
    }
    if (ev_on) cudaEventRecord(ev[5], st);
    return cudaSuccess;
}

int solve_impl(ipf_plan_s *p, const void *src, void *phi, cudaStream_t st)
{
    cudaError_t e = p->dtype == IPF_F32   ? enqueue_solve<float>(p, src, phi, st)
                    : p->dtype == IPF_F64 ? enqueue_solve<double>(p, src, phi, st)
                                          : enqueue_solve<df64>(p, src, phi, st);
    return cuda_status(e);
}

// Host-buffer solve, pipelined over chunks of z planes.  The x and y passes
// (and their inverses) treat z planes independently, so chunk k's forward
// x/y passes start as soon as its copy has landed while later chunks are
// still in flight on the copy stream; only the z pass needs every plane.
// On the way back, chunk k's potential is copied out while later chunks'
// inverse passes run.
template <typename T>
cudaError_t enqueue_solve_host(ipf_plan_s *p, const void *h_src, void *h_phi, int max_chunks, cudaStream_t st)
{
    using IoT = typename IoReal<T>::type;
    const int Nx = (int)p->N[0], Ny = (int)p->N[1], Nz = (int)p->N[2];
    const int Lx = (int)(p->M[0] / 2), My = (int)p->M[1], Mz = (int)p->M[2];
    const size_t plane = (size_t)Nx * Ny, wplane = (size_t)My * Lx;
    const int chunks = Nz < max_chunks ? Nz : max_chunks;
    // chunks of whole z blocks (the workspace's blocks start every 2^zsh planes)
    const int zb = 1 << p->zsh;
    const int per = ((Nz + chunks - 1) / chunks + zb - 1) / zb * zb;
    const int s = p->stage_set;
    p->stage_set = (s + 1) % ipf_plan_s::kSets;
    IoT *stage = (IoT *)p->stage[s];
    const char *hs = (const char *)h_src;
    char *hp = (char *)h_phi;
    char *W = (char *)p->W;
    const size_t cs = 2 * sizeof(T);  // bytes of one workspace complex
    // the set's previous potential has left before its staging is refilled
    cudaError_t e = cudaStreamWaitEvent(p->h2d_st, p->ev_free[s], 0);
    // test hook: NaN bytes in every workspace element before the passes
    if (e == cudaSuccess && (p->flags & IPF_FLAG_TEST_CANARY)) e = cudaMemsetAsync(p->W, 0xff, p->W_bytes, st);
    for (int k = 0; k < chunks && e == cudaSuccess; ++k) {
        const int z0 = k * per, nz = z0 + per <= Nz ? per : Nz - z0;
        if (nz <= 0) break;
        e = cudaMemcpyAsync(stage + z0 * plane, hs + z0 * plane * sizeof(IoT), nz * plane * sizeof(IoT),
                            cudaMemcpyHostToDevice, p->h2d_st);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[s][k], p->h2d_st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_in[s][k], 0);
        if (e == cudaSuccess)
            e = launch_x_forward<T>(Lx, stage + z0 * plane, W + z0 * wplane * cs, p->tw_x, p->rtw, Nx, Ny, My,
                                    (int64_t)nz * Ny, p->zsh, st);
        if (e == cudaSuccess)
            e = launch_y_forward<T>(My, W + z0 * wplane * cs, p->tw_y, Ny, Lx, nz, p->zsh, p->status, p->yvar[0],
                                    st);
    }
    if (e == cudaSuccess)
        e = launch_z_convolve<T>(Mz, p->W, p->tw_z, (const T *)p->spec->G, (const T *)p->spec->Gs, (T)p->gscale, Nz,
                                 My, Lx, p->zsh, p->status, runout_bytes(p), st);
    for (int k = 0; k < chunks && e == cudaSuccess; ++k) {
        const int z0 = k * per, nz = z0 + per <= Nz ? per : Nz - z0;
        if (nz <= 0) break;
        e = launch_y_inverse<T>(My, W + z0 * wplane * cs, p->tw_y, Ny, Lx, nz, p->zsh, p->status, p->yvar[1], st);
        if (e == cudaSuccess)
            e = launch_x_inverse<T>(Lx, W + z0 * wplane * cs, stage + z0 * plane, p->tw_x, p->rtw, Nx, Ny, My,
                                    (int64_t)nz * Ny, p->zsh, st);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[s][k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h_st, p->ev_out[s][k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hp + z0 * plane * sizeof(IoT), stage + z0 * plane, nz * plane * sizeof(IoT),
                                cudaMemcpyDeviceToHost, p->d2h_st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_free[s], p->d2h_st);
    return e;
}

// Staging buffers, copy streams and events of the host-buffer solves,
// created on the plan's first such solve.
int host_solve_setup(ipf_plan_s *p)
{
    const size_t bytes = elem_size(p->dtype) * (size_t)p->N[0] * (size_t)p->N[1] * (size_t)p->N[2];
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < ipf_plan_s::kSets && e == cudaSuccess; ++s)
        if (!p->stage[s]) {
            e = dev_alloc(&p->stage[s], bytes, "staging");
            if (e != cudaSuccess) p->stage[s] = nullptr;
        }
    if (e == cudaSuccess && !p->h2d_st) {
        e = cudaStreamCreateWithFlags(&p->h2d_st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h_st, cudaStreamNonBlocking);
        for (int s = 0; s < ipf_plan_s::kSets && e == cudaSuccess; ++s) {
            e = cudaEventCreateWithFlags(&p->ev_free[s], cudaEventDisableTiming);
            for (int k = 0; k < ipf_plan_s::kChunks && e == cudaSuccess; ++k) {
                e = cudaEventCreateWithFlags(&p->ev_in[s][k], cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_out[s][k], cudaEventDisableTiming);
            }
        }
    }
    return cuda_status(e);
}

// chunks: z-plane chunks of the copies (more chunks overlap a lone solve's
// copies with its own passes better; fewer keep the host's enqueue work per
// solve small when solves overlap one another)
int enqueue_host(ipf_plan_s *p, const void *h_src, void *h_phi, int chunks, cudaStream_t st)
{
    int rc = host_solve_setup(p);
    if (rc) return rc;
    const cudaError_t e = p->dtype == IPF_F32   ? enqueue_solve_host<float>(p, h_src, h_phi, chunks, st)
                          : p->dtype == IPF_F64 ? enqueue_solve_host<double>(p, h_src, h_phi, chunks, st)
                                                : enqueue_solve_host<df64>(p, h_src, h_phi, chunks, st);
    return cuda_status(e);
}

bool aligned16(const void *ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// Internal streams a batch is spread over, created once per device on the
// first multi-solve batch (so that first batch should precede any capture).
struct BatchLanes {
    static constexpr int kLanes = 8;
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t fork = nullptr, join[kLanes] = {};
    std::mutex mu;
};
std::mutex g_lanes_mu;
BatchLanes *g_lanes[64] = {};

// ISOFFT_BATCH_FUSED=1 in the environment runs the small FP32 grids of a
// batch in one launch per pass (batch.cu) instead of their own passes on the
// library's streams.  Off by default: one launch per pass streams every
// grid's workspace through HBM between passes, while the per-grid passes
// keep a grid's workspace in L2 from one pass to the next and measured
// faster (config 4: 0.94 vs 1.38 ms per batch of 64).  Read at every call.
// ISOFFT_BATCH_FUSED: 1 = one launch per pass, 2 = one launch for the
// batch, anything else = per-grid passes on the library's streams
int batch_fused_mode()
{
    const char *v = getenv("ISOFFT_BATCH_FUSED");
    return v && (v[0] == '1' || v[0] == '2') && v[1] == 0 ? v[0] - '0' : 0;
}

int batch_lanes(BatchLanes **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return IPF_CUDA_ERROR;
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    if (!g_lanes[dev]) {
        BatchLanes *b = new (std::nothrow) BatchLanes();
        if (!b) return IPF_OUT_OF_MEMORY;
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int l = 0; l < BatchLanes::kLanes && e == cudaSuccess; ++l) {
            e = cudaStreamCreateWithFlags(&b->lane[l], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_status(e);  // leaked on failure: creation of streams is not retried
        g_lanes[dev] = b;
    }
    *out = g_lanes[dev];
    return IPF_OK;
}

}  // namespace

extern "C" {

int ipf_plan_create(ipf_plan_t *out, const int64_t n[3], const double h[3], int dtype, uint32_t flags,
                    int verbosity, void *stream)
{
    if (!out) return IPF_INVALID_ARG;
    *out = nullptr;
    int rc = validate(n, h, dtype);
    if (rc) return rc;
    if (flags & ~(uint32_t)(IPF_FLAG_PASS_EVENTS | IPF_FLAG_Y_TILES | IPF_FLAG_Y_STREAM | IPF_FLAG_TEST_WAIT_RUNOUT |
                            IPF_FLAG_TEST_CANARY | IPF_FLAG_Y_TILES_NARROW))
        return IPF_INVALID_ARG;
    {
        const uint32_t forms = flags & (IPF_FLAG_Y_TILES | IPF_FLAG_Y_STREAM | IPF_FLAG_Y_TILES_NARROW);
        if (forms & (forms - 1)) return IPF_INVALID_ARG;  // at most one form forced
    }
    if (verbosity < IPF_CONSOLE_ERROR || verbosity > IPF_CONSOLE_INFO_2) return IPF_INVALID_ARG;
    const int ev = env_verbosity();
    if (ev >= 0) verbosity = ev;
    cudaStream_t st = (cudaStream_t)stream;
    ipf_plan_s *p = new (std::nothrow) ipf_plan_s();
    if (!p) return IPF_OUT_OF_MEMORY;
    for (int a = 0; a < 3; ++a) {
        p->N[a] = n[a];
        p->M[a] = choose_mesh(n[a]);
        p->h[a] = h[a];
    }
    p->dtype = dtype;
    p->flags = flags;
    p->verbosity = verbosity;
    p->spec = nullptr;
    {
        const char *nv = getenv("ISOFFT_NVTX");
        p->nvtx = nv && nv[0] == '1';
    }
    cudaError_t ce = cudaGetDevice(&p->device);
    if (ce != cudaSuccess) {
        delete p;
        return cuda_status(ce);
    }
    double hmin;
    normalized_widths(h, p->key.hn, &hmin);
    p->gscale = hmin * hmin;
    p->key.device = p->device;
    p->key.dtype = dtype;
    for (int a = 0; a < 3; ++a) p->key.M[a] = p->M[a];
    p->zsh = plan_zsh(p->M[2], p->N[2]);

    p->W_bytes = 2 * elem_size(dtype) * (size_t)p->N[2] * (size_t)p->M[1] * (size_t)(p->M[0] / 2);
    ce = dev_alloc(&p->W, p->W_bytes, "workspace");
    if (ce != cudaSuccess) {
        rc = cuda_status(ce);
        ipf_plan_destroy(p);
        return rc;
    }
    rc = dtype == IPF_F32   ? upload_tables<float>(p, st)
         : dtype == IPF_F64 ? upload_tables<double>(p, st)
                            : upload_tables<df64>(p, st);
    if (!rc) rc = acquire_spectrum(p, st);
    if (!rc)
        rc = dtype == IPF_F32   ? tune_y<float>(p, st)
             : dtype == IPF_F64 ? tune_y<double>(p, st)
                                : tune_y<df64>(p, st);
    if (!rc && (flags & IPF_FLAG_PASS_EVENTS)) {
        for (int s = 0; s < ipf_plan_s::kSlots && !rc; ++s)
            for (int i = 0; i < 6 && !rc; ++i) rc = cuda_status(cudaEventCreate(&p->ev[s][i]));
        p->have_events = !rc;
    }
    if (rc) {
        ipf_plan_destroy(p);
        return rc;
    }
    logf(IPF_CONSOLE_INFO_2, p->verbosity, "plan %lldx%lldx%lld on mesh %lldx%lldx%lld, workspace %zu bytes",
         (long long)n[0], (long long)n[1], (long long)n[2], (long long)p->M[0], (long long)p->M[1],
         (long long)p->M[2], p->W_bytes);
    *out = p;
    return IPF_OK;
}

int ipf_plan_destroy(ipf_plan_t p)
{
    if (!p) return IPF_OK;
    release_spectrum(p);
    if (p->W) cudaFree(p->W);
    if (p->tables) cudaFree(p->tables);
    for (int s = 0; s < ipf_plan_s::kSets; ++s) {
        if (p->stage[s]) cudaFree(p->stage[s]);
        if (p->ev_free[s]) cudaEventDestroy(p->ev_free[s]);
        for (int k = 0; k < ipf_plan_s::kChunks; ++k) {
            if (p->ev_in[s][k]) cudaEventDestroy(p->ev_in[s][k]);
            if (p->ev_out[s][k]) cudaEventDestroy(p->ev_out[s][k]);
        }
    }
    if (p->h2d_st) cudaStreamDestroy(p->h2d_st);
    if (p->d2h_st) cudaStreamDestroy(p->d2h_st);
    for (int s = 0; s < ipf_plan_s::kSlots; ++s)
        for (int i = 0; i < 6; ++i)
            if (p->ev[s][i]) cudaEventDestroy(p->ev[s][i]);
    delete p;
    return IPF_OK;
}

int ipf_plan_padded_shape(const ipf_plan_t p, int64_t m[3])
{
    if (!p || !m) return IPF_INVALID_ARG;
    for (int a = 0; a < 3; ++a) m[a] = p->M[a];
    return IPF_OK;
}

int ipf_plan_workspace_bytes(const ipf_plan_t p, size_t *bytes)
{
    if (!p || !bytes) return IPF_INVALID_ARG;
    *bytes = p->W_bytes;
    return IPF_OK;
}

int ipf_plan_spectrum_bytes(const ipf_plan_t p, size_t *bytes)
{
    if (!p || !bytes || !p->spec) return IPF_INVALID_ARG;
    *bytes = p->spec->bytes;
    return IPF_OK;
}

int ipf_estimate_bytes(const int64_t n[3], const double h[3], int dtype, size_t *bytes)
{
    if (!bytes) return IPF_INVALID_ARG;
    int rc = validate(n, h, dtype);
    if (rc) return rc;
    int64_t M[3];
    for (int a = 0; a < 3; ++a) M[a] = choose_mesh(n[a]);
    size_t w = 2 * elem_size(dtype) * (size_t)n[2] * (size_t)M[1] * (size_t)(M[0] / 2);
    SpecKey key;
    double hmin;
    normalized_widths(h, key.hn, &hmin);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetLastError();
    key.device = dev;
    key.dtype = dtype;
    for (int a = 0; a < 3; ++a) key.M[a] = M[a];
    bool cached;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        cached = g_cache.count(key) != 0;
    }
    *bytes = w + (cached ? 0 : spectrum_bytes(M, dtype));
    return IPF_OK;
}

int ipf_solve(ipf_plan_t p, const void *d_src, void *d_phi, void *stream)
{
    if (!p || !d_src || !d_phi) return IPF_INVALID_ARG;
    if (!aligned16(d_src) || !aligned16(d_phi)) return IPF_INVALID_ARG;
    return solve_impl(p, d_src, d_phi, (cudaStream_t)stream);
}


int ipf_solve_host(ipf_plan_t p, const void *h_src, void *h_phi, void *stream)
{
    if (!p || !h_src || !h_phi) return IPF_INVALID_ARG;
    const int rc = enqueue_host(p, h_src, h_phi, ipf_plan_s::kChunks, (cudaStream_t)stream);
    if (rc) return rc;
    return ipf_plan_host_wait(p);
}

int ipf_solve_host_async(ipf_plan_t p, const void *h_src, void *h_phi, void *stream)
{
    if (!p || !h_src || !h_phi) return IPF_INVALID_ARG;
    return enqueue_host(p, h_src, h_phi, ipf_plan_s::kAsyncChunks, (cudaStream_t)stream);
}

int ipf_plan_host_wait(ipf_plan_t p)
{
    if (!p) return IPF_INVALID_ARG;
    if (!p->d2h_st) return IPF_OK;  // no host-buffer solve yet
    const cudaError_t e = cudaStreamSynchronize(p->d2h_st);
    if (e != cudaSuccess) return cuda_status(e);
    return read_status(p, p->d2h_st);
}

int ipf_plan_check(ipf_plan_t p, void *stream)
{
    if (!p) return IPF_INVALID_ARG;
    return read_status(p, (cudaStream_t)stream);
}

int ipf_submit_batch(const ipf_plan_t *plans, int count, const void *const *d_src, void *const *d_phi,
                     void *stream)
{
    if (count < 0 || (count > 0 && (!plans || !d_src || !d_phi))) return IPF_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !d_src[i] || !d_phi[i]) return IPF_INVALID_ARG;
        if (!aligned16(d_src[i]) || !aligned16(d_phi[i])) return IPF_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return IPF_INVALID_ARG;
    }
    if (count == 0) return IPF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (count == 1) return solve_impl(plans[0], d_src[0], d_phi[0], st);
    // small FP32 grids: one launch per pass over all of them (batch.cu)
    std::vector<BatchGridDesc> fused;
    std::vector<int> rest;
    const int mode = batch_fused_mode();
    unsigned *bstatus = nullptr;  // the first batched plan's status word
    for (int i = 0; i < count; ++i) {
        const ipf_plan_s *p = plans[i];
        // the run-out test hook joins a one-launch batch (its dependency
        // wait runs out there); other hooked plans keep their own passes
        const uint32_t hooks = IPF_FLAG_PASS_EVENTS | IPF_FLAG_TEST_CANARY | (mode == 2 ? 0u : IPF_FLAG_TEST_WAIT_RUNOUT);
        const bool plain = !(p->flags & hooks);
        if (mode && plain && batch_fits(p->dtype == IPF_F32, p->M)) {
            if (!bstatus) bstatus = p->status;
            fused.push_back({d_src[i], d_phi[i], p->W, p->tw_x, p->rtw, p->tw_y, p->tw_z, p->spec->G, p->spec->Gs,
                             p->gscale, (int)p->N[0], (int)p->N[1], (int)p->N[2], (int)p->M[0], (int)p->M[1],
                             (int)p->M[2], (p->flags & IPF_FLAG_TEST_WAIT_RUNOUT) ? 1 : 0});
        } else {
            rest.push_back(i);
        }
    }
    if (fused.size() == 1) {  // a single grid runs its own kernels
        for (int i = 0; i < count; ++i)
            if (std::find(rest.begin(), rest.end(), i) == rest.end()) rest.push_back(i);
        fused.clear();
    }
    if (rest.empty()) return cuda_status(batch_enqueue(fused.data(), (int)fused.size(), mode, bstatus, st));
    BatchLanes *bl = nullptr;
    int rc = batch_lanes(&bl);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(bl->mu);
    // fork: every lane waits for the work already on the caller's stream
    cudaError_t e = cudaEventRecord(bl->fork, st);
    if (e != cudaSuccess) return cuda_status(e);
    const int nrest = (int)rest.size();
    const int lanes = nrest < BatchLanes::kLanes ? nrest : BatchLanes::kLanes;
    for (int l = 0; l < lanes; ++l) {
        e = cudaStreamWaitEvent(bl->lane[l], bl->fork, 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (!fused.empty()) {
        e = batch_enqueue(fused.data(), (int)fused.size(), mode, bstatus, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // the other solves longest first, each to the least-loaded lane
    std::vector<int> order(rest);
    std::vector<double> cost(count, 0.0), load(lanes, 0.0);
    for (int i : rest) {
        const ipf_plan_s *p = plans[i];
        cost[i] = (double)p->M[0] * p->M[1] * p->N[2] * (p->dtype == IPF_F64 ? 16.0 : (p->dtype == IPF_DF64 ? 6.0 : 1.0));
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i : order) {
        int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost[i];
        rc = solve_impl(plans[i], d_src[i], d_phi[i], bl->lane[l]);
        if (rc) return rc;
    }
    // join: the caller's stream waits for every lane
    for (int l = 0; l < lanes; ++l) {
        e = cudaEventRecord(bl->join[l], bl->lane[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, bl->join[l], 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return IPF_OK;
}

int ipf_plan_pass_times(ipf_plan_t p, float ms[5])
{
    if (!p || !ms || !p->have_events) return IPF_INVALID_ARG;
    while (p->folded < p->solves) {
        cudaError_t e = fold_slot(p, p->folded);
        if (e != cudaSuccess) return cuda_status(e);
        p->folded += 1;
    }
    if (p->pass_n == 0) return IPF_NOT_READY;
    for (int i = 0; i < 5; ++i) ms[i] = (float)(p->pass_sum[i] / (double)p->pass_n);
    for (int i = 0; i < 5; ++i) p->pass_sum[i] = 0.0;
    p->pass_n = 0;
    return IPF_OK;
}

int ipf_greens_cache_bytes(size_t *bytes)
{
    if (!bytes) return IPF_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    size_t b = 0;
    for (auto &kv : g_cache) b += kv.second.bytes;
    *bytes = b;
    return IPF_OK;
}

int ipf_greens_cache_trim(size_t budget)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    size_t b = 0;
    for (auto &kv : g_cache) b += kv.second.bytes;
    while (b > budget) {
        auto victim = g_cache.end();
        for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
            if (it->second.ready && it->second.refs == 0 &&
                (victim == g_cache.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == g_cache.end()) break;
        b -= victim->second.bytes;
        free_entry(victim->second);
        g_cache.erase(victim);
    }
    return IPF_OK;
}

int ipf_launch_count(uint64_t *count)
{
    if (!count) return IPF_INVALID_ARG;
    *count = g_launches.load();
    return IPF_OK;
}

int ipf_last_cuda_error(void) { return g_last_cuda; }

int ipf_plan_variants(const ipf_plan_t p, int v[2])
{
    if (!p || !v) return IPF_INVALID_ARG;
    v[0] = p->yvar[0];
    v[1] = p->yvar[1];
    return IPF_OK;
}

const char *ipf_status_string(int s)
{
    switch (s) {
    case IPF_OK: return "ok";
    case IPF_INVALID_ARG: return "invalid argument";
    case IPF_UNSUPPORTED_SIZE: return "unsupported size";
    case IPF_OUT_OF_MEMORY: return "out of memory";
    case IPF_CUDA_ERROR: return "CUDA error";
    case IPF_TIMEOUT: return "timeout";
    case IPF_BUDGET_EXCEEDED: return "memory budget exceeded";
    case IPF_NOT_READY: return "not ready";
    default: return "unknown status";
    }
}

}  // extern "C"
