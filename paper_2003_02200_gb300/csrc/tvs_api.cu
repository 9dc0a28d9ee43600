// tvs_api.cu -- host side of the C ABI declared in include/tvs.h: argument
// checks, the direction table, chunking of the directions under the HBM
// budget, kernel launches and per-kernel timing.
#include "tvs.h"
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace tvs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(TVS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TVS_CUDA(call, where)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

constexpr int kMaxDim = 16384;        // longest walk axis the staged sweep supports
constexpr int kMaxChunkDirs = 1024;   // directions per chunk (bounds the item table in smem)
constexpr long long kMaxChunkItems = 1LL << 30;  // sweep warp items per chunk
constexpr double kTwo32 = 4294967296.0;

// ---------------------------------------------------------- directions --
// Direction k of n: theta_k = k*pi/n from +j (east) toward +i (south).  Alg. 6
// covers 0..45 degrees; the rest of the half-plane reuses it through a D4 view
// chosen by integer tests on k, with the reduced angle alpha = pi*m/(2n):
//   4k <  n : identity,                  m = 2k
//   4k < 2n : transpose,                 m = n - 2k
//   4k < 3n : transpose + mirror columns, m = 2k - n
//   else    : mirror rows,               m = 2n - 2k
// tan(alpha) is held in 32.32 fixed point; g = 1 + t^2 is the (1/cos s)^2
// factor of Alg. 7 for that t.
struct HostDir {
    int frame, m, H, W, D, R;
    unsigned long long t_fx;
    double t, g;
    long long K;  // LLONG_MAX = unlimited
};

int make_direction(int n, int k, int rows, int cols, double step, double max_range, HostDir* d)
{
    if (n < 1 || k < 0 || k >= n || rows < 2 || cols < 2 || !(step > 0.0) || std::isnan(max_range))
        return TVS_ERR_ARG;
    const long long k4 = 4LL * k;
    if (k4 < n) { d->frame = 0; d->m = 2 * k; d->H = rows; d->W = cols; }
    else if (k4 < 2LL * n) { d->frame = 1; d->m = n - 2 * k; d->H = cols; d->W = rows; }
    else if (k4 < 3LL * n) { d->frame = 2; d->m = 2 * k - n; d->H = cols; d->W = rows; }
    else { d->frame = 3; d->m = 2 * n - 2 * k; d->H = rows; d->W = cols; }
    const double alpha = M_PI * (double)d->m / (2.0 * (double)n);
    d->t_fx = (unsigned long long)std::llround(std::tan(alpha) * kTwo32);
    d->t = (double)d->t_fx / kTwo32;
    d->g = 1.0 + d->t * d->t;
    if (!(max_range > 0.0) || std::isinf(max_range)) {
        d->K = LLONG_MAX;
    } else {
        const double kk = std::floor(max_range / (step * std::sqrt(d->g)));
        d->K = kk >= 9.0e18 ? LLONG_MAX : (long long)kk;
    }
    d->D = (int)(((unsigned long long)(d->W - 1) * d->t_fx) >> 32);
    d->R = d->H + d->D;
    return TVS_OK;
}

// Usable columns of skewed row p (base row p - D): 0 <= (p-D) + j*t <= H-1.
void host_row_range(const HostDir& d, int p, int* lo, int* hi)
{
    const long long b = (long long)p - d.D;
    long long l = 0, h;
    if (d.t_fx == 0ull) {
        h = (b >= 0 && b <= d.H - 1) ? d.W - 1 : -1;
    } else {
        if (b < 0) l = (long long)((((unsigned long long)(-b) << 32) + d.t_fx - 1ull) / d.t_fx);
        const long long top = (long long)d.H - 1 - b;
        h = top < 0 ? -1 : (long long)(((unsigned long long)top << 32) / d.t_fx);
        if (h > d.W - 1) h = d.W - 1;
    }
    if (l > h) { l = 0; h = -1; }
    *lo = (int)l;
    *hi = (int)h;
}

// Warp items per skewed row and walk direction: a row of W samples has
// ceil(W / P) groups, paired into ceil(groups / 2) lane slots, 32 per item.
int sweep_chunks(int W)
{
    const int groups = (W + POVS_PER_LANE - 1) / POVS_PER_LANE;
    return ((groups + 1) / 2 + 31) / 32;
}

long long sum_min(long long L, long long K)
{
    // sum_{x=0}^{L-1} min(x, K)
    if (L <= 0) return 0;
    if (L - 1 <= K) return (L - 1) * L / 2;
    return K * (K + 1) / 2 + (L - 1 - K) * K;
}

struct DirWork {
    long long evals;        // targets visited (work count)
    long long samples;      // usable samples (virtual POVs)
};

DirWork direction_work(const HostDir& d)
{
    DirWork w{0, 0};
    const long long K = d.K == LLONG_MAX ? (long long)d.W : std::min<long long>(d.K, d.W);
    for (int p = 0; p < d.R; ++p) {
        int lo, hi;
        host_row_range(d, p, &lo, &hi);
        const long long L = hi - lo + 1;
        if (L <= 0) continue;
        w.samples += L;
        w.evals += 2 * sum_min(L, K);
    }
    return w;
}

int check_job(int rows, int cols, double step_m, double obs_height_m, int n_sectors, double max_range_m)
{
    if (rows < 2 || cols < 2) return fail(TVS_ERR_ARG, "rows and cols must be >= 2");
    if (rows > kMaxDim || cols > kMaxDim)
        return fail(TVS_ERR_ARG, "rows and cols must be <= 16384 (shared-memory row staging limit)");
    if (!(step_m > 0.0) || !std::isfinite(step_m)) return fail(TVS_ERR_ARG, "step_m must be finite and > 0");
    if (!std::isfinite(obs_height_m)) return fail(TVS_ERR_ARG, "obs_height_m must be finite");
    if (n_sectors < 1 || n_sectors > 1 << 20) return fail(TVS_ERR_ARG, "n_sectors must be in [1, 2^20]");
    if (std::isnan(max_range_m)) return fail(TVS_ERR_ARG, "max_range_m is NaN");
    return TVS_OK;
}

// ------------------------------------------------------------ profiling --
enum KernelId { K_ROWMAP = 0, K_SKEW, K_SWEEP, K_UNSKEW, K_FINAL, K_COUNT };
const char* kKernelName[K_COUNT] = {"rowmap", "skew", "sweep", "unskew", "unskew_finalize"};
const char* kKernelUnit[K_COUNT] = {"bytes", "bytes", "evals", "bytes", "bytes"};

struct Pending {
    int kernel;
    cudaEvent_t start, stop;
    double units;
};

}  // namespace

struct tvs_ctx {
    int device = 0;
    size_t budget = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;   // the handle's own stream (host-memory API)
    char* ws = nullptr;              // device scratch
    size_t ws_bytes = 0;
    int smem_optin = 0;              // max dynamic shared memory per block
    char* pinned = nullptr;          // pinned staging of the per-call table upload
    size_t pinned_bytes = 0;
    cudaEvent_t pinned_done = nullptr;  // the last upload from `pinned` has been read
    bool profiling = false;
    std::vector<Pending> pending;
    tvs_kernel_stats stats[K_COUNT];
};

namespace {

struct Timer {
    tvs_ctx* h;
    int kernel;
    cudaStream_t s;
    double units;
    cudaEvent_t a = nullptr, b = nullptr;
    Timer(tvs_ctx* h_, int k, cudaStream_t s_, double u) : h(h_), kernel(k), s(s_), units(u)
    {
        if (h->profiling && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, s);
    }
    ~Timer()
    {
        if (a && b) {
            cudaEventRecord(b, s);
            h->pending.push_back(Pending{kernel, a, b, units});
        }
    }
};

void drain_pending(tvs_ctx* h)
{
    for (auto& p : h->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            tvs_kernel_stats& s = h->stats[p.kernel];
            s.launches += 1;
            s.total_ms += ms;
            s.units += p.units;
        }
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    h->pending.clear();
}

void reset_stats(tvs_ctx* h)
{
    for (int k = 0; k < K_COUNT; ++k) {
        std::memset(&h->stats[k], 0, sizeof(tvs_kernel_stats));
        std::snprintf(h->stats[k].name, sizeof(h->stats[k].name), "%s", kKernelName[k]);
        std::snprintf(h->stats[k].unit, sizeof(h->stats[k].unit), "%s", kKernelUnit[k]);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ensure_scratch(tvs_ctx* h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return TVS_OK;
    if (h->ws) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize before scratch growth");
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return fail(TVS_ERR_OOM, std::string("cudaMalloc of scratch failed: ") + cudaGetErrorString(e));
    }
    h->ws_bytes = bytes;
    return TVS_OK;
}

// One planned chunk of directions [k0, k1).
struct Chunk {
    int k0, k1;
    size_t slab_elems;   // sum of R * Wp over the chunk
    long long rows;      // sum of R
    int items;           // sweep warp items
    int max_R, max_tiles, wmax, dmax;
    double evals, skew_bytes, unskew_bytes, rowmap_bytes;
};

struct Plan {
    std::vector<HostDir> dirs;
    std::vector<DirDev> dev;        // per direction, slab / row offsets relative to its chunk
    std::vector<Chunk> chunks;
    size_t max_slab = 0;            // largest chunk slab (elements)
    long long max_rows = 0;         // largest chunk row count
    int max_items1 = 0;             // largest chunk direction count + 1
    int istart_total = 0;           // sum over chunks of (directions + 1)
};

size_t chunk_bytes(size_t slab, long long rows, int ndir)
{
    // skewed heights + forward measures + backward measures, row tables, item table
    return align256(slab * 4) * 3 + align256((size_t)rows * 4) * 2 + align256((size_t)(ndir + 1) * 4);
}

// Split the n directions into consecutive chunks whose scratch fits `avail`
// bytes; chunk sizes are kept multiples of FP32_GROUP so that the FP32 group
// sums (and so the result bits) do not depend on the chunking.
int make_plan(int rows, int cols, double step, double max_range, int n, size_t avail, Plan* plan,
              int only_k = -1)
{
    plan->dirs.resize(n);
    plan->dev.resize(n);
    for (int k = 0; k < n; ++k) {
        int rc = make_direction(n, k, rows, cols, step, max_range, &plan->dirs[k]);
        if (rc) return fail(rc, "bad direction arguments");
    }
    int k = only_k >= 0 ? only_k : 0;
    const int kend = only_k >= 0 ? only_k + 1 : n;
    while (k < kend) {
        Chunk c{};
        c.k0 = k;
        size_t slab = 0;
        long long nrows = 0;
        int kk = k;
        int last_ok = -1;
        long long items_acc = 0;
        size_t slab_ok = 0;
        long long rows_ok = 0;
        while (kk < kend) {
            const HostDir& d = plan->dirs[kk];
            const size_t wp = (size_t)((d.W + 3) & ~3);
            const size_t s2 = slab + (size_t)d.R * wp;
            const long long r2 = nrows + d.R;
            const long long it2 = items_acc + 2LL * d.R * sweep_chunks(d.W);
            if (kk > k && (chunk_bytes(s2, r2, kk - k + 1) > avail || kk - k >= kMaxChunkDirs ||
                           it2 > kMaxChunkItems))
                break;
            items_acc = it2;
            slab = s2;
            nrows = r2;
            ++kk;
            if ((kk - k) % FP32_GROUP == 0 || kk == kend) { last_ok = kk; slab_ok = slab; rows_ok = nrows; }
        }
        if (kk == k) return fail(TVS_ERR_OOM, "one direction does not fit the HBM budget");
        if (chunk_bytes(slab, nrows, kk - k) > avail)
            return fail(TVS_ERR_OOM, "one direction does not fit the HBM budget");
        if (last_ok > k && kk < kend) { kk = last_ok; slab = slab_ok; nrows = rows_ok; }
        c.k1 = kk;
        size_t off = 0;
        long long roff = 0;
        int items = 0;
        c.max_R = 0; c.max_tiles = 0; c.wmax = 0; c.dmax = 0;
        c.evals = c.skew_bytes = c.unskew_bytes = c.rowmap_bytes = 0;
        for (int q = c.k0; q < c.k1; ++q) {
            const HostDir& d = plan->dirs[q];
            DirDev& v = plan->dev[q];
            std::memset(&v, 0, sizeof(v));
            v.t_fx = d.t_fx;
            v.slab = (long long)off;
            v.frame = d.frame; v.H = d.H; v.W = d.W; v.Wp = (d.W + 3) & ~3;
            v.D = d.D; v.R = d.R;
            v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
            v.row_off = (int)roff;
            v.chunks = sweep_chunks(d.W);
            v.gidx = q;
            v.g = (float)d.g;
            off += (size_t)d.R * v.Wp;
            roff += d.R;
            items += 2 * d.R * v.chunks;
            c.max_R = std::max(c.max_R, d.R);
            c.max_tiles = std::max(c.max_tiles, ((d.R + SKEW_TP - 1) / SKEW_TP) * ((d.W + SKEW_TJ - 1) / SKEW_TJ));
            c.wmax = std::max(c.wmax, d.W);
            c.dmax = std::max(c.dmax, v.K);
            const DirWork w = direction_work(d);
            c.evals += (double)w.evals;
            c.skew_bytes += 4.0 * rows * cols + 4.0 * (double)w.samples;
            c.unskew_bytes += 4.0 * (double)w.samples;
            c.rowmap_bytes += 8.0 * d.R;
        }
        c.slab_elems = off;
        c.rows = roff;
        c.items = items;
        plan->max_slab = std::max(plan->max_slab, off);
        plan->max_rows = std::max(plan->max_rows, roff);
        plan->max_items1 = std::max(plan->max_items1, c.k1 - c.k0 + 1);
        plan->istart_total += c.k1 - c.k0 + 1;
        plan->chunks.push_back(c);
        k = kk;
    }
    const size_t nch = plan->chunks.size();
    for (size_t q = 0; q < nch; ++q) {
        Chunk& c = plan->chunks[q];
        const double cells = (double)rows * cols;
        c.unskew_bytes += (q == 0 ? 0.0 : 8.0 * cells) + (q + 1 == nch ? 4.0 * cells : 8.0 * cells);
    }
    return TVS_OK;
}

// Scratch layout of a job (offsets in bytes from h->ws).
struct Layout {
    size_t dem, out, dirs, istart, rowlo, rowhi, sdem, cvf, cvb, vs64, part, counter, total;
};

Layout make_layout(const Plan& plan, int n, int rows, int cols, bool host_io, bool need_vs64, int nsplit)
{
    Layout L{};
    size_t o = 0;
    const size_t cells = (size_t)rows * cols;
    L.dem = o;     if (host_io) o += align256(cells * 4);
    L.out = o;     if (host_io) o += align256(cells * 4);
    L.dirs = o;    o += align256((size_t)n * sizeof(DirDev));
    L.istart = o;  o += align256((size_t)plan.istart_total * 4);
    L.rowlo = o;   o += align256((size_t)plan.max_rows * 4);
    L.rowhi = o;   o += align256((size_t)plan.max_rows * 4);
    L.sdem = o;    o += align256(plan.max_slab * 4);
    L.cvf = o;     o += align256(plan.max_slab * 4);
    L.cvb = o;     o += align256(plan.max_slab * 4);
    L.vs64 = o;    if (need_vs64) o += align256(cells * 8);
    L.part = o;    if (nsplit > 1) o += align256((size_t)nsplit * cells * 8);
    L.counter = o; o += 256;
    L.total = o;
    return L;
}

size_t fixed_bytes(int n, int rows, int cols, bool host_io, int num_sms)
{
    const size_t cells = (size_t)rows * cols;
    const int nsplit = unskew_splits(rows, cols, n, num_sms);
    return (host_io ? 2 * align256(cells * 4) : 0) + align256((size_t)n * sizeof(DirDev)) +
           align256(cells * 8) + (nsplit > 1 ? align256((size_t)nsplit * cells * 8) : 0) + 4096 +
           align256((size_t)(2 * n + 1) * 4);
}

// Copy two host tables into device memory with one asynchronous copy from the
// handle's pinned staging buffer.  The buffer is reused by the next call only
// after the copy that read it has run (event), so the host never blocks on
// the GPU work queued before the copy.
int upload_header(tvs_ctx* h, const void* a, size_t a_bytes, const void* b, size_t b_bytes, void* d_a,
                  void* d_b, cudaStream_t s)
{
    const size_t bytes = a_bytes + b_bytes;
    if (h->pinned_done) TVS_CUDA(cudaEventSynchronize(h->pinned_done), "wait for staging buffer");
    if (bytes > h->pinned_bytes) {
        if (h->pinned) cudaFreeHost(h->pinned);
        h->pinned = nullptr;
        h->pinned_bytes = 0;
        TVS_CUDA(cudaHostAlloc((void**)&h->pinned, bytes, cudaHostAllocDefault), "cudaHostAlloc");
        h->pinned_bytes = bytes;
    }
    std::memcpy(h->pinned, a, a_bytes);
    std::memcpy(h->pinned + a_bytes, b, b_bytes);
    // d_a and d_b are adjacent in the scratch layout only by accident; copy separately.
    TVS_CUDA(cudaMemcpyAsync(d_a, h->pinned, a_bytes, cudaMemcpyHostToDevice, s), "copy direction table");
    TVS_CUDA(cudaMemcpyAsync(d_b, h->pinned + a_bytes, b_bytes, cudaMemcpyHostToDevice, s), "copy item table");
    if (!h->pinned_done) TVS_CUDA(cudaEventCreateWithFlags(&h->pinned_done, cudaEventDisableTiming), "event");
    TVS_CUDA(cudaEventRecord(h->pinned_done, s), "record staging event");
    return TVS_OK;
}

// Enqueue the whole job: per chunk rowmap -> skew -> sweep -> unskew.
int run_job(tvs_ctx* h, const float* d_dem, int rows, int cols, double step, double h0, int n,
            double max_range, float* d_out, cudaStream_t s, bool host_io, const float* host_dem,
            float* host_out)
{
    const size_t fixed = fixed_bytes(n, rows, cols, host_io, h->num_sms);
    if (fixed >= h->budget) return fail(TVS_ERR_OOM, "the DEM does not fit the HBM budget");
    Plan plan;
    int rc = make_plan(rows, cols, step, max_range, n, h->budget - fixed, &plan);
    if (rc) return rc;
    const bool need_vs64 = plan.chunks.size() > 1;
    int max_nd = 0;
    for (const Chunk& c : plan.chunks) max_nd = std::max(max_nd, c.k1 - c.k0);
    const int nsplit = unskew_splits(rows, cols, max_nd, h->num_sms);
    const Layout L = make_layout(plan, n, rows, cols, host_io, need_vs64, nsplit);
    rc = ensure_scratch(h, L.total);
    if (rc) return rc;
    char* ws = h->ws;
    DirDev* d_dirs = reinterpret_cast<DirDev*>(ws + L.dirs);
    int* d_istart = reinterpret_cast<int*>(ws + L.istart);
    int* d_rowlo = reinterpret_cast<int*>(ws + L.rowlo);
    int* d_rowhi = reinterpret_cast<int*>(ws + L.rowhi);
    float* d_sdem = reinterpret_cast<float*>(ws + L.sdem);
    int* d_cvf = reinterpret_cast<int*>(ws + L.cvf);
    int* d_cvb = reinterpret_cast<int*>(ws + L.cvb);
    double* d_vs64 = need_vs64 ? reinterpret_cast<double*>(ws + L.vs64) : nullptr;
    double* d_part = nsplit > 1 ? reinterpret_cast<double*>(ws + L.part) : nullptr;
    unsigned* d_counter = reinterpret_cast<unsigned*>(ws + L.counter);
    const size_t cells = (size_t)rows * cols;
    if (host_io) {
        d_dem = reinterpret_cast<const float*>(ws + L.dem);
        d_out = reinterpret_cast<float*>(ws + L.out);
        TVS_CUDA(cudaMemcpyAsync((void*)d_dem, host_dem, cells * 4, cudaMemcpyHostToDevice, s), "copy dem");
    }
    // One upload per call: the direction table, then every chunk's item table.
    std::vector<int> istart(plan.istart_total, 0);
    std::vector<int> istart_at(plan.chunks.size(), 0);
    {
        int at = 0;
        for (size_t q = 0; q < plan.chunks.size(); ++q) {
            const Chunk& c = plan.chunks[q];
            istart_at[q] = at;
            for (int i = 0; i < c.k1 - c.k0; ++i) {
                const DirDev& v = plan.dev[c.k0 + i];
                istart[at + i + 1] = istart[at + i] + 2 * v.R * v.chunks;
            }
            at += c.k1 - c.k0 + 1;
        }
    }
    const size_t dir_bytes = (size_t)n * sizeof(DirDev);
    rc = upload_header(h, plan.dev.data(), dir_bytes, istart.data(), istart.size() * 4, d_dirs, d_istart, s);
    if (rc) return rc;
    const double scale = (M_PI / (2.0 * (double)n)) * (step * step);
    const float h0f = (float)h0;
    for (size_t q = 0; q < plan.chunks.size(); ++q) {
        const Chunk& c = plan.chunks[q];
        const int nd = c.k1 - c.k0;
        const int* c_istart = d_istart + istart_at[q];
        const int c_items = istart[istart_at[q] + nd];
        const DirDev* cd = d_dirs + c.k0;
        {
            Timer t(h, K_ROWMAP, s, c.rowmap_bytes);
            TVS_CUDA(launch_rowmap(cd, nd, c.max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        }
        {
            Timer t(h, K_SKEW, s, c.skew_bytes);
            TVS_CUDA(launch_skew(d_dem, rows, cols, cd, nd, c.max_tiles, d_rowlo, d_rowhi, d_sdem, s),
                     "skew launch");
        }
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        {
            Timer t(h, K_SWEEP, s, c.evals);
            TVS_CUDA(launch_sweep(cd, c_istart, nd, c_items, d_sdem, d_rowlo, d_rowhi, d_cvf, d_cvb, h0f,
                                  c.wmax, c.dmax, d_counter, h->num_sms, h->smem_optin, s),
                     "sweep launch");
        }
        {
            Timer t(h, K_UNSKEW, s, c.unskew_bytes);
            TVS_CUDA(launch_unskew(d_cvf, d_cvb, rows, cols, cd, nd, nsplit, d_part, d_vs64, d_out, q == 0,
                                   q + 1 == plan.chunks.size(), scale, s),
                     "unskew launch");
        }
        if (unskew_effective_splits(nd, nsplit) > 1) {
            const double cells_b = (double)rows * cols * 8.0 * (unskew_effective_splits(nd, nsplit) + 1);
            Timer t(h, K_FINAL, s, cells_b);
            TVS_CUDA(launch_unskew_finalize(rows, cols, nd, nsplit, d_part, d_vs64, d_out, q == 0,
                                            q + 1 == plan.chunks.size(), scale, s),
                     "unskew finalize launch");
        }
    }
    if (host_io) {
        TVS_CUDA(cudaMemcpyAsync(host_out, d_out, cells * 4, cudaMemcpyDeviceToHost, s), "copy out");
        TVS_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return TVS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// ================================================================== C ABI ==
extern "C" {

int tvs_abi_version(void) { return TVS_ABI_VERSION; }

const char* tvs_last_error(tvs_handle) { return g_err.c_str(); }

int tvs_create(tvs_handle* out, int device, size_t hbm_budget_bytes)
{
    if (!out) return fail(TVS_ERR_ARG, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaGetDeviceCount");
    }
    if (device < 0 || device >= count) return fail(TVS_ERR_ARG, "device index out of range");
    DeviceGuard g(device);
    tvs_ctx* h = new tvs_ctx();
    h->device = device;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDeviceProperties"); }
    h->num_sms = prop.multiProcessorCount;
    h->smem_optin = (int)prop.sharedMemPerBlockOptin;
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaMemGetInfo"); }
    if (hbm_budget_bytes == 0) hbm_budget_bytes = std::min<size_t>((size_t)16 << 30, (size_t)(0.6 * free_b));
    h->budget = hbm_budget_bytes;
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
    reset_stats(h);
    *out = h;
    return TVS_OK;
}

void tvs_destroy(tvs_handle h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    for (auto& p : h->pending) { cudaEventDestroy(p.start); cudaEventDestroy(p.stop); }
    if (h->ws) cudaFree(h->ws);
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->pinned_done) cudaEventDestroy(h->pinned_done);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int tvs_total_viewshed(tvs_handle h, const float* dem, int rows, int cols, double step_m,
                       double obs_height_m, int n_sectors, double max_range_m, float* out)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    if (!dem || !out) return fail(TVS_ERR_ARG, "dem or out is NULL");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    const size_t cells = (size_t)rows * cols;
    for (size_t q = 0; q < cells; ++q)
        if (!std::isfinite(dem[q])) return fail(TVS_ERR_ARG, "dem holds a non-finite value");
    DeviceGuard g(h->device);
    return run_job(h, nullptr, rows, cols, step_m, obs_height_m, n_sectors, max_range_m, nullptr,
                   h->stream, true, dem, out);
}

int tvs_total_viewshed_device(tvs_handle h, const float* d_dem, int rows, int cols, double step_m,
                              double obs_height_m, int n_sectors, double max_range_m, float* d_out,
                              void* cuda_stream)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    if (!d_dem || !d_out) return fail(TVS_ERR_ARG, "d_dem or d_out is NULL");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    const size_t bytes = (size_t)rows * cols * 4;
    const char* a = reinterpret_cast<const char*>(d_dem);
    const char* b = reinterpret_cast<const char*>(d_out);
    if (a < b + bytes && b < a + bytes) return fail(TVS_ERR_ARG, "d_dem and d_out overlap");
    DeviceGuard g(h->device);
    return run_job(h, d_dem, rows, cols, step_m, obs_height_m, n_sectors, max_range_m, d_out,
                   reinterpret_cast<cudaStream_t>(cuda_stream), false, nullptr, nullptr);
}

int tvs_direction(int n_sectors, int k, int rows, int cols, double step_m, double max_range_m,
                  tvs_direction_info* info)
{
    if (!info) return fail(TVS_ERR_ARG, "info is NULL");
    HostDir d;
    if (make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d))
        return fail(TVS_ERR_ARG, "bad direction arguments");
    info->frame = d.frame; info->m = d.m; info->H = d.H; info->W = d.W; info->D = d.D; info->R = d.R;
    info->t_fx = d.t_fx; info->t = d.t; info->g = d.g;
    info->K = d.K == LLONG_MAX ? INT64_MAX : d.K;
    return TVS_OK;
}

int64_t tvs_count_evals(int rows, int cols, int n_sectors, double step_m, double max_range_m)
{
    if (check_job(rows, cols, step_m, 0.0, n_sectors, max_range_m)) return TVS_ERR_ARG;
    int64_t E = 0;
    for (int k = 0; k < n_sectors; ++k) {
        HostDir d;
        make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d);
        E += direction_work(d).evals;
    }
    return E;
}

int tvs_debug_rowmap(tvs_handle h, int rows, int cols, int n_sectors, int k, int32_t* dest,
                     uint32_t* frac, int32_t* jlo, int32_t* jhi, int32_t* R)
{
    if (!h || !dest || !frac || !jlo || !jhi || !R) return fail(TVS_ERR_ARG, "NULL argument");
    int rc = check_job(rows, cols, 1.0, 0.0, n_sectors, 0.0);
    if (rc) return rc;
    if (k < 0 || k >= n_sectors) return fail(TVS_ERR_ARG, "k out of range");
    DeviceGuard g(h->device);
    HostDir d;
    make_direction(n_sectors, k, rows, cols, 1.0, 0.0, &d);
    DirDev v{};
    v.t_fx = d.t_fx; v.frame = d.frame; v.H = d.H; v.W = d.W; v.Wp = (d.W + 3) & ~3;
    v.D = d.D; v.R = d.R; v.K = d.W; v.row_off = 0; v.chunks = 1; v.gidx = k; v.g = (float)d.g;
    const size_t need = align256(sizeof(DirDev)) + 4 * align256((size_t)std::max(d.R, d.W) * 4);
    rc = ensure_scratch(h, need);
    if (rc) return rc;
    char* ws = h->ws;
    DirDev* d_dir = reinterpret_cast<DirDev*>(ws);
    const size_t slot = align256((size_t)std::max(d.R, d.W) * 4);
    int* d_dest = reinterpret_cast<int*>(ws + align256(sizeof(DirDev)));
    unsigned* d_frac = reinterpret_cast<unsigned*>(ws + align256(sizeof(DirDev)) + slot);
    int* d_lo = reinterpret_cast<int*>(ws + align256(sizeof(DirDev)) + 2 * slot);
    int* d_hi = reinterpret_cast<int*>(ws + align256(sizeof(DirDev)) + 3 * slot);
    cudaStream_t s = h->stream;
    TVS_CUDA(cudaMemcpyAsync(d_dir, &v, sizeof(v), cudaMemcpyHostToDevice, s), "copy direction");
    TVS_CUDA(launch_colmap(d_dir, d_dest, d_frac, s), "colmap launch");
    TVS_CUDA(launch_rowmap(d_dir, 1, d.R, d_lo, d_hi, s), "rowmap launch");
    TVS_CUDA(cudaMemcpyAsync(dest, d_dest, (size_t)d.W * 4, cudaMemcpyDeviceToHost, s), "copy dest");
    TVS_CUDA(cudaMemcpyAsync(frac, d_frac, (size_t)d.W * 4, cudaMemcpyDeviceToHost, s), "copy frac");
    TVS_CUDA(cudaMemcpyAsync(jlo, d_lo, (size_t)d.R * 4, cudaMemcpyDeviceToHost, s), "copy jlo");
    TVS_CUDA(cudaMemcpyAsync(jhi, d_hi, (size_t)d.R * 4, cudaMemcpyDeviceToHost, s), "copy jhi");
    TVS_CUDA(cudaStreamSynchronize(s), "synchronize");
    *R = d.R;
    return TVS_OK;
}

int tvs_debug_direction_cv(tvs_handle h, const float* dem, int rows, int cols, double step_m,
                           double obs_height_m, int n_sectors, double max_range_m, int k,
                           int32_t* cv, int32_t* R, int32_t* W)
{
    if (!h || !dem || !cv || !R || !W) return fail(TVS_ERR_ARG, "NULL argument");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    if (k < 0 || k >= n_sectors) return fail(TVS_ERR_ARG, "k out of range");
    DeviceGuard g(h->device);
    Plan plan;
    rc = make_plan(rows, cols, step_m, max_range_m, n_sectors, (size_t)1 << 62, &plan, k);
    if (rc) return rc;
    const Chunk& c = plan.chunks[0];
    const DirDev& v = plan.dev[k];
    const size_t cells = (size_t)rows * cols;
    const size_t o_dem = 0, o_dir = align256(cells * 4), o_is = o_dir + align256(sizeof(DirDev));
    const size_t o_lo = o_is + 256, o_hi = o_lo + align256((size_t)v.R * 4);
    const size_t o_s = o_hi + align256((size_t)v.R * 4), o_cv = o_s + align256(c.slab_elems * 4);
    const size_t o_cb = o_cv + align256(c.slab_elems * 4);
    const size_t o_cnt = o_cb + align256(c.slab_elems * 4), total = o_cnt + 256;
    rc = ensure_scratch(h, total);
    if (rc) return rc;
    char* ws = h->ws;
    cudaStream_t s = h->stream;
    float* d_dem = reinterpret_cast<float*>(ws + o_dem);
    DirDev* d_dir = reinterpret_cast<DirDev*>(ws + o_dir);
    int* d_is = reinterpret_cast<int*>(ws + o_is);
    int* d_lo = reinterpret_cast<int*>(ws + o_lo);
    int* d_hi = reinterpret_cast<int*>(ws + o_hi);
    float* d_s = reinterpret_cast<float*>(ws + o_s);
    int* d_cv = reinterpret_cast<int*>(ws + o_cv);
    int* d_cb = reinterpret_cast<int*>(ws + o_cb);
    unsigned* d_cnt = reinterpret_cast<unsigned*>(ws + o_cnt);
    const int is_host[2] = {0, 2 * v.R * v.chunks};
    TVS_CUDA(cudaMemcpyAsync(d_dem, dem, cells * 4, cudaMemcpyHostToDevice, s), "copy dem");
    TVS_CUDA(cudaMemcpyAsync(d_dir, &v, sizeof(v), cudaMemcpyHostToDevice, s), "copy direction");
    TVS_CUDA(cudaMemcpyAsync(d_is, is_host, sizeof(is_host), cudaMemcpyHostToDevice, s), "copy items");
    TVS_CUDA(launch_rowmap(d_dir, 1, v.R, d_lo, d_hi, s), "rowmap launch");
    TVS_CUDA(launch_skew(d_dem, rows, cols, d_dir, 1, c.max_tiles, d_lo, d_hi, d_s, s), "skew launch");
    TVS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), s), "reset work counter");
    TVS_CUDA(launch_sweep(d_dir, d_is, 1, is_host[1], d_s, d_lo, d_hi, d_cv, d_cb, (float)obs_height_m, v.W,
                          v.K, d_cnt, h->num_sms, h->smem_optin, s),
             "sweep launch");
    std::vector<int> slab(c.slab_elems), slabb(c.slab_elems), lo(v.R), hi(v.R);
    TVS_CUDA(cudaMemcpyAsync(slab.data(), d_cv, c.slab_elems * 4, cudaMemcpyDeviceToHost, s), "copy cv");
    TVS_CUDA(cudaMemcpyAsync(slabb.data(), d_cb, c.slab_elems * 4, cudaMemcpyDeviceToHost, s), "copy cv");
    TVS_CUDA(cudaMemcpyAsync(lo.data(), d_lo, (size_t)v.R * 4, cudaMemcpyDeviceToHost, s), "copy jlo");
    TVS_CUDA(cudaMemcpyAsync(hi.data(), d_hi, (size_t)v.R * 4, cudaMemcpyDeviceToHost, s), "copy jhi");
    TVS_CUDA(cudaStreamSynchronize(s), "synchronize");
    for (int p = 0; p < v.R; ++p)
        for (int j = 0; j < v.W; ++j)
            cv[(size_t)p * v.W + j] = (j >= lo[p] && j <= hi[p])
                                          ? slab[(size_t)p * v.Wp + j] + slabb[(size_t)p * v.Wp + j] : -1;
    *R = v.R;
    *W = v.W;
    return TVS_OK;
}

int tvs_profile_enable(tvs_handle h, int on)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    drain_pending(h);
    if (on) reset_stats(h);
    h->profiling = on != 0;
    return TVS_OK;
}

int tvs_profile_read(tvs_handle h, tvs_kernel_stats* stats, int max, int* count)
{
    if (!h || !count || (max > 0 && !stats)) return fail(TVS_ERR_ARG, "NULL argument");
    DeviceGuard g(h->device);
    drain_pending(h);
    const int n = std::min(max, (int)K_COUNT);
    for (int k = 0; k < n; ++k) stats[k] = h->stats[k];
    *count = n;
    return TVS_OK;
}

}  // extern "C"

// ================================================ no-allocation entry point ==
// For callers that cannot allocate device memory themselves: a framework
// whose caching allocator owns the whole GPU budget, or a latency-bound loop
// that must not pay the device-wide synchronisation cudaMalloc and cudaFree
// imply.  All scratch of this entry point lives in one file-scope device array
// of fixed size, reserved when the library's module is loaded and held by
// every GPU that loads it until the process exits.  It has no counterpart in
// the paper.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB
constexpr int kNoAllocMaxDirs = 1024;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
char* g_noalloc_base[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `device` (current), resolved once per
// device.  A host-side reference to g_noalloc_scratch is only a stand-in, so
// host code must pass this address to kernels.
int noalloc_scratch(int device, char** base)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(TVS_ERR_ARG, "device index out of range");
    if (!g_noalloc_base[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
        g_noalloc_base[device] = static_cast<char*>(p);
    }
    *base = g_noalloc_base[device];
    return TVS_OK;
}

}  // namespace

extern "C" int tvs_total_viewshed_device_noalloc(const float* d_dem, int rows, int cols, double step_m,
                                                 double obs_height_m, int n_sectors, double max_range_m,
                                                 float* d_out, void* cuda_stream)
{
    if (!d_dem || !d_out) return fail(TVS_ERR_ARG, "d_dem or d_out is NULL");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    if (n_sectors > kNoAllocMaxDirs)
        return fail(TVS_ERR_ARG, "the no-allocation entry point takes at most 1024 directions");
    const size_t cells = (size_t)rows * cols;
    const char* a = reinterpret_cast<const char*>(d_dem);
    const char* b = reinterpret_cast<const char*>(d_out);
    if (a < b + cells * 4 && b < a + cells * 4) return fail(TVS_ERR_ARG, "d_dem and d_out overlap");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    int device = 0;
    TVS_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    char* base = nullptr;
    rc = noalloc_scratch(device, &base);
    if (rc) return rc;
    int num_sms = 0, smem_optin = 0;
    TVS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
    TVS_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device),
             "device attribute");

    // Direction table and chunking, on the stack: chunks of consecutive
    // directions whose skewed slabs fit what the fixed part leaves.
    DirDev dirs[kNoAllocMaxDirs];
    int istart[2 * kNoAllocMaxDirs + 1];
    int chunk_k0[kNoAllocMaxDirs + 1];
    int nchunks = 0;
    const int nsplit = unskew_splits(rows, cols, std::min(n_sectors, FP32_GROUP * 64), num_sms);
    const size_t o_dirs = 0;
    const size_t o_istart = o_dirs + align256((size_t)n_sectors * sizeof(DirDev));
    const size_t o_vs64 = o_istart + align256((size_t)(2 * n_sectors + 1) * 4);
    const size_t o_part = o_vs64 + align256(cells * 8);
    const size_t o_counter = o_part + (nsplit > 1 ? align256((size_t)nsplit * cells * 8) : 0);
    const size_t o_chunk = o_counter + 256;
    if (o_chunk >= kNoAllocScratchBytes)
        return fail(TVS_ERR_OOM, "the DEM does not fit the 64 MiB no-allocation scratch");
    const size_t avail = kNoAllocScratchBytes - o_chunk;
    size_t max_rows = 0, max_slab = 0;
    {
        int k = 0;
        while (k < n_sectors) {
            size_t slab = 0, nrows = 0;
            int kk = k;
            while (kk < n_sectors) {
                HostDir d;
                make_direction(n_sectors, kk, rows, cols, step_m, max_range_m, &d);
                const size_t wp = (size_t)((d.W + 3) & ~3);
                const size_t s2 = slab + (size_t)d.R * wp, r2 = nrows + d.R;
                const size_t need = 2 * align256(r2 * 4) + 3 * align256(s2 * 4);
                if (need > avail || 2LL * (long long)r2 * sweep_chunks(d.W) > kMaxChunkItems) break;
                DirDev& v = dirs[kk];
                std::memset(&v, 0, sizeof(v));
                v.t_fx = d.t_fx; v.slab = (long long)slab; v.frame = d.frame; v.H = d.H; v.W = d.W;
                v.Wp = (int)wp; v.D = d.D; v.R = d.R;
                v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
                v.row_off = (int)nrows; v.chunks = sweep_chunks(d.W); v.gidx = kk; v.g = (float)d.g;
                slab = s2;
                nrows = r2;
                ++kk;
            }
            if (kk == k)
                return fail(TVS_ERR_OOM, "one direction of this DEM does not fit the 64 MiB no-allocation scratch");
            chunk_k0[nchunks++] = k;
            max_rows = std::max(max_rows, nrows);
            max_slab = std::max(max_slab, slab);
            k = kk;
        }
        chunk_k0[nchunks] = n_sectors;
        int at = 0;
        for (int c = 0; c < nchunks; ++c) {
            istart[at] = 0;
            for (int q = chunk_k0[c]; q < chunk_k0[c + 1]; ++q) {
                istart[at + 1] = istart[at] + 2 * dirs[q].R * dirs[q].chunks;
                ++at;
            }
            ++at;
        }
    }
    DirDev* d_dirs = reinterpret_cast<DirDev*>(base + o_dirs);
    int* d_istart = reinterpret_cast<int*>(base + o_istart);
    double* d_vs64 = reinterpret_cast<double*>(base + o_vs64);
    double* d_part = nsplit > 1 ? reinterpret_cast<double*>(base + o_part) : nullptr;
    unsigned* d_counter = reinterpret_cast<unsigned*>(base + o_counter);
    int* d_rowlo = reinterpret_cast<int*>(base + o_chunk);
    int* d_rowhi = reinterpret_cast<int*>(base + o_chunk + align256(max_rows * 4));
    const size_t o_sdem = o_chunk + 2 * align256(max_rows * 4);
    float* d_sdem = reinterpret_cast<float*>(base + o_sdem);
    int* d_cvf = reinterpret_cast<int*>(base + o_sdem + align256(max_slab * 4));
    int* d_cvb = reinterpret_cast<int*>(base + o_sdem + 2 * align256(max_slab * 4));

    // Stack tables are staged by the runtime before these calls return.
    TVS_CUDA(cudaMemcpyAsync(d_dirs, dirs, (size_t)n_sectors * sizeof(DirDev), cudaMemcpyHostToDevice, s),
             "copy direction table");
    TVS_CUDA(cudaMemcpyAsync(d_istart, istart, (size_t)(n_sectors + nchunks) * 4, cudaMemcpyHostToDevice, s),
             "copy item table");
    const double scale = (M_PI / (2.0 * (double)n_sectors)) * (step_m * step_m);
    int at = 0;
    for (int c = 0; c < nchunks; ++c) {
        const int k0 = chunk_k0[c], nd = chunk_k0[c + 1] - k0;
        int max_R = 0, max_tiles = 0, wmax = 0, dmax = 0;
        for (int q = k0; q < k0 + nd; ++q) {
            dmax = std::max(dmax, dirs[q].K);
            max_R = std::max(max_R, dirs[q].R);
            max_tiles = std::max(max_tiles, ((dirs[q].R + SKEW_TP - 1) / SKEW_TP) * ((dirs[q].W + SKEW_TJ - 1) / SKEW_TJ));
            wmax = std::max(wmax, dirs[q].W);
        }
        const DirDev* cd = d_dirs + k0;
        const int first = c == 0, last = c + 1 == nchunks;
        TVS_CUDA(launch_rowmap(cd, nd, max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        TVS_CUDA(launch_skew(d_dem, rows, cols, cd, nd, max_tiles, d_rowlo, d_rowhi, d_sdem, s), "skew launch");
        // the shared array keeps the previous call's contents: the work counter must start at zero
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        TVS_CUDA(launch_sweep(cd, d_istart + at, nd, istart[at + nd], d_sdem, d_rowlo, d_rowhi, d_cvf, d_cvb,
                              (float)obs_height_m, wmax, dmax, d_counter, num_sms, smem_optin, s),
                 "sweep launch");
        TVS_CUDA(launch_unskew(d_cvf, d_cvb, rows, cols, cd, nd, nsplit, d_part, d_vs64, d_out, first, last,
                               scale, s),
                 "unskew launch");
        TVS_CUDA(launch_unskew_finalize(rows, cols, nd, nsplit, d_part, d_vs64, d_out, first, last, scale, s),
                 "unskew finalize launch");
        at += nd + 1;
    }
    return TVS_OK;
}
