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

// Tunable launch choices (see tvs_tuning in tvs.h).
struct Tuning {
    int small_pov_below_w = 768;   // walk axes shorter than this use SMALL_POV groups
    int sweep_max_warps = 0;       // 0 = as many as shared memory allows (up to SWEEP_MAX_WARPS)
    int unskew_ctas_per_sm = 2;    // split a chunk's directions below this many unskew CTAs per SM
};

int pov_for(const Tuning& tn, int W) { return W < tn.small_pov_below_w ? SMALL_POV : LARGE_POV; }

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
    Tuning tuning;
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
        if (h && h->profiling && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
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

// A DEM of a call: device pointers and parameters.
struct JobSpec {
    const float* dem;
    float* out;
    int rows, cols, n;
    double step, h0, max_range;
};

// A planned chunk: the consecutive (job, direction) instances [i0, i1).
struct Chunk {
    int i0, i1;
    size_t slab_elems;       // sum of R * Wp over the chunk
    long long rows;          // sum of R
    int items;               // sweep warp items
    int max_R, max_tiles, wmax, dmax;
    int cj_beg, ncj;         // the chunk's entries of the chunk-job table
    int total_tiles, max_split;
    long long total_cells, part_elems;
    int istart_at;           // offset of the chunk's item table
    double evals, skew_bytes, unskew_bytes, rowmap_bytes, final_bytes;
};

struct BatchPlan {
    std::vector<JobSpec> jobs;
    std::vector<int> inst_job, inst_k;   // per instance
    std::vector<HostDir> hdirs;          // per instance
    std::vector<DirDev> dirs;            // per instance (slab / row offsets relative to its chunk)
    std::vector<Chunk> chunks;
    std::vector<ChunkJob> cj;            // every chunk's job entries, chunk after chunk
    std::vector<int> istart;             // every chunk's item table
    std::vector<long long> vs64_off;     // per job, -1 when the job lives in one chunk
    long long vs64_elems = 0;
    size_t max_slab = 0;
    long long max_rows = 0, max_part = 0;
    double evals = 0;
};

size_t chunk_bytes(size_t slab, long long rows, int ninst)
{
    // skewed heights + forward measures + backward measures, row tables, item table
    return align256(slab * 4) * 3 + align256((size_t)rows * 4) * 2 + align256((size_t)(ninst + 1) * 4);
}

// Upper bound of the FP64 partials of a split unskew: splits only happen when
// a chunk's jobs have fewer than 2 cell tiles per SM, so the partials cover at
// most about 4 tiles of 1024 cells per SM.
size_t part_bound(int num_sms) { return align256((size_t)(4 * num_sms + 4) * UNSKEW_TI * UNSKEW_TJ * 8); }

// Plans the instances of `jobs` (job after job, directions in order) into
// chunks whose scratch fits `avail` bytes.  Cuts fall on multiples of
// FP32_GROUP directions of a job where possible, so a job's FP32 group sums do
// not depend on the chunking.  only_k >= 0 keeps only direction only_k of a
// single job (test hook).
int plan_batch(const std::vector<JobSpec>& jobs, size_t avail, int num_sms, const Tuning& tn, BatchPlan* plan,
               int only_k = -1)
{
    plan->jobs = jobs;
    for (int j = 0; j < (int)jobs.size(); ++j) {
        const JobSpec& J = jobs[j];
        for (int k = 0; k < J.n; ++k) {
            if (only_k >= 0 && k != only_k) continue;
            HostDir d;
            if (make_direction(J.n, k, J.rows, J.cols, J.step, J.max_range, &d))
                return fail(TVS_ERR_ARG, "bad direction arguments");
            plan->hdirs.push_back(d);
            plan->inst_job.push_back(j);
            plan->inst_k.push_back(k);
        }
    }
    const int ninst = (int)plan->hdirs.size();
    plan->dirs.resize(ninst);
    int i = 0;
    while (i < ninst) {
        size_t slab = 0, slab_ok = 0;
        long long nrows = 0, rows_ok = 0, items = 0;
        int ii = i, last_ok = -1;
        while (ii < ninst) {
            const HostDir& d = plan->hdirs[ii];
            const size_t wp = (size_t)((d.W + 3) & ~3);
            const size_t s2 = slab + (size_t)d.R * wp;
            const long long r2 = nrows + d.R;
            const long long it2 = items + 2LL * d.R * sweep_chunks(d.W, pov_for(tn, d.W));
            if (ii > i && (chunk_bytes(s2, r2, ii - i + 1) > avail || ii - i >= kMaxChunkDirs ||
                           it2 > kMaxChunkItems))
                break;
            slab = s2;
            nrows = r2;
            items = it2;
            ++ii;
            const int kk = plan->inst_k[ii - 1], jj = plan->inst_job[ii - 1];
            if ((kk + 1) % FP32_GROUP == 0 || kk + 1 == jobs[jj].n || ii == ninst) {
                last_ok = ii; slab_ok = slab; rows_ok = nrows;
            }
        }
        if (chunk_bytes(slab, nrows, ii - i) > avail)
            return fail(TVS_ERR_OOM, "one direction does not fit the HBM budget");
        if (last_ok > i && ii < ninst) { ii = last_ok; slab = slab_ok; nrows = rows_ok; }
        Chunk c{};
        c.i0 = i;
        c.i1 = ii;
        plan->chunks.push_back(c);
        i = ii;
    }
    const int njobs = (int)jobs.size();
    std::vector<int> first_chunk(njobs, -1), last_chunk(njobs, -1);
    for (int q = 0; q < (int)plan->chunks.size(); ++q)
        for (int t = plan->chunks[q].i0; t < plan->chunks[q].i1; ++t) {
            const int j = plan->inst_job[t];
            if (first_chunk[j] < 0) first_chunk[j] = q;
            last_chunk[j] = q;
        }
    plan->vs64_off.assign(njobs, -1);
    for (int j = 0; j < njobs; ++j)
        if (first_chunk[j] >= 0 && first_chunk[j] != last_chunk[j]) {
            plan->vs64_off[j] = plan->vs64_elems;
            plan->vs64_elems += (long long)jobs[j].rows * jobs[j].cols;
        }
    for (int q = 0; q < (int)plan->chunks.size(); ++q) {
        Chunk& c = plan->chunks[q];
        size_t off = 0;
        long long roff = 0;
        c.istart_at = (int)plan->istart.size();
        plan->istart.push_back(0);
        for (int t = c.i0; t < c.i1; ++t) {
            const HostDir& d = plan->hdirs[t];
            const JobSpec& J = jobs[plan->inst_job[t]];
            DirDev& v = plan->dirs[t];
            std::memset(&v, 0, sizeof(v));
            v.t_fx = d.t_fx;
            v.slab = (long long)off;
            v.frame = d.frame; v.H = d.H; v.W = d.W; v.Wp = (d.W + 3) & ~3;
            v.D = d.D; v.R = d.R;
            v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
            v.row_off = (int)roff;
            v.pov = pov_for(tn, d.W);
            v.chunks = sweep_chunks(d.W, v.pov);
            v.gidx = plan->inst_k[t];
            v.job = plan->inst_job[t];
            v.g = (float)d.g;
            v.h0 = (float)J.h0;
            off += (size_t)d.R * v.Wp;
            roff += d.R;
            c.items += 2 * d.R * v.chunks;
            plan->istart.push_back(c.items);
            c.max_R = std::max(c.max_R, d.R);
            c.max_tiles = std::max(c.max_tiles, ((d.R + SKEW_TP - 1) / SKEW_TP) * ((d.W + SKEW_TJ - 1) / SKEW_TJ));
            c.wmax = std::max(c.wmax, d.W);
            c.dmax = std::max(c.dmax, v.K);
            const DirWork w = direction_work(d);
            c.evals += (double)w.evals;
            c.skew_bytes += 4.0 * J.rows * J.cols + 4.0 * (double)w.samples;
            c.unskew_bytes += 8.0 * (double)w.samples;
            c.rowmap_bytes += 8.0 * d.R;
        }
        c.slab_elems = off;
        c.rows = roff;
        plan->evals += c.evals;
        plan->max_slab = std::max(plan->max_slab, off);
        plan->max_rows = std::max(plan->max_rows, roff);
        // the chunk's jobs, in instance order (a job's instances are contiguous)
        c.cj_beg = (int)plan->cj.size();
        long long tiles = 0;
        for (int t = c.i0; t < c.i1;) {
            int u = t;
            while (u < c.i1 && plan->inst_job[u] == plan->inst_job[t]) ++u;
            tiles += unskew_tiles(jobs[plan->inst_job[t]].rows, jobs[plan->inst_job[t]].cols);
            t = u;
        }
        c.total_tiles = (int)tiles;
        int tile_beg = 0;
        long long cell_beg = 0;
        for (int t = c.i0; t < c.i1;) {
            int u = t;
            const int j = plan->inst_job[t];
            while (u < c.i1 && plan->inst_job[u] == j) ++u;
            const JobSpec& J = jobs[j];
            ChunkJob e{};
            e.job = j;
            e.dbeg = t - c.i0;
            e.dcnt = u - t;
            e.tile_beg = tile_beg;
            e.tiles_x = unskew_tiles_x(J.cols);
            e.first = first_chunk[j] == q;
            e.last = last_chunk[j] == q;
            const int want = unskew_splits(tiles, e.dcnt, num_sms, tn.unskew_ctas_per_sm);
            e.per_split = unskew_per_split(e.dcnt, want);
            e.nsplit = unskew_effective_splits(e.dcnt, want);
            e.cell_beg = cell_beg;
            const long long cells = (long long)J.rows * J.cols;
            e.part_off = -1;
            if (e.nsplit > 1) { e.part_off = c.part_elems; c.part_elems += e.nsplit * cells; }
            c.max_split = std::max(c.max_split, e.nsplit);
            c.total_cells += cells;
            c.final_bytes += e.nsplit > 1 ? 8.0 * cells * (e.nsplit + 1) : 0.0;
            c.unskew_bytes += (e.first ? 0.0 : 8.0 * cells) + (e.last ? 4.0 * cells : 8.0 * cells);
            tile_beg += unskew_tiles(J.rows, J.cols);
            cell_beg += cells;
            plan->cj.push_back(e);
            t = u;
        }
        c.ncj = (int)plan->cj.size() - c.cj_beg;
        plan->max_part = std::max(plan->max_part, c.part_elems);
    }
    return TVS_OK;
}

// Scratch layout of a planned batch (byte offsets).  The header (directions,
// jobs, chunk-job entries, item tables) is one contiguous block, uploaded with
// one copy.
struct Layout {
    size_t hdr, dirs, jobs, cj, istart, hdr_bytes;
    size_t io_dem, io_out, counter, vs64, part, rowlo, rowhi, sdem, cvf, cvb, total;
};

Layout make_layout(const BatchPlan& plan, bool host_io)
{
    Layout L{};
    size_t o = 0;
    L.hdr = o;
    L.dirs = o;    o += align256(plan.dirs.size() * sizeof(DirDev));
    L.jobs = o;    o += align256(plan.jobs.size() * sizeof(JobDev));
    L.cj = o;      o += align256(plan.cj.size() * sizeof(ChunkJob));
    L.istart = o;  o += align256(plan.istart.size() * 4);
    L.hdr_bytes = o - L.hdr;
    const size_t cells = host_io ? (size_t)plan.jobs[0].rows * plan.jobs[0].cols : 0;
    L.io_dem = o;  o += align256(cells * 4);
    L.io_out = o;  o += align256(cells * 4);
    L.counter = o; o += 256;
    L.vs64 = o;    o += align256((size_t)plan.vs64_elems * 8);
    L.part = o;    o += align256((size_t)plan.max_part * 8);
    L.rowlo = o;   o += align256((size_t)plan.max_rows * 4);
    L.rowhi = o;   o += align256((size_t)plan.max_rows * 4);
    L.sdem = o;    o += align256(plan.max_slab * 4);
    L.cvf = o;     o += align256(plan.max_slab * 4);
    L.cvb = o;     o += align256(plan.max_slab * 4);
    L.total = o;
    return L;
}

// Bytes a batch needs besides its chunks' slabs (header, host copies of a
// single job, FP64 totals of every job, partials bound, counter).
size_t fixed_bytes(const std::vector<JobSpec>& jobs, bool host_io, int num_sms)
{
    size_t ninst = 0, cells = 0;
    for (const JobSpec& J : jobs) { ninst += J.n; cells += (size_t)J.rows * J.cols; }
    size_t b = align256(ninst * sizeof(DirDev)) + align256(jobs.size() * sizeof(JobDev)) +
               align256((jobs.size() + ninst) * sizeof(ChunkJob)) + align256((2 * ninst + 1) * 4) + 4096;
    if (host_io) b += 2 * align256((size_t)jobs[0].rows * jobs[0].cols * 4);
    return b + align256(cells * 8) + part_bound(num_sms);
}

// Host image of the header for the scratch at `base`.
void build_header(const BatchPlan& plan, const Layout& L, char* base, bool host_io, std::vector<char>* img)
{
    img->assign(L.hdr_bytes, 0);
    std::memcpy(img->data() + (L.dirs - L.hdr), plan.dirs.data(), plan.dirs.size() * sizeof(DirDev));
    std::vector<JobDev> jd(plan.jobs.size());
    for (size_t j = 0; j < plan.jobs.size(); ++j) {
        const JobSpec& J = plan.jobs[j];
        jd[j].dem = host_io ? reinterpret_cast<const float*>(base + L.io_dem) : J.dem;
        jd[j].out = host_io ? reinterpret_cast<float*>(base + L.io_out) : J.out;
        jd[j].vs64 = plan.vs64_off[j] >= 0 ? reinterpret_cast<double*>(base + L.vs64) + plan.vs64_off[j] : nullptr;
        jd[j].scale = (M_PI / (2.0 * (double)J.n)) * (J.step * J.step);
        jd[j].rows = J.rows;
        jd[j].cols = J.cols;
    }
    std::memcpy(img->data() + (L.jobs - L.hdr), jd.data(), jd.size() * sizeof(JobDev));
    std::memcpy(img->data() + (L.cj - L.hdr), plan.cj.data(), plan.cj.size() * sizeof(ChunkJob));
    std::memcpy(img->data() + (L.istart - L.hdr), plan.istart.data(), plan.istart.size() * 4);
}

// Enqueue every chunk of a planned batch whose header already sits at base +
// L.hdr: per chunk row map -> skew -> sweep -> unskew (-> finalize).
int enqueue_chunks(tvs_ctx* h, const BatchPlan& plan, const Layout& L, char* base, int num_sms, int smem_optin,
                   int max_warps, cudaStream_t s)
{
    const DirDev* d_dirs = reinterpret_cast<const DirDev*>(base + L.dirs);
    const JobDev* d_jobs = reinterpret_cast<const JobDev*>(base + L.jobs);
    const ChunkJob* d_cj = reinterpret_cast<const ChunkJob*>(base + L.cj);
    const int* d_istart = reinterpret_cast<const int*>(base + L.istart);
    unsigned* d_counter = reinterpret_cast<unsigned*>(base + L.counter);
    double* d_part = reinterpret_cast<double*>(base + L.part);
    int* d_rowlo = reinterpret_cast<int*>(base + L.rowlo);
    int* d_rowhi = reinterpret_cast<int*>(base + L.rowhi);
    float* d_sdem = reinterpret_cast<float*>(base + L.sdem);
    int* d_cvf = reinterpret_cast<int*>(base + L.cvf);
    int* d_cvb = reinterpret_cast<int*>(base + L.cvb);
    for (const Chunk& c : plan.chunks) {
        const int nd = c.i1 - c.i0;
        const DirDev* cd = d_dirs + c.i0;
        {
            Timer t(h, K_ROWMAP, s, c.rowmap_bytes);
            TVS_CUDA(launch_rowmap(cd, nd, c.max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        }
        {
            Timer t(h, K_SKEW, s, c.skew_bytes);
            TVS_CUDA(launch_skew(d_jobs, cd, nd, c.max_tiles, d_sdem, s), "skew launch");
        }
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        {
            Timer t(h, K_SWEEP, s, c.evals);
            TVS_CUDA(launch_sweep(cd, d_istart + c.istart_at, nd, c.items, d_sdem, d_rowlo, d_rowhi, d_cvf, d_cvb,
                                  c.wmax, c.dmax, d_counter, num_sms, smem_optin, max_warps, s),
                     "sweep launch");
        }
        {
            Timer t(h, K_UNSKEW, s, c.unskew_bytes);
            TVS_CUDA(launch_unskew(d_cvf, d_cvb, d_jobs, cd, d_cj + c.cj_beg, c.ncj, c.total_tiles, c.max_split,
                                   d_part, s),
                     "unskew launch");
        }
        if (c.max_split > 1) {
            Timer t(h, K_FINAL, s, c.final_bytes);
            TVS_CUDA(launch_unskew_finalize(d_jobs, d_cj + c.cj_beg, c.ncj, c.total_cells, d_part, s),
                     "unskew finalize launch");
        }
    }
    return TVS_OK;
}

// Copy a header image to the device through the handle's pinned staging
// buffer.  The buffer is reused by the next call only after the copy that
// read it has run (event), so the host never blocks on earlier GPU work.
int upload_header(tvs_ctx* h, const std::vector<char>& img, void* dst, cudaStream_t s)
{
    if (h->pinned_done) TVS_CUDA(cudaEventSynchronize(h->pinned_done), "wait for staging buffer");
    if (img.size() > h->pinned_bytes) {
        if (h->pinned) cudaFreeHost(h->pinned);
        h->pinned = nullptr;
        h->pinned_bytes = 0;
        TVS_CUDA(cudaHostAlloc((void**)&h->pinned, img.size(), cudaHostAllocDefault), "cudaHostAlloc");
        h->pinned_bytes = img.size();
    }
    std::memcpy(h->pinned, img.data(), img.size());
    TVS_CUDA(cudaMemcpyAsync(dst, h->pinned, img.size(), cudaMemcpyHostToDevice, s), "copy tables");
    if (!h->pinned_done) TVS_CUDA(cudaEventCreateWithFlags(&h->pinned_done, cudaEventDisableTiming), "event");
    TVS_CUDA(cudaEventRecord(h->pinned_done, s), "record staging event");
    return TVS_OK;
}

// Plan, size the scratch and enqueue a batch on the handle.  With host_io the
// single job's DEM is copied in from host memory and its map copied back.
int run_batch(tvs_ctx* h, const std::vector<JobSpec>& jobs, cudaStream_t s, bool host_io, const float* host_dem,
              float* host_out)
{
    const size_t fixed = fixed_bytes(jobs, host_io, h->num_sms);
    if (fixed >= h->budget) return fail(TVS_ERR_OOM, "the DEMs do not fit the HBM budget");
    BatchPlan plan;
    int rc = plan_batch(jobs, h->budget - fixed, h->num_sms, h->tuning, &plan);
    if (rc) return rc;
    const Layout L = make_layout(plan, host_io);
    rc = ensure_scratch(h, L.total);
    if (rc) return rc;
    char* base = h->ws;
    std::vector<char> img;
    build_header(plan, L, base, host_io, &img);
    if (host_io) {
        const size_t bytes = (size_t)jobs[0].rows * jobs[0].cols * 4;
        TVS_CUDA(cudaMemcpyAsync(base + L.io_dem, host_dem, bytes, cudaMemcpyHostToDevice, s), "copy dem");
    }
    rc = upload_header(h, img, base + L.hdr, s);
    if (rc) return rc;
    rc = enqueue_chunks(h, plan, L, base, h->num_sms, h->smem_optin, h->tuning.sweep_max_warps, s);
    if (rc) return rc;
    if (host_io) {
        const size_t bytes = (size_t)jobs[0].rows * jobs[0].cols * 4;
        TVS_CUDA(cudaMemcpyAsync(host_out, base + L.io_out, bytes, cudaMemcpyDeviceToHost, s), "copy out");
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
    const std::vector<JobSpec> jobs{JobSpec{nullptr, nullptr, rows, cols, n_sectors, step_m, obs_height_m,
                                            max_range_m}};
    return run_batch(h, jobs, h->stream, true, dem, out);
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
    const std::vector<JobSpec> jobs{JobSpec{d_dem, d_out, rows, cols, n_sectors, step_m, obs_height_m,
                                            max_range_m}};
    return run_batch(h, jobs, reinterpret_cast<cudaStream_t>(cuda_stream), false, nullptr, nullptr);
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
    const std::vector<JobSpec> jobs{JobSpec{nullptr, nullptr, rows, cols, n_sectors, step_m, obs_height_m,
                                            max_range_m}};
    BatchPlan plan;
    rc = plan_batch(jobs, (size_t)1 << 62, h->num_sms, h->tuning, &plan, k);
    if (rc) return rc;
    const Chunk& c = plan.chunks[0];
    const DirDev& v = plan.dirs[0];
    const Layout L = make_layout(plan, true);
    rc = ensure_scratch(h, L.total);
    if (rc) return rc;
    char* ws = h->ws;
    cudaStream_t s = h->stream;
    std::vector<char> img;
    build_header(plan, L, ws, true, &img);
    const size_t cells = (size_t)rows * cols;
    TVS_CUDA(cudaMemcpyAsync(ws + L.io_dem, dem, cells * 4, cudaMemcpyHostToDevice, s), "copy dem");
    rc = upload_header(h, img, ws + L.hdr, s);
    if (rc) return rc;
    const DirDev* d_dir = reinterpret_cast<const DirDev*>(ws + L.dirs);
    const JobDev* d_jobs = reinterpret_cast<const JobDev*>(ws + L.jobs);
    int* d_lo = reinterpret_cast<int*>(ws + L.rowlo);
    int* d_hi = reinterpret_cast<int*>(ws + L.rowhi);
    float* d_s = reinterpret_cast<float*>(ws + L.sdem);
    int* d_cv = reinterpret_cast<int*>(ws + L.cvf);
    int* d_cb = reinterpret_cast<int*>(ws + L.cvb);
    unsigned* d_cnt = reinterpret_cast<unsigned*>(ws + L.counter);
    TVS_CUDA(launch_rowmap(d_dir, 1, v.R, d_lo, d_hi, s), "rowmap launch");
    TVS_CUDA(launch_skew(d_jobs, d_dir, 1, c.max_tiles, d_s, s), "skew launch");
    TVS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), s), "reset work counter");
    TVS_CUDA(launch_sweep(d_dir, reinterpret_cast<const int*>(ws + L.istart), 1, c.items, d_s, d_lo, d_hi, d_cv,
                          d_cb, v.W, v.K, d_cnt, h->num_sms, h->smem_optin, h->tuning.sweep_max_warps, s),
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
    ChunkJob cjs[kNoAllocMaxDirs];
    int nchunks = 0;
    const int tiles = unskew_tiles(rows, cols);
    const Tuning tn;
    const int nsplit_max = unskew_splits(tiles, n_sectors, num_sms, tn.unskew_ctas_per_sm);
    const size_t o_dirs = 0;
    const size_t o_job = o_dirs + align256((size_t)n_sectors * sizeof(DirDev));
    const size_t o_cj = o_job + align256(sizeof(JobDev));
    const size_t o_istart = o_cj + align256((size_t)n_sectors * sizeof(ChunkJob));
    const size_t o_vs64 = o_istart + align256((size_t)(2 * n_sectors + 1) * 4);
    const size_t o_part = o_vs64 + align256(cells * 8);
    const size_t o_counter = o_part + (nsplit_max > 1 ? align256((size_t)nsplit_max * cells * 8) : 0);
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
                if (need > avail || 2LL * (long long)r2 * sweep_chunks(d.W, pov_for(tn, d.W)) > kMaxChunkItems) break;
                DirDev& v = dirs[kk];
                std::memset(&v, 0, sizeof(v));
                v.t_fx = d.t_fx; v.slab = (long long)slab; v.frame = d.frame; v.H = d.H; v.W = d.W;
                v.Wp = (int)wp; v.D = d.D; v.R = d.R;
                v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
                v.pov = pov_for(tn, d.W);
                v.row_off = (int)nrows; v.chunks = sweep_chunks(d.W, v.pov); v.gidx = kk; v.job = 0;
                v.g = (float)d.g; v.h0 = (float)obs_height_m;
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
            const int nd = chunk_k0[c + 1] - chunk_k0[c];
            ChunkJob& e = cjs[c];
            std::memset(&e, 0, sizeof(e));
            e.job = 0; e.dbeg = 0; e.dcnt = nd; e.tile_beg = 0; e.tiles_x = unskew_tiles_x(cols);
            e.first = c == 0; e.last = c + 1 == nchunks;
            const int want = unskew_splits(tiles, nd, num_sms, tn.unskew_ctas_per_sm);
            e.per_split = unskew_per_split(nd, want);
            e.nsplit = unskew_effective_splits(nd, want);
            e.cell_beg = 0;
            e.part_off = 0;
        }
    }
    JobDev job;
    job.dem = d_dem;
    job.out = d_out;
    job.vs64 = nchunks > 1 ? reinterpret_cast<double*>(base + o_vs64) : nullptr;
    job.scale = (M_PI / (2.0 * (double)n_sectors)) * (step_m * step_m);
    job.rows = rows;
    job.cols = cols;
    DirDev* d_dirs = reinterpret_cast<DirDev*>(base + o_dirs);
    JobDev* d_job = reinterpret_cast<JobDev*>(base + o_job);
    ChunkJob* d_cj = reinterpret_cast<ChunkJob*>(base + o_cj);
    int* d_istart = reinterpret_cast<int*>(base + o_istart);
    double* d_part = reinterpret_cast<double*>(base + o_part);
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
    TVS_CUDA(cudaMemcpyAsync(d_job, &job, sizeof(JobDev), cudaMemcpyHostToDevice, s), "copy job table");
    TVS_CUDA(cudaMemcpyAsync(d_cj, cjs, (size_t)nchunks * sizeof(ChunkJob), cudaMemcpyHostToDevice, s),
             "copy chunk table");
    TVS_CUDA(cudaMemcpyAsync(d_istart, istart, (size_t)(n_sectors + nchunks) * 4, cudaMemcpyHostToDevice, s),
             "copy item table");
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
        TVS_CUDA(launch_rowmap(cd, nd, max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        TVS_CUDA(launch_skew(d_job, cd, nd, max_tiles, d_sdem, s), "skew launch");
        // the shared array keeps the previous call's contents: the work counter must start at zero
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        TVS_CUDA(launch_sweep(cd, d_istart + at, nd, istart[at + nd], d_sdem, d_rowlo, d_rowhi, d_cvf, d_cvb,
                              wmax, dmax, d_counter, num_sms, smem_optin, tn.sweep_max_warps, s),
                 "sweep launch");
        TVS_CUDA(launch_unskew(d_cvf, d_cvb, d_job, cd, d_cj + c, 1, tiles, cjs[c].nsplit, d_part, s),
                 "unskew launch");
        if (cjs[c].nsplit > 1)
            TVS_CUDA(launch_unskew_finalize(d_job, d_cj + c, 1, (long long)cells, d_part, s),
                     "unskew finalize launch");
        at += nd + 1;
    }
    return TVS_OK;
}

// ================================================================ batches ==
namespace {

int check_jobs(const tvs_job* jobs, int njobs, std::vector<JobSpec>* out)
{
    if (!jobs || njobs < 1) return fail(TVS_ERR_ARG, "jobs is NULL or njobs < 1");
    for (int j = 0; j < njobs; ++j) {
        const tvs_job& J = jobs[j];
        const std::string pre = "job " + std::to_string(j) + ": ";
        if (!J.d_dem || !J.d_out) return fail(TVS_ERR_ARG, pre + "d_dem or d_out is NULL");
        const int rc = check_job(J.rows, J.cols, J.step_m, J.obs_height_m, J.n_sectors, J.max_range_m);
        if (rc) return fail(rc, pre + g_err);
        const size_t bytes = (size_t)J.rows * J.cols * 4;
        const char* a = reinterpret_cast<const char*>(J.d_dem);
        const char* b = reinterpret_cast<const char*>(J.d_out);
        if (a < b + bytes && b < a + bytes) return fail(TVS_ERR_ARG, pre + "d_dem and d_out overlap");
        out->push_back(JobSpec{J.d_dem, J.d_out, J.rows, J.cols, J.n_sectors, J.step_m, J.obs_height_m,
                               J.max_range_m});
    }
    return TVS_OK;
}

}  // namespace

struct tvs_batch {
    tvs_ctx* h = nullptr;
    BatchPlan plan;
    Layout L{};
    char* ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
};

extern "C" {

int tvs_total_viewshed_batch(tvs_handle h, const tvs_job* jobs, int njobs, void* cuda_stream)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    std::vector<JobSpec> specs;
    int rc = check_jobs(jobs, njobs, &specs);
    if (rc) return rc;
    DeviceGuard g(h->device);
    return run_batch(h, specs, reinterpret_cast<cudaStream_t>(cuda_stream), false, nullptr, nullptr);
}

void tvs_batch_destroy(tvs_batch_handle b)
{
    if (!b) return;
    DeviceGuard g(b->h->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

int tvs_batch_create(tvs_handle h, const tvs_job* jobs, int njobs, size_t hbm_budget_bytes,
                     tvs_batch_handle* out)
{
    if (!h || !out) return fail(TVS_ERR_ARG, "handle or out is NULL");
    *out = nullptr;
    std::vector<JobSpec> specs;
    int rc = check_jobs(jobs, njobs, &specs);
    if (rc) return rc;
    DeviceGuard g(h->device);
    const size_t budget = hbm_budget_bytes ? hbm_budget_bytes : h->budget;
    const size_t fixed = fixed_bytes(specs, false, h->num_sms);
    if (fixed >= budget) return fail(TVS_ERR_OOM, "the DEMs do not fit the HBM budget");
    tvs_batch* b = new tvs_batch();
    b->h = h;
    rc = plan_batch(specs, budget - fixed, h->num_sms, h->tuning, &b->plan);
    if (rc) { delete b; return rc; }
    b->L = make_layout(b->plan, false);
    cudaError_t e = cudaMalloc(&b->ws, b->L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->ws = nullptr;
        tvs_batch_destroy(b);
        return fail(TVS_ERR_OOM, std::string("cudaMalloc of batch scratch failed: ") + cudaGetErrorString(e));
    }
    std::vector<char> img;
    build_header(b->plan, b->L, b->ws, false, &img);
    e = cudaMemcpy(b->ws + b->L.hdr, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { tvs_batch_destroy(b); return cuda_fail(e, "copy batch tables"); }
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { tvs_batch_destroy(b); return cuda_fail(e, "cudaStreamCreate"); }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cap); tvs_batch_destroy(b); return cuda_fail(e, "begin capture"); }
    rc = enqueue_chunks(nullptr, b->plan, b->L, b->ws, h->num_sms, h->smem_optin, h->tuning.sweep_max_warps, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    b->graph = graph;
    if (rc) { tvs_batch_destroy(b); return rc; }
    if (e != cudaSuccess) { tvs_batch_destroy(b); return cuda_fail(e, "end capture"); }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) { b->exec = nullptr; tvs_batch_destroy(b); return cuda_fail(e, "instantiate graph"); }
    for (const Chunk& c : b->plan.chunks) b->kernels += 4 + (c.max_split > 1 ? 1 : 0);
    *out = b;
    return TVS_OK;
}

int tvs_batch_launch(tvs_batch_handle b, void* cuda_stream)
{
    if (!b) return fail(TVS_ERR_ARG, "batch is NULL");
    DeviceGuard g(b->h->device);
    TVS_CUDA(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(cuda_stream)), "graph launch");
    return TVS_OK;
}

int tvs_batch_get_info(tvs_batch_handle b, tvs_batch_info* info)
{
    if (!b || !info) return fail(TVS_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->jobs = (int32_t)b->plan.jobs.size();
    info->chunks = (int32_t)b->plan.chunks.size();
    info->kernels_per_launch = b->kernels;
    info->evals = b->plan.evals;
    info->scratch_bytes = (double)b->L.total;
    return TVS_OK;
}

}  // extern "C"

// ============================================================== tuning ==
extern "C" {

int tvs_get_tuning(tvs_handle h, tvs_tuning* t)
{
    if (!h || !t) return fail(TVS_ERR_ARG, "NULL argument");
    std::memset(t, 0, sizeof(*t));
    t->small_pov_below_w = h->tuning.small_pov_below_w;
    t->sweep_max_warps = h->tuning.sweep_max_warps;
    t->unskew_ctas_per_sm = h->tuning.unskew_ctas_per_sm;
    return TVS_OK;
}

int tvs_set_tuning(tvs_handle h, const tvs_tuning* t)
{
    if (!h || !t) return fail(TVS_ERR_ARG, "NULL argument");
    if (t->small_pov_below_w < 0 || t->sweep_max_warps < 0 || t->sweep_max_warps > SWEEP_MAX_WARPS ||
        t->unskew_ctas_per_sm < 1)
        return fail(TVS_ERR_ARG, "tuning out of range");
    h->tuning.small_pov_below_w = t->small_pov_below_w;
    h->tuning.sweep_max_warps = t->sweep_max_warps;
    h->tuning.unskew_ctas_per_sm = t->unskew_ctas_per_sm;
    return TVS_OK;
}

int tvs_autotune(tvs_handle h, const tvs_job* jobs, int njobs, tvs_tuning* best, double* best_ms)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    std::vector<JobSpec> specs;
    int rc = check_jobs(jobs, njobs, &specs);
    if (rc) return rc;
    DeviceGuard g(h->device);
    cudaStream_t s = h->stream;
    cudaEvent_t a = nullptr, b = nullptr;
    TVS_CUDA(cudaEventCreate(&a), "event");
    TVS_CUDA(cudaEventCreate(&b), "event");
    const bool prof = h->profiling;
    h->profiling = false;
    auto time_of = [&](const Tuning& tn, float* ms) -> int {
        h->tuning = tn;
        int r = run_batch(h, specs, s, false, nullptr, nullptr);   // warm-up (and scratch growth)
        if (r) return r;
        cudaEventRecord(a, s);
        r = run_batch(h, specs, s, false, nullptr, nullptr);
        if (r) return r;
        cudaEventRecord(b, s);
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
        e = cudaEventElapsedTime(ms, a, b);
        if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
        return TVS_OK;
    };
    Tuning cur = h->tuning;
    float cur_ms = 0.f;
    rc = time_of(cur, &cur_ms);
    const int povs[] = {0, 384, 768, 1536, 1 << 30};
    const int warps[] = {0, 12, 8};
    const int unskews[] = {1, 2, 4};
    for (int stage = 0; stage < 3 && !rc; ++stage) {
        const int* opts = stage == 0 ? povs : stage == 1 ? warps : unskews;
        const int nopt = stage == 0 ? 5 : 3;
        for (int o = 0; o < nopt && !rc; ++o) {
            Tuning tn = cur;
            if (stage == 0) tn.small_pov_below_w = opts[o];
            if (stage == 1) tn.sweep_max_warps = opts[o];
            if (stage == 2) tn.unskew_ctas_per_sm = opts[o];
            float ms = 0.f;
            rc = time_of(tn, &ms);
            if (!rc && ms < cur_ms) { cur = tn; cur_ms = ms; }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->profiling = prof;
    h->tuning = cur;
    if (rc) return rc;
    if (best) tvs_get_tuning(h, best);
    if (best_ms) *best_ms = cur_ms;
    return TVS_OK;
}

}  // extern "C"
