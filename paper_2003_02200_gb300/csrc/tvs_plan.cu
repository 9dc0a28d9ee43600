// tvs_plan.cu -- host-side planning: the direction table, chunking of (job,
// direction) instances under a byte budget, the scratch layout and the launch
// sequence of a planned batch, and per-kernel timing.
#include "tvs_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace tvs {

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

namespace {

constexpr double kTwo32 = 4294967296.0;

const char* kKernelName[K_COUNT] = {"rowmap", "sweep", "unskew", "unskew_finalize",
                                   "points", "map_flags", "map_raster"};
const char* kKernelUnit[K_COUNT] = {"bytes", "evals", "bytes", "bytes", "evals", "evals", "cells"};

long long sum_min(long long L, long long K)
{
    // sum_{x=0}^{L-1} min(x, K)
    if (L <= 0) return 0;
    if (L - 1 <= K) return (L - 1) * L / 2;
    return K * (K + 1) / 2 + (L - 1 - K) * K;
}

}  // namespace

// ---------------------------------------------------------- directions --
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

// Same row ranges as host_row_range, walked in order of p: lo and hi only
// decrease as p grows, so after one division each they are stepped down by
// comparisons (O(R + W) per direction instead of two divisions per row).
DirWork direction_work(const HostDir& d)
{
    DirWork w{0, 0};
    const long long K = d.K == LLONG_MAX ? (long long)d.W : std::min<long long>(d.K, d.W);
    if (d.t_fx == 0ull) {
        w.samples = (long long)d.H * d.W;
        w.evals = (long long)d.H * 2 * sum_min(d.W, K);
        return w;
    }
    const unsigned long long T = d.t_fx;
    const unsigned long long last = (unsigned long long)(d.W - 1) * T;
    // rows with b in [0, H-1-c] span the whole walk axis (c = ceil((W-1) t))
    const long long c = (long long)((last + 0xFFFFFFFFull) >> 32);
    const long long full = std::max(0LL, (long long)d.H - c);
    w.samples += full * d.W;
    w.evals += full * 2 * sum_min(d.W, K);
    long long lo = -1, hi = -1;
    bool lo_set = false, hi_set = false;
    for (int p = 0; p < d.R; ++p) {
        const long long b = (long long)p - d.D;
        if (b >= 0 && b < full) { p += (int)(full - b) - 1; continue; }
        long long l = 0, h;
        if (b < 0) {
            const unsigned long long need = (unsigned long long)(-b) << 32;   // smallest j: j T >= need
            if (!lo_set) { lo = (long long)((need + T - 1ull) / T); lo_set = true; }
            while (lo > 0 && (unsigned long long)(lo - 1) * T >= need) --lo;
            l = lo;
        }
        const long long top = (long long)d.H - 1 - b;
        if (top < 0) {
            h = -1;
        } else {
            const unsigned long long lim = (unsigned long long)top << 32;     // largest j: j T <= lim
            if (last <= lim) {
                h = d.W - 1;
            } else {
                if (!hi_set) { hi = (long long)(lim / T); hi_set = true; }
                while (hi >= 0 && (unsigned long long)hi * T > lim) --hi;
                h = hi;
            }
        }
        const long long L = h - l + 1;
        if (L <= 0) continue;
        w.samples += L;
        w.evals += 2 * sum_min(L, K);
    }
    return w;
}

void job_work(int n, int rows, int cols, double step, double max_range, int k0, int k1, std::vector<DirWork>* out)
{
    out->assign(std::max(0, k1 - k0), DirWork{0, 0});
    std::map<std::pair<int, int>, DirWork> memo;   // (m, view shape) -> work
    for (int k = k0; k < k1; ++k) {
        HostDir d;
        if (make_direction(n, k, rows, cols, step, max_range, &d)) continue;
        const int shape = rows == cols ? 0 : (d.frame == 1 || d.frame == 2);
        const auto key = std::make_pair(d.m, shape);
        auto it = memo.find(key);
        if (it == memo.end()) it = memo.emplace(key, direction_work(d)).first;
        (*out)[k - k0] = it->second;
    }
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
Timer::Timer(tvs_ctx* h_, int k, cudaStream_t s_, double u) : h(h_), kernel(k), s(s_), units(u)
{
    if (h && h->profiling && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
        cudaEventRecord(a, s);
}

Timer::~Timer()
{
    if (a && b) {
        cudaEventRecord(b, s);
        h->pending.push_back(Pending{kernel, a, b, units});
    }
}

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

DeviceGuard::DeviceGuard(int dev)
{
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
}

DeviceGuard::~DeviceGuard()
{
    if (prev >= 0) cudaSetDevice(prev);
}

}  // namespace tvs

// --------------------------------------------------------------- plans --
namespace tvs {

size_t chunk_bytes(size_t slab, long long rows, int ninst)
{
    // forward measures + backward measures, row tables, item table (the sweep
    // gathers its rows from the DEM: no skewed heights are stored)
    return align256(slab * 4) * 2 + align256((size_t)rows * 4) * 2 + align256((size_t)(ninst + 1) * 4);
}

// A chunk splits only when its jobs have fewer than c = unskew_ctas_per_sm
// (at most 4) cell tiles per SM, into at most ceil(c * SMs / tiles) ranges, so
// its partials cover at most (c * SMs + tiles) < 2 c SMs tiles of 1024 cells,
// 16 bytes per cell.
size_t part_bound(int num_sms) { return align256((size_t)(8 * num_sms + 8) * UNSKEW_TI * UNSKEW_TJ * 16); }

// Cuts fall on multiples of FP32_GROUP directions of a job where the budget
// allows, so a job's FP32 group sums (and, the totals being exact, its result)
// do not depend on the chunking.
int plan_batch(const std::vector<JobSpec>& jobs, size_t avail, int num_sms, const Tuning& tn, BatchPlan* plan,
               int only_k, int smem_optin)
{
    plan->jobs = jobs;
    const int njobs = (int)jobs.size();
    std::vector<int> kend(njobs);
    // instances are planned largest DEM first (stable), so that a chunk holds
    // DEMs of similar row lengths; the results do not depend on the order
    std::vector<int> order(njobs);
    for (int j = 0; j < njobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return std::max(jobs[a].rows, jobs[a].cols) > std::max(jobs[b].rows, jobs[b].cols);
    });
    for (int j = 0; j < njobs; ++j) {
        const JobSpec& J = jobs[j];
        kend[j] = J.k1 < 0 ? J.n : J.k1;
        if (J.k0 < 0 || kend[j] > J.n || J.k0 > kend[j]) return fail(TVS_ERR_ARG, "direction range out of bounds");
    }
    for (int oj = 0; oj < njobs; ++oj) {
        const int j = order[oj];
        const JobSpec& J = jobs[j];
        for (int k = J.k0; k < kend[j]; ++k) {
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
    // work of every instance (from the caller's table, else counted once per distinct direction)
    std::vector<DirWork> inst_work(ninst);
    {
        std::vector<DirWork> tmp;
        for (int t = 0; t < ninst;) {
            int u = t;
            const int j = plan->inst_job[t];
            while (u < ninst && plan->inst_job[u] == j) ++u;
            const JobSpec& J = jobs[j];
            if (J.work) {
                for (int q = t; q < u; ++q) inst_work[q] = J.work[plan->inst_k[q]];
            } else {
                job_work(J.n, J.rows, J.cols, J.step, J.max_range, plan->inst_k[t], plan->inst_k[u - 1] + 1, &tmp);
                for (int q = t; q < u; ++q) inst_work[q] = tmp[plan->inst_k[q] - plan->inst_k[t]];
            }
            t = u;
        }
    }
    // a certified launch is sized for its longest rows: a chunk also ends
    // where the next DEM's rows take another layout class of the sweep
    auto job_class = [&](int j) {
        if (smem_optin <= 0 || tn.fp32_decisions) return 0;
        const int w = std::max(jobs[j].rows, jobs[j].cols);
        return cert_sweep_class(w, w, tn.prune, 64, smem_optin);
    };
    int i = 0;
    while (i < ninst) {
        size_t slab = 0, slab_ok = 0;
        long long nrows = 0, rows_ok = 0, items = 0;
        int ii = i, last_ok = -1;
        const int cls = job_class(plan->inst_job[i]);
        while (ii < ninst) {
            const HostDir& d = plan->hdirs[ii];
            const size_t wp = (size_t)((d.W + 3) & ~3);
            const size_t s2 = slab + (size_t)d.R * wp;
            const long long r2 = nrows + d.R;
            const long long it2 = items + 2LL * d.R;
            if (ii > i && (chunk_bytes(s2, r2, ii - i + 1) > avail || ii - i >= kMaxChunkDirs ||
                           it2 > kMaxChunkItems ||
                           (plan->inst_job[ii] != plan->inst_job[ii - 1] && job_class(plan->inst_job[ii]) != cls)))
                break;
            slab = s2;
            nrows = r2;
            items = it2;
            ++ii;
            const int kk = plan->inst_k[ii - 1], jj = plan->inst_job[ii - 1];
            if ((kk + 1) % FP32_GROUP == 0 || kk + 1 == kend[jj] || ii == ninst) {
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
    // Cost-sorted queue: within each chunk the jobs are ordered by their longest
    // side, largest first, so that the sweep's persistent warps, which claim
    // items in order, end the launch on the short rows of the smallest DEMs.
    // A job's instances stay contiguous and in direction order.
    for (const Chunk& c : plan->chunks) {
        std::vector<std::pair<int, int>> blocks;   // [t, u) of one job
        for (int t = c.i0; t < c.i1;) {
            int u = t;
            while (u < c.i1 && plan->inst_job[u] == plan->inst_job[t]) ++u;
            blocks.emplace_back(t, u);
            t = u;
        }
        if (blocks.size() < 2) continue;
        auto side = [&](const std::pair<int, int>& b) {
            const JobSpec& J = jobs[plan->inst_job[b.first]];
            return std::max(J.rows, J.cols);
        };
        std::stable_sort(blocks.begin(), blocks.end(),
                         [&](const std::pair<int, int>& a, const std::pair<int, int>& b) { return side(a) > side(b); });
        std::vector<HostDir> hd;
        std::vector<int> ij, ik;
        std::vector<DirWork> iw;
        for (const auto& b : blocks)
            for (int t = b.first; t < b.second; ++t) {
                hd.push_back(plan->hdirs[t]);
                ij.push_back(plan->inst_job[t]);
                ik.push_back(plan->inst_k[t]);
                iw.push_back(inst_work[t]);
            }
        for (int t = c.i0; t < c.i1; ++t) {
            plan->hdirs[t] = hd[t - c.i0];
            plan->inst_job[t] = ij[t - c.i0];
            plan->inst_k[t] = ik[t - c.i0];
            inst_work[t] = iw[t - c.i0];
        }
    }
    std::vector<int> first_chunk(njobs, -1), last_chunk(njobs, -1);
    for (int q = 0; q < (int)plan->chunks.size(); ++q)
        for (int t = plan->chunks[q].i0; t < plan->chunks[q].i1; ++t) {
            const int j = plan->inst_job[t];
            if (first_chunk[j] < 0) first_chunk[j] = q;
            last_chunk[j] = q;
        }
    plan->acc_off.assign(njobs, -1);
    for (int j = 0; j < njobs; ++j) {
        if (first_chunk[j] < 0 || jobs[j].acc) continue;
        const bool whole = jobs[j].k0 == 0 && kend[j] == jobs[j].n;
        if (!whole) return fail(TVS_ERR_ARG, "a partial direction range needs caller-owned totals");
        if (first_chunk[j] != last_chunk[j]) {
            plan->acc_off[j] = plan->acc_elems;
            plan->acc_elems += (long long)jobs[j].rows * jobs[j].cols;
        }
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
            v.pov = pov_mode(tn, d.W);
            v.p4_pct = tn.p4_cost_pct;
            v.gidx = plan->inst_k[t];
            v.job = plan->inst_job[t];
            v.g = (float)d.g;
            v.h0 = (float)J.h0;
            v.h0_lo = (float)(J.h0 - (double)v.h0);
            off += (size_t)d.R * v.Wp;
            roff += d.R;
            c.items += 2 * d.R;
            plan->istart.push_back(c.items);
            c.max_R = std::max(c.max_R, d.R);
            c.wmax = std::max(c.wmax, d.W);
            c.dmax = std::max(c.dmax, v.K);
            const DirWork w = inst_work[t];
            c.evals += (double)w.evals;
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
            e.first = first_chunk[j] == q && J.k0 == 0;
            e.last = last_chunk[j] == q && kend[j] == J.n;
            const int want = unskew_splits(tiles, e.dcnt, num_sms, tn.unskew_ctas_per_sm);
            e.per_split = unskew_per_split(e.dcnt, want);
            e.nsplit = unskew_effective_splits(e.dcnt, want);
            e.cell_beg = cell_beg;
            const long long cells = (long long)J.rows * J.cols;
            e.part_off = -1;
            if (e.nsplit > 1) { e.part_off = c.part_elems; c.part_elems += e.nsplit * cells; }
            c.max_split = std::max(c.max_split, e.nsplit);
            c.total_cells += cells;
            c.final_bytes += e.nsplit > 1 ? 16.0 * cells * (e.nsplit + 1) : 0.0;
            c.unskew_bytes += (e.first ? 0.0 : 16.0 * cells) + (e.last ? 4.0 * cells : 16.0 * cells);
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

// Entries of the flagged-walk buffer for these jobs: 1 in 64 of their walks
// (flags run between 1 in 700 and 1 in 250 on fractal terrain; walks beyond
// the buffer are walked in the sweep itself, at a cost), at least 4096, at
// most `cap` and FLAG_BUF_ENTRIES.
size_t flag_entries(const std::vector<JobSpec>& jobs, size_t cap)
{
    double walks = 0.0;
    for (const JobSpec& J : jobs) {
        const int nd = J.k1 > J.k0 ? J.k1 - J.k0 : J.n;   // the job's directions in this call
        walks += 2.0 * (double)J.rows * (double)J.cols * (double)nd;
    }
    return (size_t)std::min<double>((double)std::min<size_t>(cap, FLAG_BUF_ENTRIES), std::max(4096.0, walks / 64.0));
}

size_t budget_flags(size_t budget)
{
    return std::min<size_t>((size_t)FLAG_BUF_ENTRIES, budget / 16 / FLAG_ENTRY_BYTES);
}

Layout make_layout(const BatchPlan& plan, bool host_io, size_t max_flags)
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
    L.counter = o; o += 256;   // work counter at 0, flag-buffer counters at 64
    L.flag_cap = flag_entries(plan.jobs, max_flags);
    L.flags = o;   o += align256(L.flag_cap * FLAG_ENTRY_BYTES);
    L.acc = o;     o += align256((size_t)plan.acc_elems * 16);
    L.part = o;    o += align256((size_t)plan.max_part * 16);
    L.rowlo = o;   o += align256((size_t)plan.max_rows * 4);
    L.rowhi = o;   o += align256((size_t)plan.max_rows * 4);
    L.cvf = o;     o += align256(plan.max_slab * 4);
    L.cvb = o;     o += align256(plan.max_slab * 4);
    L.total = o;
    return L;
}

// Header, host copies of a single job, exact totals of every job, partials
// bound, counter.
size_t fixed_bytes(const std::vector<JobSpec>& jobs, bool host_io, int num_sms, size_t max_flags)
{
    size_t ninst = 0, cells = 0;
    for (const JobSpec& J : jobs) { ninst += J.n; cells += (size_t)J.rows * J.cols; }
    size_t b = align256(ninst * sizeof(DirDev)) + align256(jobs.size() * sizeof(JobDev)) +
               align256((jobs.size() + ninst) * sizeof(ChunkJob)) + align256((2 * ninst + 1) * 4) + 4096;
    if (host_io) b += 2 * align256((size_t)jobs[0].rows * jobs[0].cols * 4);
    b += align256(flag_entries(jobs, max_flags) * FLAG_ENTRY_BYTES);
    return b + align256(cells * 16) + part_bound(num_sms);
}

void build_header(const BatchPlan& plan, const Layout& L, char* base, bool host_io, std::vector<char>* img)
{
    img->assign(L.hdr_bytes, 0);
    std::memcpy(img->data() + (L.dirs - L.hdr), plan.dirs.data(), plan.dirs.size() * sizeof(DirDev));
    std::vector<JobDev> jd(plan.jobs.size());
    for (size_t j = 0; j < plan.jobs.size(); ++j) {
        const JobSpec& J = plan.jobs[j];
        jd[j].dem = host_io ? reinterpret_cast<const float*>(base + L.io_dem) : J.dem;
        jd[j].out = host_io ? reinterpret_cast<float*>(base + L.io_out) : J.out;
        jd[j].acc = J.acc ? J.acc
                          : plan.acc_off[j] >= 0 ? reinterpret_cast<__int128*>(base + L.acc) + plan.acc_off[j]
                                                 : nullptr;
        jd[j].scale = (M_PI / (2.0 * (double)J.n)) * (J.step * J.step);
        jd[j].h0 = J.h0;
        jd[j].rows = J.rows;
        jd[j].cols = J.cols;
    }
    std::memcpy(img->data() + (L.jobs - L.hdr), jd.data(), jd.size() * sizeof(JobDev));
    std::memcpy(img->data() + (L.cj - L.hdr), plan.cj.data(), plan.cj.size() * sizeof(ChunkJob));
    std::memcpy(img->data() + (L.istart - L.hdr), plan.istart.data(), plan.istart.size() * 4);
}

int enqueue_chunks(tvs_ctx* h, const BatchPlan& plan, const Layout& L, char* base, int num_sms, int smem_optin,
                   const Tuning& tn, cudaStream_t s, int* kernels, cudaEvent_t before_unskew)
{
    const DirDev* d_dirs = reinterpret_cast<const DirDev*>(base + L.dirs);
    const JobDev* d_jobs = reinterpret_cast<const JobDev*>(base + L.jobs);
    const ChunkJob* d_cj = reinterpret_cast<const ChunkJob*>(base + L.cj);
    const int* d_istart = reinterpret_cast<const int*>(base + L.istart);
    unsigned* d_counter = reinterpret_cast<unsigned*>(base + L.counter);
    unsigned* d_fcount = reinterpret_cast<unsigned*>(base + L.counter + 64);
    int4* d_flags = reinterpret_cast<int4*>(base + L.flags);
    __int128* d_part = reinterpret_cast<__int128*>(base + L.part);
    int* d_rowlo = reinterpret_cast<int*>(base + L.rowlo);
    int* d_rowhi = reinterpret_cast<int*>(base + L.rowhi);
    int* d_cvf = reinterpret_cast<int*>(base + L.cvf);
    int* d_cvb = reinterpret_cast<int*>(base + L.cvb);
    int launched = 0;
    for (const Chunk& c : plan.chunks) {
        const int nd = c.i1 - c.i0;
        const DirDev* cd = d_dirs + c.i0;
        {
            Timer t(h, K_ROWMAP, s, c.rowmap_bytes);
            TVS_CUDA(launch_rowmap(cd, nd, c.max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        }
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        {
            Timer t(h, K_SWEEP, s, c.evals);
            TVS_CUDA(launch_sweep(cd, d_jobs, d_istart + c.istart_at, nd, c.items, d_rowlo, d_rowhi, d_cvf, d_cvb,
                                  c.wmax, c.dmax, tn.prune, !tn.fp32_decisions, d_counter, d_flags, d_fcount,
                                  (int)L.flag_cap, num_sms, smem_optin, tn.sweep_max_warps, s),
                     "sweep launch");
        }
        if (before_unskew) {
            TVS_CUDA(cudaStreamWaitEvent(s, before_unskew, 0), "order unskews");
            before_unskew = nullptr;
        }
        {
            Timer t(h, K_UNSKEW, s, c.unskew_bytes);
            TVS_CUDA(launch_unskew(d_cvf, d_cvb, d_jobs, cd, d_cj + c.cj_beg, c.ncj, c.total_tiles, c.max_split,
                                   d_part, s),
                     "unskew launch");
        }
        // row map, sweep, unskew, and the exact pass that a certified sweep
        // with a flag buffer launches after itself
        launched += (!tn.fp32_decisions && d_flags && L.flag_cap > 0) ? 4 : 3;
        if (c.max_split > 1) {
            Timer t(h, K_FINAL, s, c.final_bytes);
            TVS_CUDA(launch_unskew_finalize(d_jobs, d_cj + c.cj_beg, c.ncj, c.total_cells, d_part, s),
                     "unskew finalize launch");
            ++launched;
        }
    }
    if (kernels) *kernels = launched;
    return TVS_OK;
}

// The buffer is reused by the next call only after the copy that read it has
// run (event), so the host never blocks on earlier GPU work.
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

int run_batch(tvs_ctx* h, const std::vector<JobSpec>& jobs, cudaStream_t s, bool host_io, const float* host_dem,
              float* host_out)
{
    const size_t mf = budget_flags(h->budget);
    const size_t fixed = fixed_bytes(jobs, host_io, h->num_sms, mf);
    if (fixed >= h->budget) return fail(TVS_ERR_OOM, "the DEMs do not fit the HBM budget");
    BatchPlan plan;
    int rc = plan_batch(jobs, h->budget - fixed, h->num_sms, h->tuning, &plan, -1, h->smem_optin);
    if (rc) return rc;
    const Layout L = make_layout(plan, host_io, mf);
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
    rc = enqueue_chunks(h, plan, L, base, h->num_sms, h->smem_optin, h->tuning, s);
    if (rc) return rc;
    if (host_io) {
        const size_t bytes = (size_t)jobs[0].rows * jobs[0].cols * 4;
        TVS_CUDA(cudaMemcpyAsync(host_out, base + L.io_out, bytes, cudaMemcpyDeviceToHost, s), "copy out");
        TVS_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return TVS_OK;
}

}  // namespace tvs
