// tvs_api.cu -- the C ABI declared in include/tvs.h for single DEMs, batches,
// prepared (graph-replayed) batches, tuning and the no-allocation entry point.
// Planning and launch sequencing live in tvs_plan.cu, the request server in
// tvs_server.cu.
#include "tvs.h"
#include "tvs_host.h"
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
    std::vector<DirWork> w;
    job_work(n_sectors, rows, cols, step_m, max_range_m, 0, n_sectors, &w);
    int64_t E = 0;
    for (const DirWork& x : w) E += x.evals;
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
    v.D = d.D; v.R = d.R; v.K = d.W; v.row_off = 0; v.gidx = k; v.g = (float)d.g;
    v.pov = LARGE_POV; v.p4_pct = 100;
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

int tvs_debug_plan(const int32_t* rows, const int32_t* cols, const int32_t* n_sectors, const double* step_m,
                   const double* max_range_m, int njobs, uint64_t budget_bytes, int num_sms, int smem_optin,
                   int prune, int fp32_decisions, int32_t* inst_job, int32_t* inst_k, int32_t* inst_chunk,
                   int inst_cap, int32_t* ninst, int32_t* nchunks)
{
    if (!rows || !cols || !n_sectors || !step_m || !max_range_m || !inst_job || !inst_k || !inst_chunk || !ninst ||
        !nchunks)
        return fail(TVS_ERR_ARG, "NULL argument");
    if (njobs <= 0 || num_sms <= 0 || smem_optin < 0) return fail(TVS_ERR_ARG, "njobs and num_sms must be positive");
    std::vector<JobSpec> jobs;
    long long total = 0;
    for (int j = 0; j < njobs; ++j) {
        const int rc = check_job(rows[j], cols[j], step_m[j], 0.0, n_sectors[j], max_range_m[j]);
        if (rc) return rc;
        jobs.push_back(JobSpec{nullptr, nullptr, rows[j], cols[j], n_sectors[j], step_m[j], 0.0, max_range_m[j]});
        total += n_sectors[j];
    }
    if (total > inst_cap) return fail(TVS_ERR_ARG, "inst_cap is below the jobs' total number of directions");
    Tuning tn;
    tn.prune = prune != 0;
    tn.fp32_decisions = fp32_decisions != 0;
    // the budget split of a batch call (run_batch): fixed parts first, the rest for chunks
    const size_t budget = (size_t)budget_bytes;
    const size_t fixed = fixed_bytes(jobs, false, num_sms, budget_flags(budget));
    if (fixed >= budget) return fail(TVS_ERR_OOM, "the DEMs do not fit the HBM budget");
    BatchPlan plan;
    const int rc = plan_batch(jobs, budget - fixed, num_sms, tn, &plan, -1, smem_optin);
    if (rc) return rc;
    const int n = (int)plan.inst_job.size();
    for (int q = 0; q < (int)plan.chunks.size(); ++q)
        for (int t = plan.chunks[q].i0; t < plan.chunks[q].i1; ++t) {
            inst_job[t] = plan.inst_job[t];
            inst_k[t] = plan.inst_k[t];
            inst_chunk[t] = q;
        }
    *ninst = n;
    *nchunks = (int)plan.chunks.size();
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
    int* d_cv = reinterpret_cast<int*>(ws + L.cvf);
    int* d_cb = reinterpret_cast<int*>(ws + L.cvb);
    unsigned* d_cnt = reinterpret_cast<unsigned*>(ws + L.counter);
    TVS_CUDA(launch_rowmap(d_dir, 1, v.R, d_lo, d_hi, s), "rowmap launch");
    TVS_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), s), "reset work counter");
    TVS_CUDA(launch_sweep(d_dir, d_jobs, reinterpret_cast<const int*>(ws + L.istart), 1, c.items, d_lo, d_hi, d_cv,
                          d_cb, v.W, v.K, h->tuning.prune, !h->tuning.fp32_decisions, d_cnt, nullptr, nullptr, 0,
                          h->num_sms, h->smem_optin, h->tuning.sweep_max_warps, s),
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

// Host-side planning tables of the no-allocation entry point.  They live in
// static storage rather than on the calling thread's stack (about 140 KB at
// 1024 directions, more than some worker threads have) and are used by one
// call at a time under g_noalloc_call_mu.  That is host memory, so the entry
// point still allocates nothing on the device.
struct NoAllocTables {
    DirDev dirs[kNoAllocMaxDirs];
    int istart[2 * kNoAllocMaxDirs + 1];
    int chunk_k0[kNoAllocMaxDirs + 1];
    ChunkJob cjs[kNoAllocMaxDirs];
};
std::mutex g_noalloc_call_mu;
NoAllocTables g_noalloc_tables;

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
    // The tables below reach the device through copies from host memory that
    // is reused by the next call, so a captured call would replay stale
    // tables: refuse capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce == cudaErrorStreamCaptureImplicit || (ce == cudaSuccess && cap != cudaStreamCaptureStatusNone)) {
        cudaGetLastError();
        return fail(TVS_ERR_ARG, "the no-allocation entry point cannot be captured into a CUDA graph");
    }
    TVS_CUDA(ce, "cudaStreamIsCapturing");
    int device = 0;
    TVS_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    char* base = nullptr;
    rc = noalloc_scratch(device, &base);
    if (rc) return rc;
    int num_sms = 0, smem_optin = 0;
    TVS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
    TVS_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device),
             "device attribute");

    // Direction table and chunking: chunks of consecutive directions whose
    // skewed slabs fit what the fixed part leaves.  The tables are static
    // host storage used by one call at a time.
    std::lock_guard<std::mutex> call_lock(g_noalloc_call_mu);
    DirDev* dirs = g_noalloc_tables.dirs;
    int* istart = g_noalloc_tables.istart;
    int* chunk_k0 = g_noalloc_tables.chunk_k0;
    ChunkJob* cjs = g_noalloc_tables.cjs;
    int nchunks = 0;
    const int tiles = unskew_tiles(rows, cols);
    const Tuning tn;
    const int nsplit_max = unskew_splits(tiles, n_sectors, num_sms, tn.unskew_ctas_per_sm);
    const size_t o_dirs = 0;
    const size_t o_job = o_dirs + align256((size_t)n_sectors * sizeof(DirDev));
    const size_t o_cj = o_job + align256(sizeof(JobDev));
    const size_t o_istart = o_cj + align256((size_t)n_sectors * sizeof(ChunkJob));
    const size_t o_acc = o_istart + align256((size_t)(2 * n_sectors + 1) * 4);
    const size_t o_part = o_acc + align256(cells * 16);
    const size_t o_counter = o_part + (nsplit_max > 1 ? align256((size_t)nsplit_max * cells * 16) : 0);
    const size_t o_chunk = o_counter + 256;
    if (o_chunk >= kNoAllocScratchBytes)
        return fail(TVS_ERR_OOM, "the DEM does not fit the 64 MiB no-allocation scratch");
    const size_t avail = kNoAllocScratchBytes - o_chunk;
    size_t max_rows = 0, max_slab = 0;
    {
        int k = 0;
        while (k < n_sectors) {
            size_t slab = 0, nrows = 0, slab_ok = 0, rows_ok = 0;
            int kk = k, kk_ok = -1;
            while (kk < n_sectors) {
                HostDir d;
                make_direction(n_sectors, kk, rows, cols, step_m, max_range_m, &d);
                const size_t wp = (size_t)((d.W + 3) & ~3);
                const size_t s2 = slab + (size_t)d.R * wp, r2 = nrows + d.R;
                // every chunk uses one layout sized by the largest row count
                // and the largest slab of all chunks, which may come from
                // different chunks: check the layout this chunk will really get
                const size_t need = 2 * align256(std::max(max_rows, r2) * 4) + 2 * align256(std::max(max_slab, s2) * 4);
                if (need > avail || 2LL * (long long)r2 > kMaxChunkItems) break;
                DirDev& v = dirs[kk];
                std::memset(&v, 0, sizeof(v));
                v.t_fx = d.t_fx; v.slab = (long long)slab; v.frame = d.frame; v.H = d.H; v.W = d.W;
                v.Wp = (int)wp; v.D = d.D; v.R = d.R;
                v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
                v.pov = pov_mode(tn, d.W);
                v.p4_pct = tn.p4_cost_pct;
                v.row_off = (int)nrows; v.gidx = kk; v.job = 0;
                v.g = (float)d.g; v.h0 = (float)obs_height_m;
                v.h0_lo = (float)(obs_height_m - (double)v.h0);
                slab = s2;
                nrows = r2;
                ++kk;
                if (kk % FP32_GROUP == 0 || kk == n_sectors) { kk_ok = kk; slab_ok = slab; rows_ok = nrows; }
            }
            if (kk == k)
                return fail(TVS_ERR_OOM, "one direction of this DEM does not fit the 64 MiB no-allocation scratch");
            // cut on a group boundary when one fits, so the FP32 group sums match the allocating path
            if (kk < n_sectors && kk_ok > k) { kk = kk_ok; slab = slab_ok; nrows = rows_ok; }
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
                istart[at + 1] = istart[at] + 2 * dirs[q].R;
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
    job.acc = nchunks > 1 ? reinterpret_cast<__int128*>(base + o_acc) : nullptr;
    job.scale = (M_PI / (2.0 * (double)n_sectors)) * (step_m * step_m);
    job.h0 = obs_height_m;
    job.rows = rows;
    job.cols = cols;
    DirDev* d_dirs = reinterpret_cast<DirDev*>(base + o_dirs);
    JobDev* d_job = reinterpret_cast<JobDev*>(base + o_job);
    ChunkJob* d_cj = reinterpret_cast<ChunkJob*>(base + o_cj);
    int* d_istart = reinterpret_cast<int*>(base + o_istart);
    __int128* d_part = reinterpret_cast<__int128*>(base + o_part);
    unsigned* d_counter = reinterpret_cast<unsigned*>(base + o_counter);
    int* d_rowlo = reinterpret_cast<int*>(base + o_chunk);
    int* d_rowhi = reinterpret_cast<int*>(base + o_chunk + align256(max_rows * 4));
    const size_t o_slabs = o_chunk + 2 * align256(max_rows * 4);
    int* d_cvf = reinterpret_cast<int*>(base + o_slabs);
    int* d_cvb = reinterpret_cast<int*>(base + o_slabs + align256(max_slab * 4));
    if (o_slabs + 2 * align256(max_slab * 4) > kNoAllocScratchBytes)
        return fail(TVS_ERR_OOM, "the job's layout does not fit the 64 MiB no-allocation scratch");

    // Copies from pageable host memory: the runtime has staged the tables
    // before each call returns, so the next call may reuse them.
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
        int max_R = 0, wmax = 0, dmax = 0;
        for (int q = k0; q < k0 + nd; ++q) {
            dmax = std::max(dmax, dirs[q].K);
            max_R = std::max(max_R, dirs[q].R);
            wmax = std::max(wmax, dirs[q].W);
        }
        const DirDev* cd = d_dirs + k0;
        TVS_CUDA(launch_rowmap(cd, nd, max_R, d_rowlo, d_rowhi, s), "rowmap launch");
        // the shared array keeps the previous call's contents: the work counter must start at zero
        TVS_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s), "reset work counter");
        TVS_CUDA(launch_sweep(cd, d_job, d_istart + at, nd, istart[at + nd], d_rowlo, d_rowhi, d_cvf, d_cvb, wmax,
                              dmax, tn.prune, !tn.fp32_decisions, d_counter, nullptr, nullptr, 0, num_sms,
                              smem_optin, tn.sweep_max_warps, s),
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
    const size_t mf = budget_flags(budget);
    const size_t fixed = fixed_bytes(specs, false, h->num_sms, mf);
    if (fixed >= budget) return fail(TVS_ERR_OOM, "the DEMs do not fit the HBM budget");
    tvs_batch* b = new tvs_batch();
    b->h = h;
    rc = plan_batch(specs, budget - fixed, h->num_sms, h->tuning, &b->plan, -1, h->smem_optin);
    if (rc) { delete b; return rc; }
    b->L = make_layout(b->plan, false, mf);
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
    rc = enqueue_chunks(nullptr, b->plan, b->L, b->ws, h->num_sms, h->smem_optin, h->tuning, cap);
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
    t->p4_cost_pct = h->tuning.p4_cost_pct;
    t->prune = h->tuning.prune;
    t->fp32_decisions = h->tuning.fp32_decisions;
    return TVS_OK;
}

int tvs_set_tuning(tvs_handle h, const tvs_tuning* t)
{
    if (!h || !t) return fail(TVS_ERR_ARG, "NULL argument");
    if (t->small_pov_below_w < 0 || t->sweep_max_warps < 0 || t->sweep_max_warps > SWEEP_MAX_WARPS ||
        t->unskew_ctas_per_sm < 1 || t->unskew_ctas_per_sm > 4 || t->p4_cost_pct < 0 || t->p4_cost_pct > (1 << 20) ||
        t->prune < 0 || t->prune > 1 || t->fp32_decisions < 0 || t->fp32_decisions > 1)
        return fail(TVS_ERR_ARG, "tuning out of range");
    h->tuning.small_pov_below_w = t->small_pov_below_w;
    h->tuning.sweep_max_warps = t->sweep_max_warps;
    h->tuning.unskew_ctas_per_sm = t->unskew_ctas_per_sm;
    h->tuning.p4_cost_pct = t->p4_cost_pct ? t->p4_cost_pct : Tuning().p4_cost_pct;
    h->tuning.prune = t->prune;
    h->tuning.fp32_decisions = t->fp32_decisions;
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
    const int prunes[] = {1, 0};
    const int costs[] = {100, 107, 115, 130, 1 << 20};
    const int povs[] = {0, 256, 512};
    const int warps[] = {0, 12, 8};
    const int unskews[] = {1, 2, 4};
    for (int stage = 0; stage < 5 && !rc; ++stage) {
        const int* opts = stage == 0 ? prunes : stage == 1 ? costs : stage == 2 ? povs : stage == 3 ? warps : unskews;
        const int nopt = stage == 0 ? 2 : stage == 1 ? 5 : 3;
        for (int o = 0; o < nopt && !rc; ++o) {
            Tuning tn = cur;
            if (stage == 0) tn.prune = opts[o];
            if (stage == 1) tn.p4_cost_pct = opts[o];
            if (stage == 2) tn.small_pov_below_w = opts[o];
            if (stage == 3) tn.sweep_max_warps = opts[o];
            if (stage == 4) tn.unskew_ctas_per_sm = opts[o];
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
