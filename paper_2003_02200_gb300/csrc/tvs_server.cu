// tvs_server.cu -- request server with continuous batching (the "request
// server" part of include/tvs.h).
//
// Threads: callers submit from any thread; one scheduler thread admits
// requests into the resident arena and enqueues steps; one completion thread
// waits for finished outputs to reach the caller's buffers, stamps them and
// frees their arena space.
//
// Streams: one per lane (a step runs on one lane), one for the DEM uploads and
// one for the output downloads.  Within a step the pipeline is ordered by its
// lane's stream.  Across steps two orders matter:
//   * a step's skew reads DEMs: the lane waits for each request's upload event;
//   * steps add into the same running totals: each step's first unskew waits
//     for the end of the step enqueued before it, so totals are updated in
//     step order (the additions are exact, but the first and last writes of a
//     request must come in order);
// while the row map, skew and sweep of a step overlap the previous step's tail.
#include "tvs.h"
#include "tvs_host.h"
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace tvs;

namespace {

constexpr int kMaxStepJobs = 512;          // requests in one step (bounds the header)
constexpr size_t kAccBytes = 16;           // exact running total per cell

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, total) in 256-byte granules; free ranges are
// coalesced on release.
class Arena {
public:
    void reset(size_t total)
    {
        free_.clear();
        total_ = total;
        used_ = peak_ = 0;
        if (total) free_[0] = total;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t total() const { return total_; }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
    int64_t id = 0;
    const float* host_dem = nullptr;
    float* host_out = nullptr;
    JobSpec spec{};
    std::vector<DirWork> work;        // per direction (spec.work points here)
    // per-direction prefix sums of the step costs: evals, slab elements, rows, sweep items
    std::vector<double> cum_evals;
    std::vector<long long> cum_slab, cum_rows, cum_items;
    int next_k = 0;                   // first direction not yet in a step
    int state = TVS_REQ_QUEUED;
    int error = TVS_OK;
    std::string message;
    double t_submit = 0, t_admit = -1, t_first = -1, t_done = -1;
    int steps = 0;
    double key = 0;                   // deadline policy: submit time + evals / rate
    double evals_total = 0;           // work count of the request
    size_t off = 0, bytes = 0;        // arena range
    cudaEvent_t loaded = nullptr;     // DEM upload done
    cudaEvent_t finished = nullptr;   // output download done
    bool resident = false;
};

struct Lane {
    cudaStream_t stream = nullptr;
    char* scratch = nullptr;          // inside the server's allocation
    size_t bytes = 0;
    char* pinned = nullptr;           // header staging, reused once the lane's step is done
    size_t pinned_bytes = 0;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t seq = 0;                 // step number of the lane's current step
};

}  // namespace

struct tvs_server {
    int device = 0;
    int num_sms = 0, smem_optin = 0;
    tvs_server_config cfg{};
    Tuning tuning;
    Clock::time_point t0;

    char* pool = nullptr;             // one device allocation: lanes, then the arena
    Arena arena;
    char* arena_base = nullptr;
    std::vector<Lane> lanes;
    cudaStream_t upload = nullptr, download = nullptr;
    cudaEvent_t last_step_done = nullptr;   // end of the most recently enqueued step (a lane's `done`)
    uint64_t step_seq = 0;

    std::mutex mu;
    std::condition_variable cv_sched;     // submissions, completions, stop
    std::condition_variable cv_done;      // request completions (waiters)
    std::condition_variable cv_complete;  // the completion thread's queue
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<Request*> queue;           // submitted, not admitted
    std::vector<Request*> active;         // admitted, not finished
    std::deque<Request*> finishing;       // downloads enqueued, in stream order
    int64_t next_id = 1;
    bool stopping = false, stop_completion = false;
    bool broken = false;
    std::string broken_msg;
    tvs_server_stats st{};

    std::thread scheduler, completer;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void mark_failed(tvs_server* S, Request* r, int code, const std::string& msg)
{
    r->state = TVS_REQ_FAILED;
    r->error = code;
    r->message = msg;
    r->t_done = S->now();
    S->st.failed += 1;
}

// Everything not finished fails (a CUDA error left the server unusable).
void break_server(tvs_server* S, const std::string& msg)
{
    S->broken = true;
    S->broken_msg = msg;
    for (Request* r : S->queue) mark_failed(S, r, TVS_ERR_CUDA, msg);
    S->queue.clear();
    for (Request* r : S->active)
        if (r->state != TVS_REQ_DONE && r->state != TVS_REQ_FAILED) mark_failed(S, r, TVS_ERR_CUDA, msg);
    S->cv_done.notify_all();
}

// Admit queued requests in submission order while the arena has room.
void admit(tvs_server* S)
{
    while (!S->queue.empty() && (int)S->active.size() < S->cfg.max_active) {
        Request* r = S->queue.front();
        const size_t cells = (size_t)r->spec.rows * r->spec.cols;
        const size_t need = align256(cells * kAccBytes) + align256(cells * 4) * 2;
        size_t off = 0;
        if (!S->arena.alloc(need, &off)) break;   // head of line waits for room
        r->off = off;
        r->bytes = need;
        r->resident = true;
        char* base = S->arena_base + off;
        r->spec.acc = reinterpret_cast<__int128*>(base);
        r->spec.dem = reinterpret_cast<const float*>(base + align256(cells * kAccBytes));
        r->spec.out = reinterpret_cast<float*>(base + align256(cells * kAccBytes) + align256(cells * 4));
        cudaError_t e = cudaMemcpyAsync(const_cast<float*>(r->spec.dem), r->host_dem, cells * 4,
                                        cudaMemcpyHostToDevice, S->upload);
        if (e == cudaSuccess) e = cudaEventRecord(r->loaded, S->upload);
        S->queue.pop_front();
        S->active.push_back(r);
        if (e != cudaSuccess) {
            break_server(S, std::string("DEM upload: ") + cudaGetErrorString(e));
            return;
        }
        r->state = TVS_REQ_ADMITTED;
        r->t_admit = S->now();
    }
}

// Slices of the next step, in policy order: whole groups of FP32_GROUP
// directions until the step holds about step_evals evaluations or a lane's
// scratch, the direction table or the job table is full.  The first group is
// always taken, so every step makes progress.
struct Slice {
    Request* r;
    int k0, k1;
};

std::vector<Slice> pick_slices(tvs_server* S, size_t slot_avail)
{
    std::vector<Request*> cand;
    for (Request* r : S->active)
        if (r->state == TVS_REQ_ADMITTED || r->state == TVS_REQ_RUNNING)
            if (r->next_k < r->spec.n) cand.push_back(r);
    auto remaining = [](const Request* r) { return r->cum_evals.back() - r->cum_evals[r->next_k]; };
    std::stable_sort(cand.begin(), cand.end(), [&](const Request* a, const Request* b) {
        switch (S->cfg.policy) {
        case TVS_POLICY_FIFO: return a->id < b->id;
        case TVS_POLICY_SRPT: return remaining(a) < remaining(b);
        default: return a->key < b->key;
        }
    });
    std::vector<Slice> out;
    double ev = 0.0;
    long long slab = 0, rows = 0, items = 0;
    int ndirs = 0;
    bool full = false;
    for (Request* r : cand) {
        if (full || (int)out.size() >= kMaxStepJobs) break;
        int k = r->next_k;
        while (k < r->spec.n) {
            const int g1 = std::min(r->spec.n, (k / FP32_GROUP + 1) * FP32_GROUP);
            const double gev = r->cum_evals[g1] - r->cum_evals[k];
            const long long gslab = r->cum_slab[g1] - r->cum_slab[k];
            const long long grows = r->cum_rows[g1] - r->cum_rows[k];
            const long long gitems = r->cum_items[g1] - r->cum_items[k];
            const bool first = out.empty() && k == r->next_k;
            const bool fits = chunk_bytes((size_t)(slab + gslab), rows + grows, ndirs + (g1 - k)) <= slot_avail &&
                              ndirs + (g1 - k) <= kMaxChunkDirs && items + gitems <= kMaxChunkItems;
            if (!first && (!fits || ev + gev > S->cfg.step_evals)) { full = true; break; }
            ev += gev; slab += gslab; rows += grows; items += gitems; ndirs += g1 - k;
            k = g1;
        }
        if (k > r->next_k) out.push_back(Slice{r, r->next_k, k});
    }
    return out;
}

// Entries of a lane's flagged-walk buffer: an eighth of the lane, at most
// FLAG_BUF_ENTRIES.
size_t lane_flags(size_t lane_bytes)
{
    return std::min<size_t>((size_t)FLAG_BUF_ENTRIES, lane_bytes / 8 / FLAG_ENTRY_BYTES);
}

// Bytes of a lane's scratch that the header, counters, flagged-walk buffer
// and partials may take.
size_t lane_fixed_bytes(int num_sms, size_t lane_bytes)
{
    return align256((size_t)kMaxChunkDirs * sizeof(DirDev)) + align256((size_t)kMaxStepJobs * sizeof(JobDev)) +
           align256((size_t)(kMaxStepJobs + kMaxChunkDirs) * sizeof(ChunkJob)) +
           align256((size_t)(2 * kMaxChunkDirs + 2) * 4) + 256 + align256(lane_flags(lane_bytes) * FLAG_ENTRY_BYTES) +
           part_bound(num_sms) + 4096;
}

// Plan and enqueue one step on a free lane.  Called with the lock held.
int enqueue_step(tvs_server* S, Lane& lane, const std::vector<Slice>& slices)
{
    if (S->cfg.fail_after_steps > 0 && S->st.steps >= S->cfg.fail_after_steps)
        return fail(TVS_ERR_CUDA, "injected step failure (fail_after_steps)");
    std::vector<JobSpec> jobs;
    jobs.reserve(slices.size());
    for (const Slice& sl : slices) {
        JobSpec J = sl.r->spec;
        J.k0 = sl.k0;
        J.k1 = sl.k1;
        jobs.push_back(J);
    }
    BatchPlan plan;
    const size_t fixed = lane_fixed_bytes(S->num_sms, lane.bytes);
    int rc = plan_batch(jobs, lane.bytes - fixed, S->num_sms, S->tuning, &plan, -1, S->smem_optin);
    if (rc) return rc;
    const Layout L = make_layout(plan, false, lane_flags(lane.bytes));
    if (L.total > lane.bytes) return fail(TVS_ERR_OOM, "step does not fit its lane");
    std::vector<char> img;
    build_header(plan, L, lane.scratch, false, &img);
    if (img.size() > lane.pinned_bytes) {
        if (lane.pinned) cudaFreeHost(lane.pinned);
        lane.pinned = nullptr;
        lane.pinned_bytes = 0;
        TVS_CUDA(cudaHostAlloc((void**)&lane.pinned, img.size(), cudaHostAllocDefault), "cudaHostAlloc");
        lane.pinned_bytes = img.size();
    }
    std::memcpy(lane.pinned, img.data(), img.size());
    TVS_CUDA(cudaMemcpyAsync(lane.scratch + L.hdr, lane.pinned, img.size(), cudaMemcpyHostToDevice, lane.stream),
             "copy step tables");
    for (const Slice& sl : slices) TVS_CUDA(cudaStreamWaitEvent(lane.stream, sl.r->loaded, 0), "wait for DEM");
    int kernels = 0;
    rc = enqueue_chunks(nullptr, plan, L, lane.scratch, S->num_sms, S->smem_optin, S->tuning, lane.stream, &kernels,
                        S->last_step_done);
    if (rc) return rc;
    TVS_CUDA(cudaEventRecord(lane.done, lane.stream), "record step end");
    S->last_step_done = lane.done;
    lane.busy = true;
    lane.seq = ++S->step_seq;
    // downloads of the requests this step completes
    bool waited = false;
    const double t = S->now();
    for (const Slice& sl : slices) {
        Request* r = sl.r;
        r->next_k = sl.k1;
        r->steps += 1;
        if (r->t_first < 0) r->t_first = t;
        r->state = TVS_REQ_RUNNING;
        if (sl.k1 < r->spec.n) continue;
        if (!waited) {
            TVS_CUDA(cudaStreamWaitEvent(S->download, lane.done, 0), "order download");
            waited = true;
        }
        const size_t bytes = (size_t)r->spec.rows * r->spec.cols * 4;
        TVS_CUDA(cudaMemcpyAsync(r->host_out, r->spec.out, bytes, cudaMemcpyDeviceToHost, S->download),
                 "download output");
        TVS_CUDA(cudaEventRecord(r->finished, S->download), "record download");
        S->finishing.push_back(r);
    }
    if (waited) S->cv_complete.notify_one();
    S->st.steps += 1;
    S->st.kernels += kernels;
    S->st.evals += plan.evals;
    S->st.max_step_jobs = std::max<int32_t>(S->st.max_step_jobs, (int32_t)slices.size());
    return TVS_OK;
}

void scheduler_loop(tvs_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        for (Lane& ln : S->lanes) {
            if (!ln.busy) continue;
            const cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaSuccess) ln.busy = false;
            else if (q != cudaErrorNotReady && !S->broken) break_server(S, std::string("step: ") + cudaGetErrorString(q));
        }
        if (!S->broken) admit(S);
        Lane* free_lane = nullptr;
        for (Lane& ln : S->lanes)
            if (!ln.busy) { free_lane = &ln; break; }
        bool work = false;
        if (!S->broken)
            for (Request* r : S->active)
                if ((r->state == TVS_REQ_ADMITTED || r->state == TVS_REQ_RUNNING) && r->next_k < r->spec.n) {
                    work = true;
                    break;
                }
        if (work && free_lane) {
            const std::vector<Slice> slices =
                pick_slices(S, free_lane->bytes - lane_fixed_bytes(S->num_sms, free_lane->bytes));
            const int rc = enqueue_step(S, *free_lane, slices);
            if (rc) break_server(S, "step enqueue failed: " + g_err);
            continue;
        }
        bool any_busy = false;
        for (const Lane& ln : S->lanes) any_busy |= ln.busy;
        if (S->stopping && S->queue.empty() && !work && !any_busy) break;
        if (!free_lane) {
            // every lane has a step in flight: wait for the oldest one
            Lane* oldest = nullptr;
            for (Lane& ln : S->lanes)
                if (ln.busy && (!oldest || ln.seq < oldest->seq)) oldest = &ln;
            cudaEvent_t ev = oldest->done;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
            continue;
        }
        if (any_busy && S->stopping) {
            // shutting down with nothing left to plan: let the running steps end
            for (Lane& ln : S->lanes)
                if (ln.busy) {
                    cudaEvent_t ev = ln.done;
                    lk.unlock();
                    cudaEventSynchronize(ev);
                    lk.lock();
                    break;
                }
            continue;
        }
        // a free lane and nothing to plan: sleep until a submission, a completion (arena room) or a stop
        S->cv_sched.wait(lk);
    }
}

void completion_loop(tvs_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_complete.wait(lk, [&] { return !S->finishing.empty() || S->stop_completion; });
        if (S->finishing.empty()) break;
        Request* r = S->finishing.front();
        cudaEvent_t ev = r->finished;
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(ev);
        lk.lock();
        S->finishing.pop_front();
        if (r->state != TVS_REQ_FAILED) {
            if (e == cudaSuccess) {
                r->state = TVS_REQ_DONE;
                r->t_done = S->now();
                S->st.completed += 1;
            } else {
                mark_failed(S, r, TVS_ERR_CUDA, std::string("output download: ") + cudaGetErrorString(e));
            }
        }
        if (r->resident) {
            S->arena.release(r->off, r->bytes);
            r->resident = false;
        }
        S->active.erase(std::remove(S->active.begin(), S->active.end(), r), S->active.end());
        r->cum_evals.clear(); r->cum_slab.clear(); r->cum_rows.clear(); r->cum_items.clear();
        r->work.clear();
        r->spec.work = nullptr;
        if (r->loaded) { cudaEventDestroy(r->loaded); r->loaded = nullptr; }
        if (r->finished) { cudaEventDestroy(r->finished); r->finished = nullptr; }
        S->cv_done.notify_all();
        S->cv_sched.notify_one();
    }
}

}  // namespace

// ================================================================== C ABI ==
namespace {

void destroy_server(tvs_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (Request* r : S->queue) mark_failed(S, r, TVS_ERR_STATE, "the server shut down before admission");
        S->queue.clear();
        S->cv_sched.notify_all();
        S->cv_done.notify_all();
    }
    if (S->scheduler.joinable()) S->scheduler.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop_completion = true;
        S->cv_complete.notify_all();
    }
    if (S->completer.joinable()) S->completer.join();
    cudaSetDevice(S->device);
    cudaDeviceSynchronize();
    for (auto& kv : S->reqs) {
        Request* r = kv.second.get();
        if (r->loaded) cudaEventDestroy(r->loaded);
        if (r->finished) cudaEventDestroy(r->finished);
    }
    for (Lane& ln : S->lanes) {
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.pinned) cudaFreeHost(ln.pinned);
    }
    if (S->upload) cudaStreamDestroy(S->upload);
    if (S->download) cudaStreamDestroy(S->download);
    if (S->pool) cudaFree(S->pool);
    delete S;
}

}  // namespace

extern "C" {

int tvs_server_create(int device, const tvs_server_config* cfg_in, tvs_server_handle* out)
{
    if (!out) return fail(TVS_ERR_ARG, "out is NULL");
    *out = nullptr;
    tvs_server_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.step_evals < 0 || cfg.rate_hint < 0 || cfg.max_active < 0 || cfg.lanes < 0 || cfg.lanes > 2 ||
        cfg.fail_after_steps < 0 ||
        cfg.policy < 0 || cfg.policy > TVS_POLICY_SRPT || !std::isfinite(cfg.step_evals) ||
        !std::isfinite(cfg.rate_hint))
        return fail(TVS_ERR_ARG, "server config out of range");
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaGetDeviceCount");
    }
    if (device < 0 || device >= count) return fail(TVS_ERR_ARG, "device index out of range");
    DeviceGuard g(device);
    cudaDeviceProp prop;
    TVS_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    size_t free_b = 0, total_b = 0;
    TVS_CUDA(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    if (cfg.hbm_budget_bytes == 0) cfg.hbm_budget_bytes = std::min<size_t>((size_t)80 << 30, (size_t)(0.85 * free_b));
    if (cfg.lanes == 0) cfg.lanes = 2;
    if (cfg.step_slot_bytes == 0)
        cfg.step_slot_bytes = std::min<size_t>((size_t)4 << 30, cfg.hbm_budget_bytes / 8);
    cfg.step_slot_bytes = align256(cfg.step_slot_bytes);
    if (cfg.step_evals == 0) cfg.step_evals = 1.6e11;
    if (cfg.rate_hint == 0) cfg.rate_hint = 5e12;
    if (cfg.max_active == 0) cfg.max_active = 256;
    const int num_sms = prop.multiProcessorCount;
    if (cfg.step_slot_bytes < lane_fixed_bytes(num_sms, cfg.step_slot_bytes) + ((size_t)1 << 20))
        return fail(TVS_ERR_ARG, "step_slot_bytes is too small for a step");
    const size_t lanes_bytes = cfg.step_slot_bytes * (size_t)cfg.lanes;
    if (cfg.hbm_budget_bytes <= lanes_bytes + ((size_t)1 << 20))
        return fail(TVS_ERR_OOM, "the HBM budget leaves no arena beside the step slots");

    tvs_server* S = new tvs_server();
    S->device = device;
    S->num_sms = num_sms;
    S->smem_optin = (int)prop.sharedMemPerBlockOptin;
    S->cfg = cfg;
    S->t0 = Clock::now();
    e = cudaMalloc(&S->pool, cfg.hbm_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        S->pool = nullptr;
        destroy_server(S);
        return fail(TVS_ERR_OOM, std::string("cudaMalloc of the server budget failed: ") + cudaGetErrorString(e));
    }
    S->lanes.resize(cfg.lanes);
    for (int q = 0; q < cfg.lanes; ++q) {
        Lane& ln = S->lanes[q];
        ln.scratch = S->pool + (size_t)q * cfg.step_slot_bytes;
        ln.bytes = cfg.step_slot_bytes;
        e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming);
        if (e != cudaSuccess) { destroy_server(S); return cuda_fail(e, "lane stream or event"); }
    }
    S->arena_base = S->pool + lanes_bytes;
    S->arena.reset(cfg.hbm_budget_bytes - lanes_bytes);
    S->st.arena_bytes = (double)S->arena.total();
    S->st.lanes = cfg.lanes;
    e = cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->download, cudaStreamNonBlocking);
    if (e != cudaSuccess) { destroy_server(S); return cuda_fail(e, "server streams"); }
    S->scheduler = std::thread(scheduler_loop, S);
    S->completer = std::thread(completion_loop, S);
    *out = S;
    return TVS_OK;
}

void tvs_server_destroy(tvs_server_handle s) { destroy_server(s); }

double tvs_server_clock(tvs_server_handle s) { return s ? s->now() : 0.0; }

int tvs_server_submit(tvs_server_handle S, const float* dem, int rows, int cols, double step_m,
                      double obs_height_m, int n_sectors, double max_range_m, float* out, int64_t* ticket)
{
    if (!S || !dem || !out || !ticket) return fail(TVS_ERR_ARG, "NULL argument");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    const size_t cells = (size_t)rows * cols;
    for (size_t q = 0; q < cells; ++q)
        if (!std::isfinite(dem[q])) return fail(TVS_ERR_ARG, "dem holds a non-finite value");
    const size_t need = align256(cells * kAccBytes) + align256(cells * 4) * 2;
    if (need > S->arena.total()) return fail(TVS_ERR_OOM, "the request can never fit the server's arena");
    auto r = std::make_unique<Request>();
    r->host_dem = dem;
    r->host_out = out;
    r->spec = JobSpec{nullptr, nullptr, rows, cols, n_sectors, step_m, obs_height_m, max_range_m};
    job_work(n_sectors, rows, cols, step_m, max_range_m, 0, n_sectors, &r->work);
    r->spec.work = r->work.data();
    r->cum_evals.assign(n_sectors + 1, 0.0);
    r->cum_slab.assign(n_sectors + 1, 0);
    r->cum_rows.assign(n_sectors + 1, 0);
    r->cum_items.assign(n_sectors + 1, 0);
    size_t worst_group = 0;
    for (int k = 0; k < n_sectors; ++k) {
        HostDir d;
        make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d);
        const long long wp = (d.W + 3) & ~3;
        r->cum_evals[k + 1] = r->cum_evals[k] + (double)r->work[k].evals;
        r->cum_slab[k + 1] = r->cum_slab[k] + (long long)d.R * wp;
        r->cum_rows[k + 1] = r->cum_rows[k] + d.R;
        r->cum_items[k + 1] = r->cum_items[k] + 2LL * d.R;
        if ((k + 1) % FP32_GROUP == 0 || k + 1 == n_sectors) {
            const int g0 = (k / FP32_GROUP) * FP32_GROUP;
            worst_group = std::max(worst_group,
                                   chunk_bytes((size_t)(r->cum_slab[k + 1] - r->cum_slab[g0]),
                                               r->cum_rows[k + 1] - r->cum_rows[g0], k + 1 - g0));
        }
    }
    if (worst_group + lane_fixed_bytes(S->num_sms, S->cfg.step_slot_bytes) > S->cfg.step_slot_bytes)
        return fail(TVS_ERR_OOM, "8 directions of this DEM do not fit a step slot (raise step_slot_bytes)");
    {
        DeviceGuard g(S->device);
        TVS_CUDA(cudaEventCreateWithFlags(&r->loaded, cudaEventDisableTiming), "event");
        cudaError_t e = cudaEventCreateWithFlags(&r->finished, cudaEventDisableTiming);
        if (e != cudaSuccess) { cudaEventDestroy(r->loaded); return cuda_fail(e, "event"); }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping || S->broken) {
        cudaEventDestroy(r->loaded);
        cudaEventDestroy(r->finished);
        return fail(TVS_ERR_STATE, S->broken ? "the server failed: " + S->broken_msg : "the server is shutting down");
    }
    r->id = S->next_id++;
    r->t_submit = S->now();
    r->evals_total = r->cum_evals.back();
    r->key = r->t_submit + r->evals_total / S->cfg.rate_hint;
    *ticket = r->id;
    S->queue.push_back(r.get());
    S->reqs.emplace(r->id, std::move(r));
    S->st.submitted += 1;
    S->cv_sched.notify_one();
    return TVS_OK;
}

int tvs_server_wait(tvs_server_handle S, int64_t ticket, double timeout_s)
{
    if (!S) return fail(TVS_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TVS_ERR_ARG, "unknown ticket");
    Request* r = it->second.get();
    auto finished = [&] { return r->state == TVS_REQ_DONE || r->state == TVS_REQ_FAILED; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
        return fail(TVS_ERR_TIMEOUT, "the request is not finished");
    }
    if (r->state == TVS_REQ_FAILED) return fail(r->error, r->message);
    return TVS_OK;
}

int tvs_server_query(tvs_server_handle S, int64_t ticket, tvs_request_info* info)
{
    if (!S || !info) return fail(TVS_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TVS_ERR_ARG, "unknown ticket");
    const Request* r = it->second.get();
    std::memset(info, 0, sizeof(*info));
    info->state = r->state;
    info->error = r->error;
    info->steps = r->steps;
    info->n_sectors = r->spec.n;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_first = r->t_first;
    info->t_done = r->t_done;
    info->evals = r->evals_total;
    std::snprintf(info->message, sizeof(info->message), "%s", r->message.c_str());
    return TVS_OK;
}

int tvs_server_forget(tvs_server_handle S, int64_t ticket)
{
    if (!S) return fail(TVS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TVS_ERR_ARG, "unknown ticket");
    Request* r = it->second.get();
    if (r->state != TVS_REQ_DONE && r->state != TVS_REQ_FAILED)
        return fail(TVS_ERR_STATE, "the request is not finished");
    for (Request* f : S->finishing)
        if (f == r) return fail(TVS_ERR_STATE, "the request's download is still being waited for");
    if (r->resident) return fail(TVS_ERR_STATE, "the request still holds arena space");
    if (r->loaded) cudaEventDestroy(r->loaded);
    if (r->finished) cudaEventDestroy(r->finished);
    S->reqs.erase(it);
    return TVS_OK;
}

int tvs_server_get_stats(tvs_server_handle S, tvs_server_stats* stats)
{
    if (!S || !stats) return fail(TVS_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *stats = S->st;
    stats->arena_peak_bytes = (double)S->arena.peak();
    stats->queued = (int32_t)S->queue.size();
    stats->active = (int32_t)S->active.size();
    return TVS_OK;
}

}  // extern "C"
