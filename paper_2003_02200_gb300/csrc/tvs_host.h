// tvs_host.h -- host-side planning shared by the C ABI entry points
// (tvs_api.cu) and the request server (tvs_server.cu): argument checks, the
// direction table, chunking of (job, direction) instances under a byte budget,
// the scratch layout of a planned batch and the launch sequence of its chunks.
#pragma once

#include "tvs.h"
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <climits>
#include <string>
#include <vector>

namespace tvs {

// Error message of the calling thread's last failed call (tvs_last_error).
extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define TVS_CUDA(call, where)                                    \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::tvs::cuda_fail(e_, where); \
    } while (0)

constexpr int kMaxDim = 16384;        // longest walk axis the staged sweep supports
constexpr int kMaxChunkDirs = 4096;   // directions per chunk (bounds the item table in smem)
constexpr long long kMaxChunkItems = 1LL << 30;  // sweep warp items per chunk

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

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

int make_direction(int n, int k, int rows, int cols, double step, double max_range, HostDir* d);
// Usable columns [lo, hi] of skewed row p (hi < lo when none).
void host_row_range(const HostDir& d, int p, int* lo, int* hi);

struct DirWork {
    long long evals;        // targets visited (work count)
    long long samples;      // usable samples (virtual POVs)
};
DirWork direction_work(const HostDir& d);
// Work of directions [k0, k1) of an n-direction job, out[k - k0].  Directions
// with the same reduced angle and the same view shape (k and n - k always; all
// four frames when rows == cols) share one count.
void job_work(int n, int rows, int cols, double step, double max_range, int k0, int k1, std::vector<DirWork>* out);

// Argument checks of one job (sets the thread's error message).
int check_job(int rows, int cols, double step_m, double obs_height_m, int n_sectors, double max_range_m);

// ------------------------------------------------------------ profiling --
enum KernelId { K_ROWMAP = 0, K_SWEEP, K_UNSKEW, K_FINAL, K_POINTS, K_MAP_FLAGS, K_MAP_RASTER, K_COUNT };

// Tunable launch choices (see tvs_tuning in tvs.h).
struct Tuning {
    int small_pov_below_w = 0;     // directions whose walk axis is shorter than this use SMALL_POV groups
    int sweep_max_warps = 0;       // 0 = as many as shared memory allows (up to SWEEP_MAX_WARPS)
    int unskew_ctas_per_sm = 2;    // split a chunk's directions below this many unskew CTAs per SM
    int p4_cost_pct = 107;         // per-row group choice: SMALL_POV step cost relative to LARGE_POV, percent
    int prune = 1;                 // exact horizon pruning in the sweep
    int fp32_decisions = 0;        // 1: FP32 visibility decisions, 0: certified (exact) ones
};

// Group-size mode of a direction (DirDev::pov): forced SMALL_POV below the
// threshold, else chosen per row.
inline int pov_mode(const Tuning& tn, int W) { return W < tn.small_pov_below_w ? SMALL_POV : 0; }

struct Pending {
    int kernel;
    cudaEvent_t start, stop;
    double units;
};

// --------------------------------------------------------------- plans --
// A DEM of a call: device pointers and parameters, and the directions
// [k0, k1) of it that the call covers (k1 < 0: all of them).  A call that
// covers only part of a job's directions passes `acc`, the job's exact running
// totals (one __int128 per cell), which earlier calls have filled when k0 > 0.
struct JobSpec {
    const float* dem;
    float* out;
    int rows, cols, n;
    double step, h0, max_range;
    int k0 = 0, k1 = -1;
    __int128* acc = nullptr;
    const DirWork* work = nullptr;   // work of all n directions when the caller has it, else NULL
};

// A planned chunk: the consecutive (job, direction) instances [i0, i1).
struct Chunk {
    int i0, i1;
    size_t slab_elems;       // sum of R * Wp over the chunk
    long long rows;          // sum of R
    int items;               // sweep warp items
    int max_R, wmax, dmax;
    int cj_beg, ncj;         // the chunk's entries of the chunk-job table
    int total_tiles, max_split;
    long long total_cells, part_elems;
    int istart_at;           // offset of the chunk's item table
    double evals, unskew_bytes, rowmap_bytes, final_bytes;
};

struct BatchPlan {
    std::vector<JobSpec> jobs;
    std::vector<int> inst_job, inst_k;   // per instance
    std::vector<HostDir> hdirs;          // per instance
    std::vector<DirDev> dirs;            // per instance (slab / row offsets relative to its chunk)
    std::vector<Chunk> chunks;
    std::vector<ChunkJob> cj;            // every chunk's job entries, chunk after chunk
    std::vector<int> istart;             // every chunk's item table
    std::vector<long long> acc_off;      // per job: offset of its totals in the plan's own buffer, or -1
    long long acc_elems = 0;
    size_t max_slab = 0;
    long long max_rows = 0, max_part = 0;
    double evals = 0;
};

// Scratch bytes of a chunk's slabs, row tables and item table.
size_t chunk_bytes(size_t slab, long long rows, int ninst);
// Upper bound of the partial totals of a split unskew.
size_t part_bound(int num_sms);

// Plans the instances of `jobs` (job after job, directions in order) into
// chunks whose scratch fits `avail` bytes.  only_k >= 0 keeps only direction
// only_k of a single job (test hook).
int plan_batch(const std::vector<JobSpec>& jobs, size_t avail, int num_sms, const Tuning& tn, BatchPlan* plan,
               int only_k = -1, int smem_optin = 0);

// Scratch layout of a planned batch (byte offsets from the scratch base).  The
// header (directions, jobs, chunk-job entries, item tables) is one contiguous
// block, uploaded with one copy.
struct Layout {
    size_t hdr, dirs, jobs, cj, istart, hdr_bytes;
    size_t io_dem, io_out, counter, flags, flag_cap, acc, part, rowlo, rowhi, cvf, cvb, total;
};

// max_flags bounds the flagged-walk buffer's entries (see flag_entries).
Layout make_layout(const BatchPlan& plan, bool host_io, size_t max_flags = FLAG_BUF_ENTRIES);
// Bytes a batch needs besides its chunks' slabs.
size_t fixed_bytes(const std::vector<JobSpec>& jobs, bool host_io, int num_sms, size_t max_flags);
// The flagged-walk buffer entries a scratch budget allows: a sixteenth of it.
size_t budget_flags(size_t budget);
// Host image of the header for the scratch at `base`.
void build_header(const BatchPlan& plan, const Layout& L, char* base, bool host_io, std::vector<char>* img);

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

}  // namespace tvs

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
    tvs::Tuning tuning;
    bool profiling = false;
    std::vector<tvs::Pending> pending;
    tvs_kernel_stats stats[tvs::K_COUNT];
};

namespace tvs {

// Times the launches enqueued during its lifetime when `h` profiles.
struct Timer {
    tvs_ctx* h;
    int kernel;
    cudaStream_t s;
    double units;
    cudaEvent_t a = nullptr, b = nullptr;
    Timer(tvs_ctx* h_, int k, cudaStream_t s_, double u);
    ~Timer();
};

void drain_pending(tvs_ctx* h);
void reset_stats(tvs_ctx* h);
int ensure_scratch(tvs_ctx* h, size_t bytes);

// Enqueue every chunk of a planned batch whose header already sits at base +
// L.hdr: per chunk row map -> skew -> sweep -> unskew (-> finalize).  `h` may
// be NULL (no profiling).  Returns the number of kernels enqueued in *kernels
// when it is not NULL.  When before_unskew is not NULL the stream waits for it
// before the first unskew (the request server orders the unskews of steps on
// different streams that add to the same totals).
int enqueue_chunks(tvs_ctx* h, const BatchPlan& plan, const Layout& L, char* base, int num_sms, int smem_optin,
                   const Tuning& tn, cudaStream_t s, int* kernels = nullptr, cudaEvent_t before_unskew = nullptr);

// Copy a header image to the device through the handle's pinned staging buffer.
int upload_header(tvs_ctx* h, const std::vector<char>& img, void* dst, cudaStream_t s);

// Plan, size the scratch and enqueue a batch on the handle.  With host_io the
// single job's DEM is copied in from host memory and its map copied back.
int run_batch(tvs_ctx* h, const std::vector<JobSpec>& jobs, cudaStream_t s, bool host_io, const float* host_dem,
              float* host_out);

}  // namespace tvs
