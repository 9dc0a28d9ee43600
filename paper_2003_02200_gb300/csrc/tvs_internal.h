// tvs_internal.h -- types shared by the host orchestration and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tvs {

// Sweep tiling.  A warp item is one skewed row and one walk direction; the
// row's POVs form groups of consecutive samples that the 32 lanes take from a
// queue.  A row is swept with groups of SMALL_POV samples (blocks of
// SMALL_UNROLL steps) or of LARGE_POV samples (blocks of LARGE_UNROLL steps),
// chosen per row by row_pov.
constexpr int SMALL_POV = 4;
constexpr int SMALL_UNROLL = 16;
constexpr int LARGE_POV = 8;
constexpr int LARGE_UNROLL = 28;
#ifndef TVS_SWEEP_MAX_WARPS
#define TVS_SWEEP_MAX_WARPS 16
#endif
constexpr int SWEEP_MAX_WARPS = TVS_SWEEP_MAX_WARPS;
// Left pad of a staged row (floats); a multiple of 4, at most 32 (one lane
// per pad sample fills it), and at least a certified block's step count (a
// backward block's window starts that many samples before its group).
constexpr int ROW_PADL = 32;
// Right pad: the last window of a block reads up to P + U floats past a target.
constexpr int ROW_PADR = LARGE_POV + 2 * LARGE_UNROLL + 8;
// Directions whose FP32 partial sums are added once into the FP64 total.
constexpr int FP32_GROUP = 8;

// Unskew tile: DEM cells per CTA (rows x columns).
constexpr int UNSKEW_TI = 32;
constexpr int UNSKEW_TJ = 32;

// One direction of one job as the kernels see it (section 4.1 step 1, Alg. 6
// extended to the four eighths of the half-plane by a D4 view of the DEM).
struct DirDev {
    unsigned long long t_fx;   // llround(tan(alpha) * 2^32), 0 .. 2^32
    long long slab;            // element offset of this direction's skewed slab
    int frame;                 // 0 identity, 1 transpose, 2 transpose+mirror cols, 3 mirror rows
    int H, W;                  // view shape; W is the walk axis
    int Wp;                    // row pitch of the skewed slab (W rounded up to 4)
    int D;                     // dest(W - 1)
    int R;                     // skewed rows, H + D; row p has base row p - D
    int K;                     // walk limit in steps, clipped to [0, W]
    int row_off;               // offset of this direction in the row tables
    int gidx;                  // direction index k within its job
    int job;                   // index of the job in the job table
    float g;                   // 1 + t^2
    float h0;                  // observer height of the job, rounded to single precision
    float h0_lo;               // h0 - (double)h0 above, rounded (h0 to about 2^-48)
    int pov;                   // group size of every row (SMALL_POV or LARGE_POV), 0 = chosen per row
    int p4_pct;                // row_pov's relative cost of a SMALL_POV step, percent
};

// Lane steps of the sweep of one row of L samples (walk limit K) with groups
// of P POVs: `total` over all groups (unrounded walk lengths) and `longest`
// (group 0).  A row's 32 lanes share its groups, so it takes about
// max(total / 32, longest) steps of P POVs.
__host__ __device__ inline void row_steps(int L, int K, int P, long long* total, long long* longest)
{
    const long long c = K - 1, G = (L + P - 1) / P;
    *longest = c < L - 2 ? (c > 0 ? c : 0) : (L - 2 > 0 ? L - 2 : 0);
    if (c <= 0 || L < 3) { *total = 0; return; }
    // groups with L - 2 - gP >= c walk c steps, the rest L - 2 - gP while positive
    long long n1 = L - 2 - c >= 0 ? (L - 2 - c) / P + 1 : 0;
    if (n1 > G) n1 = G;
    long long glast = (L - 3) / P;
    if (glast > G - 1) glast = G - 1;
    long long t = n1 * c;
    if (glast >= n1) {
        const long long cnt = glast - n1 + 1;
        t += cnt * (L - 2) - (long long)P * (n1 + glast) * cnt / 2;
    }
    *total = t;
}

// Group size of a row of L samples with walk limit K: `mode` forces one
// (SMALL_POV or LARGE_POV); mode 0 takes the smaller of
// max(total / 32, longest) x P x step cost, a SMALL_POV step costing p4_pct
// percent of a LARGE_POV step per POV.  Only speed depends on it: the
// measures are exact integers.
__host__ __device__ inline int row_pov(int L, int K, int mode, int p4_pct)
{
    if (mode) return mode;
    long long t8, l8, t4, l4;
    row_steps(L, K, LARGE_POV, &t8, &l8);
    row_steps(L, K, SMALL_POV, &t4, &l4);
    const long long s8 = (t8 + 31) / 32 > l8 ? (t8 + 31) / 32 : l8;
    const long long s4 = (t4 + 31) / 32 > l4 ? (t4 + 31) / 32 : l4;
    return s4 * SMALL_POV * p4_pct < s8 * LARGE_POV * 100 ? SMALL_POV : LARGE_POV;
}

// Per-cell totals are exact: each FP32 group sum (FP32_GROUP directions) is
// converted to a signed fixed-point integer with ACC_FRAC_BITS fractional bits
// and added in 128-bit integer arithmetic, so a total does not depend on the
// order in which chunks, CTAs or steps add their groups.
constexpr int ACC_FRAC_BITS = 56;

// One DEM of a call (a batch holds several).
struct JobDev {
    const float* dem;          // rows x cols elevations (device)
    float* out;                // rows x cols visible areas (device)
    __int128* acc;             // exact running totals when the job spans several chunks, else NULL
    double scale;              // (pi / (2n)) * step^2
    double h0;                 // observer height (the FP64 walks of the certified sweep)
    int rows, cols;
};

// One job's share of a chunk of directions, for the unskew and its finalize.
struct ChunkJob {
    long long cell_beg;        // first cell of the job in the chunk's flattened cell space
    long long part_off;        // exact partials of a split unskew: offset in the partials buffer
    int job;                   // index in the job table
    int dbeg, dcnt;            // the job's directions in the chunk (chunk-local)
    int tile_beg;              // first unskew tile of the job in the chunk's flattened tiles
    int tiles_x;               // cell tiles per DEM row
    int first, last;           // the chunk is the job's first / last one
    int nsplit;                // direction ranges of the unskew (1 = no partials)
    int per_split;             // directions per range (a multiple of FP32_GROUP)
    int pad_;
};

// Launchers (tvs_kernels.cu).  All are asynchronous on `stream`.
cudaError_t launch_rowmap(const DirDev* d_dirs, int ndir, int max_R, int* rowlo, int* rowhi,
                          cudaStream_t stream);
cudaError_t launch_colmap(const DirDev* d_dir, int* dest, unsigned* frac, cudaStream_t stream);
// Sweep of a chunk (tvs_sweep.cu): one warp item per skewed row and walk
// direction (items 2p and 2p + 1 of a direction are row p forward and
// backward), its row gathered from the job's DEM; `prune` turns exact horizon
// pruning on, `cert` certified (exact) visibility decisions instead of FP32
// ones.  With cert and a flag buffer (flag_cap entries, flag_count two
// counters) the walks the sweep cannot certify are walked exactly by a second
// kernel on the same stream; without one (or once it is full) the sweep's
// warps walk them themselves.
cudaError_t launch_sweep(const DirDev* d_dirs, const JobDev* d_jobs, const int* d_item_start, int ndir,
                         int total_items, const int* rowlo, const int* rowhi, int* cv_fwd, int* cv_bwd, int wmax,
                         int dmax, int prune, int cert, unsigned* counter, int4* flag_buf, unsigned* flag_count,
                         int flag_cap, int num_sms, int smem_optin, int max_warps, cudaStream_t stream);
// Layout class of a certified sweep launch (rows up to wmax samples, walks
// up to dmax steps, ndir directions): the warps of its one-row-per-warp
// kernel (16 or 12), or 0 when its rows go to warp pairs.  Chunks of a batch
// are cut where the class changes, so that short rows do not run in a launch
// sized for long ones.
int cert_sweep_class(int wmax, int dmax, int prune, int ndir, int smem_optin);
// Entries of a launch's flagged-walk buffer (16 bytes each), at most.
constexpr int FLAG_BUF_ENTRIES = 1 << 24;
constexpr int FLAG_ENTRY_BYTES = 16;
// Unskew of a chunk: `total_tiles` flattened cell tiles over the chunk's jobs
// (ncj entries of d_cj, sorted by tile_beg), `max_split` the largest nsplit.
cudaError_t launch_unskew(const int* cv_fwd, const int* cv_bwd, const JobDev* d_jobs, const DirDev* d_dirs,
                          const ChunkJob* d_cj, int ncj, int total_tiles, int max_split, __int128* part,
                          cudaStream_t stream);
// Adds the exact partials of the chunk's split jobs (a no-op entry for the others).
cudaError_t launch_unskew_finalize(const JobDev* d_jobs, const ChunkJob* d_cj, int ncj, long long total_cells,
                                   const __int128* part, cudaStream_t stream);

// Number of direction ranges for one job of a chunk whose jobs have
// `chunk_tiles` cell tiles in all (1 when the chunk fills the GPU).
int unskew_splits(long long chunk_tiles, int ndir, int num_sms, int ctas_per_sm);
int unskew_per_split(int ndir, int nsplit);
int unskew_effective_splits(int ndir, int nsplit);
int unskew_tiles_x(int cols);
int unskew_tiles(int rows, int cols);

}  // namespace tvs
