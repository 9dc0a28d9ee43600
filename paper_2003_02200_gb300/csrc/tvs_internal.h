// tvs_internal.h -- types shared by the host orchestration and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tvs {

// Sweep tiling.  Each lane walks two groups of consecutive samples (a group
// and its mirror), 32 lanes per warp item.  A row is swept with groups of
// SMALL_POV samples (blocks of SMALL_UNROLL steps) or of LARGE_POV samples
// (blocks of LARGE_UNROLL steps), chosen per row by row_pov.
constexpr int SMALL_POV = 4;
constexpr int SMALL_UNROLL = 16;
constexpr int LARGE_POV = 8;
constexpr int LARGE_UNROLL = 24;
#ifndef TVS_SWEEP_MAX_WARPS
#define TVS_SWEEP_MAX_WARPS 16
#endif
constexpr int SWEEP_MAX_WARPS = TVS_SWEEP_MAX_WARPS;
// Left pad of a staged row (floats); a multiple of 4.
constexpr int ROW_PADL = 16;
// Right pad: the last window of a block reads up to P + U floats past a target.
constexpr int ROW_PADR = LARGE_POV + 2 * LARGE_UNROLL + 8;
// Directions whose FP32 partial sums are added once into the FP64 total.
constexpr int FP32_GROUP = 8;

// Skew tile: rows x columns of the skewed layout per CTA.
constexpr int SKEW_TP = 64;
constexpr int SKEW_TJ = 32;
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
    int chunks;                // warp items per skewed row and walk direction (the most any row needs)
    int gidx;                  // direction index k within its job
    int job;                   // index of the job in the job table
    float g;                   // 1 + t^2
    float h0;                  // observer height of the job
    int pov;                   // group size of every row (SMALL_POV or LARGE_POV), 0 = chosen per row
    int p4_pct;                // row_pov's relative cost of a SMALL_POV step, percent
};

// Lane slots of a row of L samples swept with groups of P POVs (two mirrored
// groups per slot), and the warp items they take.
__host__ __device__ inline int row_slots(int L, int P) { return ((L + P - 1) / P + 1) / 2; }
__host__ __device__ inline int row_chunks(int L, int P) { return (row_slots(L, P) + 31) / 32; }

// Steps lane 0 of a row walks (groups 0 and G-1, each rounded up to blocks of
// U steps): about every lane's share, since mirrored groups balance.
__host__ __device__ inline long long lane_steps(int L, int K, int P, int U)
{
    const int G = (L + P - 1) / P;
    const int a = (K - 1 < L - 2) ? K - 1 : L - 2;
    const int t = L - 2 - (G - 1) * P;
    const int b = G > 1 ? ((K - 1 < t) ? K - 1 : t) : 0;
    return (a > 0 ? (long long)((a + U - 1) / U) * U : 0) + (b > 0 ? (long long)((b + U - 1) / U) * U : 0);
}

// Group size of a row of L samples with walk limit K: `mode` forces one
// (SMALL_POV or LARGE_POV); mode 0 takes the smaller of items x lane steps x
// P x step cost, a SMALL_POV step costing p4_pct percent of a LARGE_POV step
// per POV.  Only speed depends on it: the measures are exact integers.
__host__ __device__ inline int row_pov(int L, int K, int mode, int p4_pct)
{
    if (mode) return mode;
    const long long c8 = (long long)row_chunks(L, LARGE_POV) * lane_steps(L, K, LARGE_POV, LARGE_UNROLL) *
                         LARGE_POV * 100;
    const long long c4 = (long long)row_chunks(L, SMALL_POV) * lane_steps(L, K, SMALL_POV, SMALL_UNROLL) *
                         SMALL_POV * p4_pct;
    return c4 < c8 ? SMALL_POV : LARGE_POV;
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
cudaError_t launch_skew(const JobDev* d_jobs, const DirDev* d_dirs, int ndir, int max_tiles, float* sdem,
                        cudaStream_t stream);
// Warp items per skewed row and walk direction of a direction whose rows
// have at most W samples: the most any row length up to W needs.
int sweep_chunks(int W, int K, int mode, int p4_pct);
cudaError_t launch_sweep(const DirDev* d_dirs, const int* d_item_start, int ndir, int total_items,
                         const float* sdem, const int* rowlo, const int* rowhi, int* cv_fwd, int* cv_bwd,
                         int wmax, int dmax, unsigned* counter, int num_sms, int smem_optin, int max_warps,
                         cudaStream_t stream);
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
