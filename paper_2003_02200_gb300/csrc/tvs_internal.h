// tvs_internal.h -- types shared by the host orchestration and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tvs {

// Warp work item of the sweep: 32 lanes x POVS_PER_LANE consecutive samples.
// Each lane walks two groups of POVS_PER_LANE consecutive samples (a group and
// its mirror), so a warp item covers 64 groups of one skewed row.  The tile
// constants can be set at compile time (-DTVS_POVS_PER_LANE=8, ...).
#ifndef TVS_POVS_PER_LANE
#define TVS_POVS_PER_LANE 8
#endif
#ifndef TVS_SWEEP_UNROLL
#define TVS_SWEEP_UNROLL 24
#endif
#ifndef TVS_SWEEP_MAX_WARPS
#define TVS_SWEEP_MAX_WARPS 16
#endif
constexpr int POVS_PER_LANE = TVS_POVS_PER_LANE;
constexpr int SWEEP_UNROLL = TVS_SWEEP_UNROLL;
constexpr int WARP_POVS = 64 * POVS_PER_LANE;
constexpr int SWEEP_MAX_WARPS = TVS_SWEEP_MAX_WARPS;
// Left pad of a staged row (floats); a multiple of 4.
constexpr int ROW_PADL = 16;
// Right pad: the last window of a block reads up to P + U floats past a target.
constexpr int ROW_PADR = POVS_PER_LANE + 2 * SWEEP_UNROLL + 8;
// Directions whose FP32 partial sums are added once into the FP64 total.
constexpr int FP32_GROUP = 8;

// Skew tile: rows x columns of the skewed layout per CTA.
constexpr int SKEW_TP = 64;
constexpr int SKEW_TJ = 32;
// Unskew tile: DEM cells per CTA (rows x columns).
constexpr int UNSKEW_TI = 32;
constexpr int UNSKEW_TJ = 32;

// One direction as the kernels see it (section 4.1 step 1, Alg. 6 extended to
// the four eighths of the half-plane by a D4 view of the DEM).
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
    int chunks;                // warp items per skewed row and walk direction, ceil(W / WARP_POVS)
    int gidx;                  // global direction index k
    float g;                   // 1 + t^2
    int pad_;
};

struct KernelTimer;  // host-side event bookkeeping (tvs_api.cu)

// Launchers (tvs_kernels.cu).  All are asynchronous on `stream`.
cudaError_t launch_rowmap(const DirDev* d_dirs, int ndir, int max_R, int* rowlo, int* rowhi,
                          cudaStream_t stream);
cudaError_t launch_colmap(const DirDev* d_dir, int* dest, unsigned* frac, cudaStream_t stream);
cudaError_t launch_skew(const float* dem, int rows, int cols, const DirDev* d_dirs, int ndir,
                        int max_tiles, const int* rowlo, const int* rowhi, float* sdem,
                        cudaStream_t stream);
cudaError_t launch_sweep(const DirDev* d_dirs, const int* d_item_start, int ndir, int total_items,
                         const float* sdem, const int* rowlo, const int* rowhi, int* cv_fwd, int* cv_bwd,
                         float h0, int wmax, int dmax, unsigned* counter, int num_sms, int smem_optin,
                         cudaStream_t stream);
// Number of direction ranges the unskew splits a chunk into for a DEM of this
// size (1 for DEMs with enough cell tiles to fill the GPU).
int unskew_splits(int rows, int cols, int ndir, int num_sms);
int unskew_per_split(int ndir, int nsplit);
int unskew_effective_splits(int ndir, int nsplit);
// Adds the per-range FP64 partials of a split unskew (no-op when nsplit <= 1).
cudaError_t launch_unskew_finalize(int rows, int cols, int ndir, int nsplit, const double* part, double* vs64,
                                   float* out, int first_chunk, int last_chunk, double scale,
                                   cudaStream_t stream);
cudaError_t launch_unskew(const int* cv_fwd, const int* cv_bwd, int rows, int cols, const DirDev* d_dirs,
                          int ndir, int nsplit, double* part, double* vs64, float* out, int first_chunk,
                          int last_chunk, double scale, cudaStream_t stream);


}  // namespace tvs
