// tvs_kernels.cu -- sm_103a kernels of the sDEM total viewshed.
//
//   rowmap : usable column range [jlo, jhi] of every skewed row (section 4.1
//            step 1(b): the limits of the skewed structure).
//   (the relocation of Kernel-1 and the sweep of Kernel-2 live in
//   tvs_sweep.cu: the sweep gathers its rows from the DEM itself)
//   unskew : blends the per-sample measures back onto DEM cells and sums the
//            directions (Kernel-3, Alg. 9), with the Pappus / step^2 scale of
//            Alg. 1 applied once at the end.
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace tvs {

namespace {

__device__ __forceinline__ int dest_of(unsigned long long t_fx, int j)
{
    return (int)(((unsigned long long)j * t_fx) >> 32);
}

// ---------------------------------------------------------------- rowmap --
// Skewed row p holds the line with base row b = p - D: sample j sits at view
// row b + j*t (t = t_fx / 2^32) and is usable iff 0 <= b + j*t <= H - 1,
// i.e. j*t_fx >= -b*2^32 and j*t_fx <= (H-1-b)*2^32 (exact integers).
__global__ void rowmap_kernel(const DirDev* __restrict__ dirs, int* __restrict__ rowlo,
                              int* __restrict__ rowhi)
{
    const DirDev d = dirs[blockIdx.y];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d.R; p += gridDim.x * blockDim.x) {
        const long long b = (long long)p - d.D;
        long long lo, hi;
        if (d.t_fx == 0ull) {
            lo = 0;
            hi = (b >= 0 && b <= d.H - 1) ? d.W - 1 : -1;
        } else {
            lo = 0;
            if (b < 0) {
                const unsigned long long num = (unsigned long long)(-b) << 32;
                lo = (long long)((num + d.t_fx - 1ull) / d.t_fx);
            }
            const long long top = (long long)d.H - 1 - b;
            hi = top < 0 ? -1 : (long long)(((unsigned long long)top << 32) / d.t_fx);
            if (hi > d.W - 1) hi = d.W - 1;
        }
        if (lo > hi) { lo = 0; hi = -1; }
        rowlo[d.row_off + p] = (int)lo;
        rowhi[d.row_off + p] = (int)hi;
    }
}

__global__ void colmap_kernel(const DirDev* __restrict__ dir, int* __restrict__ dest,
                              unsigned* __restrict__ frac)
{
    const DirDev d = *dir;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.W; j += gridDim.x * blockDim.x) {
        const unsigned long long y = (unsigned long long)j * d.t_fx;
        dest[j] = (int)(y >> 32);
        frac[j] = (unsigned)(y & 0xFFFFFFFFull);
    }
}

// ---------------------------------------------------------------- unskew --
// CTA = UNSKEW_TI x UNSKEW_TJ DEM cells and one range of the chunk's
// directions; for each direction the skewed rows those cells blend (both
// virtual POVs of every cell) are staged in shared memory with coalesced row
// reads, then every cell takes g * ((1-r) cv_hi + r cv_lo) (Kernel-3 weights;
// a virtual POV whose sample falls outside the DEM is dropped and the other
// takes weight 1), cv being the forward plus the backward measure.  Partial
// sums are FP32 over groups of FP32_GROUP consecutive directions; each group
// sum is added exactly (fixed point, 128-bit integers) to the cell's total.
// With one range per CTA the total goes to the job's running totals (or, for
// the job's last directions, through the FP64 (pi/(2n)) step^2 scale to the
// FP32 output); with several ranges each writes a partial total that
// unskew_finalize adds.  Integer addition being exact, the result does not
// depend on the ranges, the chunking or the other jobs of a chunk.
constexpr int UNSKEW_ROWS = UNSKEW_TI + UNSKEW_TJ + 4;
constexpr int UNSKEW_PITCH = UNSKEW_TJ + 1;
constexpr int UNSKEW_THREADS = 256;
constexpr int UNSKEW_CELLS = UNSKEW_TI * UNSKEW_TJ / UNSKEW_THREADS;

struct UnskewParams {
    const int* cvf;
    const int* cvb;
    const DirDev* dirs;
    const JobDev* jobs;
    const ChunkJob* cj;
    __int128* part;
    long long total_cells;
    int ncj;
};

// x * 2^ACC_FRAC_BITS as an integer, from the bit pattern of a finite float:
// exact for |x| >= 2^-(ACC_FRAC_BITS - 23) and |x| < 2^67 (every non-zero
// group sum this pipeline forms is in that range: blend weights are at least
// 2^-32 and totals stay below 2^52), truncated toward zero below.
__device__ __forceinline__ __int128 acc_of(float x)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    unsigned long long m = b & 0x7fffffu;
    if (e != 0) m |= 0x800000u;
    const int sh = (e == 0 ? 1 : e) - 150 + ACC_FRAC_BITS;     // x = m * 2^(sh - ACC_FRAC_BITS)
    __int128 v;
    if (sh >= 0) v = (__int128)m << min(sh, 100);
    else v = sh > -32 ? (__int128)(m >> -sh) : (__int128)0;
    return (b >> 31) ? -v : v;
}

// FP32 visible area of an exact total: total * 2^-ACC_FRAC_BITS * scale.
__device__ __forceinline__ float area_of(__int128 v, double scale)
{
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    // hi * 2^64 is exact (totals stay below 2^108); (double)lo and the sum round once each
    const double t = __dadd_rn(__dmul_rn((double)hi, 0x1p64), (double)lo);
    return __double2float_rn(__dmul_rn(__dmul_rn(t, 0x1p-56), scale));
}
static_assert(ACC_FRAC_BITS == 56, "area_of scales by 2^-56");

// Entry of the chunk's job table that holds flattened index t (entries are
// sorted by tile_beg or by cell_beg; `cells` selects which).
__device__ __forceinline__ int find_chunk_job(const ChunkJob* __restrict__ cj, int ncj, long long t, bool cells)
{
    int lo = 0, hi = ncj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long beg = cells ? cj[mid].cell_beg : (long long)cj[mid].tile_beg;
        if (beg <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Asynchronous global -> shared copies of 4 bytes and of 16 bytes (both
// addresses 16-byte aligned).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(sa), "l"(gmem) : "memory");
}

// Row pitch of a staged window.  In views 0 and 3 a warp's lanes blend 32
// consecutive view columns of one view row, whose skewed rows step down with
// the column: pitch 32 keeps each lane on its own bank, and rows of 128 bytes
// take 16-byte copies (the window starts at a tile column, a multiple of 32,
// in rows padded to a multiple of 4).  In views 1 and 2 the lanes blend 32
// consecutive view rows at one column: pitch 33 keeps them on distinct banks
// (4-byte copies).
__device__ __forceinline__ int unskew_pitch(int frame) { return frame == 0 || frame == 3 ? 32 : UNSKEW_PITCH; }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// The staged window of one direction for a tile: skewed rows pmin.. (np of
// them) and view columns vj0.. (nj of them) of the direction's slabs.
struct UnskewWin {
    int pmin, np, vj0, nj;
};

__device__ __forceinline__ UnskewWin unskew_window(const DirDev& d, int iD0, int iD1, int jD0, int jD1)
{
    int vi0, vi1, vj0, vj1;
    switch (d.frame) {
    case 0:  vi0 = iD0; vi1 = iD1; vj0 = jD0; vj1 = jD1; break;
    case 1:  vi0 = jD0; vi1 = jD1; vj0 = iD0; vj1 = iD1; break;
    case 2:  vi0 = jD0; vi1 = jD1; vj0 = d.W - 1 - iD1; vj1 = d.W - 1 - iD0; break;
    default: vi0 = d.H - 1 - iD1; vi1 = d.H - 1 - iD0; vj0 = jD0; vj1 = jD1; break;
    }
    UnskewWin w;
    w.pmin = max(vi0 - dest_of(d.t_fx, vj1) + d.D - 1, 0);
    const int pmax = min(vi1 - dest_of(d.t_fx, vj0) + d.D, d.R - 1);
    w.np = pmax - w.pmin + 1;
    w.vj0 = vj0;
    w.nj = vj1 - vj0 + 1;
    return w;
}

// Copies (asynchronously) the forward and backward measures of a window.
__device__ __forceinline__ void unskew_stage(const UnskewParams& up, const DirDev& d, const UnskewWin& w, int* SF,
                                             int* SB)
{
    const long long off = d.slab + (long long)w.pmin * d.Wp + w.vj0;
    if (d.frame == 0 || d.frame == 3) {
        // 8 chunks of 4 columns per row; the last may read up to 3 padding
        // columns of the row (vj0 + 4 ceil(nj / 4) <= Wp)
        for (int idx = threadIdx.x; idx < w.np * 8; idx += UNSKEW_THREADS) {
            const int r = idx >> 3, q4 = (idx & 7) * 4;
            if (q4 < w.nj) {
                const long long a = off + (long long)r * d.Wp + q4;
                cp_async16(SF + r * 32 + q4, up.cvf + a);
                cp_async16(SB + r * 32 + q4, up.cvb + a);
            }
        }
    } else {
        for (int idx = threadIdx.x; idx < w.np * 32; idx += UNSKEW_THREADS) {
            const int r = idx >> 5, cc = idx & 31;
            if (cc < w.nj) {
                const long long a = off + (long long)r * d.Wp + cc;
                cp_async4(SF + r * UNSKEW_PITCH + cc, up.cvf + a);
                cp_async4(SB + r * UNSKEW_PITCH + cc, up.cvb + a);
            }
        }
    }
}

// Directions are double-buffered: while the cells of a tile blend one
// direction's staged rows, the next direction's rows are in flight.
__global__ void __launch_bounds__(UNSKEW_THREADS, 4) unskew_kernel(UnskewParams up)
{
    __shared__ __align__(16) int SF[2][UNSKEW_ROWS * UNSKEW_PITCH];
    __shared__ __align__(16) int SB[2][UNSKEW_ROWS * UNSKEW_PITCH];
    static_assert((UNSKEW_ROWS * UNSKEW_PITCH * 4) % 16 == 0, "second buffers stay 16-byte aligned");
    const ChunkJob c = up.cj[find_chunk_job(up.cj, up.ncj, blockIdx.x, false)];
    if ((int)blockIdx.z >= c.nsplit) return;
    const JobDev J = up.jobs[c.job];
    const int rows = J.rows, cols = J.cols;
    const int tile = blockIdx.x - c.tile_beg;
    const int ty = tile / c.tiles_x, tx = tile - ty * c.tiles_x;
    const int iD0 = ty * UNSKEW_TI, jD0 = tx * UNSKEW_TJ;
    const int iD1 = min(iD0 + UNSKEW_TI, rows) - 1, jD1 = min(jD0 + UNSKEW_TJ, cols) - 1;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int kbeg = c.dbeg + blockIdx.z * c.per_split;
    const int kend = min(kbeg + c.per_split, c.dbeg + c.dcnt);
    float acc32[UNSKEW_CELLS];
    __int128 accx[UNSKEW_CELLS];
#pragma unroll
    for (int m = 0; m < UNSKEW_CELLS; ++m) { acc32[m] = 0.f; accx[m] = 0; }
    int group = kbeg < kend ? up.dirs[kbeg].gidx / FP32_GROUP : 0;

    DirDev d_next;
    UnskewWin w_next{0, 0, 0, 0};
    if (kbeg < kend) {
        d_next = up.dirs[kbeg];
        w_next = unskew_window(d_next, iD0, iD1, jD0, jD1);
        unskew_stage(up, d_next, w_next, SF[0], SB[0]);
    }
    cp_async_commit();
    for (int kk = kbeg; kk < kend; ++kk) {
        const int buf = (kk - kbeg) & 1;
        const DirDev d = d_next;
        const UnskewWin w = w_next;
        if (kk + 1 < kend) {
            d_next = up.dirs[kk + 1];
            w_next = unskew_window(d_next, iD0, iD1, jD0, jD1);
            unskew_stage(up, d_next, w_next, SF[buf ^ 1], SB[buf ^ 1]);
        }
        cp_async_commit();
        cp_async_wait<1>();          // every group but the one just issued has landed
        __syncthreads();
        if (d.gidx / FP32_GROUP != group) {
#pragma unroll
            for (int m = 0; m < UNSKEW_CELLS; ++m) { accx[m] += acc_of(acc32[m]); acc32[m] = 0.f; }
            group = d.gidx / FP32_GROUP;
        }
        const int* F = SF[buf];
        const int* B = SB[buf];
        const int pitch = unskew_pitch(d.frame);
#pragma unroll
        for (int m = 0; m < UNSKEW_CELLS; ++m) {
            const int iD = iD0 + ly + 8 * m, jD = jD0 + lx;
            if (iD > iD1 || jD > jD1) continue;
            int i, j;
            switch (d.frame) {
            case 0:  i = iD; j = jD; break;
            case 1:  i = jD; j = iD; break;
            case 2:  i = jD; j = d.W - 1 - iD; break;
            default: i = d.H - 1 - iD; j = jD; break;
            }
            const unsigned long long y = (unsigned long long)j * d.t_fx;
            const int dest = (int)(y >> 32);
            const unsigned fr = (unsigned)(y & 0xFFFFFFFFull);
            const int hi = (i - dest + d.D - w.pmin) * pitch + (j - w.vj0);   // line through i + r
            const int lo = hi - pitch;                                       // line through i - 1 + r
            float val;
            if (fr == 0u) {
                val = (float)(F[hi] + B[hi]);
            } else {
                const bool hi_ok = i <= d.H - 2, lo_ok = i >= 1;
                if (hi_ok && lo_ok) {
                    const float r = __fmul_rn(__uint2float_rn(fr), 0x1p-32f);
                    val = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, r), (float)(F[hi] + B[hi])),
                                    __fmul_rn(r, (float)(F[lo] + B[lo])));
                } else if (hi_ok) {
                    val = (float)(F[hi] + B[hi]);
                } else {
                    val = (float)(F[lo] + B[lo]);
                }
            }
            acc32[m] = __fadd_rn(acc32[m], __fmul_rn(d.g, val));
        }
        __syncthreads();             // the buffer is refilled two directions later
    }
    cp_async_wait<0>();
    const long long cells = (long long)rows * cols;
#pragma unroll
    for (int m = 0; m < UNSKEW_CELLS; ++m) {
        const int iD = iD0 + ly + 8 * m, jD = jD0 + lx;
        if (iD > iD1 || jD > jD1) continue;
        const long long idx = (long long)iD * cols + jD;
        __int128 tot = accx[m] + acc_of(acc32[m]);
        if (c.nsplit > 1) {
            up.part[c.part_off + (long long)blockIdx.z * cells + idx] = tot;
            continue;
        }
        if (!c.first) tot += J.acc[idx];
        if (c.last) J.out[idx] = area_of(tot, J.scale);
        else J.acc[idx] = tot;
    }
}

__global__ void unskew_finalize(UnskewParams up)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < up.total_cells;
         t += (long long)gridDim.x * blockDim.x) {
        const ChunkJob c = up.cj[find_chunk_job(up.cj, up.ncj, t, true)];
        if (c.nsplit <= 1) continue;
        const JobDev J = up.jobs[c.job];
        const long long cells = (long long)J.rows * J.cols;
        const long long idx = t - c.cell_beg;
        __int128 tot = 0;
        for (int z = 0; z < c.nsplit; ++z) tot += up.part[c.part_off + z * cells + idx];
        if (!c.first) tot += J.acc[idx];
        if (c.last) J.out[idx] = area_of(tot, J.scale);
        else J.acc[idx] = tot;
    }
}

}  // namespace

// -------------------------------------------------------------- launchers --
cudaError_t launch_rowmap(const DirDev* d_dirs, int ndir, int max_R, int* rowlo, int* rowhi,
                          cudaStream_t stream)
{
    if (ndir <= 0) return cudaSuccess;
    dim3 grid((max_R + 255) / 256, ndir);
    rowmap_kernel<<<grid, 256, 0, stream>>>(d_dirs, rowlo, rowhi);
    return cudaGetLastError();
}

cudaError_t launch_colmap(const DirDev* d_dir, int* dest, unsigned* frac, cudaStream_t stream)
{
    colmap_kernel<<<64, 256, 0, stream>>>(d_dir, dest, frac);
    return cudaGetLastError();
}

int unskew_per_split(int ndir, int nsplit)
{
    const int groups = (ndir + FP32_GROUP - 1) / FP32_GROUP;
    nsplit = std::max(1, std::min(nsplit, groups));
    return ((groups + nsplit - 1) / nsplit) * FP32_GROUP;
}

int unskew_effective_splits(int ndir, int nsplit)
{
    const int per = unskew_per_split(ndir, nsplit);
    return (ndir + per - 1) / per;
}

int unskew_tiles_x(int cols) { return (cols + UNSKEW_TJ - 1) / UNSKEW_TJ; }

int unskew_tiles(int rows, int cols) { return unskew_tiles_x(cols) * ((rows + UNSKEW_TI - 1) / UNSKEW_TI); }

int unskew_splits(long long chunk_tiles, int ndir, int num_sms, int ctas_per_sm)
{
    const long long want = ((long long)std::max(ctas_per_sm, 1) * num_sms + chunk_tiles - 1) / std::max(chunk_tiles, 1LL);
    const int groups = (ndir + FP32_GROUP - 1) / FP32_GROUP;
    return (int)std::max<long long>(1, std::min<long long>(want, groups));
}

cudaError_t launch_unskew(const int* cv_fwd, const int* cv_bwd, const JobDev* d_jobs, const DirDev* d_dirs,
                          const ChunkJob* d_cj, int ncj, int total_tiles, int max_split, __int128* part,
                          cudaStream_t stream)
{
    if (ncj <= 0 || total_tiles <= 0) return cudaSuccess;
    UnskewParams up{};
    up.cvf = cv_fwd; up.cvb = cv_bwd; up.dirs = d_dirs; up.jobs = d_jobs; up.cj = d_cj; up.part = part;
    up.ncj = ncj;
    dim3 grid(total_tiles, 1, std::max(max_split, 1));
    unskew_kernel<<<grid, UNSKEW_THREADS, 0, stream>>>(up);
    return cudaGetLastError();
}

cudaError_t launch_unskew_finalize(const JobDev* d_jobs, const ChunkJob* d_cj, int ncj, long long total_cells,
                                   const __int128* part, cudaStream_t stream)
{
    if (ncj <= 0 || total_cells <= 0) return cudaSuccess;
    UnskewParams up{};
    up.jobs = d_jobs; up.cj = d_cj; up.ncj = ncj; up.part = const_cast<__int128*>(part);
    up.total_cells = total_cells;
    const int blocks = (int)std::min<long long>((total_cells + 255) / 256, 4096);
    unskew_finalize<<<blocks, 256, 0, stream>>>(up);
    return cudaGetLastError();
}

}  // namespace tvs
