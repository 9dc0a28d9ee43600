// tvs_points.cu -- singular and multiple viewsheds of a list of points of view
// (section 2.1 of the paper: the singular viewshed of Alg. 1-3 and the
// multiple viewshed of several POVs; the paper's first experiment measures the
// accumulated viewshed of 10 random POVs).
//
// Two readings of a POV's lines of sight:
//   TVS_POINTS_SDEM   the sDEM discretisation of the total viewshed: the POV is
//                     blended from the two sampled lines through whole rows
//                     that straddle it (Kernel-3 weights), so the area is bit
//                     for bit the value the total viewshed map holds for the
//                     cell (same samples, slopes, FP32 group sums and exact
//                     totals);
//   TVS_POINTS_DIRECT Alg. 1-3 by definition: every line passes through the
//                     POV cell itself (no virtual POVs); comparing it with the
//                     sDEM value measures the discretisation, as section 5
//                     compares sDEM with TVS.
//
// One warp per (POV, group of FP32_GROUP directions): lane = 4 kk + 2 v + s
// walks direction 8 g + kk, virtual POV v (hi / lo; DIRECT uses v = 0 only),
// forward (s = 0) or backward (s = 1).  The walk is the sweep's: targets
// d = 1 .. n (n = min(usable samples, K)), visible iff the FP32 slope
// (z - h) * rcp(d) is strictly above the running maximum, and
// cv = 1 + sum_{d < n} v_d (2d + 1) for n >= 1 (the last target only closes a
// segment).  Lane 0 adds the group's terms g * blend(cv) in direction order in
// FP32 and stores the group sum as an exact partial; a finalize kernel adds
// each POV's partials and applies the (pi/(2n)) step^2 scale.
#include "tvs.h"
#include "tvs_host.h"
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace tvs {
namespace {

struct PointsParams {
    const float* dem;
    const DirDev* dirs;     // the job's n directions (t_fx, frame, H, W, K, g)
    const int* pov;         // npov (row, col) pairs of DEM cells
    __int128* part;         // npov x ngroups exact group sums
    float* area;            // npov visible areas
    double scale;           // (pi / (2n)) step^2
    int rows, cols, n, ngroups, npov, mode;
    float h0;
};

// View value V[i][j] of the direction's D4 view, read from the row-major DEM.
__device__ __forceinline__ float view_at(const float* dem, int cols, const DirDev& d, long long i, long long j)
{
    switch (d.frame) {
    case 0:  return dem[i * cols + j];
    case 1:  return dem[j * cols + i];
    case 2:  return dem[(d.W - 1 - j) * cols + i];
    default: return dem[(d.H - 1 - i) * cols + j];
    }
}

// Row a and 32-bit fraction of the sample at column j of a line: through
// base row b at column 0 (SDEM: y = j t) or through view cell (i0, j0)
// (DIRECT: y = (j - j0) t, either sign).
__device__ __forceinline__ void line_pos(const DirDev& d, bool direct, long long base, int j0, int j, long long* a,
                                         unsigned* fr)
{
    const long long y = (long long)(direct ? j - j0 : j) * (long long)d.t_fx;   // |y| < 2^47
    const long long q = y >> 32;                                                 // floor, arithmetic shift
    *a = base + q;
    *fr = (unsigned)(y - q * 4294967296LL);
}

// Blended height of a usable sample (Alg. 6, the skew kernel's arithmetic).
__device__ __forceinline__ float sample_at(const float* dem, int cols, const DirDev& d, long long a, unsigned fr, int j)
{
    const float va = view_at(dem, cols, d, a, j);
    if (fr == 0u) return va;
    const float r = __fmul_rn(__uint2float_rn(fr), 0x1p-32f);
    const float wa = __fsub_rn(1.0f, r);
    return __fadd_rn(__fmul_rn(wa, va), __fmul_rn(r, view_at(dem, cols, d, a + 1, j)));
}

__device__ __forceinline__ bool usable(const DirDev& d, long long a, unsigned fr, int j)
{
    if (j < 0 || j >= d.W || a < 0) return false;
    return fr == 0u ? a <= d.H - 1 : a + 1 <= d.H - 1;
}

__device__ __forceinline__ __int128 acc_of(float x)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    unsigned long long m = b & 0x7fffffu;
    if (e != 0) m |= 0x800000u;
    const int sh = (e == 0 ? 1 : e) - 150 + ACC_FRAC_BITS;
    __int128 v;
    if (sh >= 0) v = (__int128)m << min(sh, 100);
    else v = sh > -32 ? (__int128)(m >> -sh) : (__int128)0;
    return (b >> 31) ? -v : v;
}

__device__ __forceinline__ float area_of(__int128 v, double scale)
{
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    const double t = __dadd_rn(__dmul_rn((double)hi, 0x1p64), (double)lo);
    return __double2float_rn(__dmul_rn(__dmul_rn(t, 0x1p-56), scale));
}
static_assert(ACC_FRAC_BITS == 56, "area_of scales by 2^-56");

__global__ void __launch_bounds__(32) points_kernel(PointsParams pp)
{
    const int lane = threadIdx.x;
    const int q = (int)(blockIdx.x / (unsigned)pp.ngroups), grp = (int)(blockIdx.x % (unsigned)pp.ngroups);
    const int kk = lane >> 2, v = (lane >> 1) & 1, s = lane & 1;
    const int k = grp * FP32_GROUP + kk;
    const bool direct = pp.mode == TVS_POINTS_DIRECT;
    int cv = 0;                      // this lane's half-line measure
    bool valid = false;              // this lane's line exists
    float r = 0.f;                   // blend weight of the lo line (SDEM)
    bool hi_ok = true, lo_ok = false;
    unsigned fr0 = 0u;
    DirDev d;
    if (k < pp.n) {
        d = pp.dirs[k];
        const int iD = pp.pov[2 * q], jD = pp.pov[2 * q + 1];
        int i, j0;
        switch (d.frame) {
        case 0:  i = iD; j0 = jD; break;
        case 1:  i = jD; j0 = iD; break;
        case 2:  i = jD; j0 = d.W - 1 - iD; break;
        default: i = d.H - 1 - iD; j0 = jD; break;
        }
        long long base;              // the line: base row at column 0 (SDEM) or the cell row (DIRECT)
        if (direct) {
            valid = v == 0;
            base = i;
        } else {
            const unsigned long long y = (unsigned long long)j0 * d.t_fx;
            const int dest = (int)(y >> 32);
            fr0 = (unsigned)(y & 0xFFFFFFFFull);
            hi_ok = fr0 == 0u || i <= d.H - 2;
            lo_ok = fr0 != 0u && i >= 1;
            r = __fmul_rn(__uint2float_rn(fr0), 0x1p-32f);
            valid = v == 0 ? hi_ok : lo_ok;
            base = (long long)i - dest - v;
        }
        if (valid) {
            long long a;
            unsigned fr;
            line_pos(d, direct, base, j0, j0, &a, &fr);
            const float h = __fadd_rn(direct ? view_at(pp.dem, pp.cols, d, i, j0)
                                             : sample_at(pp.dem, pp.cols, d, a, fr, j0), pp.h0);
            const int dir = s ? -1 : 1;
            // targets d = 1 .. n, n = min(usable samples, K); a target's 2d + 1 is
            // committed once the next target exists (the last one only closes a segment)
            int n = 0, pend = 0;
            long long sum = 0;
            float M = __int_as_float(0xff800000);
            for (int dd = 1; dd <= d.K; ++dd) {
                const int j = j0 + dir * dd;
                line_pos(d, direct, base, j0, j, &a, &fr);
                if (!usable(d, a, fr, j)) break;
                sum += pend;
                const float z = sample_at(pp.dem, pp.cols, d, a, fr, j);
                const float t = __fmul_rn(__fsub_rn(z, h), __frcp_rn((float)dd));
                pend = t > M ? 2 * dd + 1 : 0;
                M = fmaxf(M, t);
                n = dd;
            }
            cv = n >= 1 ? (int)(1 + sum) : 0;
        }
    }
    // cv_fwd + cv_bwd of each line, then the direction's blend (Kernel-3)
    const int both = cv + __shfl_xor_sync(0xffffffffu, cv, 1);
    const float T = (float)both;
    const float T_other = __shfl_xor_sync(0xffffffffu, T, 2);   // the other virtual POV of the direction
    float val = 0.f;
    if (lane % 4 == 0 && k < pp.n) {
        if (direct || fr0 == 0u) val = T;
        else if (hi_ok && lo_ok) val = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, r), T), __fmul_rn(r, T_other));
        else if (hi_ok) val = T;
        else val = T_other;
    }
    const float term = (lane % 4 == 0 && k < pp.n) ? __fmul_rn(d.g, val) : 0.f;
    // FP32 sum of the group's terms in direction order, then one exact partial
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < FP32_GROUP; ++m) {
        const float tm = __shfl_sync(0xffffffffu, term, 4 * m);
        if (grp * FP32_GROUP + m < pp.n) acc = __fadd_rn(acc, tm);
    }
    if (lane == 0) pp.part[(long long)q * pp.ngroups + grp] = acc_of(acc);
}

__global__ void points_finalize(PointsParams pp)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= pp.npov) return;
    __int128 tot = 0;
    for (int g = 0; g < pp.ngroups; ++g) tot += pp.part[(long long)q * pp.ngroups + g];
    pp.area[q] = area_of(tot, pp.scale);
}

// ------------------------------------------------------------ visibility map --
// flags[(q * 2n + slot) * cap + d] = 1 when target d of a half-line of POV q
// is visible: slot k walks +j of direction k's view, slot n + k walks -j, both
// along the line through the POV cell itself (the direct reading).
struct MapParams {
    const float* dem;
    const DirDev* dirs;
    const int* pov;
    unsigned char* flags;
    int* count;
    int rows, cols, n, npov, cap;
    float h0;
};

__global__ void __launch_bounds__(64) map_flags_kernel(MapParams mp)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (q, slot)
    if (t >= (long long)mp.npov * 2 * mp.n) return;
    const int q = (int)(t / (2 * mp.n)), slot = (int)(t % (2 * mp.n));
    const int k = slot % mp.n, dir = slot < mp.n ? 1 : -1;
    const DirDev d = mp.dirs[k];
    const int iD = mp.pov[2 * q], jD = mp.pov[2 * q + 1];
    int i, j0;
    switch (d.frame) {
    case 0:  i = iD; j0 = jD; break;
    case 1:  i = jD; j0 = iD; break;
    case 2:  i = jD; j0 = d.W - 1 - iD; break;
    default: i = d.H - 1 - iD; j0 = jD; break;
    }
    unsigned char* f = mp.flags + t * mp.cap;
    const float h = __fadd_rn(view_at(mp.dem, mp.cols, d, i, j0), mp.h0);
    float M = __int_as_float(0xff800000);
    for (int dd = 1; dd <= d.K && dd < mp.cap; ++dd) {
        const int j = j0 + dir * dd;
        long long a;
        unsigned fr;
        line_pos(d, true, i, j0, j, &a, &fr);
        if (!usable(d, a, fr, j)) break;
        const float z = sample_at(mp.dem, mp.cols, d, a, fr, j);
        const float th = __fmul_rn(__fsub_rn(z, h), __frcp_rn((float)dd));
        f[dd] = th > M ? 1 : 0;
        M = fmaxf(M, th);
    }
}

// View coordinates of DEM cell (iD, jD) in direction d's view.
__device__ __forceinline__ void to_view(const DirDev& d, int iD, int jD, int* i, int* j)
{
    switch (d.frame) {
    case 0:  *i = iD; *j = jD; break;
    case 1:  *i = jD; *j = iD; break;
    case 2:  *i = jD; *j = d.W - 1 - iD; break;
    default: *i = d.H - 1 - iD; *j = jD; break;
    }
}

// One thread per cell: the sector of each POV it falls in (nearest of the 2n
// half-line axes k' pi / n, from a double-precision angle) and the flag of
// the target at the cell's walk-axis column.
__global__ void map_raster_kernel(MapParams mp)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (long long)mp.rows * mp.cols) return;
    const int iD = (int)(c / mp.cols), jD = (int)(c % mp.cols);
    int seen = 0;
    for (int q = 0; q < mp.npov; ++q) {
        const int i0 = mp.pov[2 * q], j0 = mp.pov[2 * q + 1];
        if (iD == i0 && jD == j0) { ++seen; continue; }
        const double qq = atan2((double)(iD - i0), (double)(jD - j0)) * (double)mp.n / 3.141592653589793;
        long long kp = (long long)floor(qq + 0.5);
        kp = ((kp % (2 * mp.n)) + 2 * mp.n) % (2 * mp.n);
        const int k = (int)(kp % mp.n);
        const DirDev d = mp.dirs[k];
        // +j of the view points along theta_k in views 0 and 1, along theta_k + pi in views 2 and 3
        const bool plus = (d.frame <= 1) == (kp < mp.n);
        int iv, jv, iv0, jv0;
        to_view(d, iD, jD, &iv, &jv);
        to_view(d, i0, j0, &iv0, &jv0);
        const int dd = plus ? jv - jv0 : jv0 - jv;
        const long long slot = plus ? k : mp.n + k;
        if (dd >= 1 && dd < mp.cap) seen += mp.flags[((long long)q * 2 * mp.n + slot) * mp.cap + dd];
    }
    mp.count[c] = seen;
}

}  // namespace
}  // namespace tvs

using namespace tvs;

extern "C" int tvs_visibility_map(tvs_handle h, const float* d_dem, int rows, int cols, double step_m,
                                  double obs_height_m, int n_sectors, double max_range_m, const int32_t* pov_ij,
                                  int npov, int32_t* d_count, void* cuda_stream)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    if (!d_dem || !pov_ij || !d_count) return fail(TVS_ERR_ARG, "d_dem, pov_ij or d_count is NULL");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    if (npov < 1) return fail(TVS_ERR_ARG, "npov must be >= 1");
    for (int q = 0; q < npov; ++q)
        if (pov_ij[2 * q] < 0 || pov_ij[2 * q] >= rows || pov_ij[2 * q + 1] < 0 || pov_ij[2 * q + 1] >= cols)
            return fail(TVS_ERR_ARG, "POV " + std::to_string(q) + " lies outside the DEM");
    const int cap = std::max(rows, cols) + 1;
    const size_t flag_bytes = (size_t)npov * 2 * n_sectors * cap;
    if (flag_bytes > ((size_t)1 << 34)) return fail(TVS_ERR_OOM, "too many POVs x directions for the flag table");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::vector<DirDev> dirs(n_sectors);
    for (int k = 0; k < n_sectors; ++k) {
        HostDir d;
        make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d);
        DirDev& v = dirs[k];
        std::memset(&v, 0, sizeof(v));
        v.t_fx = d.t_fx; v.frame = d.frame; v.H = d.H; v.W = d.W; v.Wp = (d.W + 3) & ~3; v.D = d.D; v.R = d.R;
        v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
        v.gidx = k; v.g = (float)d.g; v.h0 = (float)obs_height_m;
    }
    const size_t o_dirs = 0, o_pov = align256((size_t)n_sectors * sizeof(DirDev));
    const size_t hdr = o_pov + align256((size_t)npov * 8);
    const size_t o_flags = hdr;
    const size_t total = o_flags + align256(flag_bytes);
    rc = ensure_scratch(h, total);
    if (rc) return rc;
    std::vector<char> img(hdr, 0);
    std::memcpy(img.data() + o_dirs, dirs.data(), dirs.size() * sizeof(DirDev));
    std::memcpy(img.data() + o_pov, pov_ij, (size_t)npov * 8);
    rc = upload_header(h, img, h->ws, s);
    if (rc) return rc;
    TVS_CUDA(cudaMemsetAsync(h->ws + o_flags, 0, flag_bytes, s), "clear visibility flags");
    MapParams mp{};
    mp.dem = d_dem;
    mp.dirs = reinterpret_cast<const DirDev*>(h->ws + o_dirs);
    mp.pov = reinterpret_cast<const int*>(h->ws + o_pov);
    mp.flags = reinterpret_cast<unsigned char*>(h->ws + o_flags);
    mp.count = d_count;
    mp.rows = rows; mp.cols = cols; mp.n = n_sectors; mp.npov = npov; mp.cap = cap;
    mp.h0 = (float)obs_height_m;
    const long long walks = (long long)npov * 2 * n_sectors;
    map_flags_kernel<<<(unsigned)((walks + 63) / 64), 64, 0, s>>>(mp);
    TVS_CUDA(cudaGetLastError(), "visibility flags launch");
    const long long cells = (long long)rows * cols;
    map_raster_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(mp);
    TVS_CUDA(cudaGetLastError(), "visibility raster launch");
    return TVS_OK;
}

extern "C" int tvs_viewshed_points(tvs_handle h, const float* d_dem, int rows, int cols, double step_m,
                                   double obs_height_m, int n_sectors, double max_range_m, const int32_t* pov_ij,
                                   int npov, int mode, float* d_area, void* cuda_stream)
{
    if (!h) return fail(TVS_ERR_ARG, "handle is NULL");
    if (!d_dem || !pov_ij || !d_area) return fail(TVS_ERR_ARG, "d_dem, pov_ij or d_area is NULL");
    int rc = check_job(rows, cols, step_m, obs_height_m, n_sectors, max_range_m);
    if (rc) return rc;
    if (npov < 1) return fail(TVS_ERR_ARG, "npov must be >= 1");
    if (mode != TVS_POINTS_SDEM && mode != TVS_POINTS_DIRECT) return fail(TVS_ERR_ARG, "unknown mode");
    for (int q = 0; q < npov; ++q)
        if (pov_ij[2 * q] < 0 || pov_ij[2 * q] >= rows || pov_ij[2 * q + 1] < 0 || pov_ij[2 * q + 1] >= cols)
            return fail(TVS_ERR_ARG, "POV " + std::to_string(q) + " lies outside the DEM");
    const int ngroups = (n_sectors + FP32_GROUP - 1) / FP32_GROUP;
    if ((long long)npov * ngroups >= (1LL << 31)) return fail(TVS_ERR_ARG, "too many POVs x directions");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::vector<DirDev> dirs(n_sectors);
    for (int k = 0; k < n_sectors; ++k) {
        HostDir d;
        make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d);
        DirDev& v = dirs[k];
        std::memset(&v, 0, sizeof(v));
        v.t_fx = d.t_fx; v.frame = d.frame; v.H = d.H; v.W = d.W; v.Wp = (d.W + 3) & ~3; v.D = d.D; v.R = d.R;
        v.K = d.K == LLONG_MAX ? d.W : (int)std::min<long long>(d.K, d.W);
        v.gidx = k; v.g = (float)d.g; v.h0 = (float)obs_height_m;
    }
    const size_t o_dirs = 0, o_pov = align256((size_t)n_sectors * sizeof(DirDev));
    const size_t hdr = o_pov + align256((size_t)npov * 8);
    const size_t o_part = hdr;
    const size_t total = o_part + align256((size_t)npov * ngroups * 16);
    rc = ensure_scratch(h, total);
    if (rc) return rc;
    std::vector<char> img(hdr, 0);
    std::memcpy(img.data() + o_dirs, dirs.data(), dirs.size() * sizeof(DirDev));
    std::memcpy(img.data() + o_pov, pov_ij, (size_t)npov * 8);
    rc = upload_header(h, img, h->ws, s);
    if (rc) return rc;
    PointsParams pp{};
    pp.dem = d_dem;
    pp.dirs = reinterpret_cast<const DirDev*>(h->ws + o_dirs);
    pp.pov = reinterpret_cast<const int*>(h->ws + o_pov);
    pp.part = reinterpret_cast<__int128*>(h->ws + o_part);
    pp.area = d_area;
    pp.scale = (M_PI / (2.0 * (double)n_sectors)) * (step_m * step_m);
    pp.rows = rows; pp.cols = cols; pp.n = n_sectors; pp.ngroups = ngroups; pp.npov = npov; pp.mode = mode;
    pp.h0 = (float)obs_height_m;
    points_kernel<<<(unsigned)(npov * ngroups), 32, 0, s>>>(pp);
    TVS_CUDA(cudaGetLastError(), "points launch");
    points_finalize<<<(npov + 127) / 128, 128, 0, s>>>(pp);
    TVS_CUDA(cudaGetLastError(), "points finalize launch");
    return TVS_OK;
}
