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
// d = 1 .. n (n = min(usable samples, K)), visible iff the target's slope is
// strictly above the running maximum -- the exact decision (certified walks,
// the default) or the FP32 one, (z - h) * rcp(d) (fp32_decisions) -- and
// cv = 1 + sum_{d < n} v_d (2d + 1) for n >= 1 (the last target only closes a
// segment).  Lane 0 adds the group's terms g * blend(cv) in direction order in
// FP32 and stores the group sum as an exact partial; a finalize kernel adds
// each POV's partials and applies the (pi/(2n)) step^2 scale.
#include "tvs.h"
#include "tvs_host.h"
#include "tvs_internal.h"
#include "tvs_df.cuh"

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
    float* term;            // npov x n direction terms g * blend(cv)
    __int128* part;         // npov x ngroups exact group sums
    float* area;            // npov visible areas
    double scale;           // (pi / (2n)) step^2
    int rows, cols, n, ngroups, npov, mode;
    float h0;
    float h0_lo;            // h0 - (double)h0 above, rounded
    double h0d;             // h0 (the FP64 walks)
    int cert;               // certified (exact) visibility decisions
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

// The line of one (direction k, virtual POV v) of POV q: its view, the POV's
// view cell (i, j0), the line's base (SDEM: base row at column 0; DIRECT: the
// cell row), and the blend data of the direction (fr0, r, hi_ok, lo_ok).
struct PointLine {
    DirDev d;
    int i, j0;
    long long base;
    unsigned fr0;
    float r;
    bool hi_ok, lo_ok, valid;
};

__device__ __forceinline__ PointLine point_line(const PointsParams& pp, int q, int k, int v)
{
    PointLine L;
    L.fr0 = 0u; L.r = 0.f; L.hi_ok = true; L.lo_ok = false; L.valid = false; L.base = 0; L.i = 0; L.j0 = 0;
    if (k >= pp.n) return L;
    L.d = pp.dirs[k];
    const DirDev& d = L.d;
    const int iD = pp.pov[2 * q], jD = pp.pov[2 * q + 1];
    switch (d.frame) {
    case 0:  L.i = iD; L.j0 = jD; break;
    case 1:  L.i = jD; L.j0 = iD; break;
    case 2:  L.i = jD; L.j0 = d.W - 1 - iD; break;
    default: L.i = d.H - 1 - iD; L.j0 = jD; break;
    }
    if (pp.mode == TVS_POINTS_DIRECT) {
        L.valid = v == 0;
        L.base = L.i;
    } else {
        const unsigned long long y = (unsigned long long)L.j0 * d.t_fx;
        const int dest = (int)(y >> 32);
        L.fr0 = (unsigned)(y & 0xFFFFFFFFull);
        L.hi_ok = L.fr0 == 0u || L.i <= d.H - 2;
        L.lo_ok = L.fr0 != 0u && L.i >= 1;
        L.r = __fmul_rn(__uint2float_rn(L.fr0), 0x1p-32f);
        L.valid = v == 0 ? L.hi_ok : L.lo_ok;
        L.base = (long long)L.i - dest - v;
    }
    return L;
}

// Targets per lane per chunk of a warp's half-line walk.
constexpr int WALK_TPL = 8;
constexpr int WALK_CHUNK = 32 * WALK_TPL;

// DEM offset of view cell (a, j) of a direction: o + a sa + j sj.
struct ViewAddr {
    int o, sa, sj;
};

__device__ __forceinline__ ViewAddr view_addr(const DirDev& d, int cols)
{
    switch (d.frame) {
    case 0:  return {0, cols, 1};
    case 1:  return {0, 1, cols};
    case 2:  return {(d.W - 1) * cols, 1, -cols};
    default: return {(d.H - 1) * cols, -cols, 1};
    }
}

// Fills rtab[d] = rcp(d) for d = 1 .. dmax (the CTA's threads share it).
__device__ __forceinline__ void fill_rcp(float* rtab, int dmax)
{
    for (int m = threadIdx.x + 1; m <= dmax; m += blockDim.x) rtab[m] = __frcp_rn((float)m);
}

// One half-line walked by a whole warp, WALK_CHUNK targets at a time: lane l
// takes targets d = c + 8 l + 1 .. c + 8 l + 8 of chunk c (their samples are
// independent loads), with each target's FP32 slope the serial walk's.  The
// running maximum before a target is the maximum of the slopes before it:
// a warp max-scan of the lanes' own maxima gives each lane the maximum before
// its first target, and a serial pass over its 8 targets does the rest
// (maximum is exact, so every visibility decision is the serial one).  The
// walk ends at the first unusable target or at K.  Returns the walk's measure
// cv = 1 + sum_{d < n} v_d (2d + 1) (0 for n = 0) on every lane; with `flags`
// each target's visibility is also stored at flags[d] (d < cap).
__device__ __forceinline__ int walk_half_line(const float* __restrict__ dem, int cols, const DirDev& d,
                                              const float* __restrict__ rtab, long long base, int j0, bool direct,
                                              int dir, float h, unsigned char* flags, int cap, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const float NEG = __int_as_float(0xff800000);
    const ViewAddr va = view_addr(d, cols);
    float M = NEG;
    int sum = 0;                      // this lane's sum of v_d (2d + 1) over its targets
    int n = 0, lastvis = 0;           // targets so far; visibility of the latest one
    for (int c = 0;; c += WALK_CHUNK) {
        float t[WALK_TPL];
        int firstbad = WALK_TPL;      // the lane's first unusable target
        // the lane's first target and its line position y = (j, or j - j0) t_fx,
        // stepped by +-t_fx from target to target: row base + floor(y / 2^32)
        const int d0 = c + WALK_TPL * lane + 1;
        int j = j0 + dir * d0;
        long long y = (long long)(direct ? dir * d0 : j) * (long long)d.t_fx;
        const long long ystep = dir * (long long)d.t_fx;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            const int dd = d0 + m;
            const long long a = base + (y >> 32);
            const unsigned fr = (unsigned)y;
            const bool ok = dd <= d.K && usable(d, a, fr, j);
            t[m] = NEG;
            if (ok) {
                const int at = va.o + (int)a * va.sa + j * va.sj;
                float z = dem[at];
                if (fr != 0u) {
                    const float r = __fmul_rn(__uint2float_rn(fr), 0x1p-32f);
                    z = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, r), z), __fmul_rn(r, dem[at + va.sa]));
                }
                t[m] = __fmul_rn(__fsub_rn(z, h), rtab[dd]);
            }
            if (!ok && firstbad == WALK_TPL) firstbad = m;
            y += ystep;
            j += dir;
        }
        // the walk ends at the first unusable target, as the serial walk does
        const unsigned bad = __ballot_sync(FULL, firstbad < WALK_TPL);
        const int badlane = bad ? __ffs(bad) - 1 : 32;
        const int cnt = badlane == 32 ? WALK_CHUNK
                                      : WALK_TPL * badlane + __shfl_sync(FULL, firstbad, badlane);
        const int mine = min(max(cnt - WALK_TPL * lane, 0), WALK_TPL);
        float lm = NEG;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m)
            if (m < mine) lm = fmaxf(lm, t[m]);
        float pm = lm;                // inclusive prefix maximum over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(FULL, pm, o);
            if (lane >= o) pm = fmaxf(pm, y);
        }
        const float before = __shfl_up_sync(FULL, pm, 1);
        float run = lane == 0 ? M : fmaxf(M, before);
        unsigned vbits = 0u;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            if (m < mine) {
                const int dd = c + WALK_TPL * lane + m + 1;
                const bool vis = t[m] > run;
                run = fmaxf(run, t[m]);
                if (vis) { sum += 2 * dd + 1; vbits |= 1u << m; }
                if (flags && dd < cap) flags[dd] = vis ? 1 : 0;
            }
        }
        if (cnt > 0) {
            const int last = cnt - 1;
            lastvis = (__shfl_sync(FULL, vbits, last / WALK_TPL) >> (last % WALK_TPL)) & 1u;
            n = c + cnt;
        }
        M = fmaxf(M, __shfl_sync(FULL, pm, 31));
        if (cnt < WALK_CHUNK) break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    // the last target only closes a segment: its own 2n + 1 is not counted
    return n >= 1 ? 1 + sum - (lastvis ? 2 * n + 1 : 0) : 0;
}

// ----------------------------------------------------- certified walks --
// With certified decisions (the library default) a half-line is walked with
// double-float heights (the blend of Alg. 6 to about 2^-43 of the heights) and
// double-float slopes, warp-cooperatively as walk_half_line does; each
// decision is proved by a margin (slope errors <= 2^-45 |theta| + 2 eta / d),
// and when one is not, the warp walks the half-line again in FP64 exactly as
// the FP64 definition does ((1 - r) a + r b, h = z + h0, (z - h) / d, strict
// comparison with the running maximum).  Either way every decision is the one
// exact arithmetic takes (up to FP64 rounding, which the FP64 walk shares with
// the definition), so an sDEM point's area is the certified map's value.

// A half-line: direction, observer's view cell (i0 = base row for DIRECT),
// line base, walk direction.
struct LineRef {
    const float* dem;
    int cols;
    DirDev d;
    long long base;
    int j0, dir;
    bool direct;
};

// Position of the target at distance dd: false when it is not part of the walk.
__device__ __forceinline__ bool line_target(const LineRef& L, int dd, long long* a, unsigned* fr, int* j)
{
    *j = L.j0 + L.dir * dd;
    line_pos(L.d, L.direct, L.base, L.j0, *j, a, fr);
    return dd <= L.d.K && usable(L.d, *a, *fr, *j);
}

__device__ __forceinline__ double z64_of(const LineRef& L, long long a, unsigned fr, int j)
{
    const double lo = (double)view_at(L.dem, L.cols, L.d, a, j);
    if (fr == 0u) return lo;
    const double hi = (double)view_at(L.dem, L.cols, L.d, a + 1, j);
    const double r = __dmul_rn((double)fr, 0x1p-32);
    return __dadd_rn(__dmul_rn(__dsub_rn(1.0, r), lo), __dmul_rn(r, hi));
}

// The FP64 walk: the measure cv (0 for no target) on every lane, flags as
// walk_half_line stores them.
__device__ __noinline__ int walk_fp64(const LineRef& L, double h, unsigned char* flags, int cap, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const double NEG = -__longlong_as_double(0x7ff0000000000000LL);
    double M = NEG;
    int sum = 0, n = 0, lastvis = 0;
    for (int c = 0;; c += WALK_CHUNK) {
        double t[WALK_TPL];
        int firstbad = WALK_TPL;
        const int d0 = c + WALK_TPL * lane + 1;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            long long a;
            unsigned fr;
            int j;
            const bool ok = line_target(L, d0 + m, &a, &fr, &j);
            t[m] = NEG;
            if (ok) t[m] = __ddiv_rn(__dsub_rn(z64_of(L, a, fr, j), h), (double)(d0 + m));
            if (!ok && firstbad == WALK_TPL) firstbad = m;
        }
        const unsigned bad = __ballot_sync(FULL, firstbad < WALK_TPL);
        const int badlane = bad ? __ffs(bad) - 1 : 32;
        const int cnt = badlane == 32 ? WALK_CHUNK : WALK_TPL * badlane + __shfl_sync(FULL, firstbad, badlane);
        const int mine = min(max(cnt - WALK_TPL * lane, 0), WALK_TPL);
        double lm = NEG;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m)
            if (m < mine) lm = fmax(lm, t[m]);
        double pm = lm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(FULL, pm, o);
            if (lane >= o) pm = fmax(pm, y);
        }
        const double before = __shfl_up_sync(FULL, pm, 1);
        double run = lane == 0 ? M : fmax(M, before);
        unsigned vbits = 0u;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            if (m < mine) {
                const int dd = d0 + m;
                const bool vis = t[m] > run;
                run = fmax(run, t[m]);
                if (vis) { sum += 2 * dd + 1; vbits |= 1u << m; }
                if (flags && dd < cap) flags[dd] = vis ? 1 : 0;
            }
        }
        if (cnt > 0) {
            const int last = cnt - 1;
            lastvis = (__shfl_sync(FULL, vbits, last / WALK_TPL) >> (last % WALK_TPL)) & 1u;
            n = c + cnt;
        }
        M = fmax(M, __shfl_sync(FULL, pm, 31));
        if (cnt < WALK_CHUNK) break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    return n >= 1 ? 1 + sum - (lastvis ? 2 * n + 1 : 0) : 0;
}

// The double-float walk with its margins; *esc (warp-uniform) when a
// decision fell inside its margin (the measure and flags are then the FP64
// walk's to write).  hh + hl is the observer, zobs the |elevations| it blends.
__device__ __noinline__ int walk_df(const LineRef& L, float hh, float hl, float zobs, float h0abs,
                                    unsigned char* flags, int cap, int lane, bool* esc_out)
{
    const unsigned FULL = 0xffffffffu;
    const float NEG = __int_as_float(0xff800000);
    float rh = NEG, rl = 0.f;
    int rd = 1;
    float zmax = zobs;
    int sum = 0, n = 0, lastvis = 0;
    bool esc = false;
    for (int c = 0;; c += WALK_CHUNK) {
        float th[WALK_TPL], tl[WALK_TPL], iv[WALK_TPL];
        int firstbad = WALK_TPL;
        const int d0 = c + WALK_TPL * lane + 1;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            long long a;
            unsigned fr;
            int j;
            const bool ok = line_target(L, d0 + m, &a, &fr, &j);
            th[m] = NEG; tl[m] = 0.f;
            iv[m] = __frcp_rn((float)(d0 + m));
            if (ok) {
                const float va = view_at(L.dem, L.cols, L.d, a, j);
                const float vb = fr ? view_at(L.dem, L.cols, L.d, a + 1, j) : va;
                float zh, zl;
                df::df_blend(va, vb, fr, zh, zl);
                zmax = fmaxf(zmax, fmaxf(fabsf(va), fabsf(vb)));
                df::df_slope_iv(zh, zl, hh, hl, d0 + m, iv[m], th[m], tl[m]);
            }
            if (!ok && firstbad == WALK_TPL) firstbad = m;
        }
        const unsigned bad = __ballot_sync(FULL, firstbad < WALK_TPL);
        const int badlane = bad ? __ffs(bad) - 1 : 32;
        const int cnt = badlane == 32 ? WALK_CHUNK : WALK_TPL * badlane + __shfl_sync(FULL, firstbad, badlane);
        const int mine = min(max(cnt - WALK_TPL * lane, 0), WALK_TPL);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(FULL, zmax, o));
        const float eta = 0x1p-42f * (zmax + h0abs) + 0x1p-126f;
        float mh = NEG, ml = 0.f;
        int md = 1;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m)
            if (m < mine && df::df_gt(th[m], tl[m], mh, ml)) { mh = th[m]; ml = tl[m]; md = d0 + m; }
        float ph = mh, pl = ml;
        int pd = md;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float qh = __shfl_up_sync(FULL, ph, o);
            const float ql = __shfl_up_sync(FULL, pl, o);
            const int qd = __shfl_up_sync(FULL, pd, o);
            if (lane >= o && df::df_gt(qh, ql, ph, pl)) { ph = qh; pl = ql; pd = qd; }
        }
        float ch = __shfl_up_sync(FULL, ph, 1);
        float cl = __shfl_up_sync(FULL, pl, 1);
        int cd = __shfl_up_sync(FULL, pd, 1);
        if (lane == 0 || df::df_gt(rh, rl, ch, cl)) { ch = rh; cl = rl; cd = rd; }
        float icd = __frcp_rn((float)cd);
        unsigned vbits = 0u;
#pragma unroll
        for (int m = 0; m < WALK_TPL; ++m) {
            if (m < mine) {
                const int dd = d0 + m;
                bool vis = true;                   // the first target (no earlier one) is visible
                if (ch > NEG) {
                    float s, e;
                    df::two_sum(th[m], -ch, s, e);
                    const float dh = __fadd_rn(s, __fadd_rn(e, __fsub_rn(tl[m], cl)));
                    const float marg = __fmaf_rn(0x1p-40f, fabsf(th[m]) + fabsf(ch), 4.04f * eta * (iv[m] + icd)) +
                                       0x1p-120f;
                    if (!(fabsf(dh) > marg)) esc = true;
                    vis = dh > 0.f;
                }
                if (df::df_gt(th[m], tl[m], ch, cl)) { ch = th[m]; cl = tl[m]; cd = dd; icd = iv[m]; }
                if (vis) { sum += 2 * dd + 1; vbits |= 1u << m; }
                if (flags && dd < cap) flags[dd] = vis ? 1 : 0;
            }
        }
        if (cnt > 0) {
            const int last = cnt - 1;
            lastvis = (__shfl_sync(FULL, vbits, last / WALK_TPL) >> (last % WALK_TPL)) & 1u;
            n = c + cnt;
        }
        const float lh = __shfl_sync(FULL, ph, 31), ll = __shfl_sync(FULL, pl, 31);
        const int ld = __shfl_sync(FULL, pd, 31);
        if (df::df_gt(lh, ll, rh, rl)) { rh = lh; rl = ll; rd = ld; }
        if (cnt < WALK_CHUNK) break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
    *esc_out = __any_sync(FULL, esc);
    return n >= 1 ? 1 + sum - (lastvis ? 2 * n + 1 : 0) : 0;
}

// Certified measure of a half-line whose observer stands on the sample
// (a0, fr0) of view column j0 (DIRECT: the cell itself, fr0 = 0).
__device__ __forceinline__ int walk_exact(const LineRef& L, long long a0, unsigned fr0, float h0, float h0_lo,
                                          double h0d, unsigned char* flags, int cap, int lane)
{
    const float va = view_at(L.dem, L.cols, L.d, a0, L.j0);
    const float vb = fr0 ? view_at(L.dem, L.cols, L.d, a0 + 1, L.j0) : va;
    float zh, zl, hh, hl;
    df::df_blend(va, vb, fr0, zh, zl);
    {
        float s, e;
        df::two_sum(zh, h0, s, e);
        e = __fadd_rn(e, __fadd_rn(zl, h0_lo));
        df::two_sum(s, e, hh, hl);
    }
    bool esc = false;
    const int cv = walk_df(L, hh, hl, fmaxf(fabsf(va), fabsf(vb)), fabsf(h0), flags, cap, lane, &esc);
    if (!esc) return cv;
    return walk_fp64(L, __dadd_rn(z64_of(L, a0, fr0, L.j0), h0d), flags, cap, lane);
}

// Directions per CTA of the points kernel (4 warps each: 2 lines x 2 sides).
constexpr int POINTS_DIRS = 2;

// One CTA of 4 POINTS_DIRS warps per (POV q, POINTS_DIRS consecutive
// directions): warp 4 kk + 2 v + s walks direction k0 + kk, virtual POV v
// (hi / lo; DIRECT uses v = 0 only), forward (s = 0) or backward (s = 1).
// Then one thread per direction blends its lines' measures (Kernel-3) and
// stores the direction's term g * blend.
__global__ void __launch_bounds__(128 * POINTS_DIRS) points_kernel(PointsParams pp)
{
    __shared__ int cvs[4 * POINTS_DIRS];
    extern __shared__ float rtab[];   // rcp(d), d = 1 .. max(rows, cols)
    fill_rcp(rtab, max(pp.rows, pp.cols));
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per_pov = (pp.n + POINTS_DIRS - 1) / POINTS_DIRS;
    const int q = (int)(blockIdx.x / (unsigned)per_pov);
    const int k0 = (int)(blockIdx.x % (unsigned)per_pov) * POINTS_DIRS;
    const bool direct = pp.mode == TVS_POINTS_DIRECT;
    {
        const int kk = w >> 2, v = (w >> 1) & 1, s = w & 1;
        const PointLine L = point_line(pp, q, k0 + kk, v);
        int cv = 0;
        if (L.valid) {
            long long a;
            unsigned fr;
            line_pos(L.d, direct, L.base, L.j0, L.j0, &a, &fr);
            if (pp.cert) {
                const LineRef R{pp.dem, pp.cols, L.d, L.base, L.j0, s ? -1 : 1, direct};
                cv = walk_exact(R, a, fr, pp.h0, pp.h0_lo, pp.h0d, nullptr, 0, lane);
            } else {
                const float h = __fadd_rn(direct ? view_at(pp.dem, pp.cols, L.d, L.i, L.j0)
                                                 : sample_at(pp.dem, pp.cols, L.d, a, fr, L.j0), pp.h0);
                cv = walk_half_line(pp.dem, pp.cols, L.d, rtab, L.base, L.j0, direct, s ? -1 : 1, h, nullptr, 0,
                                    lane);
            }
        }
        if (lane == 0) cvs[w] = cv;
    }
    __syncthreads();
    if (threadIdx.x >= POINTS_DIRS) return;
    const int kk = threadIdx.x, k = k0 + kk;
    if (k >= pp.n) return;
    // cv_fwd + cv_bwd of each line, then the direction's blend (Kernel-3)
    const PointLine L = point_line(pp, q, k, 0);
    const float T = (float)(cvs[4 * kk] + cvs[4 * kk + 1]);             // hi line
    const float T_other = (float)(cvs[4 * kk + 2] + cvs[4 * kk + 3]);   // lo line
    float val;
    if (direct || L.fr0 == 0u) val = T;
    else if (L.hi_ok && L.lo_ok) val = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, L.r), T), __fmul_rn(L.r, T_other));
    else if (L.hi_ok) val = T;
    else val = T_other;
    pp.term[(long long)q * pp.n + k] = __fmul_rn(L.d.g, val);
}

// One thread per (POV, group of FP32_GROUP directions): the FP32 sum of the
// group's terms in direction order, stored as one exact partial (the total
// viewshed map's unskew adds its groups the same way).
__global__ void points_groups(PointsParams pp)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)pp.npov * pp.ngroups) return;
    const int q = (int)(t / pp.ngroups), grp = (int)(t % pp.ngroups);
    const float* term = pp.term + (long long)q * pp.n;
    float acc = 0.f;
    for (int k = grp * FP32_GROUP; k < min(pp.n, (grp + 1) * FP32_GROUP); ++k) acc = __fadd_rn(acc, term[k]);
    pp.part[t] = acc_of(acc);
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
    float h0_lo;
    double h0d;
    int cert;
};

// One warp per (POV, slot), walking the half-line as the points kernel does.
__global__ void __launch_bounds__(256) map_flags_kernel(MapParams mp)
{
    extern __shared__ float rtab[];   // rcp(d), d = 1 .. max(rows, cols)
    fill_rcp(rtab, max(mp.rows, mp.cols));
    __syncthreads();
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // (q, slot)
    const int lane = threadIdx.x & 31;
    if (t >= (long long)mp.npov * 2 * mp.n) return;                                // warp-uniform
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
    if (mp.cert) {
        const LineRef R{mp.dem, mp.cols, d, i, j0, dir, true};
        walk_exact(R, i, 0u, mp.h0, mp.h0_lo, mp.h0d, mp.flags + t * mp.cap, mp.cap, lane);
        return;
    }
    const float h = __fadd_rn(view_at(mp.dem, mp.cols, d, i, j0), mp.h0);
    walk_half_line(mp.dem, mp.cols, d, rtab, i, j0, true, dir, h, mp.flags + t * mp.cap, mp.cap, lane);
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
// half-line axes k' pi / n to the direction of the cell, the double-precision
// decision kp = floor(atan2(di, dj) n / pi + 1/2) mod 2n) and the flag of the
// target at the cell's walk-axis column.  The decision is taken from a
// single-precision angle when it is far from a sector boundary: atan2f is
// within a few ulp of the angle (|angle| <= pi, ulp 2^-22), so with the three
// roundings of q = angle (n / pi) + 1/2 the single-precision q is within
// about 4.1e-7 n of the double one; a cell whose q lies within
// 4e-6 n + 1e-6 of a boundary takes the double-precision angle instead.
__global__ void map_raster_kernel(MapParams mp)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (long long)mp.rows * mp.cols) return;
    const int iD = (int)(c / mp.cols), jD = (int)(c % mp.cols);
    const float scale = (float)((double)mp.n / 3.141592653589793);
    const float margin = 4e-6f * (float)mp.n + 1e-6f;
    int seen = 0;
    for (int q = 0; q < mp.npov; ++q) {
        const int i0 = mp.pov[2 * q], j0 = mp.pov[2 * q + 1];
        if (iD == i0 && jD == j0) { ++seen; continue; }
        const float x = __fadd_rn(__fmul_rn(atan2f((float)(iD - i0), (float)(jD - j0)), scale), 0.5f);
        const float fl = floorf(x);
        const float fx = x - fl;                  // exact
        long long kp;
        if (fx > margin && fx < 1.0f - margin) {
            kp = (long long)fl;
        } else {
            const double qq = atan2((double)(iD - i0), (double)(jD - j0)) * (double)mp.n / 3.141592653589793;
            kp = (long long)floor(qq + 0.5);
        }
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

extern "C" int64_t tvs_count_point_evals(int rows, int cols, int n_sectors, double step_m, double max_range_m,
                                         const int32_t* pov_ij, int npov, int mode)
{
    if (!pov_ij || npov < 1) return TVS_ERR_ARG;
    if (mode != TVS_POINTS_SDEM && mode != TVS_POINTS_DIRECT) return TVS_ERR_ARG;
    if (check_job(rows, cols, step_m, 0.0, n_sectors, max_range_m)) return TVS_ERR_ARG;
    for (int q = 0; q < npov; ++q)
        if (pov_ij[2 * q] < 0 || pov_ij[2 * q] >= rows || pov_ij[2 * q + 1] < 0 || pov_ij[2 * q + 1] >= cols)
            return TVS_ERR_ARG;
    int64_t total = 0;
    for (int k = 0; k < n_sectors; ++k) {
        HostDir d;
        make_direction(n_sectors, k, rows, cols, step_m, max_range_m, &d);
        const long long K = d.K == LLONG_MAX ? (long long)d.W : std::min<long long>(d.K, d.W);
        for (int q = 0; q < npov; ++q) {
            const int iD = pov_ij[2 * q], jD = pov_ij[2 * q + 1];
            int i, j0;
            switch (d.frame) {
            case 0:  i = iD; j0 = jD; break;
            case 1:  i = jD; j0 = iD; break;
            case 2:  i = jD; j0 = d.W - 1 - iD; break;
            default: i = d.H - 1 - iD; j0 = jD; break;
            }
            if (mode == TVS_POINTS_DIRECT) {
                // 0 <= i + (j - j0) t <= H - 1 and 0 <= j < W, t = t_fx 2^-32
                long long f = d.W - 1 - j0, b = j0;
                if (d.t_fx != 0ull) {
                    f = std::min<long long>(f, (long long)(((unsigned long long)(d.H - 1 - i) << 32) / d.t_fx));
                    b = std::min<long long>(b, (long long)(((unsigned long long)i << 32) / d.t_fx));
                }
                total += std::min(f, K) + std::min(b, K);
                continue;
            }
            const unsigned long long y = (unsigned long long)j0 * d.t_fx;
            const int dest = (int)(y >> 32);
            const bool frac = (y & 0xFFFFFFFFull) != 0ull;
            for (int v = 0; v < 2; ++v) {
                const bool ok = v == 0 ? (!frac || i <= d.H - 2) : (frac && i >= 1);
                if (!ok) continue;
                int lo, hi;
                host_row_range(d, i - dest - v + d.D, &lo, &hi);
                total += std::min<long long>(hi - j0, K) + std::min<long long>(j0 - lo, K);
            }
        }
    }
    return total;
}

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
    mp.h0_lo = (float)(obs_height_m - (double)mp.h0);
    mp.h0d = obs_height_m;
    mp.cert = !h->tuning.fp32_decisions;
    const long long walks = (long long)npov * 2 * n_sectors;
    const size_t rtab_bytes = ((size_t)std::max(rows, cols) + 1) * sizeof(float);
    TVS_CUDA(cudaFuncSetAttribute(map_flags_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rtab_bytes),
             "visibility flags shared memory");
    {
        const double evals = h->profiling ? (double)tvs_count_point_evals(rows, cols, n_sectors, step_m, max_range_m,
                                                                          pov_ij, npov, TVS_POINTS_DIRECT)
                                          : 0.0;
        Timer t(h, K_MAP_FLAGS, s, evals);
        map_flags_kernel<<<(unsigned)((walks * 32 + 255) / 256), 256, rtab_bytes, s>>>(mp);
    }
    TVS_CUDA(cudaGetLastError(), "visibility flags launch");
    const long long cells = (long long)rows * cols;
    {
        Timer t(h, K_MAP_RASTER, s, (double)cells * npov);
        map_raster_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(mp);
    }
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
    if ((long long)npov * n_sectors >= (1LL << 31)) return fail(TVS_ERR_ARG, "too many POVs x directions");
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
    const size_t o_term = o_part + align256((size_t)npov * ngroups * 16);
    const size_t total = o_term + align256((size_t)npov * n_sectors * 4);
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
    pp.term = reinterpret_cast<float*>(h->ws + o_term);
    pp.area = d_area;
    pp.scale = (M_PI / (2.0 * (double)n_sectors)) * (step_m * step_m);
    pp.rows = rows; pp.cols = cols; pp.n = n_sectors; pp.ngroups = ngroups; pp.npov = npov; pp.mode = mode;
    pp.h0 = (float)obs_height_m;
    pp.h0_lo = (float)(obs_height_m - (double)pp.h0);
    pp.h0d = obs_height_m;
    pp.cert = !h->tuning.fp32_decisions;
    const size_t rtab_bytes = ((size_t)std::max(rows, cols) + 1) * sizeof(float);
    TVS_CUDA(cudaFuncSetAttribute(points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rtab_bytes),
             "points shared memory");
    {
        const double evals = h->profiling ? (double)tvs_count_point_evals(rows, cols, n_sectors, step_m, max_range_m,
                                                                          pov_ij, npov, mode)
                                          : 0.0;
        Timer t(h, K_POINTS, s, evals);
        const long long ctas = (long long)npov * ((n_sectors + POINTS_DIRS - 1) / POINTS_DIRS);
        points_kernel<<<(unsigned)ctas, 128 * POINTS_DIRS, rtab_bytes, s>>>(pp);
        const long long groups = (long long)npov * ngroups;
        points_groups<<<(unsigned)((groups + 127) / 128), 128, 0, s>>>(pp);
        points_finalize<<<(npov + 127) / 128, 128, 0, s>>>(pp);
    }
    TVS_CUDA(cudaGetLastError(), "points launch");
    return TVS_OK;
}
