// tvs_sweep.cu -- the sweep of the sDEM total viewshed (Kernel-2, Alg. 7 and
// 8) with the relocation of Kernel-1 (Alg. 6) fused into its row staging.
//
// A warp item is one skewed row and one walk direction.  The warp gathers the
// row's samples straight from the DEM (section 4.1 step 1(a): sample j of
// line b blends view rows a = b + dest(j) and a + 1 with weights 1 - r(j) and
// r(j)), so the skewed DEM never reaches HBM, then every usable sample of the
// row walks it (forward items walk the row, backward items its reverse).
//
// Two decision modes:
//
//  * FP32 decisions (the paper's kernel precision: "float" heights and
//    slopes in Alg. 6-8): the staged height is (1-r)*a + r*b in single
//    precision and a target is visible iff fl(fl(z - h) * fl(1/d)) is
//    strictly above the running maximum.
//
//  * Certified decisions (the default): every visibility decision is the one
//    exact arithmetic takes on the exact blended heights, which is what the
//    FP64 definition decides (it rounds some 10^-16 away from exact).  The
//    row is staged as a double-float (hi + lo) pair per sample.  The fast
//    path still decides in FP32, on height differences formed against a
//    per-group reference, and proves each decision with a margin derived
//    below; a decision inside the margin flags its POV, and flagged POVs are
//    walked again exactly (double-float slopes with their own margin, and the
//    FP64 definition itself for what that margin cannot settle).
#include "tvs.h"
#include "tvs_internal.h"
#include "tvs_df.cuh"

#include <cuda_runtime.h>

#include <algorithm>

namespace tvs {

// Index checks of the sweep.  Every index the staging, the per-block margins,
// the flagged-POV list and the exact walks use is checked against its buffer
// (not the inner step loop, whose indices follow from the block's): a
// violation records the first offending index in g_sweep_check (code, index,
// bound, CTA) and skips the access instead of faulting.  Read and cleared by
// tvs_debug_sweep_check.
__device__ int g_sweep_check[4];
// Event counts of the certified sweep: exact walks (flagged POVs), of them
// FP64 walks, SM clock cycles warps spent in exact walks, and cycles warps
// spent in the certified sweep kernels in all.
__device__ unsigned long long g_sweep_stats[4];

__device__ __forceinline__ bool in_range(long long idx, long long bound, int code)
{
    if (idx >= 0 && idx < bound) return true;
    if (atomicCAS(&g_sweep_check[0], 0, code) == 0) {
        g_sweep_check[1] = (int)idx;
        g_sweep_check[2] = (int)bound;
        g_sweep_check[3] = (int)blockIdx.x;
    }
    return false;
}

namespace {

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float pos_inf() { return __int_as_float(0x7f800000); }

struct SweepParams {
    const DirDev* dirs;
    const JobDev* jobs;
    const int* item_start;
    const int* rowlo;
    const int* rowhi;
    int* cv_fwd;       // forward measure of every sample (slab layout)
    int* cv_bwd;       // backward measure of every sample (slab layout)
    unsigned* counter;
    int4* flag_buf;    // certified: flagged walks for the exact pass (NULL: walked in the sweep)
    unsigned* flag_count;
    int flag_cap;
    int ndir;
    int total_items;
    int inv_len;       // entries of the per-distance table (float4 each)
    int tab_slots;     // float4 slots the table takes (the certified kernels skew it)
    int istart_len;    // ints of the item-start table (multiple of 4)
    int half;          // floats of one staged row array (multiple of 4)
    int per_pair;      // floats of a warp pair's shared area (certified)
    int zs_len;        // floats of the row's suffix maxima (0 without pruning)
    int fl_cap;        // entries of the flagged-POV list (certified only)
    int per_warp;      // floats of a warp's shared area
};

// ------------------------------------------------------ row geometry --
// DEM index of view cell (a, j) of direction d and the index step from view
// row a to view row a + 1 (the four D4 views of section 4.1 / Alg. 6).
__device__ __forceinline__ long long view_index(const DirDev& d, int cols, int a, int j, int* step)
{
    switch (d.frame) {
    case 0:  *step = cols;  return (long long)a * cols + j;
    case 1:  *step = 1;     return (long long)j * cols + a;
    case 2:  *step = 1;     return (long long)(d.W - 1 - j) * cols + a;
    default: *step = -cols; return (long long)(d.H - 1 - a) * cols + j;
    }
}

// The paper's single-precision blend of Kernel-1: r = float(fr) 2^-32,
// (1 - r) a + r b with every operation rounded.
__device__ __forceinline__ float blend32(float va, float vb, unsigned fr)
{
    if (fr == 0u) return va;
    const float r = __fmul_rn(__uint2float_rn(fr), 0x1p-32f);
    const float wa = __fsub_rn(1.0f, r);
    return __fadd_rn(__fmul_rn(wa, va), __fmul_rn(r, vb));
}

// A sweep work item: (direction, skewed row, walk direction).
struct ItemRow {
    long long rowbase;   // slab offset of the row's first usable sample
    int dir, p, jlo;
    int L, K, pov;
    float h0;
    bool rev;
};

// Decodes item into its row; false when the row is empty.
__device__ __forceinline__ bool decode_item(const SweepParams& sp, const int* istart, int item, ItemRow* it)
{
    int lo = 0, hi = sp.ndir - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (istart[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const DirDev& d = sp.dirs[lo];
    const int rem = item - istart[lo];
    const int p = rem >> 1;
    it->rev = (rem & 1) != 0;
    const int jlo = sp.rowlo[d.row_off + p], jhi = sp.rowhi[d.row_off + p];
    it->dir = lo;
    it->p = p;
    it->jlo = jlo;
    it->L = jhi - jlo + 1;
    it->K = d.K;
    it->h0 = d.h0;
    it->pov = row_pov(it->L, d.K, d.pov, d.p4_pct);
    it->rowbase = d.slab + (long long)p * d.Wp + jlo;
    return it->L > 0;
}

// Stages the item's row from the DEM: FP32 heights into Fh, or with CERT hi
// parts into Fh and lo parts into Fl, reversed for backward items unless
// rev_ok is false (rows that both walk directions share stay in row order).  The last sample and ROW_PADR samples after
// it hold -inf (lo 0): the last target of a walk never adds area, so it may be
// a sentinel that is never visible.  With CERT the first sample and the
// ROW_PADL samples before it are sentinels too (the last target of a backward
// walk), and the real hi and lo parts of the two end samples, which are POVs,
// go to ends[0..3] (first hi, first lo, last hi, last lo).  Returns (CERT) the
// row's largest |elevation| read, for the blend's error bound.
template <bool CERT>
__device__ __forceinline__ float stage_row(const SweepParams& sp, const ItemRow& it, float* Fh, float* Fl,
                                           float* ends, int lane, int part = 0, int parts = 1, bool rev_ok = true)
{
    const DirDev& d = sp.dirs[it.dir];
    const float* __restrict__ dem = sp.jobs[d.job].dem;
    const int cols = sp.jobs[d.job].cols;
    const long long cells = (long long)sp.jobs[d.job].rows * cols;
    const int b = it.p - d.D;
    const unsigned long long t_fx = d.t_fx;
    const bool rev = rev_ok && it.rev;
    const float NEG = neg_inf();
    float zmax = 0.f;
    constexpr int B = 4;
    for (int x0 = lane + 32 * B * part; x0 < it.L; x0 += 32 * B * parts) {
        float va[B], vb[B];
        unsigned fr[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int x = x0 + 32 * k;
            va[k] = 0.f; vb[k] = 0.f; fr[k] = 0u;
            if (x < it.L) {
                const int j = it.jlo + (rev ? it.L - 1 - x : x);
                const unsigned long long y = (unsigned long long)j * t_fx;
                const int a = b + (int)(y >> 32);
                fr[k] = (unsigned)y;
                int st;
                const long long idx = view_index(d, cols, a, j, &st);
                va[k] = in_range(idx, cells, 1) ? dem[idx] : 0.f;
                vb[k] = fr[k] != 0u ? (in_range(idx + st, cells, 2) ? dem[idx + st] : 0.f) : va[k];
            }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int x = x0 + 32 * k;
            if (x >= it.L || !in_range(ROW_PADL + x, sp.half, 3)) continue;
            if (CERT) {
                float zh, zl;
                df::df_blend(va[k], vb[k], fr[k], zh, zl);
                const bool end = x == 0 || x == it.L - 1;
                if (x == 0) { ends[0] = zh; ends[1] = zl; }
                if (x == it.L - 1) { ends[2] = zh; ends[3] = zl; }
                Fh[ROW_PADL + x] = end ? NEG : zh;
                Fl[ROW_PADL + x] = end ? 0.f : zl;
                zmax = fmaxf(zmax, fmaxf(fabsf(va[k]), fabsf(vb[k])));
            } else {
                Fh[ROW_PADL + x] = x == it.L - 1 ? NEG : blend32(va[k], vb[k], fr[k]);
            }
        }
    }
    for (int m = lane; part == 0 && m < ROW_PADR; m += 32) {
        if (!in_range(ROW_PADL + it.L + m, sp.half, 4)) continue;
        Fh[ROW_PADL + it.L + m] = NEG;
        if (CERT) Fl[ROW_PADL + it.L + m] = 0.f;
    }
    if (CERT) {
        if (part == 0 && lane < ROW_PADL) { Fh[lane] = NEG; Fl[lane] = 0.f; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    }
    return zmax;
}

// ------------------------------------------------ FP32-decision sweep --
__device__ __forceinline__ float fset_gt(float a, float b)
{
    // 1.0f if a > b (strict; false for NaN), else 0.0f
    float v;
    asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(v) : "f"(a), "f"(b));
    return v;
}

// Distance entry (1/d, 1/d, 2d + 1, 2d + 1) as the table holds it.
__device__ __forceinline__ float4 dist_entry(int d)
{
    const float r = __frcp_rn((float)d);
    const float c = (float)(2 * d + 1);
    return make_float4(r, r, c, c);
}

// U steps of one lane's P POVs.  POV q at step u (distance d = e + 1 + u)
// sees target w[q + u + 1]; its slope is (target - h_q) * (1/d) in single
// precision, it is visible iff that slope is strictly above the running
// maximum M_q, and a visible target adds 2d + 1 to the POV's measure.  Two
// POVs share one packed multiply and one packed accumulate; the comparison and
// the maximum are scalar.  tab[u] holds (1/d, 1/d, 2d + 1, 2d + 1); a
// range-limited walk's last block counts only its first `nvalid` steps.
// With FAR the block's entries are computed (distances e + 1 .. e + U, past
// the end of a capped table) instead of read from tab[0 .. U).
template <int P, int U, bool MASKED, bool FAR>
__device__ __forceinline__ void sweep_block(const float* w, const float4* __restrict__ tab, int e, const float* h,
                                            float* M, float2* acc2, int nvalid)
{
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const float4 t4 = FAR ? dist_entry(e + u + 1) : tab[u];
        const float2 iv = make_float2(t4.x, t4.y);
        float2 cpair = make_float2(t4.z, t4.w);
        if (MASKED && u >= nvalid) cpair = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < P; q += 2) {
            const float2 d = make_float2(__fsub_rn(w[q + u + 1], h[q]), __fsub_rn(w[q + u + 2], h[q + 1]));
            const float2 t = __fmul2_rn(d, iv);
            const float2 v = make_float2(fset_gt(t.x, M[q]), fset_gt(t.y, M[q + 1]));
            acc2[q / 2] = __ffma2_rn(v, cpair, acc2[q / 2]);
            M[q] = fmaxf(M[q], t.x);
            M[q + 1] = fmaxf(M[q + 1], t.y);
        }
    }
}

// Walks of more than LONG_WALK steps (rows longer than the constant, with a
// range beyond it) move their FP32 partial measures into integers every
// FLUSH_STEPS steps: a measure is a sum of odd integers 2d + 1 and stays exact
// in FP32 only below 2^24 (a walk of D steps sums to at most D^2 + 2D, and
// FLUSH_STEPS steps at d < 16384 add at most 1.1e7).  Shorter walks never
// flush (the LONG = false instantiation).
constexpr int LONG_WALK = 4000;
constexpr int FLUSH_STEPS = 336;   // a multiple of SMALL_UNROLL, LARGE_UNROLL and 24
// Suffix maxima of a staged row are kept at every ZS_STRIDE-th sample; pruning
// checks every PRUNE_EVERY blocks.
constexpr int ZS_STRIDE = 4;
constexpr int PRUNE_EVERY = 1;

// A warp item is one skewed row and one walk direction.  Its G groups of P
// consecutive POVs are taken in order (longest walks first) from a warp-local
// queue by whichever lane is free, so lanes stay busy whatever the walk
// lengths (and wherever pruning ends a walk early).  F holds the row (or the
// reversed row for backward walks) with -inf at its last sample and after it:
// the last target of a walk never adds area (its segment closes there), so it
// may be a sentinel that is never visible.  A walk's measure is
// cv = 1 + sum_{d=1}^{n-1} v_d (2d + 1) for n >= 1 targets, which is Alg. 8's
// sum of d^2 - open^2 over its closed segments plus the segment still open at
// the end (closed at the last target).
//
// PRUNE (exact horizon pruning): every PRUNE_EVERY blocks a lane stops its
// group's walks once min_q M_q >= B, B = fl(A * (1/d)) if A >= 0 else 0, where
// d is the next target distance and A = fl(Zmax - min_q h_q) with Zmax an upper
// bound of every remaining target (the suffix maximum ZS).  Rounding to nearest
// is monotone, so every remaining slope fl(fl(z - h_q) * fl(1/d')) is at most
// fl(A * fl(1/d)) when A >= 0 (d' >= d) and at most 0 when A < 0: no remaining
// target can be strictly above its POV's running maximum, and the walk's
// measure is already complete.  The result is bit for bit the same.
//
// With LONG, `spill` is the lane's column (stride 32) of P integers.
template <int P, int U, bool LONG, bool PRUNE>
__device__ __forceinline__ void sweep_row(const float* __restrict__ F, const float* __restrict__ ZS,
                                          const float4* __restrict__ tab, int tabn, int* __restrict__ cvrow,
                                          int* __restrict__ spill, int L, int K, float h0, bool rev, int lane)
{
    // the window is read as float4 from F + ROW_PADL + x0 + e (x0 = g P, e a
    // multiple of U): both must keep it 16-byte aligned
    static_assert(P % 4 == 0 && U % 4 == 0, "window loads must stay 16-byte aligned");
    const unsigned FULL = 0xffffffffu;
    const unsigned below = (1u << lane) - 1u;
    const float NEG = neg_inf();
    const int G = (L + P - 1) / P;
    const int klim = K - 1;          // last target distance that still adds area
    float h[P], M[P];
    float2 acc2[P / 2];
    float hmin = 0.f;
    int g = lane, next = 32;         // the lane's group; the first group nobody has taken
    int x0 = 0, e = 0, dlim = -1, seg = FLUSH_STEPS;
    int pc = 1;                      // blocks until the next pruning check
    bool klimited = false;

    auto start = [&]() {
        x0 = g * P;
        const int rowlim = L - 2 - x0;   // last target adding area, POV q = 0
        dlim = min(klim, rowlim);
        klimited = klim < rowlim;
        e = 0;
        seg = FLUSH_STEPS;
        pc = 1;
#pragma unroll
        for (int q = 0; q < P; ++q) { h[q] = __fadd_rn(F[ROW_PADL + x0 + q], h0); M[q] = NEG; }
#pragma unroll
        for (int q = 0; q < P / 2; ++q) acc2[q] = make_float2(0.f, 0.f);
        if (PRUNE) {
            hmin = h[0];
#pragma unroll
            for (int q = 1; q < P; ++q) hmin = fminf(hmin, h[q]);
        }
        if (LONG) {
#pragma unroll
            for (int q = 0; q < P; ++q) spill[32 * q] = 0;
        }
    };
    if (g < G) start();
    for (;;) {
        const bool fin = g < G && e >= dlim;
        const unsigned need = __ballot_sync(FULL, fin);
        if (need) {
            if (fin) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int x = x0 + q;
                    if (x < L) {
                        const int n = min(L - 1 - x, K);
                        const float s = q % 2 ? acc2[q / 2].y : acc2[q / 2].x;
                        cvrow[rev ? L - 1 - x : x] = n >= 1 ? 1 + (int)s + (LONG ? spill[32 * q] : 0) : 0;
                    }
                }
            }
            if (fin) {
                g = next + __popc(need & below);
                if (g < G) start(); else g = G;
            }
            next += __popc(need);
            if (!__any_sync(FULL, g < G)) break;
            continue;
        }
        if (g < G) {
            if (LONG && e >= seg) {
                seg += FLUSH_STEPS;
#pragma unroll
                for (int q = 0; q < P; q += 2) {
                    spill[32 * q] += __float2int_rz(acc2[q / 2].x);
                    spill[32 * (q + 1)] += __float2int_rz(acc2[q / 2].y);
                    acc2[q / 2] = make_float2(0.f, 0.f);
                }
            }
            if (PRUNE && --pc < 0) {
                pc = PRUNE_EVERY - 1;
                const float A = __fsub_rn(ZS[(x0 + e + 1) / ZS_STRIDE], hmin);
                const float rd = (LONG && e >= tabn) ? __frcp_rn((float)(e + 1)) : tab[e].x;
                const float B = A >= 0.f ? __fmul_rn(A, rd) : 0.f;
                float m = M[0];
#pragma unroll
                for (int q = 1; q < P; ++q) m = fminf(m, M[q]);
                if (m >= B) { e = dlim; continue; }
            }
            const float* base = F + ROW_PADL + x0 + e;
            float w[P + U];
#pragma unroll
            for (int m = 0; m < P + U; m += 4) {
                const float4 v = *reinterpret_cast<const float4*>(base + m);
                w[m] = v.x; w[m + 1] = v.y; w[m + 2] = v.z; w[m + 3] = v.w;
            }
            // long walks may run past a capped distance table (LONG only)
            const bool far = LONG && e + U > tabn;
            if (klimited && e + U > dlim) {
                if (far) sweep_block<P, U, true, true>(w, tab, e, h, M, acc2, dlim - e);
                else sweep_block<P, U, true, false>(w, tab + e, e, h, M, acc2, dlim - e);
            } else {
                if (far) sweep_block<P, U, false, true>(w, tab, e, h, M, acc2, U);
                else sweep_block<P, U, false, false>(w, tab + e, e, h, M, acc2, U);
            }
            e += U;
        }
    }
}

// Suffix maxima of the staged row F (L samples, -inf from L - 1 on) at every
// ZS_STRIDE-th sample: ZS[j] = max F[x] over x >= ZS_STRIDE * j, for
// j <= (L - 1) / ZS_STRIDE.  Lane l scans its own segment, a warp scan joins
// the segments.
__device__ __forceinline__ void suffix_max(const float* __restrict__ F, float* __restrict__ ZS, int L, int lane)
{
    const float NEG = neg_inf();
    const int seglen = ((L + 31) / 32 + ZS_STRIDE - 1) / ZS_STRIDE * ZS_STRIDE;
    const int a = lane * seglen, b = min(a + seglen, L);
    float m = NEG;
    for (int x = b - 1; x >= a; --x) m = fmaxf(m, F[ROW_PADL + x]);
    // inclusive suffix scan of the segment maxima over the lanes
    float s = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_down_sync(0xffffffffu, s, o);
        if (lane + o < 32) s = fmaxf(s, t);
    }
    float after = __shfl_down_sync(0xffffffffu, s, 1);   // maximum of the following segments
    if (lane == 31) after = NEG;
    float run = after;
    for (int x = b - 1; x >= a; --x) {
        run = fmaxf(run, F[ROW_PADL + x]);
        if (x % ZS_STRIDE == 0) ZS[x / ZS_STRIDE] = run;   // x / ZS_STRIDE <= (L - 1) / ZS_STRIDE < zs_len
    }
}

// Prefix maxima of the staged row F (row order, certified backward walks) at
// every ZS_STRIDE-th sample: ZP[j] = max F[x] over x <= ZS_STRIDE * j +
// ZS_STRIDE - 1, for j <= (L - 1) / ZS_STRIDE.  Lane l scans its own segment,
// a warp scan joins the segments.
__device__ __forceinline__ void prefix_max(const float* __restrict__ F, float* __restrict__ ZP, int L, int lane)
{
    const float NEG = neg_inf();
    const int seglen = ((L + 31) / 32 + ZS_STRIDE - 1) / ZS_STRIDE * ZS_STRIDE;
    const int a = lane * seglen, b = min(a + seglen, L);
    float m = NEG;
    for (int x = a; x < b; ++x) m = fmaxf(m, F[ROW_PADL + x]);
    // inclusive prefix scan of the segment maxima over the lanes
    float s = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s = fmaxf(s, t);
    }
    float before = __shfl_up_sync(0xffffffffu, s, 1);   // maximum of the earlier segments
    if (lane == 0) before = NEG;
    float run = before;
    for (int x = a; x < b; ++x) {
        run = fmaxf(run, F[ROW_PADL + x]);
        if (x % ZS_STRIDE == ZS_STRIDE - 1 || x == L - 1) ZP[x / ZS_STRIDE] = run;
    }
}

// ------------------------------------------------ certified decisions --
//
// The fast path of a group of P POVs x0 .. x0 + P - 1 works on differences
// against the group's reference R = zh(x0) (the hi part of its first
// sample, a float): per block it forms, for every target t of its window,
// y_t = fl(fl(zh_t - R) + zl_t), and per POV q once g_q = fl(fl(fl(zh_q -
// R) + zl_q) + h0).  Then, for POV q and target t at distance d,
//     diff = fl(y_t - g_q),  x = fl(diff * fl(1/d)),  s = fl(x - M_q),
// visible iff s > 0 (the sign of s is exact), M_q = max(M_q, x).
//
// Error bound (u = 2^-24; D = z_t - h_q exact, theta = D / d, G = h_q - R):
//   |y_t - (z_t - R)| <= 2u |z_t - R| + 2 eta (eta: the staged heights'
//   error, which also covers the u |zl_t| <= 2^-48 |z_t| of adding zl_t
//   after the subtraction), |g_q - G| <= 3.01u |G| + 2.01u |h0| + |h0 -
//   float(h0)| + 2 eta, so |diff - D| <= 3.01u |D| + Eg with Eg = 5.02u |G|
//   + 2.01u |h0| + |h0 - float(h0)| + 4 eta, and |x - theta| <= 5.04u
//   |theta| + 1.01 Eg / d.
// M_q is the x of the last visible target a (the maximum is exact), so with
// every earlier decision right, comparing x_t with M_q errs by at most
//   5.04u (|theta_t| + |theta_a|) + 1.01 Eg (1/d_t + 1/d_a).
// When |s| >= delta the decision is right as soon as
//   delta (1 - u)(1 - 5.05u) >= 10.1u |M| + 1.02 Eg (1/d_t + 1/d_a)
// (|theta| <= |x| (1 + 5.1u) + Eg / d, |x_t| <= |M| + |x_t - M|).  Per block
// and POV the kernel takes
//   delta = CERT_REL * Mb + CERT_ABS * Eg' * (1/(e+1) + ia) + CERT_FLOOR,
// with Mb >= |M| over the whole block (the test runs after the block's
// steps, and M only rises within it, so Mb = max(|M| at its start, |M| at
// its end)), 1/(e+1) >= 1/d_t, ia >= 1/d_a (1/(e'+1) of the last block e' in
// which M rose; 1 at first), Eg' >= Eg from the group's largest |g_q|.
// Induction over the targets then makes every unflagged decision the exact
// one.  A POV with a step inside its margin is flagged: its fast-path
// measure is discarded and it is walked again exactly.
constexpr float CERT_REL = 10.2f * 0x1p-24f * 1.01f;
constexpr float CERT_ABS = 1.03f * 1.01f;
constexpr float CERT_FLOOR = 0x1p-99f;
// Group size and steps per unrolled block of every certified walk.  A
// certified step takes about 40 % more instructions than an FP32 one and its
// state per POV twice the registers: groups of 4 POVs, and blocks short
// enough that the margin of a block (which grows with its window) stays
// tight.
#ifndef TVS_CERT_UNROLL
#define TVS_CERT_UNROLL 16
#endif
// The one-row-per-warp kernel (shorter rows, every walk staged forward)
// takes longer blocks: its lanes keep one margin per window block, and 24
// steps spread that block's overhead further (1000^2: 3 % faster); on the
// paired kernel's 2000-sample rows 24-step blocks were 4 % slower.
#ifndef TVS_CERT_UNROLL_SINGLE
#define TVS_CERT_UNROLL_SINGLE 24
#endif
constexpr int CERT_UNROLL = TVS_CERT_UNROLL;                 // paired-warp kernel
constexpr int CERT_UNROLL_SINGLE = TVS_CERT_UNROLL_SINGLE;   // one-row-per-warp kernel
#ifndef TVS_CERT_POV
#define TVS_CERT_POV SMALL_POV
#endif
constexpr int CERT_POV = TVS_CERT_POV;
static_assert(CERT_POV + CERT_UNROLL <= ROW_PADR && CERT_POV + CERT_UNROLL_SINGLE <= ROW_PADR,
              "a forward block's window reads up to P + U samples on");
static_assert(CERT_UNROLL <= ROW_PADL, "a backward block's window starts up to U samples before the row");
static_assert(FLUSH_STEPS % CERT_UNROLL == 0, "long walks flush on block boundaries");
// A certified kernel with U-step blocks stores distance entry m at slot m +
// m / U.  A lane reads entries e .. e + U - 1 of its own block start e (a
// multiple of U); groups of different lengths leave the lanes of a warp at
// different e, and unskewed such reads would fall on a few of the eight
// 16-byte bank groups.  Skewed, entry u of block k sits in bank group
// ((U + 1) k + u) mod 8 (U a multiple of 8), which spreads blocks k over all
// eight.  Tables are sized for the shorter block, which needs the most slots.
constexpr int TAB_SKEW_MIN = CERT_UNROLL < CERT_UNROLL_SINGLE ? CERT_UNROLL : CERT_UNROLL_SINGLE;
static_assert(CERT_UNROLL % 8 == 0 && CERT_UNROLL_SINGLE % 8 == 0, "skewed blocks cover the eight bank groups");
__host__ __device__ constexpr int tab_slots_for(int entries, bool skew)
{
    return skew ? ((entries + entries / TAB_SKEW_MIN + 1 + 1) & ~1) : entries;
}
// Far from the POV one margin serves several window blocks: from step
// CERT_NEAR on a margin block is 2 window blocks long, from CERT_FAR on 4 and
// from CERT_FAR2 on 8 (while the group's walks have that many steps left), so
// that the finish vote, the margins and the last-rise update are taken once
// per 32, 64 or 128 steps.  Near the POV, where the margin's 1/(e+1) terms
// fall fastest, every window block takes its own.  The lanes of a warp run
// as many window blocks as the longest of their margin blocks (the others
// wait), which pays only on long rows: the paired-warp kernel takes these
// tiers, the one-row-per-warp kernel (shorter rows) one window block per
// margin.  A pruned walk checks its stopping bound once per margin block and
// most pruned walks are short, so pruned launches keep one window block per
// margin too.
#ifndef TVS_CERT_NEAR
#define TVS_CERT_NEAR 64
#endif
#ifndef TVS_CERT_FAR
#define TVS_CERT_FAR 256
#endif
#ifndef TVS_CERT_FAR2
#define TVS_CERT_FAR2 (1 << 30)
#endif
#ifndef TVS_CERT_PACKADD
#define TVS_CERT_PACKADD 1
#endif
constexpr int CERT_NEAR = TVS_CERT_NEAR;
constexpr int CERT_FAR = TVS_CERT_FAR;
constexpr int CERT_FAR2 = TVS_CERT_FAR2;

// Entries of a warp's flagged-POV list (at least 32 lanes x LARGE_POV).
constexpr int FLAG_CAP = 256;
// Targets per lane per chunk of an exact walk.
constexpr int XW_KPL = 8;

// 1.0f if s >= 2^-100 (s > 0 and outside every margin, which is at least
// CERT_FLOOR), 0.0f if s <= 0, a fraction only inside the margin.
__device__ __forceinline__ float sat_pos(float s)
{
    float v;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(v) : "f"(s), "f"(0x1p100f), "f"(0.0f));
    return v;
}

// What the exact walks of a row need.
struct ExactCtx {
    const float* H;      // staged hi parts (index 0 = first sample)
    const float* Lo;     // staged lo parts
    int L, K;
    float h0h, h0l;      // h0 = h0h + h0l (to 2^-48)
    float eta;           // bound of the staged heights' error, plus h0's split
    int* cvrow;
    bool bwd;            // walks go toward lower sample indices
    bool from_dem;       // samples blended from the DEM as needed (no staged row)
    bool rev_staged;     // the staged row is reversed: staged x is row sample L - 1 - x
    float eh0, el0;      // hi and lo parts of the first sample (a sentinel in H, Lo)
    float ehL, elL;      // and of the last one
    const DirDev* dir;
    const JobDev* job;
    int p, jlo;
    int half;            // floats of a staged row array (index bound, with ROW_PADL)
    int zs_len;          // entries of the suffix maxima
    const float4* tab;   // the distance table (skewed: entry m at m + m / tskew)
    int tabn;            // its entries
    int tskew;           // its skew: the block length of the kernel that built it
};

// fl(1/d), correctly rounded: from the distance table while it reaches d.
__device__ __forceinline__ float inv_d(const ExactCtx& c, int d)
{
    const int m = d - 1;
    return m < c.tabn ? c.tab[m + m / c.tskew].x : __frcp_rn((float)d);
}

// Hi and lo parts of sample xs (row order) blended from the DEM, as the
// staging forms them.
__device__ __forceinline__ void dem_hl(const ExactCtx& c, int xs, float& hi, float& lo)
{
    const DirDev& d = *c.dir;
    const int j = c.jlo + (c.rev_staged ? c.L - 1 - xs : xs);
    const unsigned long long y = (unsigned long long)j * d.t_fx;
    const int a = c.p - d.D + (int)(y >> 32);
    const unsigned fr = (unsigned)y;
    int st;
    const long long idx = view_index(d, c.job->cols, a, j, &st);
    const long long cells = (long long)c.job->rows * c.job->cols;
    const float va = in_range(idx, cells, 16) ? c.job->dem[idx] : 0.f;
    const float vb = fr != 0u ? (in_range(idx + st, cells, 17) ? c.job->dem[idx + st] : 0.f) : va;
    df::df_blend(va, vb, fr, hi, lo);
}

// Hi and lo parts of POV x's ground height (the end samples are sentinels in
// the staged arrays; their real parts are kept aside).
__device__ __forceinline__ void pov_hl(const ExactCtx& c, int x, float& hi, float& lo)
{
    if (c.from_dem) dem_hl(c, x, hi, lo);
    else if (x == 0) { hi = c.eh0; lo = c.el0; }
    else if (x == c.L - 1) { hi = c.ehL; lo = c.elL; }
    else { hi = c.H[x]; lo = c.Lo[x]; }
}

// FP64 height of staged sample xs (row order) exactly as the FP64 definition
// forms it: (1 - r) * a + r * b with r = fr / 2^32, every operation rounded.
__device__ __forceinline__ double z64_at(const ExactCtx& c, int xs)
{
    const DirDev& d = *c.dir;
    const int j = c.jlo + (c.rev_staged ? c.L - 1 - xs : xs);
    const unsigned long long y = (unsigned long long)j * d.t_fx;
    const int a = c.p - d.D + (int)(y >> 32);
    const unsigned fr = (unsigned)y;
    int st;
    const long long idx = view_index(d, c.job->cols, a, j, &st);
    const long long cells = (long long)c.job->rows * c.job->cols;
    if (!in_range(idx, cells, 16) || (fr != 0u && !in_range(idx + st, cells, 17))) return 0.0;
    const double lo = (double)c.job->dem[idx];
    if (fr == 0u) return lo;
    const double hi = (double)c.job->dem[idx + st];
    const double r = __dmul_rn((double)fr, 0x1p-32);
    return __dadd_rn(__dmul_rn(__dsub_rn(1.0, r), lo), __dmul_rn(r, hi));
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The FP64 walk of POV x (Alg. 8 in double precision: theta = (z - h) / d
// rounded once, strict comparison with the running maximum): sum of 2d + 1
// over the visible targets d = 1 .. last.  Warp-cooperative: 32 x XW_KPL
// targets per chunk, a warp max-scan gives each lane the running maximum
// before its first target.
__device__ __noinline__ int fp64_walk(const ExactCtx& c, int x, int last, int lane)
{
    const double h = __dadd_rn(z64_at(c, x), c.job->h0);
    const int dir = c.bwd ? -1 : 1;
    double run = -__longlong_as_double(0x7ff0000000000000LL);
    int acc = 0;
    for (int base = 1; base <= last; base += 32 * XW_KPL) {
        double th[XW_KPL];
        double m = run;
        const int d0 = base + lane * XW_KPL;
#pragma unroll
        for (int k = 0; k < XW_KPL; ++k) {
            const int d = d0 + k;
            th[k] = d <= last ? __ddiv_rn(__dsub_rn(z64_at(c, x + dir * d), h), (double)d) : run;
            m = fmax(m, th[k]);
        }
        double incl = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = fmax(incl, t);
        }
        double cur = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) cur = run;
        cur = fmax(cur, run);
#pragma unroll
        for (int k = 0; k < XW_KPL; ++k) {
            const int d = d0 + k;
            if (d > last) break;
            if (th[k] > cur) { acc += 2 * d + 1; cur = th[k]; }
        }
        run = fmax(run, __shfl_sync(0xffffffffu, incl, 31));
    }
    return warp_sum(acc);
}

// The double-float walk of POV x: the same sum, with every decision proved by
// a margin (slope error <= 2^-45 |theta| + eta / d each); a decision inside
// its margin sets *esc and the FP64 walk decides instead.
__device__ __noinline__ int df_walk(const ExactCtx& c, int x, int last, int lane, bool* esc_out)
{
    const float NEG = neg_inf();
    const int dir = c.bwd ? -1 : 1;
    float hh, hl;
    {
        float zh, zl;
        pov_hl(c, x, zh, zl);
        float s, e;
        df::two_sum(zh, c.h0h, s, e);
        e = __fadd_rn(e, __fadd_rn(zl, c.h0l));
        df::two_sum(s, e, hh, hl);
    }
    float rh = NEG, rl = 0.f;
    int rd = 1;
    int acc = 0;
    bool esc = false;
    for (int base = 1; base <= last; base += 32 * XW_KPL) {
        float th[XW_KPL], tl[XW_KPL], iv[XW_KPL];
        float mh = NEG, ml = 0.f;
        int md = 1;
        const int d0 = base + lane * XW_KPL;
#pragma unroll
        for (int k = 0; k < XW_KPL; ++k) {
            const int d = d0 + k;
            th[k] = NEG; tl[k] = 0.f; iv[k] = 1.f;
            if (d <= last && (c.from_dem || in_range(ROW_PADL + x + dir * d, c.half, 15))) {
                iv[k] = inv_d(c, d);
                float zh, zl;
                if (c.from_dem) dem_hl(c, x + dir * d, zh, zl);
                else { zh = c.H[x + dir * d]; zl = c.Lo[x + dir * d]; }
                df::df_slope_iv(zh, zl, hh, hl, d, iv[k], th[k], tl[k]);
                if (df::df_gt(th[k], tl[k], mh, ml)) { mh = th[k]; ml = tl[k]; md = d; }
            }
        }
        // inclusive max-scan over the lanes
        float ph = mh, pl = ml;
        int pd = md;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float qh = __shfl_up_sync(0xffffffffu, ph, o);
            const float ql = __shfl_up_sync(0xffffffffu, pl, o);
            const int qd = __shfl_up_sync(0xffffffffu, pd, o);
            if (lane >= o && df::df_gt(qh, ql, ph, pl)) { ph = qh; pl = ql; pd = qd; }
        }
        float ch = __shfl_up_sync(0xffffffffu, ph, 1);
        float cl = __shfl_up_sync(0xffffffffu, pl, 1);
        int cd = __shfl_up_sync(0xffffffffu, pd, 1);
        if (lane == 0 || df::df_gt(rh, rl, ch, cl)) { ch = rh; cl = rl; cd = rd; }
        float icd = inv_d(c, cd);
#pragma unroll
        for (int k = 0; k < XW_KPL; ++k) {
            const int d = d0 + k;
            if (d > last) break;
            bool v = true;                           // the first target (no earlier one) is visible
            if (ch > NEG) {
                float s, e;
                df::two_sum(th[k], -ch, s, e);
                const float dh = __fadd_rn(s, __fadd_rn(e, __fsub_rn(tl[k], cl)));
                const float marg = __fmaf_rn(0x1p-40f, fabsf(th[k]) + fabsf(ch), 4.04f * c.eta * (iv[k] + icd)) +
                                   0x1p-120f;
                if (!(fabsf(dh) > marg)) esc = true;
                v = dh > 0.f;
            }
            if (v) acc += 2 * d + 1;
            if (df::df_gt(th[k], tl[k], ch, cl)) { ch = th[k]; cl = tl[k]; cd = d; icd = iv[k]; }
        }
        const float lh = __shfl_sync(0xffffffffu, ph, 31);
        const float ll = __shfl_sync(0xffffffffu, pl, 31);
        const int ld = __shfl_sync(0xffffffffu, pd, 31);
        if (df::df_gt(lh, ll, rh, rl)) { rh = lh; rl = ll; rd = ld; }
    }
    *esc_out = __any_sync(0xffffffffu, esc);
    return warp_sum(acc);
}

// Exact measure of POV x of the staged row, written by lane 0.
__device__ __noinline__ void exact_walk(const ExactCtx& c, int x, int lane)
{
    const int n = min(c.bwd ? x : c.L - 1 - x, c.K);
    int cv;
    if (n < 2) {
        cv = n < 1 ? 0 : 1;
    } else {
        bool esc = false;
        const int s = df_walk(c, x, n - 1, lane, &esc);
        cv = 1 + (esc ? fp64_walk(c, x, n - 1, lane) : s);
        if (lane == 0) {
            atomicAdd(&g_sweep_stats[0], 1ull);
            if (esc) atomicAdd(&g_sweep_stats[1], 1ull);
        }
    }
    if (lane == 0 && in_range(x, c.L, 14)) c.cvrow[c.rev_staged ? c.L - 1 - x : x] = cv;
}

// The warp's list of flagged POVs (positions in the staged row).
struct FlagList {
    int* list;
    int count;
    int4* gbuf;          // the launch's flagged-walk buffer (NULL: walk every flag here)
    unsigned* gcount;    // its fill counter
    int gcap;            // its capacity
    int item;            // the current row's work item
    float zmax;          // and its largest |elevation| (for the staged heights' error bound)
};

__device__ __noinline__ void drain_flags(FlagList& fl, const ExactCtx& c, int lane)
{
    __syncwarp();
    const long long t0 = clock64();
    for (int i = 0; i < fl.count; ++i) exact_walk(c, fl.list[i], lane);
    fl.count = 0;
    if (lane == 0) atomicAdd(&g_sweep_stats[2], (unsigned long long)(clock64() - t0));
    __syncwarp();
}

// Warp-collective: appends every lane's flagged POVs (bits of fm, positions
// x0 + q), first walking the list exactly when it would overflow.
__device__ __forceinline__ void flag_push(FlagList& fl, const ExactCtx& c, unsigned fm, int x0, int lane)
{
    const int cnt = __popc(fm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (fl.gbuf) {
        // hand the walks to the exact pass after the sweep: (item, sample)
        // entries; when the buffer is full they are walked here instead
        unsigned at = 0u;
        if (lane == 0) at = atomicAdd(fl.gcount, (unsigned)total);
        at = __shfl_sync(0xffffffffu, at, 0);
        if ((unsigned long long)at + (unsigned long long)total <= (unsigned long long)fl.gcap) {
            unsigned pos = at + (unsigned)(incl - cnt);
            for (unsigned m = fm; m; m &= m - 1, ++pos)
                if (in_range(pos, fl.gcap, 20)) {
                    const int xs = x0 + __ffs(m) - 1;   // staged sample; the entry holds the row's
                    fl.gbuf[pos] = make_int4(fl.item, c.rev_staged ? c.L - 1 - xs : xs, __float_as_int(fl.zmax), 0);
                }
            __syncwarp();
            return;
        }
        // full: the slots reserved below the capacity are marked empty
        for (unsigned long long pos = (unsigned long long)at + lane;
             pos < (unsigned long long)at + (unsigned long long)total && pos < (unsigned long long)fl.gcap; pos += 32)
            fl.gbuf[pos] = make_int4(-1, -1, 0, 0);
        __syncwarp();
    }
    if (fl.count + total > FLAG_CAP) drain_flags(fl, c, lane);
    int pos = fl.count + incl - cnt;
    for (unsigned m = fm; m; m &= m - 1, ++pos)
        if (in_range(pos, FLAG_CAP, 13)) fl.list[pos] = x0 + __ffs(m) - 1;
    fl.count += total;
    __syncwarp();
}

// min(a, |b|, |c|).  TVS_CERT_MIN3 selects the three-input minimum of
// sm_100+ (one instruction for two steps of a POV) or two chained minima.
#ifndef TVS_CERT_MIN3
#define TVS_CERT_MIN3 1
#endif
__device__ __forceinline__ float min_abs2(float a, float b, float c)
{
#if TVS_CERT_MIN3
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(fabsf(b)), "f"(fabsf(c)));
    return r;
#else
    return fminf(fminf(a, fabsf(b)), fabsf(c));
#endif
}

// U certified steps of one lane's P POVs (see the derivation above), two
// steps at a time.  y[m] is the window's target x0 + e + m relative to R,
// ng2 the POVs' heights relative to R, negated, in pairs (q, q + 1).  mn[q]
// keeps the smallest |s| of the POV's steps: the block's margin test (mn <
// delta) runs once at its end.  With PACK the differences of a pair of POVs
// go through one packed add wherever their two targets form an aligned pair
// of the window (y[2j], y[2j + 1]: every other step); y - g and y + (-g)
// round alike.
template <int P, int U, bool MASKED, bool FAR, bool PACK>
__device__ __forceinline__ void cert_block(const float* y, const float4* __restrict__ tab, int e, const float2* ng2,
                                           float2* M2, float2* acc2, float* mn, int nvalid)
{
    static_assert(U % 2 == 0, "steps go in pairs");
#pragma unroll
    for (int u = 0; u < U; u += 2) {
        float2 sv[2][P / 2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int w = u + k;
            const float4 t4 = FAR ? dist_entry(e + w + 1) : tab[w + w / U];
            const float2 iv = make_float2(t4.x, t4.y);
            float2 cp = make_float2(t4.z, t4.w);
            if (MASKED && w >= nvalid) cp = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < P; q += 2) {
                const float2 d = (PACK && (q + w + 1) % 2 == 0)
                                     ? __fadd2_rn(make_float2(y[q + w + 1], y[q + w + 2]), ng2[q / 2])
                                     : make_float2(__fadd_rn(y[q + w + 1], ng2[q / 2].x),
                                                   __fadd_rn(y[q + w + 2], ng2[q / 2].y));
                const float2 x = __fmul2_rn(d, iv);
                const float2 sp = __ffma2_rn(make_float2(-1.f, -1.f), M2[q / 2], x);
                const float2 v = make_float2(sat_pos(sp.x), sat_pos(sp.y));
                acc2[q / 2] = __ffma2_rn(v, cp, acc2[q / 2]);
                M2[q / 2].x = fmaxf(M2[q / 2].x, x.x);
                M2[q / 2].y = fmaxf(M2[q / 2].y, x.y);
                // a masked step's |s| is +inf: it takes no part in the test
                sv[k][q / 2] = (MASKED && w >= nvalid) ? make_float2(pos_inf(), pos_inf()) : sp;
            }
        }
#pragma unroll
        for (int q = 0; q < P; q += 2) {
            mn[q] = min_abs2(mn[q], sv[0][q / 2].x, sv[1][q / 2].x);
            mn[q + 1] = min_abs2(mn[q + 1], sv[0][q / 2].y, sv[1][q / 2].y);
        }
    }
}

// Upper bound of the slopes a POV of the group can meet among targets whose
// hi heights are at most z (a suffix or prefix maximum): max(0, z + slack -
// Rh - gmin) / (e + 1), with slack covering the hi / lo split, the rounding of
// the differences and of g (2^-20 relative, plus eg).  z = -inf (sentinels
// only) gives 0.
__device__ __forceinline__ float bound_slope(float z, float Rh, float gmin, float eg, float ive)
{
    const float A = __fsub_rn(__fsub_rn(z, Rh), gmin);
    const float sl = 0x1p-20f * (fminf(fabsf(z), 0x1p100f) + fabsf(Rh) + fabsf(gmin)) + eg;
    return __fmul_rn(fmaxf(__fadd_rn(A, sl), 0.f), ive) * 1.0000039f;
}

// Certified sweep of one staged row (the lane queue of sweep_row).  eg0 =
// 2.01u |h0| + |h0 - float(h0)| + 4 eta (the parts of Eg that do not depend
// on the group).  With PRUNE a group stops once, for every POV q, the
// remaining targets' largest possible exact slope (from the suffix maxima,
// or the prefix maxima of a backward walk) is at most M_q - 2 delta_q: they
// are then not above theta_a exactly.
//
// The row is staged in row order for both walk directions.  A group covers
// the samples x0 .. x0 + P - 1 (x0 a multiple of 4, so that every window is
// 16-byte aligned); its POV q is sample x0 + q walking forward, or sample
// x0 + P - 1 - q walking backward, so that in either direction POV q's step
// w meets the window's element q + w + 1: a backward block's window is
// loaded from x0 - e - U and stored reversed.  Backward groups are taken
// from the row's end (the longest walks first).
template <int P, int U, bool LONG, bool PRUNE, bool BWD, bool TIERS>
__device__ __forceinline__ void sweep_row_cert(const ExactCtx& xc, const float* __restrict__ ZS,
                                               const float4* __restrict__ tab,
                                               int tabn, int* __restrict__ spill, float eg0, FlagList& fl, int lane)
{
    static_assert(P % 4 == 0 && U % 4 == 0, "window loads must stay 16-byte aligned");
    const unsigned FULL = 0xffffffffu;
    const unsigned below = (1u << lane) - 1u;
    const float NEG = neg_inf();
    const float* __restrict__ H = xc.H;
    const float* __restrict__ Lo = xc.Lo;
    const int L = xc.L, K = xc.K;
    const int G = (L + P - 1) / P;
    const int klim = K - 1;
    // a backward block's window is stored reversed, so its aligned register
    // pairs hold (y[2j + 1], y[2j]) and only forward walks pack the differences
    constexpr bool PACK = !BWD && TVS_CERT_PACKADD;
    float ia[P];
    float2 ng2[P / 2];               // -g of POV pairs
    float2 M2[P / 2], acc2[P / 2];   // running maxima of POV pairs (packed x - M)
#define CERT_M(q) ((q) % 2 ? M2[(q) / 2].y : M2[(q) / 2].x)
#define CERT_NG(q) ((q) % 2 ? ng2[(q) / 2].y : ng2[(q) / 2].x)
    float Rh = 0.f, gmin = 0.f, c2e = 0.f;
    unsigned mask = 0u;
    int gi = lane, next = 32;
    int x0 = 0, e = 0, dlim = -1, seg = FLUSH_STEPS;
    bool klimited = false;
    // sample of POV q of the current group, and its walk's target count
    auto pov_x = [&](int q) { return BWD ? x0 + P - 1 - q : x0 + q; };
    auto walk_n = [&](int x) { return min(BWD ? x : L - 1 - x, K); };

    auto start = [&]() {
        x0 = (BWD ? G - 1 - gi : gi) * P;
        // the group's longest walk: its first existing POV in walk order
        const int xl = BWD ? min(x0 + P - 1, L - 1) : x0;
        const int rowlim = BWD ? xl - 1 : L - 2 - xl;
        dlim = min(klim, rowlim);
        klimited = klim < rowlim;
        e = 0;
        seg = FLUSH_STEPS;
        mask = 0u;
#pragma unroll
        for (int q = 0; q < P / 2; ++q) acc2[q] = make_float2(0.f, 0.f);
        if (LONG) {
#pragma unroll
            for (int q = 0; q < P; ++q) spill[32 * q] = 0;
        }
        if (dlim < 1) return;                 // no block runs
        // every index the group's blocks use, checked once: the last block
        // starts at elast < dlim
        const int elast = (dlim - 1) / U * U;
        const int wlo = BWD ? x0 - elast - U : x0;           // lowest window start
        const int whi = BWD ? x0 - U : x0 + elast;           // highest window start
        const int zsi = BWD ? (x0 + P - 2) / ZS_STRIDE : (x0 + elast + 1) / ZS_STRIDE;
        if (!in_range(ROW_PADL + wlo, xc.half, 19) || !in_range(ROW_PADL + whi + P + U - 1, xc.half, 19) ||
            (PRUNE && !in_range(zsi, xc.zs_len, 9)) ||
            (!(LONG && elast + U > tabn) && !in_range(elast + U - 1, tabn, 11))) {
            dlim = 0;
            const unsigned all = L - x0 >= P ? (1u << P) - 1u : (1u << (L - x0)) - 1u;   // bits by sample
            mask = BWD ? __brev(all) >> (32 - P) : all;                                   // bits by POV q
            return;
        }
        float Rl;
        pov_hl(xc, x0, Rh, Rl);
        (void)Rl;
        float gmax = 0.f;
        gmin = pos_inf();
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int x = pov_x(q);
            float gq = 0.f;
            if (BWD ? (x >= 1 && x <= L - 1) : x <= L - 2) {   // POVs with a target
                float zh, zl;
                pov_hl(xc, x, zh, zl);
                gq = __fadd_rn(__fadd_rn(__fsub_rn(zh, Rh), zl), xc.h0h);
                gmin = fminf(gmin, gq);
            }
            CERT_NG(q) = -gq;
            gmax = fmaxf(gmax, fabsf(gq));
        }
        c2e = CERT_ABS * __fmaf_rn(5.1f * 0x1p-24f, gmax, eg0);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            // target 1 (a sentinel, -inf, when the POV has no target adding
            // area): M starts just below its slope, so that target is visible
            // and outside its margin, and the maximum then is its slope exactly
            const int x = pov_x(q);
            const int t = BWD ? x - 1 : x + 1;
            const float y1 = __fadd_rn(__fsub_rn(H[t], Rh), Lo[t]);
            const float x1 = __fadd_rn(y1, CERT_NG(q));
            const float C = __fmaf_rn(0x1p-6f, fabsf(x1), __fmaf_rn(4.f, c2e, 0x1p-16f));
            // a POV with no target that adds area starts at +inf: nothing is
            // visible to it, no step is inside its margin, and it never holds
            // back pruning
            const bool area = BWD ? (x >= 2 && x <= L - 1) : x <= L - 3;
            CERT_M(q) = area ? __fsub_rn(x1, C) : pos_inf();
            ia[q] = 1.f;
        }
    };
    if (gi < G) start();
    for (;;) {
        const bool fin = gi < G && e >= dlim;
        const unsigned need = __ballot_sync(FULL, fin);
        if (need) {
            if (fin) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int x = pov_x(q);
                    if (x < L && !((mask >> q) & 1u)) {
                        const int n = walk_n(x);
                        const float s = q % 2 ? acc2[q / 2].y : acc2[q / 2].x;
                        xc.cvrow[xc.rev_staged ? L - 1 - x : x] = n >= 1 ? 1 + (int)s + (LONG ? spill[32 * q] : 0) : 0;
                    }
                }
            }
            // flagged POVs as bits by sample (x0 + bit)
            const unsigned fm = fin ? (BWD ? __brev(mask) >> (32 - P) : mask) : 0u;
            if (__any_sync(FULL, fm != 0u)) flag_push(fl, xc, fm, x0, lane);
            if (fin) {
                gi = next + __popc(need & below);
                if (gi < G) start(); else gi = G;
            }
            next += __popc(need);
            if (!__any_sync(FULL, gi < G)) break;
            continue;
        }
        if (gi < G) {
            if (LONG && e >= seg) {
                seg += FLUSH_STEPS;
#pragma unroll
                for (int q = 0; q < P; q += 2) {
                    spill[32 * q] += __float2int_rz(acc2[q / 2].x);
                    spill[32 * (q + 1)] += __float2int_rz(acc2[q / 2].y);
                    acc2[q / 2] = make_float2(0.f, 0.f);
                }
            }
            // a margin block of nh window blocks of U steps.  The bounds are
            // formed branch-free: a window or suffix of sentinels only (-inf)
            // gives 0.  A margin block of several window blocks lies wholly
            // before the group's last needed step (e + nh U <= dlim), so none
            // of its window blocks is masked and every window and table entry
            // it reads lies in the ranges start() checked.
            const int nh = (!TIERS || PRUNE || LONG || e < CERT_NEAR) ? 1
                         : (e >= CERT_FAR2 && e + 8 * U <= dlim) ? 8
                         : (e >= CERT_FAR && e + 4 * U <= dlim) ? 4
                         : (e + 2 * U <= dlim) ? 2 : 1;
            const float4* __restrict__ tb = tab + e + e / U;
            const float ive = (LONG && e >= tabn) ? __frcp_rn((float)(e + 1)) : tb->x;
            float Ms[P], mn[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                Ms[q] = CERT_M(q);
                mn[q] = pos_inf();
            }
            if (PRUNE) {
                // the remaining targets (samples from x0 + e + 1 on forward, up
                // to x0 + P - 2 - e backward) have exact slopes of at most Bp;
                // delta with Mb = |M| bounds |M - theta_a| now, so once M - 2
                // delta >= Bp for every POV none of them rises above theta_a
                const float ce = __fmaf_rn(c2e, ive, CERT_FLOOR);
                const int zi = BWD ? max(x0 + P - 2 - e, 0) / ZS_STRIDE : (x0 + e + 1) / ZS_STRIDE;
                const float Bp = bound_slope(ZS[zi], Rh, gmin, 2.f * c2e, ive);
                float m = pos_inf();
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const float dq = __fmaf_rn(CERT_REL, fabsf(CERT_M(q)), __fmaf_rn(c2e, ia[q], ce));
                    m = fminf(m, __fmaf_rn(-2.f, dq, CERT_M(q)));
                }
                if (m >= Bp) { e = dlim; continue; }
            }
#pragma unroll 1
            for (int h = 0; h < nh; ++h) {
                const int eh = e + h * U;                    // this window block's first step
                const int wsh = BWD ? x0 - eh - U : x0 + eh; // its window's first sample
                const bool far = LONG && eh + U > tabn;
                const float4* __restrict__ tbh = tab + eh + eh / U;
                // the window, relative to R (reversed for a backward walk)
                float y[P + U];
                {
                    const float2 nRh = make_float2(-Rh, -Rh);
                    const float* bh = H + wsh;
                    const float* bl = Lo + wsh;
#pragma unroll
                    for (int m = 0; m < P + U; m += 4) {
                        const float4 a = *reinterpret_cast<const float4*>(bh + m);
                        const float4 b = *reinterpret_cast<const float4*>(bl + m);
                        const float2 y0 = __fadd2_rn(__fadd2_rn(make_float2(a.x, a.y), nRh), make_float2(b.x, b.y));
                        const float2 y1 = __fadd2_rn(__fadd2_rn(make_float2(a.z, a.w), nRh), make_float2(b.z, b.w));
                        const float v[4] = {y0.x, y0.y, y1.x, y1.y};
#pragma unroll
                        for (int i = 0; i < 4; ++i) y[BWD ? P + U - 1 - (m + i) : m + i] = v[i];
                    }
                }
                const bool masked = klimited && eh + U > dlim;
                if (masked) {
                    if (far) cert_block<P, U, true, true, PACK>(y, tab, eh, ng2, M2, acc2, mn, dlim - eh);
                    else cert_block<P, U, true, false, PACK>(y, tbh, eh, ng2, M2, acc2, mn, dlim - eh);
                } else {
                    if (far) cert_block<P, U, false, true, PACK>(y, tab, eh, ng2, M2, acc2, mn, U);
                    else cert_block<P, U, false, false, PACK>(y, tbh, eh, ng2, M2, acc2, mn, U);
                }
            }
            // the margin test, once the block's last M is known: M only rises
            // within the block, so max(|M| at its start, |M| at its end)
            // bounds |M| at every one of its steps
            const float ce = __fmaf_rn(c2e, ive, CERT_FLOOR);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const float dq =
                    __fmaf_rn(CERT_REL, fmaxf(fabsf(Ms[q]), fabsf(CERT_M(q))), __fmaf_rn(c2e, ia[q], ce));
                mask |= mn[q] < dq ? 1u << q : 0u;
            }
#pragma unroll
            for (int q = 0; q < P; ++q) ia[q] = CERT_M(q) > Ms[q] ? ive : ia[q];
            e += nh * U;
        }
    }
    if (fl.count > 0) drain_flags(fl, xc, lane);
#undef CERT_M
#undef CERT_NG
}

template <bool LONG, bool PRUNE>
__device__ __forceinline__ void sweep_item(const ItemRow& it, const float* F, const float* ZS, const float4* tab,
                                           int tabn, int* cvrow, int* spill, int lane)
{
    if (it.pov == SMALL_POV)
        sweep_row<SMALL_POV, SMALL_UNROLL, LONG, PRUNE>(F, ZS, tab, tabn, cvrow, spill, it.L, it.K, it.h0, it.rev,
                                                       lane);
    else
        sweep_row<LARGE_POV, LARGE_UNROLL, LONG, PRUNE>(F, ZS, tab, tabn, cvrow, spill, it.L, it.K, it.h0, it.rev,
                                                       lane);
}


// Warps per CTA of the certified kernels (pairs of warps, below): their
// per-lane state (4 POVs' maxima, heights, margins and last-visible bounds,
// the window relative to the group) takes about 160 registers, which 12 warps
// still leave every thread.  When shared memory holds CERT_WIDE_WARPS warps, a
// second instantiation bounded to 128 registers runs them: the extra warps
// hide more latency than the few spills of its group-restart path cost.
#ifndef TVS_CERT_MAX_WARPS
#define TVS_CERT_MAX_WARPS 12
#endif
constexpr int CERT_MAX_WARPS = TVS_CERT_MAX_WARPS;
#ifndef TVS_CERT_WIDE_WARPS
#define TVS_CERT_WIDE_WARPS 16
#endif
constexpr int CERT_WIDE_WARPS = TVS_CERT_WIDE_WARPS;
// The fewest warps the one-row-per-warp certified kernel runs with; longer
// rows go to warp pairs.
#ifndef TVS_CERT_SINGLE_MIN
#define TVS_CERT_SINGLE_MIN 12
#endif
static_assert(CERT_MAX_WARPS % 2 == 0 && CERT_WIDE_WARPS % 2 == 0, "certified warps come in pairs");

// The FP32-decision sweep.  PRUNE: exact horizon pruning; LONG: the launch
// holds rows with walks of more than LONG_WALK steps (every row then takes
// the flushing walk).  Per warp, shared memory holds the staged row (reversed
// for backward items), its suffix maxima (PRUNE) and the long-walk spill
// (LONG).
template <bool PRUNE, bool LONG, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) sweep_kernel(SweepParams sp)
{
    extern __shared__ __align__(16) float smem[];
    float4* tab = reinterpret_cast<float4*>(smem);
    int* istart = reinterpret_cast<int*>(smem + 4 * sp.tab_slots);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* Fh = smem + 4 * sp.tab_slots + sp.istart_len + warp * sp.per_warp;
    float* ZS = Fh + sp.half;
    int* spill = reinterpret_cast<int*>(ZS + sp.zs_len) + lane;
    // per distance d = m + 1: (1/d, 1/d, 2d + 1, 2d + 1); 1/d correctly rounded
    for (int m = threadIdx.x; m < sp.inv_len; m += blockDim.x) {
        const float r = __frcp_rn((float)(m + 1));
        const float c = (float)(2 * m + 3);
        tab[m] = make_float4(r, r, c, c);
    }
    for (int m = threadIdx.x; m <= sp.ndir; m += blockDim.x) istart[m] = sp.item_start[m];
    __syncthreads();

    int next = 0;
    if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    for (;;) {
        const int item = next;
        if (item >= sp.total_items) break;
        ItemRow it;
        const bool nonempty = decode_item(sp, istart, item, &it);
        if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
        next = __shfl_sync(0xffffffffu, next, 0);
        if (!nonempty) continue;
        __syncwarp();
        stage_row<false>(sp, it, Fh, nullptr, nullptr, lane);
        __syncwarp();   // the staged row is visible to every lane
        if (PRUNE) {
            suffix_max(Fh, ZS, it.L, lane);
            __syncwarp();
        }
        int* cvrow = (it.rev ? sp.cv_bwd : sp.cv_fwd) + it.rowbase;
        sweep_item<LONG, PRUNE>(it, Fh, ZS, tab, sp.inv_len, cvrow, spill, lane);
    }
}

// The certified sweep with one row per warp, for launches whose rows leave
// room for at least TVS_CERT_SINGLE_MIN of them (16 warps when they fit, else
// 12): a backward item's row is staged reversed and walked forward, like the
// FP32 sweep's.  Per warp, shared memory holds
// [Fh half][Fl half][suffix maxima][flag list][spill][ends 4].
template <bool PRUNE, bool LONG, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) sweep_cert_kernel(SweepParams sp)
{
    extern __shared__ __align__(16) float smem[];
    float4* tab = reinterpret_cast<float4*>(smem);
    int* istart = reinterpret_cast<int*>(smem + 4 * sp.tab_slots);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* Fh = smem + 4 * sp.tab_slots + sp.istart_len + warp * sp.per_warp;
    float* Fl = Fh + sp.half;
    float* ZS = Fl + sp.half;
    int* flist = reinterpret_cast<int*>(ZS + sp.zs_len);
    int* spill = flist + sp.fl_cap + lane;
    float* ends = Fh + sp.per_warp - 4;
    for (int m = threadIdx.x; m < sp.inv_len; m += blockDim.x) {
        const float r = __frcp_rn((float)(m + 1));
        const float c = (float)(2 * m + 3);
        tab[m + m / CERT_UNROLL_SINGLE] = make_float4(r, r, c, c);
    }
    for (int m = threadIdx.x; m <= sp.ndir; m += blockDim.x) istart[m] = sp.item_start[m];
    __syncthreads();
    FlagList fl{flist, 0, sp.flag_buf, sp.flag_count, sp.flag_cap, 0, 0.f};
    const long long t_start = clock64();

    int next = 0;
    if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    for (;;) {
        const int item = next;
        if (item >= sp.total_items) break;
        ItemRow it;
        const bool nonempty = decode_item(sp, istart, item, &it);
        if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
        next = __shfl_sync(0xffffffffu, next, 0);
        if (!nonempty) continue;
        __syncwarp();
        const float zmax = stage_row<true>(sp, it, Fh, Fl, ends, lane);
        __syncwarp();   // the staged row is visible to every lane
        if (PRUNE) suffix_max(Fh, ZS, it.L, lane);
        __syncwarp();
        fl.item = item;
        fl.zmax = zmax;
        const DirDev* d = sp.dirs + it.dir;
        ExactCtx xc;
        xc.H = Fh + ROW_PADL;
        xc.Lo = Fl + ROW_PADL;
        xc.L = it.L;
        xc.K = it.K;
        xc.h0h = it.h0;
        xc.h0l = d->h0_lo;
        xc.eta = 0x1p-42f * (zmax + fabsf(it.h0)) + 0x1p-126f;
        xc.cvrow = (it.rev ? sp.cv_bwd : sp.cv_fwd) + it.rowbase;
        xc.bwd = false;
        xc.from_dem = false;
        xc.rev_staged = it.rev;
        xc.eh0 = ends[0];
        xc.el0 = ends[1];
        xc.ehL = ends[2];
        xc.elL = ends[3];
        xc.dir = d;
        xc.job = sp.jobs + d->job;
        xc.p = it.p;
        xc.jlo = it.jlo;
        xc.half = sp.half;
        xc.zs_len = sp.zs_len;
        xc.tab = tab;
        xc.tskew = CERT_UNROLL_SINGLE;
        xc.tabn = sp.inv_len;
        const float u = 0x1p-24f;
        const float eg0 = 2.01f * u * fabsf(it.h0) + fabsf(d->h0_lo) * 1.0001f + 4.04f * xc.eta;
        sweep_row_cert<CERT_POV, CERT_UNROLL_SINGLE, LONG, PRUNE, false, false>(xc, ZS, tab, sp.inv_len, spill, eg0,
                                                                                fl, lane);
    }
    if (lane == 0) atomicAdd(&g_sweep_stats[3], (unsigned long long)(clock64() - t_start));
}

// Barrier of the two warps of pair `pair` (named barrier 1 + pair).
__device__ __forceinline__ void pair_sync(int pair)
{
    asm volatile("bar.sync %0, %1;" :: "r"(1 + pair), "r"(64) : "memory");
}

// The certified sweep with one staged row per pair of warps: warp 2k walks
// every row of the pair forward and warp 2k + 1 walks the same row backward
// (items 2p and 2p + 1), so a row's double-float samples and end samples are
// staged once and held once for both directions (half the shared memory per
// warp of one row per warp, and room for twice the warps at 2000-sample
// rows).  Both warps stage half of the row; the forward warp computes its
// suffix maxima, the backward warp its prefix maxima (pruning).  Each warp
// runs one direction's code only.  Per pair, shared memory holds [Fh
// half][Fl half][suffix maxima][prefix maxima][ends 4][exchange 4]; per warp
// the flagged-POV list and the long-walk spill.
template <bool PRUNE, bool LONG, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) sweep_pair_kernel(SweepParams sp)
{
    extern __shared__ __align__(16) float smem[];
    float4* tab = reinterpret_cast<float4*>(smem);
    int* istart = reinterpret_cast<int*>(smem + 4 * sp.tab_slots);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = warp >> 1, bwd = warp & 1;
    const int npairs = blockDim.x >> 6;
    float* base = smem + 4 * sp.tab_slots + sp.istart_len;
    float* Fh = base + pair * sp.per_pair;
    float* Fl = Fh + sp.half;
    float* ZS = Fl + sp.half + bwd * sp.zs_len;            // this warp's suffix or prefix maxima
    float* ends = Fl + sp.half + 2 * sp.zs_len;              // 4 floats
    float* xch = ends + 4;                                   // item number and the halves' zmax
    float* own = base + npairs * sp.per_pair + warp * sp.per_warp;
    int* flist = reinterpret_cast<int*>(own);
    int* spill = reinterpret_cast<int*>(own) + sp.fl_cap + lane;
    for (int m = threadIdx.x; m < sp.inv_len; m += blockDim.x) {
        const float r = __frcp_rn((float)(m + 1));
        const float c = (float)(2 * m + 3);
        tab[m + m / CERT_UNROLL] = make_float4(r, r, c, c);
    }
    for (int m = threadIdx.x; m <= sp.ndir; m += blockDim.x) istart[m] = sp.item_start[m];
    __syncthreads();
    FlagList fl{flist, 0, sp.flag_buf, sp.flag_count, sp.flag_cap, 0, 0.f};
    const long long t_start = clock64();

    for (;;) {
        if (bwd == 0 && lane == 0) reinterpret_cast<int*>(xch)[0] = (int)atomicAdd(sp.counter, 2u);
        pair_sync(pair);
        const int pitem = reinterpret_cast<const int*>(xch)[0];   // items pitem (forward), pitem + 1
        if (pitem >= sp.total_items) break;
        ItemRow it;
        const bool nonempty = decode_item(sp, istart, pitem + bwd, &it);
        fl.item = pitem + bwd;
        if (nonempty) {
            const float zpart = stage_row<true>(sp, it, Fh, Fl, ends, lane, bwd, 2, false);
            if (lane == 0) xch[1 + bwd] = zpart;
            pair_sync(pair);   // the staged row is complete
            if (PRUNE) {   // each warp's own suffix or prefix maxima
                if (bwd) prefix_max(Fh, ZS, it.L, lane);
                else suffix_max(Fh, ZS, it.L, lane);
                __syncwarp();
            }
            const float zmax = fmaxf(xch[1], xch[2]);
            fl.zmax = zmax;
            const DirDev* d = sp.dirs + it.dir;
            ExactCtx xc;
            xc.H = Fh + ROW_PADL;
            xc.Lo = Fl + ROW_PADL;
            xc.L = it.L;
            xc.K = it.K;
            xc.h0h = it.h0;
            xc.h0l = d->h0_lo;
            xc.eta = 0x1p-42f * (zmax + fabsf(it.h0)) + 0x1p-126f;
            xc.cvrow = (bwd ? sp.cv_bwd : sp.cv_fwd) + it.rowbase;
            xc.bwd = bwd != 0;
            xc.from_dem = false;
            xc.rev_staged = false;
            xc.eh0 = ends[0];
            xc.el0 = ends[1];
            xc.ehL = ends[2];
            xc.elL = ends[3];
            xc.dir = d;
            xc.job = sp.jobs + d->job;
            xc.p = it.p;
            xc.jlo = it.jlo;
            xc.half = sp.half;
            xc.zs_len = sp.zs_len;
                xc.tab = tab;
                xc.tskew = CERT_UNROLL;
            xc.tabn = sp.inv_len;
            const float u = 0x1p-24f;
            const float eg0 = 2.01f * u * fabsf(it.h0) + fabsf(d->h0_lo) * 1.0001f + 4.04f * xc.eta;
            if (bwd)
                sweep_row_cert<CERT_POV, CERT_UNROLL, LONG, PRUNE, true, true>(xc, ZS, tab, sp.inv_len, spill, eg0, fl,
                                                                               lane);
            else
                sweep_row_cert<CERT_POV, CERT_UNROLL, LONG, PRUNE, false, true>(xc, ZS, tab, sp.inv_len, spill, eg0, fl,
                                                                                lane);
        }
        pair_sync(pair);   // both walks are done with the row (and with the exchange slot)
    }
    if (lane == 0) atomicAdd(&g_sweep_stats[3], (unsigned long long)(clock64() - t_start));
}

// The exact pass of a certified launch: every walk the sweep flagged and
// handed over (an (item, sample, row |elevation| bound) entry of the flag
// buffer) is walked again exactly (double-float, FP64 past its margin) by one
// warp, which blends the walk's samples from the DEM as the staging does
// (the DEM is L2-resident while the sweep runs).  Warps claim one entry at a
// time; flag_count[0] is the buffer's fill, flag_count[1] the claim counter.
constexpr int EXACT_WARPS = 16;

__global__ void __launch_bounds__(EXACT_WARPS * 32) exact_kernel(SweepParams sp)
{
    const int lane = threadIdx.x & 31;
    const unsigned n = min(sp.flag_count[0], (unsigned)sp.flag_cap);
    const long long t_start = clock64();
    for (;;) {
        unsigned i = 0u;
        if (lane == 0) i = atomicAdd(sp.flag_count + 1, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n) break;
        const int4 en = sp.flag_buf[i];
        if (en.x < 0) continue;                 // a slot of a push that did not fit
        if (!in_range(en.x, sp.total_items, 22)) continue;
        ItemRow it;
        if (!decode_item(sp, sp.item_start, en.x, &it)) continue;
        if (!in_range(en.y, it.L, 23)) continue;
        const DirDev* d = sp.dirs + it.dir;
        ExactCtx xc;
        xc.H = nullptr;
        xc.Lo = nullptr;
        xc.L = it.L;
        xc.K = it.K;
        xc.h0h = it.h0;
        xc.h0l = d->h0_lo;
        xc.eta = 0x1p-42f * (__int_as_float(en.z) + fabsf(it.h0)) + 0x1p-126f;
        xc.cvrow = (it.rev ? sp.cv_bwd : sp.cv_fwd) + it.rowbase;
        xc.bwd = it.rev;
        xc.from_dem = true;
        xc.rev_staged = false;
        xc.eh0 = xc.el0 = xc.ehL = xc.elL = 0.f;
        xc.dir = d;
        xc.job = sp.jobs + d->job;
        xc.p = it.p;
        xc.jlo = it.jlo;
        xc.half = sp.half;
        xc.zs_len = 0;
        xc.tab = nullptr;
        xc.tabn = 0;     // 1/d by __frcp_rn
        xc.tskew = 1;
        exact_walk(xc, en.y, lane);
    }
    if (lane == 0) atomicAdd(&g_sweep_stats[2], (unsigned long long)(clock64() - t_start));
}

}  // namespace

// A long-walk launch keeps at least this many warps per CTA, shrinking the
// distance table (to no fewer than MIN_TABLE entries) when both do not fit.
constexpr int LONG_MIN_WARPS = 2;
constexpr int MIN_TABLE = 1024;

// Certified one-row-per-warp sweep warps that shared memory holds for rows
// of up to wmax samples and walks of up to dmax steps in a launch of ndir
// directions (launch_sweep runs that kernel when the count reaches
// TVS_CERT_SINGLE_MIN).
static size_t cert_single_fit(int wmax, int dmax, int prune, int ndir, int smem_optin)
{
    const int inv_len = (std::min(dmax, wmax) + 2 * LARGE_UNROLL + 8 + 1) & ~1;
    const int tab_slots = tab_slots_for(inv_len, true);
    const int istart_len = (ndir + 1 + 3) & ~3;
    const int half = (ROW_PADL + 4 + wmax + ROW_PADR + 3) & ~3;
    const int zs_len = prune ? ((wmax + ZS_STRIDE - 1) / ZS_STRIDE + 4) & ~3 : 0;
    const int single_warp = 2 * half + zs_len + FLAG_CAP + 4;
    const size_t fixed = (size_t)(4 * tab_slots + istart_len) * 4;
    return fixed >= (size_t)smem_optin ? 0 : ((size_t)smem_optin - fixed) / ((size_t)single_warp * 4);
}

int cert_sweep_class(int wmax, int dmax, int prune, int ndir, int smem_optin)
{
    if (wmax - 2 > LONG_WALK && dmax - 1 > LONG_WALK) return 0;
    const size_t fit = cert_single_fit(wmax, dmax, prune, ndir, smem_optin);
    return fit >= (size_t)CERT_WIDE_WARPS ? CERT_WIDE_WARPS : fit >= (size_t)TVS_CERT_SINGLE_MIN ? CERT_MAX_WARPS : 0;
}

cudaError_t launch_sweep(const DirDev* d_dirs, const JobDev* d_jobs, const int* d_item_start, int ndir,
                         int total_items, const int* rowlo, const int* rowhi, int* cv_fwd, int* cv_bwd, int wmax,
                         int dmax, int prune, int cert, unsigned* counter, int4* flag_buf, unsigned* flag_count,
                         int flag_cap, int num_sms, int smem_optin, int max_warps, cudaStream_t stream)
{
    if (ndir <= 0 || total_items <= 0) return cudaSuccess;
    constexpr int U = LARGE_UNROLL;
    SweepParams sp;
    sp.dirs = d_dirs; sp.jobs = d_jobs; sp.item_start = d_item_start; sp.rowlo = rowlo;
    sp.rowhi = rowhi; sp.cv_fwd = cv_fwd; sp.cv_bwd = cv_bwd; sp.counter = counter; sp.ndir = ndir;
    sp.total_items = total_items;
    const bool pass = cert && flag_buf && flag_count && flag_cap > 0;   // flagged walks in a second kernel
    sp.flag_buf = pass ? flag_buf : nullptr;
    sp.flag_count = pass ? flag_count : nullptr;
    sp.flag_cap = pass ? flag_cap : 0;
    // the distance table is read up to d = dmax + U (a walk of at most
    // min(K, W) - 1 steps, rounded up to U); dmax <= wmax
    sp.inv_len = (std::min(dmax, wmax) + 2 * U + 8 + 1) & ~1;
    sp.tab_slots = tab_slots_for(sp.inv_len, cert != 0);
    sp.istart_len = (ndir + 1 + 3) & ~3;
    sp.half = (ROW_PADL + 4 + wmax + ROW_PADR + 3) & ~3;
    const bool longw = wmax - 2 > LONG_WALK && dmax - 1 > LONG_WALK;
    sp.zs_len = prune ? ((wmax + ZS_STRIDE - 1) / ZS_STRIDE + 4) & ~3 : 0;
    sp.fl_cap = cert ? FLAG_CAP : 0;
    const int lspill = longw ? 32 * LARGE_POV : 0;
    // FP32 decisions: one row per warp.  Certified: one row per warp
    // (reversed for backward walks) when TVS_CERT_SINGLE_MIN such warps fit, else
    // one row per pair of warps (both staged arrays, suffix and prefix maxima,
    // the end samples and an exchange slot), and per warp its
    // flag list and spill: a row's samples are then held once for both walk
    // directions.
    const int single_warp = 2 * sp.half + sp.zs_len + sp.fl_cap + 4;
    const size_t single_fit = cert ? cert_single_fit(wmax, dmax, prune, ndir, smem_optin) : 0;
    const int single_min = TVS_CERT_SINGLE_MIN;
    const bool single = cert && !longw && (max_warps == 0 || max_warps >= single_min) &&
                        single_fit >= (size_t)single_min;
    const bool pairs = cert && !single;
    sp.per_pair = pairs ? 2 * sp.half + 2 * sp.zs_len + 8 : 0;
    sp.per_warp = single ? single_warp : pairs ? sp.fl_cap + lspill : sp.half + sp.zs_len + lspill;
    // shared memory of one unit: a pair of warps or one warp
    const int uw = pairs ? 2 : 1;
    const size_t unit = (size_t)(sp.per_pair + uw * sp.per_warp) * 4;
    size_t fixed = (size_t)(4 * sp.tab_slots + sp.istart_len) * 4;
    if (longw && fixed + (size_t)(LONG_MIN_WARPS / uw) * unit > (size_t)smem_optin) {
        // Rows of more than about 10^4 samples: the whole table and several
        // staged rows do not fit together.  Keep LONG_MIN_WARPS warps (or as
        // many as fit) and a table of what is left (at least MIN_TABLE
        // entries); the long-walk sweep computes the entries past its end.
        const size_t base = (size_t)sp.istart_len * 4;
        int w = LONG_MIN_WARPS / uw;
        const size_t min_tab = (size_t)tab_slots_for(MIN_TABLE, cert != 0) * 16;
        while (w > 1 && base + min_tab + (size_t)w * unit > (size_t)smem_optin) --w;
        if (base + 16 * 4 + (size_t)w * unit >= (size_t)smem_optin) return cudaErrorInvalidConfiguration;
        // slots that fit, and the most entries whose slots do
        const size_t room = ((size_t)smem_optin - base - (size_t)w * unit) / 16;
        const size_t fit = cert ? (room - 2) * TAB_SKEW_MIN / (TAB_SKEW_MIN + 1) : room;
        sp.inv_len = (int)std::min<size_t>((size_t)sp.inv_len, fit) & ~1;
        sp.tab_slots = tab_slots_for(sp.inv_len, cert != 0);
        fixed = (size_t)(4 * sp.tab_slots + sp.istart_len) * 4;
    }
    if (fixed + unit > (size_t)smem_optin) return cudaErrorInvalidConfiguration;
    // As many resident units as shared memory and registers allow, in one CTA
    // per SM (the 1/d table is shared by the CTA).
    const size_t fit = (smem_optin - fixed) / unit;
    constexpr int CW = CERT_MAX_WARPS, WW = CERT_WIDE_WARPS, FW = SWEEP_MAX_WARPS;
    void (*kern)(SweepParams);
    int most;
    if (single) {
        const bool wide = single_fit >= (size_t)WW && (max_warps == 0 || max_warps >= WW);
        most = wide ? WW : CW;
        if (wide) kern = prune ? sweep_cert_kernel<true, false, WW> : sweep_cert_kernel<false, false, WW>;
        else kern = prune ? sweep_cert_kernel<true, false, CW> : sweep_cert_kernel<false, false, CW>;
    } else if (pairs) {
        // pruned walks are short and restart groups often: the 12-warp
        // instantiation (no spills) beats 16 warps there (2000^2: 210.9
        // against 218.4 ms), while unpruned walks favour 16 (351 against 365)
        const bool wide = !longw && !prune && fit * 2 >= (size_t)WW && (max_warps == 0 || max_warps >= WW);
        most = wide ? WW : CW;
        if (wide) kern = sweep_pair_kernel<false, false, WW>;
        else kern = prune ? (longw ? sweep_pair_kernel<true, true, CW> : sweep_pair_kernel<true, false, CW>)
                          : (longw ? sweep_pair_kernel<false, true, CW> : sweep_pair_kernel<false, false, CW>);
    } else {
        most = FW;
        kern = prune ? (longw ? sweep_kernel<true, true, FW> : sweep_kernel<true, false, FW>)
                     : (longw ? sweep_kernel<false, true, FW> : sweep_kernel<false, false, FW>);
    }
    const int cap = max_warps > 0 ? std::max(std::min(max_warps, most), uw) : most;
    const int units = (int)std::min<size_t>(fit, (size_t)(cap / uw));
    const int warps = units * uw;
    const size_t smem = fixed + (size_t)units * unit;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (pass) {
        err = cudaMemsetAsync(flag_count, 0, 2 * sizeof(unsigned), stream);
        if (err != cudaSuccess) return err;
    }
    kern<<<per_sm * num_sms, warps * 32, smem, stream>>>(sp);
    err = cudaGetLastError();
    if (err != cudaSuccess || !pass) return err;
    // the exact pass: no shared memory, as many warps as registers allow
    int xper = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&xper, exact_kernel, EXACT_WARPS * 32, 0);
    if (err != cudaSuccess) return err;
    if (xper < 1) return cudaErrorInvalidConfiguration;
    exact_kernel<<<xper * num_sms, EXACT_WARPS * 32, 0, stream>>>(sp);
    return cudaGetLastError();
}

}  // namespace tvs

extern "C" int tvs_debug_sweep_stats(uint64_t* out, int clear)
{
    if (!out) return TVS_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, tvs::g_sweep_stats, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess && clear) {
        const unsigned long long zero[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(tvs::g_sweep_stats, zero, sizeof(zero));
    }
    return e == cudaSuccess ? TVS_OK : TVS_ERR_CUDA;
}

extern "C" int tvs_debug_sweep_check(int32_t* out, int clear)
{
    if (!out) return TVS_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, tvs::g_sweep_check, sizeof(int) * 4);
    if (e == cudaSuccess && clear) {
        const int zero[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(tvs::g_sweep_check, zero, sizeof(zero));
    }
    return e == cudaSuccess ? TVS_OK : TVS_ERR_CUDA;
}
