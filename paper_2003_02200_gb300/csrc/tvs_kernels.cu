// tvs_kernels.cu -- sm_103a kernels of the sDEM total viewshed.
//
//   rowmap : usable column range [jlo, jhi] of every skewed row (section 4.1
//            step 1(b): the limits of the skewed structure).
//   skew   : DEM -> skewed layout, one writer per sample (Kernel-1, Alg. 6,
//            written as a gather instead of the paper's two-way scatter).
//   sweep  : every usable sample of every skewed row walks its row forward and
//            backward (Kernel-2, Alg. 7 and 8); the hot loop, with exact
//            horizon pruning as an option.
//   unskew : blends the per-sample measures back onto DEM cells and sums the
//            directions (Kernel-3, Alg. 9), with the Pappus / step^2 scale of
//            Alg. 1 applied once at the end.
#include "tvs_internal.h"

#include <cuda_runtime.h>

#include <algorithm>

namespace tvs {

namespace {

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

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

// ------------------------------------------------------------------ skew --
// CTA = one SKEW_TP x SKEW_TJ tile of one direction's skewed slab.  The view
// rows the tile blends (at most SKEW_TP + SKEW_TJ + 1 of them) are staged in
// shared memory: for the identity / row-mirrored views they are DEM row
// segments (coalesced along the row), for the transposed views DEM column
// segments are read along DEM rows (coalesced) and transposed on the way into
// shared memory (row pitch SKEW_TJ + 1: no bank conflicts either way).
constexpr int SKEW_ROWS = SKEW_TP + SKEW_TJ + 3;
constexpr int SKEW_TILES_PER_CTA = 8;   // tiles of one direction per CTA, at most
constexpr int SKEW_PITCH = SKEW_TJ + 1;

__global__ void __launch_bounds__(256) skew_kernel(const JobDev* __restrict__ jobs,
                                                   const DirDev* __restrict__ dirs,
                                                   float* __restrict__ sdem)
{
    __shared__ float S[SKEW_ROWS * SKEW_PITCH];
    const DirDev d = dirs[blockIdx.y];
    const float* __restrict__ dem = jobs[d.job].dem;
    const int cols = jobs[d.job].cols;
    const int tiles_j = (d.W + SKEW_TJ - 1) / SKEW_TJ;
    const int tiles_p = (d.R + SKEW_TP - 1) / SKEW_TP;
    // the CTAs of a direction stride over its tiles (directions differ in
    // tile count; a grid sized for the largest would launch idle CTAs)
    for (int tile = blockIdx.x; tile < tiles_j * tiles_p; tile += gridDim.x) {
        const int pt = tile / tiles_j, jt = tile - pt * tiles_j;
        const int p0 = pt * SKEW_TP, j0 = jt * SKEW_TJ;
        const int p1 = min(p0 + SKEW_TP, d.R) - 1;
        const int j1 = min(j0 + SKEW_TJ, d.W) - 1;
        const int nj = j1 - j0 + 1;
        int amin = p0 - d.D + dest_of(d.t_fx, j0);
        int amax = p1 - d.D + dest_of(d.t_fx, j1) + 1;
        amin = max(amin, 0);
        amax = min(amax, d.H - 1);
        if (amin > amax) continue;        // uniform over the CTA
        const int na = amax - amin + 1;
        __syncthreads();                  // the previous tile's blends are done with S
        if (d.frame == 0 || d.frame == 3) {
            const bool vec = ((cols & 3) == 0) && nj == SKEW_TJ;
            if (vec) {
                // 8 lanes x 16 B per 128 B row segment, 4 row segments per warp instruction
                for (int idx = threadIdx.x; idx < na * (SKEW_TJ / 4); idx += blockDim.x) {
                    const int r = idx / (SKEW_TJ / 4), c4 = (idx - r * (SKEW_TJ / 4)) * 4;
                    const int a = amin + r;
                    const int drow = d.frame == 0 ? a : d.H - 1 - a;
                    const float4 v = *reinterpret_cast<const float4*>(dem + (long long)drow * cols + j0 + c4);
                    float* s = S + r * SKEW_PITCH + c4;
                    s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
                }
            } else {
                for (int idx = threadIdx.x; idx < na * SKEW_TJ; idx += blockDim.x) {
                    const int r = idx / SKEW_TJ, c = idx - r * SKEW_TJ;
                    const int a = amin + r;
                    const int drow = d.frame == 0 ? a : d.H - 1 - a;
                    if (c < nj) S[r * SKEW_PITCH + c] = dem[(long long)drow * cols + j0 + c];
                }
            }
        } else {
            // warp w stages view columns w, w + 8, ... (DEM rows), its lanes
            // consecutive view rows (DEM columns): coalesced reads, conflict-free
            // transposed stores (pitch 33)
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
            for (int c = warp; c < nj; c += nwarps) {
                const int j = j0 + c;
                const int drow = d.frame == 1 ? j : d.W - 1 - j;
                const float* src = dem + (long long)drow * cols + amin;
                for (int r = lane; r < na; r += 32) S[r * SKEW_PITCH + c] = src[r];
            }
        }
        __syncthreads();

        const int c = threadIdx.x % SKEW_TJ;
        const int j = j0 + c;
        if (j > j1) continue;
        const unsigned long long y = (unsigned long long)j * d.t_fx;
        const int dest = (int)(y >> 32);
        const unsigned fr = (unsigned)(y & 0xFFFFFFFFull);
        // Blend weights of Alg. 6 in single precision: r = frac * 2^-32.
        const float r = __fmul_rn(__uint2float_rn(fr), 0x1p-32f);
        const float wa = __fsub_rn(1.0f, r);
        float* out = sdem + d.slab + j;
        for (int pp = threadIdx.x / SKEW_TJ; pp < SKEW_TP; pp += blockDim.x / SKEW_TJ) {
            const int p = p0 + pp;
            if (p > p1) break;
            const int a = p - d.D + dest;
            const bool ok = a >= 0 && (fr == 0u ? a <= d.H - 1 : a + 1 <= d.H - 1);
            if (!ok) continue;
            const float va = S[(a - amin) * SKEW_PITCH + c];
            float z = va;
            if (fr != 0u) {
                const float vb = S[(a + 1 - amin) * SKEW_PITCH + c];
                z = __fadd_rn(__fmul_rn(wa, va), __fmul_rn(r, vb));
            }
            out[(long long)p * d.Wp] = z;
        }
    }
}

// ----------------------------------------------------------------- sweep --
struct SweepParams {
    const DirDev* dirs;
    const int* item_start;
    const float* sdem;
    const int* rowlo;
    const int* rowhi;
    int* cv_fwd;       // forward measure of every sample (slab layout)
    int* cv_bwd;       // backward measure of every sample (slab layout)
    unsigned* counter;
    int ndir;
    int total_items;
    int inv_len;     // entries of the per-distance table (float4 each)
    int istart_len;  // ints of the item-start table (multiple of 4)
    int half;        // floats of one staged row (multiple of 4)
    int zs_len;      // floats of the row's suffix maxima (0 without pruning)
    int per_warp;    // floats of a warp's shared area: staged row, suffix maxima, (long rows) 32 x LARGE_POV ints
};

__device__ __forceinline__ float fset_gt(float a, float b)
{
    // 1.0f if a > b (strict; false for NaN), else 0.0f
    float v;
    asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(v) : "f"(a), "f"(b));
    return v;
}

// U steps of one lane's P POVs.  POV q at step u (distance d = e + 1 + u)
// sees target w[q + u + 1]; its slope is (target - h_q) * (1/d) in single
// precision, it is visible iff that slope is strictly above the running
// maximum M_q, and a visible target adds 2d + 1 to the POV's measure.  Two
// POVs share one packed multiply and one packed accumulate; the comparison and
// the maximum are scalar.  tab[e + u] holds (1/d, 1/d, 2d + 1, 2d + 1); a
// range-limited walk's last block counts only its first `nvalid` steps.
// Distance entry (1/d, 1/d, 2d + 1, 2d + 1) as the table holds it.
__device__ __forceinline__ float4 dist_entry(int d)
{
    const float r = __frcp_rn((float)d);
    const float c = (float)(2 * d + 1);
    return make_float4(r, r, c, c);
}

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
constexpr int FLUSH_STEPS = 336;   // a multiple of SMALL_UNROLL and LARGE_UNROLL
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
        if (x % ZS_STRIDE == 0) ZS[x / ZS_STRIDE] = run;
    }
}

// A sweep work item: (direction, skewed row, walk direction).
struct ItemRow {
    long long rowbase;   // slab offset of the row's first usable sample
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
    it->L = jhi - jlo + 1;
    it->K = d.K;
    it->h0 = d.h0;
    it->pov = row_pov(it->L, d.K, d.pov, d.p4_pct);
    it->rowbase = d.slab + (long long)p * d.Wp + jlo;
    return it->L > 0;
}

// L2 prefetch of the n floats at p with one bulk request: start rounded down
// and end rounded up to 16 bytes, which stays inside the row's slab (rows
// start 16-byte aligned and are padded to a multiple of 4 floats).
__device__ __forceinline__ void prefetch_row_l2(const float* p, int n)
{
    const unsigned long long a = reinterpret_cast<unsigned long long>(p) & ~15ull;
    const unsigned long long end = (reinterpret_cast<unsigned long long>(p + n) + 15ull) & ~15ull;
    const unsigned size = (unsigned)(end - a);
    if (size == 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a), "r"(size) : "memory");
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

// PRUNE: exact horizon pruning; LONG: the launch holds rows with walks of
// more than LONG_WALK steps (every row then takes the flushing walk).
template <bool PRUNE, bool LONG>
__global__ void __launch_bounds__(SWEEP_MAX_WARPS * 32, 1) sweep_kernel(SweepParams sp)
{
    extern __shared__ __align__(16) float smem[];
    float4* tab = reinterpret_cast<float4*>(smem);
    int* istart = reinterpret_cast<int*>(smem + 4 * sp.inv_len);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* F = smem + 4 * sp.inv_len + sp.istart_len + warp * sp.per_warp;
    float* ZS = F + sp.half;
    int* spill = reinterpret_cast<int*>(ZS + sp.zs_len) + lane;
    // per distance d = m + 1: (1/d, 1/d, 2d + 1, 2d + 1); 1/d correctly rounded
    for (int m = threadIdx.x; m < sp.inv_len; m += blockDim.x) {
        const float r = __frcp_rn((float)(m + 1));
        const float c = (float)(2 * m + 3);
        tab[m] = make_float4(r, r, c, c);
    }
    for (int m = threadIdx.x; m <= sp.ndir; m += blockDim.x) istart[m] = sp.item_start[m];
    __syncthreads();
    const float NEG = neg_inf();

    // Lane 0 claims the next item while the warp works on the current one and
    // prefetches that item's skewed row into L2 (the slabs do not fit L2, so
    // otherwise every row is staged from HBM at the start of its item).
    int next = 0;
    if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    for (;;) {
        const int item = next;
        if (item >= sp.total_items) break;
        ItemRow it;
        if (!decode_item(sp, istart, item, &it)) {
            if (lane == 0) next = (int)atomicAdd(sp.counter, 1u);
            next = __shfl_sync(0xffffffffu, next, 0);
            continue;
        }
        const float* zrow = sp.sdem + it.rowbase;
        const int L = it.L;
        __syncwarp();
        // stage the row (or the reversed row): batches of loads, then stores
        constexpr int B = 8;
        for (int x0 = lane; x0 < L; x0 += 32 * B) {
            float v[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int x = x0 + 32 * b;
                v[b] = x < L ? (it.rev ? zrow[L - 1 - x] : zrow[x]) : 0.f;
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int x = x0 + 32 * b;
                if (x < L) F[ROW_PADL + x] = (x == L - 1) ? NEG : v[b];
            }
        }
        for (int m = lane; m < ROW_PADR; m += 32) F[ROW_PADL + L + m] = NEG;
        if (lane == 0) {
            next = (int)atomicAdd(sp.counter, 1u);
            ItemRow nx;
            if (next < sp.total_items && decode_item(sp, istart, next, &nx))
                prefetch_row_l2(sp.sdem + nx.rowbase, nx.L);
        }
        next = __shfl_sync(0xffffffffu, next, 0);
        __syncwarp();   // the staged row is visible to every lane
        if (PRUNE) {
            suffix_max(F, ZS, L, lane);
            __syncwarp();
        }
        int* cvrow = (it.rev ? sp.cv_bwd : sp.cv_fwd) + it.rowbase;
        sweep_item<LONG, PRUNE>(it, F, ZS, tab, sp.inv_len, cvrow, spill, lane);
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

cudaError_t launch_skew(const JobDev* d_jobs, const DirDev* d_dirs, int ndir, int max_tiles, float* sdem,
                        cudaStream_t stream)
{
    if (ndir <= 0 || max_tiles <= 0) return cudaSuccess;
    dim3 grid((max_tiles + SKEW_TILES_PER_CTA - 1) / SKEW_TILES_PER_CTA, ndir);
    skew_kernel<<<grid, 256, 0, stream>>>(d_jobs, d_dirs, sdem);
    return cudaGetLastError();
}

// A long-walk launch keeps at least this many warps per CTA, shrinking the
// distance table (to no fewer than MIN_TABLE entries) when both do not fit.
constexpr int LONG_MIN_WARPS = 2;
constexpr int MIN_TABLE = 1024;

cudaError_t launch_sweep(const DirDev* d_dirs, const int* d_item_start, int ndir, int total_items,
                         const float* sdem, const int* rowlo, const int* rowhi, int* cv_fwd, int* cv_bwd,
                         int wmax, int dmax, int prune, unsigned* counter, int num_sms, int smem_optin,
                         int max_warps, cudaStream_t stream)
{
    if (ndir <= 0 || total_items <= 0) return cudaSuccess;
    constexpr int U = LARGE_UNROLL;
    SweepParams sp;
    sp.dirs = d_dirs; sp.item_start = d_item_start; sp.sdem = sdem; sp.rowlo = rowlo;
    sp.rowhi = rowhi; sp.cv_fwd = cv_fwd; sp.cv_bwd = cv_bwd; sp.counter = counter; sp.ndir = ndir;
    sp.total_items = total_items;
    // the distance table is read up to d = dmax + U (a walk of at most
    // min(K, W) - 1 steps, rounded up to U); dmax <= wmax
    sp.inv_len = (std::min(dmax, wmax) + 2 * U + 8 + 1) & ~1;
    sp.istart_len = (ndir + 1 + 3) & ~3;
    sp.half = (ROW_PADL + 4 + wmax + ROW_PADR + 3) & ~3;
    const bool longw = wmax - 2 > LONG_WALK && dmax - 1 > LONG_WALK;
    sp.zs_len = prune ? ((wmax + ZS_STRIDE - 1) / ZS_STRIDE + 4) & ~3 : 0;
    sp.per_warp = sp.half + sp.zs_len + (longw ? 32 * LARGE_POV : 0);
    void (*kern)(SweepParams) = prune ? (longw ? sweep_kernel<true, true> : sweep_kernel<true, false>)
                                      : (longw ? sweep_kernel<false, true> : sweep_kernel<false, false>);
    const size_t per_warp = (size_t)sp.per_warp * 4;
    size_t fixed = (size_t)(4 * sp.inv_len + sp.istart_len) * 4;
    if (longw && fixed + (size_t)LONG_MIN_WARPS * per_warp > (size_t)smem_optin) {
        // Rows of more than about 10^4 samples: the whole table and several
        // staged rows do not fit together.  Keep LONG_MIN_WARPS warps (or as
        // many as fit) and a table of what is left (at least MIN_TABLE
        // entries); the long-walk sweep computes the entries past its end.
        const size_t base = (size_t)sp.istart_len * 4;
        int w = LONG_MIN_WARPS;
        while (w > 1 && base + (size_t)MIN_TABLE * 16 + (size_t)w * per_warp > (size_t)smem_optin) --w;
        if (base + (size_t)w * per_warp >= (size_t)smem_optin) return cudaErrorInvalidConfiguration;
        const size_t room = ((size_t)smem_optin - base - (size_t)w * per_warp) / 16;
        sp.inv_len = (int)std::min<size_t>((size_t)sp.inv_len, room) & ~1;
        fixed = (size_t)(4 * sp.inv_len + sp.istart_len) * 4;
    }
    if (fixed + per_warp > (size_t)smem_optin) return cudaErrorInvalidConfiguration;
    // As many resident warps as shared memory and registers allow, in one CTA per SM
    // (each warp stages its own row; the 1/d table is shared by the CTA).
    const int cap = max_warps > 0 ? std::min(max_warps, SWEEP_MAX_WARPS) : SWEEP_MAX_WARPS;
    int warps = (int)std::min<size_t>((smem_optin - fixed) / per_warp, (size_t)cap);
    const size_t smem = fixed + (size_t)warps * per_warp;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<per_sm * num_sms, warps * 32, smem, stream>>>(sp);
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
