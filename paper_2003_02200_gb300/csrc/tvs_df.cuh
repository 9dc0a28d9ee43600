// tvs_df.cuh -- double-float arithmetic shared by the certified walks of the
// sweep (tvs_sweep.cu) and of the point viewsheds (tvs_points.cu): sample
// heights of Alg. 6 as hi + lo single-precision pairs and slopes against a
// double-float observer.
#pragma once

#include <cuda_runtime.h>

namespace tvs {
namespace df {

// Error-free transformations in round-to-nearest single precision.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a + b = s + e exactly when a == 0 or exponent(a) >= exponent(b).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ bool df_gt(float ah, float al, float bh, float bl)
{
    return ah > bh || (ah == bh && al > bl);
}

// Height of the sample blending va (row a) and vb (row a + 1) with weights
// 1 - r and r, r = fr * 2^-32 (Alg. 6), as hi + lo: the difference vb - va
// and r are split exactly (TwoSum; r into its top 24 and low 8 bits), the main
// product exactly (FMA), the rest rounds at about 2^-46 of max(|va|, |vb|):
// |hi + lo - exact| <= 2^-43 max(|va|, |vb|), |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void df_blend(float va, float vb, unsigned fr, float& zh, float& zl)
{
    if (fr == 0u) { zh = va; zl = 0.f; return; }
    float dh, dl;
    two_sum(vb, -va, dh, dl);
    const float rh = __fmul_rn(__uint2float_rn(fr & 0xFFFFFF00u), 0x1p-32f);
    const float rl = __fmul_rn(__uint2float_rn(fr & 0xFFu), 0x1p-32f);
    const float ph = __fmul_rn(rh, dh);
    const float pe = __fmaf_rn(rh, dh, -ph);
    const float t = __fmaf_rn(rh, dl, __fmaf_rn(rl, dh, __fmul_rn(rl, dl)));
    float sh, se;
    two_sum(va, ph, sh, se);
    const float lo = __fadd_rn(se, __fadd_rn(pe, t));
    two_sum(sh, lo, zh, zl);
}

// Double-float slope (z - h) / d of a staged target against the observer h,
// given iv = fl(1/d) (correctly rounded, as __frcp_rn returns it).
__device__ __forceinline__ void df_slope_iv(float zh, float zl, float hh, float hl, int d, float iv, float& qh,
                                            float& ql)
{
    float s, e;
    two_sum(zh, -hh, s, e);
    e = __fadd_rn(e, __fsub_rn(zl, hl));
    float Dh, Dl;
    two_sum(s, e, Dh, Dl);
    const float fd = (float)d;
    const float q1 = __fmul_rn(Dh, iv);
    const float ph = __fmul_rn(q1, fd);
    const float pl = __fmaf_rn(q1, fd, -ph);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(Dh, ph), pl), Dl);
    fast_two_sum(q1, __fmul_rn(r, iv), qh, ql);
}

__device__ __forceinline__ void df_slope(float zh, float zl, float hh, float hl, int d, float& qh, float& ql)
{
    df_slope_iv(zh, zl, hh, hl, d, __frcp_rn((float)d), qh, ql);
}

}  // namespace df
}  // namespace tvs
