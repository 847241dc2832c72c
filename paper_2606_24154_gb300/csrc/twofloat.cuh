// twofloat.cuh -- two-float ("double-float") arithmetic on the FP32 pipe, shared by the
// mixed-precision fill (fill_mixed.cu) and the refined point evaluation (eval_acc.cu).
// Every quantity is an unevaluated sum hi + lo of two floats; sums and products keep
// their rounding errors through error-free transformations (Knuth TwoSum, FMA-based
// TwoProd), about 44 significant bits.
#pragma once
#include "eval_blocks.cuh"

namespace nb {

// All operations are the explicitly rounded intrinsics, so no contraction or reordering
// can change the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (ah + al) - (bh + bl), unnormalised
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& h, float& l) {
    float t;
    two_sum(ah, -bh, h, t);
    l = __fadd_rn(t, __fsub_rn(al, bl));
}

// a . b for three-vectors of two-float components
__device__ __forceinline__ void df_dot3(const float (&ah)[3], const float (&al)[3], const float4& bh, const float4& bl,
                                        float& h, float& l) {
    float p0, e0, p1, e1, p2, e2, t1, t2, s;
    two_prod(ah[0], bh.x, p0, e0);
    two_prod(ah[1], bh.y, p1, e1);
    two_prod(ah[2], bh.z, p2, e2);
    two_sum(p0, p1, s, t1);
    two_sum(s, p2, h, t2);
    float lo = __fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, __fadd_rn(t1, t2)));
    lo = __fmaf_rn(ah[0], bl.x, lo);
    lo = __fmaf_rn(al[0], bh.x, lo);
    lo = __fmaf_rn(ah[1], bl.y, lo);
    lo = __fmaf_rn(al[1], bh.y, lo);
    lo = __fmaf_rn(ah[2], bl.z, lo);
    lo = __fmaf_rn(al[2], bh.z, lo);
    l = lo;
}

// squared norm of (X, Y, Z), two-float components
__device__ __forceinline__ void df_norm2(float xh, float xl, float yh, float yl, float zh, float zl, float& h,
                                         float& l) {
    float px, ex, py, ey, pz, ez, s, t1, t2;
    two_prod(xh, xh, px, ex);
    two_prod(yh, yh, py, ey);
    two_prod(zh, zh, pz, ez);
    ex = __fmaf_rn(__fadd_rn(xh, xh), xl, ex);
    ey = __fmaf_rn(__fadd_rn(yh, yh), yl, ey);
    ez = __fmaf_rn(__fadd_rn(zh, zh), zl, ez);
    two_sum(px, py, s, t1);
    two_sum(s, pz, h, t2);
    l = __fadd_rn(__fadd_rn(ex, ey), __fadd_rn(ez, __fadd_rn(t1, t2)));
}

// ---------------------------------------------------------------- packed two-float nodes
// Two Gauss nodes per instruction in the packed FP32x2 forms (__fadd2_rn, __fmul2_rn,
// __ffma2_rn; a - b as fma(b, -1, a), exact like a subtraction).  Error terms of products
// come out negated, e_neg = fma(-a, b, a b) = -(a b - fl(a b)), so that no extra negation is
// needed; the running sum keeps its low part negated as well (NL = -lo).
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& t) {
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    t = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// Per-image quantities of one pair in the column element's frame, broadcast to both lanes
// (negated copies for the error terms of products).
struct PairDF2 {
    float2 xh, nxh, xl, zh, nzh, zl;  // X, Z
    float2 d2h, d2l;                  // |D|^2
};
struct NormDF2 {
    float2 nxh, nnxh, nxl, nzh, nnzh, nzl;  // local components of the row normal (x, z)
    float2 ndh, ndl;                        // n_i . D
};

// r^2 = |D|^2 + 2 (X s_x + Z s_z) + |s|^2 and 1/r for a node pair: y0 (MUFU estimate), the
// Newton correction negated (nyl = -yl), y0^2 = a exactly with its negated error nae.
__device__ __forceinline__ void node_rinv2(const PairDF2& P, const float4& q0, const float4& q1, const float4& q2,
                                           const float4& q3, float2& y0, float2& ny0, float2& nyl, float2& a,
                                           float2& na, float2& nae) {
    const float2 m1 = bc2(-1.f);
    const float2 sx = make_float2(q0.x, q0.y), sz = make_float2(q0.z, q0.w);
    const float2 s2 = make_float2(q1.x, q1.y);
    const float2 sxl = make_float2(q2.x, q2.y), szl = make_float2(q2.z, q2.w);
    const float2 s2l = make_float2(q3.x, q3.y);
    const float2 p1 = __fmul2_rn(P.xh, sx), ne1 = __ffma2_rn(P.nxh, sx, p1);
    const float2 p2 = __fmul2_rn(P.zh, sz), ne2 = __ffma2_rn(P.nzh, sz, p2);
    float2 qh, t, t2;
    two_sum2(p1, p2, qh, t);
    float2 lo = __ffma2_rn(ne1, m1, t);
    lo = __ffma2_rn(ne2, m1, lo);
    lo = __ffma2_rn(P.xh, sxl, lo);
    lo = __ffma2_rn(P.xl, sx, lo);
    lo = __ffma2_rn(P.zh, szl, lo);
    lo = __ffma2_rn(P.zl, sz, lo);
    two_sum2(qh, s2, qh, t2);
    lo = __fadd2_rn(lo, __fadd2_rn(t2, s2l));
    // |D|^2 >= |q| for d >= kFillRatioC rho (|q| <= 2 d rho + rho^2)
    const float2 r2h = __fadd2_rn(P.d2h, qh);
    const float2 t3 = sub2(qh, sub2(r2h, P.d2h));
    const float2 r2l = __fadd2_rn(P.d2l, __fadd2_rn(lo, t3));
    y0 = make_float2(rsqrtf(r2h.x), rsqrtf(r2h.y));
    ny0 = __fmul2_rn(y0, m1);
    a = __fmul2_rn(y0, y0);
    nae = __ffma2_rn(ny0, y0, a);  // a - y0^2
    na = __fmul2_rn(ny0, y0);
    const float2 b = __fmul2_rn(r2h, a);
    const float2 nbe = __ffma2_rn(r2h, na, b);  // b - r2h a
    // h = 1 - r^2 y0^2 (1 - b is exact: b within 2^-20 of 1)
    float2 h = __ffma2_rn(b, m1, bc2(1.f));
    h = __fadd2_rn(h, nbe);
    h = __ffma2_rn(r2h, nae, h);
    h = __ffma2_rn(r2l, na, h);
    nyl = __fmul2_rn(__fmul2_rn(bc2(-0.5f), y0), h);
}

}  // namespace nb
