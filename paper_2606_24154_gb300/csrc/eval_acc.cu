// eval_acc.cu -- refinement of the mixed-precision evaluation (Eq. Potential / Eq. Field
// over elements and periodic images): per-point error estimates of the FP32 pass, and a
// two-float re-evaluation of the points whose estimate exceeds the requested tolerance.
//
// Error estimate.  The FP32 pass (eval_blocks.cuh) leaves per point the scales of its FP32
// pairs' errors, built from the per-element terms b_j = |sigma_j| |sum_k Phi'_jk| (for E:
// |sigma_j| |sum_k E'_jk|_1): B = ke sum_j b_j and S = ke sqrt(sum_j b_j^2).  Its error
// comes from rounding the point-to-centroid difference and the node arithmetic to FP32
// (about u = 2^-24 relative per operation) and from the truncation of the Gauss rules.
// These do not shrink with the result, so a point whose |phi| (|E|) is small next to B --
// a potential near zero inside the plate, the weak field in the drift gap -- loses its
// relative accuracy there.  The estimate for x = phi and x = |E| is
//   gamma_r |x| + gamma_b B + gamma_s S,   gamma_r = 1e-7, gamma_b = 7e-8, gamma_s = 5e-7.
// Calibration: against the FP64 path on 133,000 points (the THGEM cell with solved and
// with structured densities, points in the gas, through the plate and 1-2 um off the Cu
// faces; the cube with solved densities on its grid and at random points; a reduced THGEM
// cell), the largest error ratios were 3.3e-8 B (phi) and 5.5e-8 B (E) on the THGEM cell
// and 7.7e-8 of the result on the cube and the reduced cell, where B and the result are
// close.  The constants cover every one of those errors by 1.7x or more (2x for phi).
// Most of the error follows B, not S: many pairs round alike (every element of a plane sees
// a point at the same z offset, identical elements carry identical FP32 node tables), so
// their errors keep one sign instead of averaging out; the S term covers the rest.  The
// estimate is statistical, not a bound.  The constants can be changed per context
// (nebem_set_error_model).
//
// Refinement.  A point is re-evaluated when its estimate exceeds tol |phi| or tol |E|,
// in two-float arithmetic (about 44 bits; the error-free transformations of twofloat.cuh),
// in two levels.  Level 1 keeps the FP32 pass's Gauss rules and tiers and its FP64 near
// pairs: their truncation, measured against the closed forms on THGEM points, stays below
// ~2e-10 of B, so its estimate is 1e-9 B.  Points whose level-1 estimate still exceeds the
// tolerance go to level 2, the rules of the mixed fill (fill_mixed.cu: truncation below
// ~3e-12 of each pair, FP64 closed forms within kFillRatioC element radii), estimate
// 1e-11 B.  In the frame of
// element j (axes ex, ey = normal, ez), a pair (point, image k) has D = P - c_j - t_k with
// local components X = (P - c_j) . ex - tau_k.x (likewise Y, Z; tau tabulated per element
// and image); a node at offset s = centroid - node (in the element plane) sees the point at
// D + s, so r^2 = |D|^2 + 2 (X s_x + Z s_z) + |s|^2 and
//   Phi' = sum w / r,   E'_local = D sum w / r^3 + (sum w s_x / r^3, 0, sum w s_z / r^3).
// Per element the image sums are rotated to the global frame and weighted by sigma_j in
// FP64.  Every flagged point's arithmetic depends on that point only, so its result does
// not depend on which other points are flagged or share the launch.
#include "twofloat.cuh"

namespace nb {

namespace {

constexpr int kAT = 128;             // threads (flagged points) per block
constexpr int kATBlocks = 4;         // resident far blocks per SM (128 registers a thread)
constexpr double kErrGammaR = 1e-7;   // FP32 pass: share of the result
constexpr double kErrGammaB = 7e-8;   // FP32 pass: share of B
constexpr double kErrGammaS = 5e-7;   // FP32 pass: share of S
constexpr double kGammaL1 = 1e-9;    // two-float, the FP32 pass's rules (truncation ~1e-10 B)
constexpr double kGammaL2 = 1e-11;   // two-float, fill-grade rules

// What a refinement pass re-evaluates: both phi and E, phi only (its E estimate was within
// the tolerance, E keeps the FP32 pass's value), or E only.
constexpr int kBoth = 0, kPhiOnly = 1, kEOnly = 2;

// Per-pair node sums S0 = sum w / r^3, S2x = sum w (2 s_x) / r^3, S2z = sum w (2 s_z) / r^3
// as packed two-float values (hi, negated lo) over the two lanes of the node pairs.
struct PairSums2 {
    float2 s0, ns0, sx, nsx, sz, nsz;
};

// Phi' (per element, accumulated over its images: ph, nph) and the pair sums of one tier's
// node pairs.  Node records as in nb_internal.h (kFillNodeRec layout): q0 = (2 s_x, 2 s_z)
// hi, q1 = (|s|^2, w) hi, q2 / q3 the lo parts.
template <int M>
__device__ __forceinline__ void nodes_acc2(const float4* __restrict__ nd, int pairs, const PairDF2& P, float2& ph,
                                           float2& nph, PairSums2& S) {
    const float2 m1 = bc2(-1.f);
    for (int q = 0; q < pairs; ++q) {
        const float4 q0 = nd[4 * q], q1 = nd[4 * q + 1], q2 = nd[4 * q + 2], q3 = nd[4 * q + 3];
        float2 y0, ny0, nyl, a, na, nae;
        node_rinv2(P, q0, q1, q2, q3, y0, ny0, nyl, a, na, nae);
        const float2 w = make_float2(q1.z, q1.w), wl = make_float2(q3.z, q3.w);
        float2 t;
        if constexpr (M != kEOnly) {
            // w / r = m - nme
            const float2 m = __fmul2_rn(w, y0);
            float2 nme = __ffma2_rn(w, ny0, m);
            nme = __ffma2_rn(w, nyl, nme);
            nme = __ffma2_rn(wl, ny0, nme);
            two_sum2(ph, m, ph, t);
            nph = __ffma2_rn(t, m1, __fadd2_rn(nph, nme));
        }
        if constexpr (M == kPhiOnly) continue;
        // y^3 = c3 - nc3e (y^2 = a - ny2l)
        const float2 ny2l = __ffma2_rn(__fadd2_rn(y0, y0), nyl, nae);
        const float2 c3 = __fmul2_rn(a, y0);
        float2 nc3e = __ffma2_rn(na, y0, c3);
        nc3e = __ffma2_rn(a, nyl, nc3e);
        nc3e = __ffma2_rn(ny2l, y0, nc3e);
        const float2 nc3 = __fmul2_rn(c3, m1);
        // w y^3 = m3 - nm3e
        const float2 m3 = __fmul2_rn(w, c3);
        float2 nm3e = __ffma2_rn(w, nc3, m3);
        nm3e = __ffma2_rn(w, nc3e, nm3e);
        nm3e = __ffma2_rn(wl, nc3, nm3e);
        two_sum2(S.s0, m3, S.s0, t);
        S.ns0 = __ffma2_rn(t, m1, __fadd2_rn(S.ns0, nm3e));
        // (w y^3) (2 s_x), (w y^3) (2 s_z)
        const float2 nm3 = __fmul2_rn(m3, m1);
        const float2 sx = make_float2(q0.x, q0.y), sz = make_float2(q0.z, q0.w);
        const float2 sxl = make_float2(q2.x, q2.y), szl = make_float2(q2.z, q2.w);
        const float2 fx = __fmul2_rn(m3, sx);
        float2 nfx = __ffma2_rn(nm3, sx, fx);
        nfx = __ffma2_rn(nm3, sxl, nfx);
        nfx = __ffma2_rn(nm3e, sx, nfx);
        two_sum2(S.sx, fx, S.sx, t);
        S.nsx = __ffma2_rn(t, m1, __fadd2_rn(S.nsx, nfx));
        const float2 fz = __fmul2_rn(m3, sz);
        float2 nfz = __ffma2_rn(nm3, sz, fz);
        nfz = __ffma2_rn(nm3, szl, nfz);
        nfz = __ffma2_rn(nm3e, sz, nfz);
        two_sum2(S.sz, fz, S.sz, t);
        S.nsz = __ffma2_rn(t, m1, __fadd2_rn(S.nsz, nfz));
    }
}

// the two lanes of a packed (hi, negated lo) sum as one two-float value, times `scale`
// (a power of two, exact)
__device__ __forceinline__ void lanes_to_df(float2 h, float2 nl, float scale, float& oh, float& ol) {
    float t;
    two_sum(h.x, h.y, oh, t);
    ol = __fsub_rn(__fsub_rn(t, nl.x), nl.y);
    oh = __fmul_rn(oh, scale);
    ol = __fmul_rn(ol, scale);
}

// (Sh, Sl) += (ah + al) (bh + bl) + (ch + cl)
__device__ __forceinline__ void df_fma_acc(float ah, float al, float bh, float bl, float ch, float cl, float& Sh,
                                           float& Sl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float h, t, t2;
    two_sum(p, ch, h, t);
    const float l = __fadd_rn(e, __fadd_rn(t, cl));
    two_sum(Sh, h, Sh, t2);
    Sl = __fadd_rn(Sl, __fadd_rn(t2, l));
}

// Two levels of re-evaluation, both two-float: level 1 takes the tiers of the FP32 pass
// (nb_internal.h FarNodes: 2x2 / 4-point, 3x3 / 6-point, 4x4, 6x6 rules at ratio_0, ratio_a,
// ratio_b, ratio_near radii; FP64 closed forms nearer), whose truncation stays near 1e-10 of
// B; level 2 takes the fill's tiers (truncation below ~3e-12 of each pair, FP64 within
// kFillRatioC radii).  Staged in shared memory per element: the level's most frequent node
// set (tier 0 for level 1, tier a for level 2) and, for level 1, the tier radii.
template <int L>
struct Level;
template <>
struct Level<1> {
    static constexpr int kStaged = 4 * kFillPairs0;  // float4 of the staged node set
    static constexpr int kStagedOff = kFillOff0;
    static constexpr int kHdr = 1;                   // FarNodes radii per element
};
template <>
struct Level<2> {
    static constexpr int kStaged = 4 * kFillPairsA;
    static constexpr int kStagedOff = 0;
    static constexpr int kHdr = 0;
};

// dynamic shared memory per tile of te elements: FillEl (9 float4), the staged node set,
// tau and image centroids (2 float4 each per image), the level-1 tier radii
__host__ __device__ constexpr int acc_tile_f4(int te, int nimg, int staged, int hdr) {
    return te * (9 + staged + 4 * nimg + hdr);
}

// Raw sums (before ke) of the far pairs of one point over the elements [e0, e1) at level L,
// with the error scales, of phi and E (M = kBoth), phi only or E only (the other sums stay
// 0); all threads of the block take part (tiles).
template <int L, int M>
__device__ __forceinline__ Sum6 acc_range(const AccView& A, int nimg, int te, float4* sm, const float (&ph)[3],
                                          const float (&pl)[3], int64_t e0, int64_t e1) {
    using Lv = Level<L>;
    FillEl* s_fe = reinterpret_cast<FillEl*>(sm);
    float4* s_na = sm + 9 * te;
    float4* s_tau = s_na + Lv::kStaged * te;
    float4* s_c = s_tau + 2 * nimg * te;
    float4* s_hdr = s_c + 2 * nimg * te;
    Sum6 acc{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t base = e0; base < e1; base += te) {
        const int cnt = (int)min((int64_t)te, e1 - base);
        __syncthreads();
        {
            const float4* src = reinterpret_cast<const float4*>(A.fe + base);
            float4* dst = reinterpret_cast<float4*>(s_fe);
            for (int i = threadIdx.x; i < 9 * cnt; i += blockDim.x) dst[i] = src[i];
        }
        for (int e = threadIdx.x; e < cnt * Lv::kStaged; e += blockDim.x) {
            const int jj = e / Lv::kStaged, q = e - jj * Lv::kStaged;
            s_na[e] = A.nodes[(base + jj) * kFillNodeRec + Lv::kStagedOff + q];
        }
        for (int i = threadIdx.x; i < 2 * cnt * nimg; i += blockDim.x) {
            s_tau[i] = A.tau[2 * base * nimg + i];
            s_c[i] = A.cjk[2 * base * nimg + i];
        }
        if (Lv::kHdr)
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_hdr[i] = A.far[base + i].hdr;
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const FillEl& F = s_fe[jj];
            const int64_t j = base + jj;
            // squared tier radii, largest first, and the nearest (FP64) radius
            const float4 hdr = Lv::kHdr ? s_hdr[jj] : F.hdr;
            const float near2 = Lv::kHdr ? hdr.w : hdr.z;
            const int na = (int)F.hdr.w;
            float dh[3], dl[3];
            df_sub(ph[0], pl[0], F.ch.x, F.cl.x, dh[0], dl[0]);
            df_sub(ph[1], pl[1], F.ch.y, F.cl.y, dh[1], dl[1]);
            df_sub(ph[2], pl[2], F.ch.z, F.cl.z, dh[2], dl[2]);
            float x0h, x0l, y0h, y0l, z0h, z0l;
            df_dot3(dh, dl, F.exh, F.exl, x0h, x0l);
            df_dot3(dh, dl, F.eyh, F.eyl, y0h, y0l);
            df_dot3(dh, dl, F.ezh, F.ezl, z0h, z0l);
            float2 fph = bc2(0.f), fnph = bc2(0.f);
            float exh = 0.f, exl = 0.f, eyh = 0.f, eyl = 0.f, ezh = 0.f, ezl = 0.f;
            for (int k = 0; k < nimg; ++k) {
                float dx, dy, dz;
                const float d2 = pair_d2(ph[0], ph[1], ph[2], pl[0], pl[1], pl[2], s_c[2 * (jj * nimg + k)],
                                         s_c[2 * (jj * nimg + k) + 1], dx, dy, dz);
                if (!(d2 >= near2)) continue;  // near pair: the level's FP64 kernel
                const float4 th = s_tau[2 * (jj * nimg + k)], tl = s_tau[2 * (jj * nimg + k) + 1];
                float xh, xl, yh, yl, zh, zl, d2h, d2l;
                df_sub(x0h, x0l, th.x, tl.x, xh, xl);
                df_sub(y0h, y0l, th.y, tl.y, yh, yl);
                df_sub(z0h, z0l, th.z, tl.z, zh, zl);
                df_norm2(xh, xl, yh, yl, zh, zl, d2h, d2l);
                PairDF2 P;
                P.xh = bc2(xh), P.nxh = bc2(-xh), P.xl = bc2(xl);
                P.zh = bc2(zh), P.nzh = bc2(-zh), P.zl = bc2(zl);
                P.d2h = bc2(d2h), P.d2l = bc2(d2l);
                const float4* nd;
                int np;
                if (d2 >= hdr.x) {  // the staged set
                    nd = s_na + jj * Lv::kStaged;
                    np = (L == 1) ? kFillPairs0 : na;
                } else if (L == 1 && d2 >= hdr.y) {
                    nd = A.nodes + j * kFillNodeRec;
                    np = na;
                } else if (d2 >= (L == 1 ? hdr.z : hdr.y)) {
                    nd = A.nodes + j * kFillNodeRec + kFillOffB;
                    np = kFillPairsB;
                } else {
                    nd = A.nodes + j * kFillNodeRec + kFillOffC;
                    np = kFillPairsC;
                }
                PairSums2 S{bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f), bc2(0.f)};
                nodes_acc2<M>(nd, np, P, fph, fnph, S);
                if constexpr (M == kPhiOnly) continue;
                float s0h, s0l, sxh, sxl, szh, szl;
                lanes_to_df(S.s0, S.ns0, 1.f, s0h, s0l);
                lanes_to_df(S.sx, S.nsx, 0.5f, sxh, sxl);
                lanes_to_df(S.sz, S.nsz, 0.5f, szh, szl);
                df_fma_acc(xh, xl, s0h, s0l, sxh, sxl, exh, exl);
                df_fma_acc(yh, yl, s0h, s0l, 0.f, 0.f, eyh, eyl);
                df_fma_acc(zh, zl, s0h, s0l, szh, szl, ezh, ezl);
            }
            // element j: image sums in FP64, rotated to the global frame, weighted by sigma_j
            const double s = A.sigma[j];
            if constexpr (M != kEOnly) {
                const double fphi = ((double)fph.x - (double)fnph.x) + ((double)fph.y - (double)fnph.y);
                acc.phi = fma(s, fphi, acc.phi);
                acc.bphi = fma(fabs(s), fabs(fphi), acc.bphi);
            }
            if constexpr (M != kPhiOnly) {
                const double lx = (double)exh + (double)exl, ly = (double)eyh + (double)eyl,
                             lz = (double)ezh + (double)ezl;
                const Elem& e = A.el[j];
                const double gx = fma(lx, e.ex[0], fma(ly, e.ey[0], lz * e.ez[0]));
                const double gy = fma(lx, e.ex[1], fma(ly, e.ey[1], lz * e.ez[1]));
                const double gz = fma(lx, e.ex[2], fma(ly, e.ey[2], lz * e.ez[2]));
                acc.x = fma(s, gx, acc.x);
                acc.y = fma(s, gy, acc.y);
                acc.z = fma(s, gz, acc.z);
                acc.bE = fma(fabs(s), fabs(gx) + fabs(gy) + fabs(gz), acc.bE);
            }
        }
    }
    return acc;
}

// ke * sums of point p at level L into phi / E, the level's estimate into err, and (level 1)
// ke * (B_phi, B_E, 0, 0) into bound for the next flag step; a quantity the pass does not
// re-evaluate (M) keeps its value and estimate, and its level-1 scale is 0, so that the
// next flag step does not take it up.
template <int L, int M>
__device__ __forceinline__ void store_acc(int64_t p, const Sum6& tot, double* __restrict__ phi,
                                          double* __restrict__ E, double* __restrict__ err,
                                          float4* __restrict__ bound) {
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const double gamma = (L == 1) ? kGammaL1 : kGammaL2;
    if (M != kEOnly && phi) phi[p] = ke * tot.phi;
    if (M != kPhiOnly && E) {
        E[3 * p] = ke * tot.x;
        E[3 * p + 1] = ke * tot.y;
        E[3 * p + 2] = ke * tot.z;
    }
    if (err) {
        if (M != kEOnly) err[2 * p] = gamma * ke * tot.bphi;
        if (M != kPhiOnly) err[2 * p + 1] = gamma * ke * tot.bE;
    }
    if (L == 1)
        bound[p] = make_float4(M != kEOnly ? (float)(ke * tot.bphi) : 0.f, M != kPhiOnly ? (float)(ke * tot.bE) : 0.f,
                               0.f, 0.f);
}

// Far part of every listed point at level L, thread per point, kAT points (a group) per
// block pass.  The G = ceil(*n_list / kAT) groups are split so that every resident block
// gets the same work: the first Gm = floor(G / gridDim) * gridDim groups are taken whole,
// round-robin; the R = G - Gm left over are cut into R * nch pieces (group, element chunk of
// kChunkEl), also round-robin, whose Sum6 go to part[chunk * cap + (group - Gm) * kAT + t]
// for k_acc_reduce.  A whole group adds its chunks' sums in chunk order, as k_acc_reduce
// does, so a point gets the same bits whichever way it is taken.  M: which quantities the
// pass re-evaluates (kBoth, kPhiOnly, kEOnly).
template <int L, int M>
__global__ void __launch_bounds__(kAT, kATBlocks)
    k_eval_acc_far(const AccView A, int nimg, int te, const double* __restrict__ pts,
                   const int32_t* __restrict__ list, const int32_t* __restrict__ n_list, int nch, int64_t cap,
                   Sum6* __restrict__ part, double* __restrict__ phi, double* __restrict__ E,
                   double* __restrict__ err, float4* __restrict__ bound) {
    extern __shared__ float4 sm[];
    const int64_t count = *n_list;
    const int64_t gb = gridDim.x;
    const int64_t G = (count + kAT - 1) / kAT;
    const int64_t Gm = (G / gb) * gb;
    for (int64_t g = blockIdx.x; g < Gm; g += gb) {
        const int64_t base = g * kAT;
        const bool active = base + threadIdx.x < count;
        const int64_t p = active ? (int64_t)list[base + threadIdx.x] : 0;
        float ph[3], pl[3];
        load_point_2f(pts, p, active, ph[0], ph[1], ph[2], pl[0], pl[1], pl[2]);
        Sum6 tot{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t e0 = 0; e0 < A.n_el; e0 += kChunkEl)
            add6(tot, acc_range<L, M>(A, nimg, te, sm, ph, pl, e0, min(e0 + (int64_t)kChunkEl, A.n_el)));
        if (active) store_acc<L, M>(p, tot, phi, E, err, bound);
    }
    const int64_t R = G - Gm;
    for (int64_t q = blockIdx.x; q < R * nch; q += gb) {
        const int64_t r = q % R, ch = q / R;  // consecutive blocks: the same chunk, other groups
        const int64_t base = (Gm + r) * kAT;
        const bool active = base + threadIdx.x < count;
        const int64_t p = active ? (int64_t)list[base + threadIdx.x] : 0;
        float ph[3], pl[3];
        load_point_2f(pts, p, active, ph[0], ph[1], ph[2], pl[0], pl[1], pl[2]);
        const int64_t e0 = ch * kChunkEl;
        const Sum6 c = acc_range<L, M>(A, nimg, te, sm, ph, pl, e0, min(e0 + (int64_t)kChunkEl, A.n_el));
        if (active) part[ch * cap + r * kAT + threadIdx.x] = c;
    }
}

// The left-over groups of k_eval_acc_far launched with gb blocks: adds each point's chunk
// sums in chunk order and stores them.
template <int L, int M>
__global__ void __launch_bounds__(256)
    k_acc_reduce(const int32_t* __restrict__ list, const int32_t* __restrict__ n_list, int64_t gb, int nch,
                 int64_t cap, const Sum6* __restrict__ part, double* __restrict__ phi, double* __restrict__ E,
                 double* __restrict__ err, float4* __restrict__ bound) {
    const int64_t count = *n_list;
    const int64_t G = (count + kAT - 1) / kAT;
    const int64_t Gm = (G / gb) * gb;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || Gm * kAT + i >= count) return;
    const int64_t p = list[Gm * kAT + i];
    Sum6 tot{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < nch; ++k) add6(tot, part[(int64_t)k * cap + i]);
    store_acc<L, M>(p, tot, phi, E, err, bound);
}

__global__ void __launch_bounds__(kEvalThreads)
    k_eval_acc_near1(const GeomView g, const ImageTable img, const double* __restrict__ pts,
                     const int32_t* __restrict__ list, const int32_t* __restrict__ n_list, double* __restrict__ phi,
                     double* __restrict__ E) {
    const int64_t count = *n_list;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        near_point(g, img, pts, list[i], phi, E);
}

// Level-2 near part (FP64 closed forms of the pairs nearer than kFillRatioC radii, found
// through the fill's cell list) of every listed point; adds ke * sum to phi / E.
__global__ void __launch_bounds__(128)
    k_eval_acc_near(const AccView A, const ImageTable img, const double* __restrict__ pts,
                    const int32_t* __restrict__ list, const int32_t* __restrict__ n_list, double* __restrict__ phi,
                    double* __restrict__ E) {
    const int64_t count = *n_list;
    const int nimg = img.n;
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = list[i];
        const double Px = pts[3 * p], Py = pts[3 * p + 1], Pz = pts[3 * p + 2];
        float phx, phy, phz, plx, ply, plz;
        split2f(Px, phx, plx);
        split2f(Py, phy, ply);
        split2f(Pz, phz, plz);
        const NearGrid& grid = A.grid;
        int cc[3];
        const double P[3] = {Px, Py, Pz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double f = floor((P[a] - grid.origin[a]) * grid.inv_h);
            f = fmin(fmax(f, -2.0), (double)grid.dims[a] + 1.0);
            cc[a] = (int)f;
        }
        double aphi = 0.0, aEx = 0.0, aEy = 0.0, aEz = 0.0;
        for (int z = max(cc[2] - 1, 0); z <= min(cc[2] + 1, grid.dims[2] - 1); ++z)
            for (int y = max(cc[1] - 1, 0); y <= min(cc[1] + 1, grid.dims[1] - 1); ++y)
                for (int x = max(cc[0] - 1, 0); x <= min(cc[0] + 1, grid.dims[0] - 1); ++x) {
                    const int64_t cell = ((int64_t)z * grid.dims[1] + y) * grid.dims[0] + x;
                    for (int32_t it = A.cell_start[cell]; it < A.cell_start[cell + 1]; ++it) {
                        const int32_t jk = A.cell_items[it];
                        const int32_t j = jk / nimg, k = jk - j * nimg;
                        float dx, dy, dz;
                        const float d2 = pair_d2(phx, phy, phz, plx, ply, plz, A.cjk[2 * (int64_t)jk],
                                                 A.cjk[2 * (int64_t)jk + 1], dx, dy, dz);
                        if (!(d2 < A.fe[j].hdr.z)) continue;  // far pair: k_eval_acc_far<2>
                        const Elem& e = A.el[j];
                        double f, ux, uy, uz;
                        elem_local_f64(e, Px - img.t[k][0], Py - img.t[k][1], Pz - img.t[k][2], false, f, ux, uy, uz);
                        const double s = A.sigma[j];
                        aphi = fma(s, f, aphi);
                        aEx = fma(s, fma(ux, e.ex[0], fma(uy, e.ey[0], uz * e.ez[0])), aEx);
                        aEy = fma(s, fma(ux, e.ex[1], fma(uy, e.ey[1], uz * e.ez[1])), aEy);
                        aEz = fma(s, fma(ux, e.ex[2], fma(uy, e.ey[2], uz * e.ez[2])), aEz);
                    }
                }
        if (phi) phi[p] += ke * aphi;
        if (E) {
            E[3 * p] += ke * aEx;
            E[3 * p + 1] += ke * aEy;
            E[3 * p + 2] += ke * aEz;
        }
    }
}

// Flags and lists (in their input order within each block) the points whose estimate
// gr |x| + gb B + gs S (x = phi or E, bound = (B_phi, B_E, S_phi, S_E)) exceeds tol |x| (when
// refine != 0): with sel < 0 every such point; with sel = kBoth, kPhiOnly or kEOnly the
// points where both quantities, phi only or E only exceed it.  Input: order[i] (or i when
// order is null) for i < n, or i < *n_dev when n_dev is given.  err (may be null) receives
// every input point's estimate.
__global__ void __launch_bounds__(256)
    k_flag(const double* __restrict__ phi, const double* __restrict__ E, const float4* __restrict__ bound,
           const int32_t* __restrict__ order, int64_t n, const int32_t* __restrict__ n_dev, double gr, double gb,
           double gs, double tol, int refine, int sel, double* __restrict__ err, int32_t* __restrict__ list,
           int32_t* __restrict__ n_list) {
    __shared__ int32_t s_warp[8];
    __shared__ int32_t s_base;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t count = n_dev ? (int64_t)*n_dev : n;
    bool f = false;
    int32_t p = 0;
    if (i < count) {
        p = order ? order[i] : (int32_t)i;
        const float4 b = bound[p];
        const double ap = phi ? fabs(phi[p]) : 0.0;
        double aE = 0.0;
        if (E) {
            const double ex = E[3 * p], ey = E[3 * p + 1], ez = E[3 * p + 2];
            aE = sqrt(ex * ex + ey * ey + ez * ez);
        }
        const double ep = gr * ap + gb * (double)b.x + gs * (double)b.z;
        const double eE = gr * aE + gb * (double)b.y + gs * (double)b.w;
        const bool fp = phi && ep > tol * ap, fe = E && eE > tol * aE;
        const int mode = (fp && fe) ? kBoth : fp ? kPhiOnly : kEOnly;
        f = refine && (fp || fe) && (sel < 0 || sel == mode);
        if (err) {
            err[2 * p] = ep;
            err[2 * p + 1] = eE;
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_warp[w] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int k = 0; k < 8; ++k) {
            const int32_t c = s_warp[k];
            s_warp[k] = run;
            run += c;
        }
        s_base = run ? atomicAdd(n_list, run) : 0;
    }
    __syncthreads();
    if (f) list[s_base + s_warp[w] + __popc(ballot & ((1u << lane) - 1u))] = p;
}

// Blocks of a far launch and the partial-sum layout of its left-over groups, from the
// largest possible list (npts points): gb resident blocks at most (kATBlocks per SM), no more than
// there are pieces; cap >= kAT * R for any list length (R < gb, and R <= the groups of npts).
struct RefineGrid {
    int64_t gb, cap;
    int nch;
};

RefineGrid refine_grid(int64_t npts, int sms, int64_t n_el) {
    RefineGrid r;
    const int64_t want = std::max<int64_t>(1, (npts + kAT - 1) / kAT);
    r.nch = (int)std::max<int64_t>(1, (n_el + kChunkEl - 1) / kChunkEl);
    r.gb = std::max<int64_t>(1, std::min<int64_t>(want * r.nch, kATBlocks * (int64_t)sms));
    r.cap = std::min(want, r.gb) * kAT;
    return r;
}

template <int L, int M>
cudaError_t launch_level(const AccView& A, const ImageTable& img, const double* pts, int64_t npts, double* phi,
                         double* E, double* err, float4* bound, const int32_t* list, const int32_t* n_list, int sms,
                         Sum6* part, cudaStream_t s) {
    using Lv = Level<L>;
    // element tile: a power of two (divides the chunk width), at most 16, within ~40 KB
    int te = 16;
    while (te > 1 && acc_tile_f4(te, img.n, Lv::kStaged, Lv::kHdr) * (int)sizeof(float4) > 40 * 1024) te /= 2;
    const size_t smem = (size_t)acc_tile_f4(te, img.n, Lv::kStaged, Lv::kHdr) * sizeof(float4);
    const RefineGrid rg = refine_grid(npts, sms, A.n_el);
    cudaError_t e =
        cudaFuncSetAttribute(k_eval_acc_far<L, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eval_acc_far<L, M><<<(unsigned)rg.gb, kAT, smem, s>>>(A, img.n, te, pts, list, n_list, rg.nch, rg.cap, part,
                                                            phi, E, err, bound);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_acc_reduce<L, M><<<(unsigned)((rg.cap + 255) / 256), 256, 0, s>>>(list, n_list, rg.gb, rg.nch, rg.cap, part,
                                                                         phi, E, err, bound);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the FP64 near pairs, added to the quantities this pass re-evaluated only
    double* nphi = (M == kEOnly) ? nullptr : phi;
    double* nE = (M == kPhiOnly) ? nullptr : E;
    const int64_t want = (npts + kAT - 1) / kAT;
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 8 * (int64_t)sms));
    if (L == 1)
        k_eval_acc_near1<<<gn, kEvalThreads, 0, s>>>(A.view, img, pts, list, n_list, nphi, nE);
    else
        k_eval_acc_near<<<gn, 128, 0, s>>>(A, img, pts, list, n_list, nphi, nE);
    return cudaGetLastError();
}

}  // namespace

ErrModel default_err_model() { return ErrModel{kErrGammaR, kErrGammaB, kErrGammaS}; }

size_t refine_part_bytes(int64_t npts, int sms, int64_t n_el) {
    const RefineGrid rg = refine_grid(npts, sms, n_el);
    return sizeof(Sum6) * (size_t)rg.cap * (size_t)rg.nch;
}

cudaError_t launch_eval_refine(const AccView& A, const ImageTable& img, const double* pts, int64_t npts,
                               double* phi, double* E, double* err, double tol, const ErrModel& em,
                               const MixedScratch& ms, int sms, cudaStream_t s, cudaEvent_t* ev, void* part_buf) {
    Sum6* part = static_cast<Sum6*>(part_buf);
    if (!part) return cudaErrorInvalidValue;
    if (npts == 0) return cudaSuccess;
    if (npts > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
    const bool refine = tol > 0.0 && (phi || E);
    // counts: [0] level 1, both quantities; [1] level 2; [2] level 1, phi only; [3] level 1, E only
    cudaError_t e = cudaMemsetAsync(ms.n_list, 0, 4 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const unsigned fb = (unsigned)((npts + 255) / 256);
    k_flag<<<fb, 256, 0, s>>>(phi, E, ms.bound, ms.order, npts, nullptr, em.gamma_r, em.gamma_b, em.gamma_s, tol,
                              refine ? 1 : 0, kBoth, err, ms.list, ms.n_list);
    e = cudaGetLastError();
    // level 1 on the flagged points, in three passes by what they need (warps then hold
    // points of one kind); it leaves their level-1 scales in ms.bound
    if (e == cudaSuccess && refine) {
        k_flag<<<fb, 256, 0, s>>>(phi, E, ms.bound, ms.order, npts, nullptr, em.gamma_r, em.gamma_b, em.gamma_s,
                                  tol, 1, kPhiOnly, nullptr, ms.list_p, ms.n_list + 2);
        k_flag<<<fb, 256, 0, s>>>(phi, E, ms.bound, ms.order, npts, nullptr, em.gamma_r, em.gamma_b, em.gamma_s,
                                  tol, 1, kEOnly, nullptr, ms.list_e, ms.n_list + 3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && refine)
        e = launch_level<1, kBoth>(A, img, pts, npts, phi, E, err, ms.bound, ms.list, ms.n_list, sms, part, s);
    if (e == cudaSuccess && refine)
        e = launch_level<1, kPhiOnly>(A, img, pts, npts, phi, E, err, ms.bound, ms.list_p, ms.n_list + 2, sms, part,
                                      s);
    if (e == cudaSuccess && refine)
        e = launch_level<1, kEOnly>(A, img, pts, npts, phi, E, err, ms.bound, ms.list_e, ms.n_list + 3, sms, part, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess && refine) {
        // level 2 on the points whose level-1 estimate still exceeds the tolerance (a quantity
        // that level 1 left alone has a level-1 scale of 0 and is not taken up again)
        const int32_t* l1[3] = {ms.list, ms.list_p, ms.list_e};
        const int32_t* c1[3] = {ms.n_list, ms.n_list + 2, ms.n_list + 3};
        for (int k = 0; k < 3; ++k)
            k_flag<<<fb, 256, 0, s>>>(phi, E, ms.bound, l1[k], npts, c1[k], 0.0, kGammaL1, 0.0, tol, 1, -1, nullptr,
                                      ms.list2, ms.n_list + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = launch_level<2, kBoth>(A, img, pts, npts, phi, E, err, nullptr, ms.list2, ms.n_list + 1, sms, part, s);
    }
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    return e;
}

}  // namespace nb
