// fill_mixed.cu -- mixed-precision influence-matrix fill (Eq. Matrix, collocation at
// centroids, periodic images):
//   conductor row i:  K_ij = ke sum_k Phi'(c_i - t_k; j)
//   interface row i:  K_ij = ke sum_k n_i . E'(c_i - t_k; j) + delta_ij diag_i
//
// Far pairs (distance to the image centroid >= kFillRatioC element radii) use Gauss rules
// whose truncation error stays below ~3e-12 of the pair (tiers in nb_internal.h), evaluated
// in two-float arithmetic: every quantity is an unevaluated sum hi + lo of two FP32 values
// and products and sums keep their rounding errors through error-free transformations
// (Dekker / Knuth TwoSum, FMA-based TwoProd), about 44 significant bits.  Near pairs use the
// FP64 closed forms of influence.cuh.  The FP32 pipe runs 64 times the FP64 rate on this
// GPU, so a two-float node (54-91 FP32 lane operations, issued two nodes per packed FP32x2
// instruction) costs about as much as one FP64 operation.
//
// Geometry of one pair in the local frame of the column element j (origin anywhere, axes
// ex, ey = normal, ez): D = c_i - (c_j + t_k) has components
//   X = (c_i - c_j) . ex - t_k . ex,  Y, Z likewise,
// the first term once per (i, j), the second (tau) tabulated per (j, k).  A node at
// offset s = centroid - node (in the element plane, local (s_x, s_z)) sees the target at
// P - node = D + s, so
//   r^2 = |D|^2 + q,  q = 2 (X s_x + Z s_z) + |s|^2,
// which needs only two products per node.  1/r comes from one MUFU rsqrt refined by one
// Newton step carried in two-float form; Phi' += w / r, n . E' += w (n . (D + s)) / r^3.
//
// Kernel k_fill_far: thread per row i, grid.y over column chunks; column tiles (element
// records, tier-a nodes, tau, image centroids) staged in shared memory.  It writes
// ke * (far sum) (+ the interface diagonal) to every entry.  Kernel k_fill_near: thread
// per row i; it visits the image centroids in the 27 grid cells around c_i (cell edge >=
// the largest near radius) and adds ke * (FP64 closed form) of every near pair.  Both
// decide "near" by the same rounded FP32 squared distance (pair_d2 of eval_blocks.cuh) on
// the same two-float inputs, so every pair is counted exactly once.
#include "twofloat.cuh"

namespace nb {

namespace {

constexpr int kFT = 128;       // threads per block (one row each)
constexpr int kFillCols = 64;  // columns per block (grid.y)

// Phi' nodes: S += w / r (sh = hi sum, nl = -lo sum), two nodes per step
__device__ __forceinline__ void nodes_phi2(const float4* __restrict__ nd, int pairs, const PairDF2& P, float2& sh,
                                           float2& nl) {
    const float2 m1 = bc2(-1.f);
    for (int q = 0; q < pairs; ++q) {
        const float4 q0 = nd[4 * q], q1 = nd[4 * q + 1], q2 = nd[4 * q + 2], q3 = nd[4 * q + 3];
        float2 y0, ny0, nyl, a, na, nae;
        node_rinv2(P, q0, q1, q2, q3, y0, ny0, nyl, a, na, nae);
        const float2 w = make_float2(q1.z, q1.w), wl = make_float2(q3.z, q3.w);
        const float2 m = __fmul2_rn(w, y0);
        float2 nme = __ffma2_rn(w, ny0, m);  // m - w y0
        nme = __ffma2_rn(w, nyl, nme);
        nme = __ffma2_rn(wl, ny0, nme);
        float2 t;
        two_sum2(sh, m, sh, t);
        nl = __ffma2_rn(t, m1, __fadd2_rn(nl, nme));
    }
}

// n . E' nodes: S += w (n . (D + s)) / r^3, with n . s = (n . ex) s_x + (n . ez) s_z
__device__ __forceinline__ void nodes_nE2(const float4* __restrict__ nd, int pairs, const PairDF2& P,
                                          const NormDF2& Nn, float2& sh, float2& nl) {
    const float2 m1 = bc2(-1.f), half = bc2(0.5f);
    for (int q = 0; q < pairs; ++q) {
        const float4 q0 = nd[4 * q], q1 = nd[4 * q + 1], q2 = nd[4 * q + 2], q3 = nd[4 * q + 3];
        float2 y0, ny0, nyl, a, na, nae;
        node_rinv2(P, q0, q1, q2, q3, y0, ny0, nyl, a, na, nae);
        const float2 sx = make_float2(q0.x, q0.y), sz = make_float2(q0.z, q0.w);
        const float2 sxl = make_float2(q2.x, q2.y), szl = make_float2(q2.z, q2.w);
        // 2 (n . s)
        const float2 p1 = __fmul2_rn(Nn.nxh, sx), ne1 = __ffma2_rn(Nn.nnxh, sx, p1);
        const float2 p2 = __fmul2_rn(Nn.nzh, sz), ne2 = __ffma2_rn(Nn.nnzh, sz, p2);
        float2 ns, t;
        two_sum2(p1, p2, ns, t);
        float2 nsl = __ffma2_rn(ne1, m1, t);
        nsl = __ffma2_rn(ne2, m1, nsl);
        nsl = __ffma2_rn(Nn.nxh, sxl, nsl);
        nsl = __ffma2_rn(Nn.nxl, sx, nsl);
        nsl = __ffma2_rn(Nn.nzh, szl, nsl);
        nsl = __ffma2_rn(Nn.nzl, sz, nsl);
        // g = n . (D + s)
        float2 gh, t2;
        two_sum2(Nn.ndh, __fmul2_rn(half, ns), gh, t2);
        const float2 gl = __fadd2_rn(__ffma2_rn(half, nsl, Nn.ndl), t2);
        // y^3 = y^2 y, y^2 = a + (ae + 2 y0 yl): negated low parts
        const float2 ny2l = __ffma2_rn(__fadd2_rn(y0, y0), nyl, nae);
        const float2 c3 = __fmul2_rn(a, y0);
        float2 nc3e = __ffma2_rn(na, y0, c3);  // c3 - a y0
        nc3e = __ffma2_rn(a, nyl, nc3e);
        nc3e = __ffma2_rn(ny2l, y0, nc3e);
        // w y^3 = m + me
        const float2 w = make_float2(q1.z, q1.w), wl = make_float2(q3.z, q3.w);
        const float2 nc3 = __fmul2_rn(c3, m1);
        const float2 m = __fmul2_rn(w, c3);
        float2 nme = __ffma2_rn(w, nc3, m);  // m - w c3
        nme = __ffma2_rn(w, nc3e, nme);
        nme = __ffma2_rn(wl, nc3, nme);
        // (w y^3) g = f + fe
        const float2 nm = __fmul2_rn(m, m1);
        const float2 f = __fmul2_rn(m, gh);
        float2 nfe = __ffma2_rn(nm, gh, f);  // f - m gh
        nfe = __ffma2_rn(nm, gl, nfe);
        nfe = __ffma2_rn(nme, gh, nfe);
        float2 t3;
        two_sum2(sh, f, sh, t3);
        nl = __ffma2_rn(t3, m1, __fadd2_rn(nl, nfe));
    }
}

__device__ __forceinline__ void stage(float4* dst, const float4* __restrict__ src, int cnt) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = src[i];
}

// Dynamic shared memory per tile of te elements: FillEl (9 float4), tier-a nodes (18 float4),
// tau and image centroids (2 float4 each per image).
__host__ __device__ constexpr int fill_tile_f4(int te, int nimg) { return te * (9 + 4 * kFillPairsA + 4 * nimg); }

__global__ void __launch_bounds__(kFT, 4)
    k_fill_far(const FillEl* __restrict__ fe, const float4* __restrict__ nodes, const float4* __restrict__ tau,
               const float4* __restrict__ cjk, const double* __restrict__ diag_in, int64_t n, int nimg, int te,
               double* __restrict__ K) {
    extern __shared__ float4 sm[];
    FillEl* s_fe = reinterpret_cast<FillEl*>(sm);
    float4* s_na = sm + 9 * te;
    float4* s_tau = s_na + 4 * kFillPairsA * te;
    float4* s_c = s_tau + 2 * nimg * te;

    const int64_t i = (int64_t)blockIdx.x * kFT + threadIdx.x;
    const bool active = i < n;
    // row data: centroid and normal (two floats each), row type
    float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f}, nh[3] = {0.f, 0.f, 0.f}, nl[3] = {0.f, 0.f, 0.f};
    bool iface = false;
    double diag = 0.0;
    if (active) {
        const FillEl r = fe[i];
        ch[0] = r.ch.x, ch[1] = r.ch.y, ch[2] = r.ch.z;
        cl[0] = r.cl.x, cl[1] = r.cl.y, cl[2] = r.cl.z;
        nh[0] = r.eyh.x, nh[1] = r.eyh.y, nh[2] = r.eyh.z;
        nl[0] = r.eyl.x, nl[1] = r.eyl.y, nl[2] = r.eyl.z;
        diag = diag_in[i];
        iface = diag != 0.0;  // interface rows carry the nonzero diagonal term
    }
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const int64_t j0 = (int64_t)blockIdx.y * kFillCols;
    const int64_t j1 = min(n, j0 + kFillCols);
    for (int64_t base = j0; base < j1; base += te) {
        const int cnt = (int)min((int64_t)te, j1 - base);
        __syncthreads();
        stage(reinterpret_cast<float4*>(s_fe), reinterpret_cast<const float4*>(fe + base), 9 * cnt);
        for (int e = threadIdx.x; e < cnt * 4 * kFillPairsA; e += blockDim.x) {
            const int jj = e / (4 * kFillPairsA), q = e - jj * 4 * kFillPairsA;
            s_na[e] = nodes[(base + jj) * kFillNodeRec + q];
        }
        stage(s_tau, tau + 2 * base * nimg, 2 * cnt * nimg);
        stage(s_c, cjk + 2 * base * nimg, 2 * cnt * nimg);
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const FillEl& E = s_fe[jj];
            const int64_t j = base + jj;
            const float4 hdr = E.hdr;
            const int na = (int)hdr.w;
            // c_i - c_j and its local components
            float dh[3], dl[3];
            df_sub(ch[0], cl[0], E.ch.x, E.cl.x, dh[0], dl[0]);
            df_sub(ch[1], cl[1], E.ch.y, E.cl.y, dh[1], dl[1]);
            df_sub(ch[2], cl[2], E.ch.z, E.cl.z, dh[2], dl[2]);
            float x0h, x0l, y0h, y0l, z0h, z0l;
            df_dot3(dh, dl, E.exh, E.exl, x0h, x0l);
            df_dot3(dh, dl, E.eyh, E.eyl, y0h, y0l);
            df_dot3(dh, dl, E.ezh, E.ezl, z0h, z0l);
            float nxh = 0.f, nxl = 0.f, nyh = 0.f, nyl = 0.f, nzh = 0.f, nzl = 0.f;
            if (iface) {
                df_dot3(nh, nl, E.exh, E.exl, nxh, nxl);
                df_dot3(nh, nl, E.eyh, E.eyl, nyh, nyl);
                df_dot3(nh, nl, E.ezh, E.ezl, nzh, nzl);
            }
            NormDF2 Nn;
            if (iface) {
                Nn.nxh = bc2(nxh), Nn.nnxh = bc2(-nxh), Nn.nxl = bc2(nxl);
                Nn.nzh = bc2(nzh), Nn.nnzh = bc2(-nzh), Nn.nzl = bc2(nzl);
            }
            float2 sh = bc2(0.f), snl = bc2(0.f);  // sum: hi, negated lo
            for (int k = 0; k < nimg; ++k) {
                float dx, dy, dz;
                const float d2 = pair_d2(ch[0], ch[1], ch[2], cl[0], cl[1], cl[2], s_c[2 * (jj * nimg + k)],
                                         s_c[2 * (jj * nimg + k) + 1], dx, dy, dz);
                if (!(d2 >= hdr.z)) continue;  // near pair: k_fill_near
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
                if (d2 >= hdr.x) {
                    nd = s_na + jj * 4 * kFillPairsA;
                    np = na;
                } else if (d2 >= hdr.y) {
                    nd = nodes + j * kFillNodeRec + kFillOffB;
                    np = kFillPairsB;
                } else {
                    nd = nodes + j * kFillNodeRec + kFillOffC;
                    np = kFillPairsC;
                }
                if (!iface) {
                    nodes_phi2(nd, np, P, sh, snl);
                } else {
                    const float Xh[3] = {xh, yh, zh}, Xl[3] = {xl, yl, zl};
                    float ndh, ndl;
                    df_dot3(Xh, Xl, make_float4(nxh, nyh, nzh, 0.f), make_float4(nxl, nyl, nzl, 0.f), ndh, ndl);
                    Nn.ndh = bc2(ndh), Nn.ndl = bc2(ndl);
                    nodes_nE2(nd, np, P, Nn, sh, snl);
                }
            }
            if (active) {
                // the two lanes' sums (hi + lo each) in FP64
                const double acc = ((double)sh.x - (double)snl.x) + ((double)sh.y - (double)snl.y);
                K[i + j * n] = (i == j) ? fma(ke, acc, diag) : ke * acc;
            }
        }
    }
}

__global__ void __launch_bounds__(128) k_fill_near(const Elem* __restrict__ el, const FillEl* __restrict__ fe,
                                                   const float4* __restrict__ cjk, int64_t n, const ImageTable img,
                                                   const NearGrid grid, const int32_t* __restrict__ cell_start,
                                                   const int32_t* __restrict__ cell_items, double* __restrict__ K) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Elem& ei = el[i];
    const double Px = ei.c[0], Py = ei.c[1], Pz = ei.c[2];
    const double nx = ei.ey[0], ny = ei.ey[1], nz = ei.ey[2];
    const bool cond = ei.bc == NEBEM_CONDUCTOR;
    const FillEl ri = fe[i];
    const int nimg = img.n;
    int cc[3];
    const double P[3] = {Px, Py, Pz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = floor((P[a] - grid.origin[a]) * grid.inv_h);
        f = fmin(fmax(f, -2.0), (double)grid.dims[a] + 1.0);
        cc[a] = (int)f;
    }
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    for (int z = max(cc[2] - 1, 0); z <= min(cc[2] + 1, grid.dims[2] - 1); ++z)
        for (int y = max(cc[1] - 1, 0); y <= min(cc[1] + 1, grid.dims[1] - 1); ++y)
            for (int x = max(cc[0] - 1, 0); x <= min(cc[0] + 1, grid.dims[0] - 1); ++x) {
                const int64_t cell = ((int64_t)z * grid.dims[1] + y) * grid.dims[0] + x;
                for (int32_t it = cell_start[cell]; it < cell_start[cell + 1]; ++it) {
                    const int32_t jk = cell_items[it];
                    const int32_t j = jk / nimg, k = jk - j * nimg;
                    float dx, dy, dz;
                    const float d2 = pair_d2(ri.ch.x, ri.ch.y, ri.ch.z, ri.cl.x, ri.cl.y, ri.cl.z, cjk[2 * (int64_t)jk],
                                             cjk[2 * (int64_t)jk + 1], dx, dy, dz);
                    if (d2 >= fe[j].hdr.z) continue;  // far pair: k_fill_far
                    const Elem& e = el[j];
                    const bool self = (i == j) && (k == img.k0);
                    double f, gx, gy, gz;
                    elem_local_f64(e, Px - img.t[k][0], Py - img.t[k][1], Pz - img.t[k][2], self, f, gx, gy, gz);
                    double v;
                    if (cond) {
                        v = f;
                    } else {
                        const double Ex = fma(gx, e.ex[0], fma(gy, e.ey[0], gz * e.ez[0]));
                        const double Ey = fma(gx, e.ex[1], fma(gy, e.ey[1], gz * e.ez[1]));
                        const double Ez = fma(gx, e.ex[2], fma(gy, e.ey[2], gz * e.ez[2]));
                        v = fma(nx, Ex, fma(ny, Ey, nz * Ez));
                    }
                    K[i + (int64_t)j * n] += ke * v;
                }
            }
}

}  // namespace

cudaError_t launch_fill_mixed(const Elem* el, const FillEl* fe, const float4* nodes, const float4* tau,
                              const float4* cjk, const double* diag, int64_t n, const ImageTable& img,
                              const NearGrid& grid, const int32_t* cell_start, const int32_t* cell_items, double* K,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    // column tile: as many elements as fit in ~40 KB (four blocks per SM), at most 16
    int te = 16;
    while (te > 1 && fill_tile_f4(te, img.n) * (int)sizeof(float4) > 40 * 1024) --te;
    const size_t smem = (size_t)fill_tile_f4(te, img.n) * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_fill_far, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 g1((unsigned)((n + kFT - 1) / kFT), (unsigned)((n + kFillCols - 1) / kFillCols));
    k_fill_far<<<g1, kFT, smem, s>>>(fe, nodes, tau, cjk, diag, n, img.n, te, K);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fill_near<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(el, fe, cjk, n, img, grid, cell_start, cell_items, K);
    return cudaGetLastError();
}

}  // namespace nb
