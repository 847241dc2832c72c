// geometry.cpp -- host-side FP64 construction of the device element table, the image
// table and the FP32 far-field Gauss nodes (Sec. 2: flat rectangular / triangular
// elements, collocation at centroids; Sec. 5 Case 2: periodic virtual copies).
#include "geometry.h"

#include <cmath>
#include <cstring>

namespace nb {

namespace {

inline void sub3(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0];
    c[1] = a[1] - b[1];
    c[2] = a[2] - b[2];
}
inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Symmetric 6-point degree-4 triangle rule (Strang-Fix / Dunavant): two orbits of
// barycentric points (a, a, 1 - 2a) with weights (fractions of the area).
const double kTriA[2] = {0.445948490915965, 0.091576213509771};
const double kTriW[2] = {0.223381589678011, 0.109951743655322};

// Strang-Fix 4-point degree-3 triangle rule: centroid with weight -27/48 and the three
// points (3/5, 1/5, 1/5) with weight 25/48.
const double kTri3B[4][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
const double kTri3W[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};

}  // namespace

void gauss_legendre01(int m, double* x, double* w) {
    for (int i = 0; i < m; ++i) {
        // initial guess (Chebyshev-like) then Newton on the Legendre recurrence
        double t = std::cos(kPi * (i + 0.75) / (m + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= m; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pm = (m == 1) ? t : p1;
            const double pm1 = (m == 1) ? 1.0 : p0;
            dp = m * (t * pm - pm1) / (t * t - 1.0);
            const double dt = pm / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2) P'^2) on [-1,1], halved for [0,1]
    }
}

int build_element(const nebem_element& r, const nebem_options& opt, Elem& e, double& diag, FarNodes& fn,
                  std::string& why) {
    std::memset(&e, 0, sizeof(e));
    std::memset(&fn, 0, sizeof(fn));
    if (r.kind != NEBEM_RECT && r.kind != NEBEM_TRI && r.kind != NEBEM_QUAD) {
        why = "unknown element kind";
        return NEBEM_INVALID_ARG;
    }
    if (r.bc != NEBEM_CONDUCTOR && r.bc != NEBEM_DIELECTRIC) {
        why = "unknown boundary-condition type";
        return NEBEM_INVALID_ARG;
    }
    const int nv = (r.kind == NEBEM_TRI) ? 3 : 4;
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(r.v[v][k])) {
                why = "non-finite vertex";
                return NEBEM_DEGENERATE_ELEMENT;
            }
    double e1[3], e2[3], n[3];
    sub3(r.v[1], r.v[0], e1);
    sub3(r.v[2], r.v[0], e2);
    cross3(e1, e2, n);
    const double l1 = std::sqrt(dot3(e1, e1));
    const double ln = std::sqrt(dot3(n, n));
    if (!(l1 > 0.0) || !(ln > 1e-300)) {
        why = "zero-area element";
        return NEBEM_DEGENERATE_ELEMENT;
    }
    for (int k = 0; k < 3; ++k) {
        e.o[k] = r.v[0][k];
        e.ex[k] = e1[k] / l1;
        e.ey[k] = n[k] / ln;
    }
    cross3(e.ey, e.ex, e.ez);
    if (r.kind == NEBEM_QUAD) {
        double e3[3], size = 0.0;
        sub3(r.v[3], r.v[0], e3);
        for (int v = 1; v < 4; ++v) {
            double d[3];
            sub3(r.v[v], r.v[0], d);
            size = std::fmax(size, std::sqrt(dot3(d, d)));
        }
        if (std::fabs(dot3(e3, e.ey)) > 1e-9 * size) {
            why = "quadrilateral is not planar";
            return NEBEM_DEGENERATE_ELEMENT;
        }
    } else if (nv == 4) {
        double e3[3], chk[3];
        sub3(r.v[3], r.v[0], e3);
        const double l3 = std::sqrt(dot3(e3, e3));
        for (int k = 0; k < 3; ++k) chk[k] = r.v[1][k] + e3[k] - r.v[2][k];
        const double scale = l1 + l3;
        if (!(l3 > 0.0) || std::fabs(dot3(e1, e3)) > 1e-9 * l1 * l3 || std::sqrt(dot3(chk, chk)) > 1e-9 * scale) {
            why = "rectangle is not planar with right angles";
            return NEBEM_DEGENERATE_ELEMENT;
        }
    }
    e.nv = nv;
    e.bc = r.bc;
    e.cond = r.conductor;
    for (int v = 0; v < nv; ++v) {
        double d[3];
        sub3(r.v[v], r.v[0], d);
        e.qx[v] = dot3(d, e.ex);
        e.qz[v] = dot3(d, e.ez);
    }
    for (int v = 0; v < nv; ++v) {
        const int w = (v + 1) % nv;
        const double dx = e.qx[w] - e.qx[v], dz = e.qz[w] - e.qz[v];
        const double len = std::sqrt(dx * dx + dz * dz);
        if (!(len > 0.0)) {
            why = "zero-length edge";
            return NEBEM_DEGENERATE_ELEMENT;
        }
        e.inv_len[v] = 1.0 / len;
    }
    for (int f = 0; f < nv - 2; ++f) {
        const double ux = e.qx[f + 1] - e.qx[0], uz = e.qz[f + 1] - e.qz[0];
        const double vx = e.qx[f + 2] - e.qx[0], vz = e.qz[f + 2] - e.qz[0];
        e.twoA[f] = ux * vz - uz * vx;
    }
    if (r.kind == NEBEM_QUAD) {
        // every corner turns counter-clockwise in the local (x, z) frame
        for (int v = 0; v < 4; ++v) {
            const int a = v, b = (v + 1) % 4, c = (v + 2) % 4;
            const double turn = (e.qx[b] - e.qx[a]) * (e.qz[c] - e.qz[b]) - (e.qz[b] - e.qz[a]) * (e.qx[c] - e.qx[b]);
            if (!(turn > 0.0)) {
                why = "quadrilateral is not convex";
                return NEBEM_DEGENERATE_ELEMENT;
            }
        }
        // area centroid of the fan triangles (v0, v1, v2) and (v0, v2, v3)
        const double A1 = 0.5 * e.twoA[0], A2 = 0.5 * e.twoA[1];
        for (int k = 0; k < 3; ++k)
            e.c[k] = (A1 * (r.v[0][k] + r.v[1][k] + r.v[2][k]) / 3.0 + A2 * (r.v[0][k] + r.v[2][k] + r.v[3][k]) / 3.0) /
                     (A1 + A2);
    } else {
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int v = 0; v < nv; ++v) s += r.v[v][k];
            e.c[k] = s / nv;
        }
    }
    double rho = 0.0;
    for (int v = 0; v < nv; ++v) {
        double d[3];
        sub3(r.v[v], e.c, d);
        rho = std::fmax(rho, std::sqrt(dot3(d, d)));
    }
    e.rho = rho;
    diag = 0.0;
    if (r.bc == NEBEM_DIELECTRIC) {
        if (!(r.eps_a > 0.0) || !(r.eps_b > 0.0) || r.eps_a == r.eps_b) {
            why = "dielectric interface needs eps_a != eps_b, both > 0";
            return NEBEM_INVALID_ARG;
        }
        diag = (r.eps_a + r.eps_b) / (2.0 * kEps0 * (r.eps_b - r.eps_a));
    }
    // FP32 far-field Gauss nodes: centroid - node, weight x area, packed in pairs.
    const double area = (r.kind == NEBEM_RECT) ? e.twoA[0]
                        : (r.kind == NEBEM_QUAD) ? 0.5 * (e.twoA[0] + e.twoA[1])
                                                 : 0.5 * e.twoA[0];
    float4 node[kNodesC];  // one tier's nodes (x, y, z = centroid - node, w = weight x area)
    auto put = [&](float4& dst, const double* g, double wt) {
        double d[3];
        sub3(e.c, g, d);
        dst.x = (float)d[0];
        dst.y = (float)d[1];
        dst.z = (float)d[2];
        dst.w = (float)(wt * area);
    };
    // pack cnt nodes of `node` into pairs at dst; returns the pair count
    auto pack = [&](int cnt, float4* dst) {
        const int np = (cnt + 1) / 2;
        for (int i = 0; i < np; ++i) {
            const float4 a = node[2 * i];
            float4 b = (2 * i + 1 < cnt) ? node[2 * i + 1] : node[2 * i];
            if (2 * i + 1 >= cnt) b.w = 0.f;
            dst[2 * i] = make_float4(a.x, b.x, a.y, b.y);
            dst[2 * i + 1] = make_float4(a.z, b.z, a.w, b.w);
        }
        return np;
    };
    int n_a = 0;
    if (nv == 4) {
        double e3[3], tw[3];
        sub3(r.v[3], r.v[0], e3);
        for (int k = 0; k < 3; ++k) tw[k] = (r.kind == NEBEM_RECT) ? 0.0 : r.v[2][k] - r.v[1][k] - e3[k];
        // tensor Gauss-Legendre on the bilinear map x(s, t) = v0 + s e1 + t e3 + s t tw,
        // weight w_s w_t |x_s x x_t| (the area for a rectangle)
        auto tensor = [&](int m, float4* dst) {
            double x[16], w[16];
            gauss_legendre01(m, x, w);
            int cnt = 0;
            float4* out = dst;
            dst = node;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    double g[3], xs[3], xt[3], jn[3];
                    for (int k = 0; k < 3; ++k) {
                        g[k] = r.v[0][k] + x[a] * e1[k] + x[b] * e3[k] + x[a] * x[b] * tw[k];
                        xs[k] = e1[k] + x[b] * tw[k];
                        xt[k] = e3[k] + x[a] * tw[k];
                    }
                    cross3(xs, xt, jn);
                    const double jac = (r.kind == NEBEM_RECT) ? area : std::sqrt(dot3(jn, jn));
                    put(dst[cnt++], g, w[a] * w[b] * jac / area);
                }
            return pack(cnt, out);
        };
        tensor(2, fn.f);
        n_a = tensor(3, fn.a);
        tensor(4, fn.b);
        tensor(6, fn.c);
    } else {
        // degree-3 four-point rule
        for (int q = 0; q < 4; ++q) {
            double g[3];
            for (int k = 0; k < 3; ++k)
                g[k] = kTri3B[q][0] * r.v[0][k] + kTri3B[q][1] * r.v[1][k] + kTri3B[q][2] * r.v[2][k];
            put(node[q], g, kTri3W[q]);
        }
        pack(4, fn.f);
        // degree-4 six-point rule
        int six = 0;
        for (int g2 = 0; g2 < 2; ++g2)
            for (int rr = 0; rr < 3; ++rr) {
                double bc[3] = {kTriA[g2], kTriA[g2], kTriA[g2]};
                bc[rr] = 1.0 - 2.0 * kTriA[g2];
                double g[3];
                for (int k = 0; k < 3; ++k) g[k] = bc[0] * r.v[0][k] + bc[1] * r.v[1][k] + bc[2] * r.v[2][k];
                put(node[six++], g, kTriW[g2]);
            }
        n_a = pack(six, fn.a);
        // collapsed (Duffy) product rules: x = v0 + s e1 + t (1 - s) e2, weight 2 ws wt (1 - s)
        auto collapsed = [&](int m, float4* dst) {
            double x[16], w[16];
            gauss_legendre01(m, x, w);
            int cnt = 0;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    const double sa = x[a], tb = x[b] * (1.0 - x[a]);
                    double g[3];
                    for (int k = 0; k < 3; ++k) g[k] = r.v[0][k] + sa * e1[k] + tb * e2[k];
                    put(node[cnt++], g, 2.0 * w[a] * w[b] * (1.0 - x[a]));
                }
            return pack(cnt, dst);
        };
        collapsed(4, fn.b);
        collapsed(6, fn.c);
    }
    // Weight totals.  Rounding the weights to FP32 leaves each tier's total off the area by
    // a relative error of order 2^-24, the same for every element of one shape (identical
    // elements of a mesh ring or a plane), so its effect on the far field would add up with
    // one sign over those elements instead of averaging out.  Tiers a-c get their largest
    // weight set so that their totals come as close to tier 0's as FP32 allows (within
    // 2^-25 of that weight), and the remaining factor area / (tier 0's total) goes into
    // wcorr, which the evaluation applies to sigma in two-float form.  The totals of a few
    // dozen FP32 numbers of similar size are exact in FP64.
    auto wsum = [](const float4* t, int np) {
        double sum = 0.0;
        for (int i = 0; i < np; ++i) sum += (double)t[2 * i + 1].z + (double)t[2 * i + 1].w;
        return sum;
    };
    const double total0 = wsum(fn.f, kPairs0);
    auto match = [&](float4* t, int np) {
        float* big = nullptr;
        for (int i = 0; i < np; ++i) {
            float* wz = &t[2 * i + 1].z;
            float* ww = &t[2 * i + 1].w;
            if (!big || std::fabs(*wz) > std::fabs(*big)) big = wz;
            if (std::fabs(*ww) > std::fabs(*big)) big = ww;
        }
        const double rest = wsum(t, np) - (double)*big;
        *big = (float)(total0 - rest);
    };
    match(fn.a, n_a);
    match(fn.b, kPairsB);
    match(fn.c, kPairsC);
    fn.wcorr = (float)(area / total0 - 1.0);
    const double r0 = opt.ratio_0 * rho, ra = opt.ratio_a * rho, rb = opt.ratio_b * rho,
                 rn = opt.ratio_near * rho;
    fn.hdr.x = (float)(r0 * r0);
    fn.hdr.y = (float)(ra * ra);
    fn.hdr.z = (float)(rb * rb);
    fn.hdr.w = (float)(rn * rn);
    fn.n_a = n_a;
    return NEBEM_OK;
}

namespace {

inline void split_f(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

inline float4 f4(float a, float b, float c, float d) {
    float4 r;
    r.x = a;
    r.y = b;
    r.z = c;
    r.w = d;
    return r;
}

// Two-float node record of the offset s = centroid - node (local frame) and weight w, for
// a node pair (a, b): see nb_internal.h.
struct FillNode {
    double sx, sz, w;
};

inline void pack_fill_pairs(const FillNode* nd, int cnt, float4* dst) {
    for (int p = 0; p < (cnt + 1) / 2; ++p) {
        const FillNode a = nd[2 * p];
        FillNode b = (2 * p + 1 < cnt) ? nd[2 * p + 1] : nd[2 * p];
        if (2 * p + 1 >= cnt) b.w = 0.0;
        float h[2][4], l[2][4];
        const FillNode* ab[2] = {&a, &b};
        for (int q = 0; q < 2; ++q) {
            split_f(2.0 * ab[q]->sx, h[q][0], l[q][0]);
            split_f(2.0 * ab[q]->sz, h[q][1], l[q][1]);
            split_f(ab[q]->sx * ab[q]->sx + ab[q]->sz * ab[q]->sz, h[q][2], l[q][2]);
            split_f(ab[q]->w, h[q][3], l[q][3]);
        }
        dst[4 * p + 0] = f4(h[0][0], h[1][0], h[0][1], h[1][1]);
        dst[4 * p + 1] = f4(h[0][2], h[1][2], h[0][3], h[1][3]);
        dst[4 * p + 2] = f4(l[0][0], l[1][0], l[0][1], l[1][1]);
        dst[4 * p + 3] = f4(l[0][2], l[1][2], l[0][3], l[1][3]);
    }
}

}  // namespace

void build_fill_tables(const std::vector<Elem>& el, const ImageTable& img, std::vector<FillEl>& fe,
                       std::vector<float4>& nodes, std::vector<float4>& tau) {
    const int64_t n = (int64_t)el.size();
    const int m = img.n;
    fe.assign((size_t)n, FillEl{});
    nodes.assign((size_t)n * kFillNodeRec, f4(0.f, 0.f, 0.f, 0.f));
    tau.assign((size_t)n * m * 2, f4(0.f, 0.f, 0.f, 0.f));
    for (int64_t j = 0; j < n; ++j) {
        const Elem& e = el[j];
        FillEl& r = fe[j];
        float h[3], l[3];
        for (int a = 0; a < 3; ++a) split_f(e.c[a], h[a], l[a]);
        r.ch = f4(h[0], h[1], h[2], 0.f);
        r.cl = f4(l[0], l[1], l[2], 0.f);
        const double* ax[3] = {e.ex, e.ey, e.ez};
        float4* dh[3] = {&r.exh, &r.eyh, &r.ezh};
        float4* dl[3] = {&r.exl, &r.eyl, &r.ezl};
        for (int v = 0; v < 3; ++v) {
            for (int a = 0; a < 3; ++a) split_f(ax[v][a], h[a], l[a]);
            *dh[v] = f4(h[0], h[1], h[2], 0.f);
            *dl[v] = f4(l[0], l[1], l[2], 0.f);
        }
        const double ra = kFillRatioA * e.rho, rb = kFillRatioB * e.rho, rc = kFillRatioC * e.rho;
        const int nv = e.nv;
        // centroid in the local frame (origin v0)
        double d[3];
        sub3(e.c, e.o, d);
        const double cx = dot3(d, e.ex), cz = dot3(d, e.ez);
        const double* qx = e.qx;
        const double* qz = e.qz;
        float4* out = nodes.data() + j * kFillNodeRec;
        FillNode nd[36];
        int cnt = 0;
        auto put = [&](double px, double pz, double w) { nd[cnt++] = FillNode{cx - px, cz - pz, w}; };
        int n_a = 0;  // tier-a node pairs
        if (nv == 4) {
            // tensor Gauss-Legendre on the bilinear map x(s, t) = q0 + s e1 + t e3 + s t tw,
            // weight ws wt |x_s x x_t|
            const double e1x = qx[1] - qx[0], e1z = qz[1] - qz[0];
            const double e3x = qx[3] - qx[0], e3z = qz[3] - qz[0];
            const double twx = qx[2] - qx[1] - e3x, twz = qz[2] - qz[1] - e3z;
            auto tensor = [&](int mq, float4* dst) {
                double x[16], w[16];
                gauss_legendre01(mq, x, w);
                cnt = 0;
                for (int a = 0; a < mq; ++a)
                    for (int b = 0; b < mq; ++b) {
                        const double px = qx[0] + x[a] * e1x + x[b] * e3x + x[a] * x[b] * twx;
                        const double pz = qz[0] + x[a] * e1z + x[b] * e3z + x[a] * x[b] * twz;
                        const double sx = e1x + x[b] * twx, sz = e1z + x[b] * twz;
                        const double tx = e3x + x[a] * twx, tz = e3z + x[a] * twz;
                        put(px, pz, w[a] * w[b] * std::fabs(sx * tz - sz * tx));
                    }
                pack_fill_pairs(nd, cnt, dst);
                return (cnt + 1) / 2;
            };
            n_a = tensor(3, out);
            tensor(4, out + kFillOffB);
            tensor(6, out + kFillOffC);
            tensor(2, out + kFillOff0);
        } else {
            const double area = 0.5 * e.twoA[0];
            cnt = 0;
            for (int g2 = 0; g2 < 2; ++g2)
                for (int rr = 0; rr < 3; ++rr) {
                    double bc[3] = {kTriA[g2], kTriA[g2], kTriA[g2]};
                    bc[rr] = 1.0 - 2.0 * kTriA[g2];
                    const double px = bc[0] * qx[0] + bc[1] * qx[1] + bc[2] * qx[2];
                    const double pz = bc[0] * qz[0] + bc[1] * qz[1] + bc[2] * qz[2];
                    put(px, pz, kTriW[g2] * area);
                }
            pack_fill_pairs(nd, cnt, out);
            n_a = (cnt + 1) / 2;
            // collapsed (Duffy) product rules: x = q0 + s e1 + t (1 - s) e2, weight 2 ws wt (1 - s) A
            auto collapsed = [&](int mq, float4* dst) {
                double x[16], w[16];
                gauss_legendre01(mq, x, w);
                cnt = 0;
                for (int a = 0; a < mq; ++a)
                    for (int b = 0; b < mq; ++b) {
                        const double sa = x[a], tb = x[b] * (1.0 - x[a]);
                        const double px = qx[0] + sa * (qx[1] - qx[0]) + tb * (qx[2] - qx[0]);
                        const double pz = qz[0] + sa * (qz[1] - qz[0]) + tb * (qz[2] - qz[0]);
                        put(px, pz, 2.0 * w[a] * w[b] * (1.0 - x[a]) * area);
                    }
                pack_fill_pairs(nd, cnt, dst);
            };
            collapsed(4, out + kFillOffB);
            collapsed(6, out + kFillOffC);
            // degree-3 four-point rule (tier 0 of the mixed evaluation)
            cnt = 0;
            for (int q = 0; q < 4; ++q) {
                const double px = kTri3B[q][0] * qx[0] + kTri3B[q][1] * qx[1] + kTri3B[q][2] * qx[2];
                const double pz = kTri3B[q][0] * qz[0] + kTri3B[q][1] * qz[1] + kTri3B[q][2] * qz[2];
                put(px, pz, kTri3W[q] * area);
            }
            pack_fill_pairs(nd, cnt, out + kFillOff0);
        }
        r.hdr = f4((float)(ra * ra), (float)(rb * rb), (float)(rc * rc), (float)n_a);
        for (int k = 0; k < m; ++k) {
            float th[3], tl[3];
            for (int v = 0; v < 3; ++v) split_f(dot3(img.t[k], ax[v]), th[v], tl[v]);
            tau[((size_t)j * m + k) * 2] = f4(th[0], th[1], th[2], 0.f);
            tau[((size_t)j * m + k) * 2 + 1] = f4(tl[0], tl[1], tl[2], 0.f);
        }
    }
}

int build_near_grid(const std::vector<Elem>& el, const ImageTable& img, double ratio_near, NearGrid& grid,
                    std::vector<int32_t>& cell_start, std::vector<int32_t>& cell_items, std::string& why) {
    const int64_t n = (int64_t)el.size(), m = img.n, total = n * m;
    if (total > (int64_t)INT32_MAX) {
        why = "too many element images for the near-pair grid";
        return NEBEM_TOO_LARGE;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, rmax = 0.0;
    std::vector<double> C((size_t)total * 3);
    for (int64_t j = 0; j < n; ++j) {
        rmax = std::fmax(rmax, ratio_near * el[j].rho);
        for (int64_t k = 0; k < m; ++k)
            for (int a = 0; a < 3; ++a) {
                const double v = el[j].c[a] + img.t[k][a];
                C[(j * m + k) * 3 + a] = v;
                lo[a] = std::fmin(lo[a], v);
                hi[a] = std::fmax(hi[a], v);
            }
    }
    double h = 1.01 * rmax;
    if (!(h > 0.0)) h = 1.0;
    // bound the cell count (16M); larger cells only cost more candidates per query
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) cells *= std::floor((hi[a] - lo[a]) / h) + 3.0;
        if (cells <= 16.0e6) break;
        h *= 1.5;
    }
    grid.inv_h = 1.0 / h;
    for (int a = 0; a < 3; ++a) {
        grid.origin[a] = lo[a] - h;
        grid.dims[a] = (int32_t)std::floor((hi[a] - grid.origin[a]) * grid.inv_h) + 2;
    }
    grid.pad = 0;
    const int64_t ncell = (int64_t)grid.dims[0] * grid.dims[1] * grid.dims[2];
    std::vector<int32_t> cell_of((size_t)total);
    cell_start.assign((size_t)ncell + 1, 0);
    for (int64_t i = 0; i < total; ++i) {
        int64_t cc[3];
        for (int a = 0; a < 3; ++a) {
            const double f = std::floor((C[i * 3 + a] - grid.origin[a]) * grid.inv_h);
            cc[a] = (int64_t)std::fmin(std::fmax(f, 0.0), (double)grid.dims[a] - 1.0);
        }
        const int64_t cell = (cc[2] * grid.dims[1] + cc[1]) * grid.dims[0] + cc[0];
        cell_of[i] = (int32_t)cell;
        cell_start[cell + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    cell_items.assign((size_t)total, 0);
    std::vector<int32_t> fillp(cell_start.begin(), cell_start.end() - 1);
    for (int64_t i = 0; i < total; ++i) cell_items[fillp[cell_of[i]]++] = (int32_t)i;  // stable: ascending j*m+k
    return NEBEM_OK;
}

int build_images(const double* lattice, int lo, int hi, ImageTable& img, std::string& why) {
    std::memset(&img, 0, sizeof(img));
    if (!lattice) {
        img.n = 1;
        img.k0 = 0;
        return NEBEM_OK;
    }
    if (hi < lo || lo > 0 || hi < 0) {
        why = "image range must contain 0";
        return NEBEM_INVALID_ARG;
    }
    const int m = hi - lo + 1;
    if (m > kMaxImgAxis) {
        why = "more than 11 images per axis";
        return NEBEM_TOO_LARGE;
    }
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(lattice[k])) {
            why = "non-finite lattice vector";
            return NEBEM_INVALID_ARG;
        }
    img.n = m * m;
    img.k0 = (0 - lo) * m + (0 - lo);
    for (int k1 = lo; k1 <= hi; ++k1)
        for (int k2 = lo; k2 <= hi; ++k2) {
            const int k = (k1 - lo) * m + (k2 - lo);
            for (int c = 0; c < 3; ++c) {
                // one rounded product per term and one rounded sum (no contraction: this
                // file is compiled with -ffp-contract=off)
                const double p1 = (double)k1 * lattice[c];
                const double p2 = (double)k2 * lattice[3 + c];
                img.t[k][c] = p1 + p2;
            }
        }
    return NEBEM_OK;
}

}  // namespace nb
