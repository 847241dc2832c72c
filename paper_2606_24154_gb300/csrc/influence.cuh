// influence.cuh -- closed-form potential and field of a uniformly charged flat polygon
// (rectangle or triangle), FP64, device code.
//
// Sec. 2.1 defines Phi'(P) = int_S dA / |P - r'| and E'(P) = int_S (P - r') dA / |P - r'|^3
// over a flat rectangle or triangle.  Both shapes are evaluated here with one boundary
// decomposition of the surface integral.  The target P has local coordinates
// (X, Y, Z); the element lies in the plane y = 0 with counter-clockwise vertices
// q_i = (qx_i, qz_i).  Per edge i (q_i -> q_i+1, unit tangent t, outward normal m):
//   d_i   signed distance from the projection (X, Z) to the edge line (inside > 0),
//   L_i = int_edge dl / R = ln((R+ + l+) / (R- + l-)),   l-/+ tangential end coordinates,
// and with Omega the solid angle subtended by the element (signed like Y):
//   Phi'  = sum_i d_i L_i - Y Omega,
//   E'_xz = sum_i m_i L_i            (in-plane part: surface gradient -> boundary term),
//   E'_y  = Omega                    (normal part).
// Omega is summed over the fan triangles (0,1,2) and (0,2,3) with the Van Oosterom -
// Strackee form tan(Omega/2) = N / D, N = 2A Y, D = R0 R1 R2 + (r0.r1) R2 + (r0.r2) R1
// + (r1.r2) R0 -- the numerator is exact (doubled area times height), so the far field
// of the normal component suffers no cancellation.  The two half-angles of a four-sided
// element are added as the argument of the product (D1 + i N1)(D2 + i N2) (one atan2).  Within 1e-4 element radii of the
// plane the solid angle is instead summed over the triangles (projection, q_i, q_i+1),
// which stays well-conditioned where the projection meets the fan diagonal.  Exactly in
// the element's plane (Y == 0) the normal field is the principal value 0.
//
// ln(l + R) with l < 0 cancels; the three cases below pick a cancellation-free ratio:
//   l- >= 0 :  (l+ + R+) / (l- + R-)
//   l+ <= 0 :  (R- - l-) / (R+ - l+)
//   else    :  (l+ + R+)(R- - l-) / rho^2,   rho^2 = d^2 + Y^2.
#pragma once
#include "nb_internal.h"

namespace nb {

template <int NV>
__device__ __forceinline__ void poly_f64(const Elem& e, double X, double Y, double Z, double& phi,
                                         double& Ex, double& Ey, double& Ez) {
    double ax[NV], az[NV], R[NV];
    const double Y2 = Y * Y;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        ax[i] = e.qx[i] - X;
        az[i] = e.qz[i] - Z;
        R[i] = sqrt(fma(ax[i], ax[i], fma(az[i], az[i], Y2)));
    }
    double sphi = 0.0, sx = 0.0, sz = 0.0;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int j = (i + 1 == NV) ? 0 : i + 1;
        const double il = e.inv_len[i];
        const double tx = (e.qx[j] - e.qx[i]) * il;
        const double tz = (e.qz[j] - e.qz[i]) * il;
        const double d = ax[i] * tz - az[i] * tx;
        const double lm = ax[i] * tx + az[i] * tz;
        const double lp = ax[j] * tx + az[j] * tz;
        const double rho2 = fma(d, d, Y2);
        const bool pos = lm >= 0.0;
        const bool neg = lp <= 0.0;
        const double a = lp + R[j];
        const double b = R[i] - lm;
        const double num = pos ? a : (neg ? b : a * b);
        const double den = pos ? (lm + R[i]) : (neg ? (R[j] - lp) : rho2);
        const double L = log(num / den);
        sphi += (d != 0.0) ? d * L : 0.0;
        sx = fma(tz, L, sx);
        sz = fma(-tx, L, sz);
    }
    double om = 0.0;
    if (Y != 0.0) {
        if (fabs(Y) >= 1e-4 * e.rho) {
            // half-angles of the fan triangles as arguments of D + i N; their sum is the
            // argument of the product, which stays inside (-pi, pi) here (the element
            // subtends less than a hemisphere by a margin of order 1e-4), so one atan2
            // of the product replaces one per triangle
            double re = 1.0, im = 0.0;
#pragma unroll
            for (int f = 0; f < NV - 2; ++f) {
                const int i1 = f + 1, i2 = f + 2;
                const double d01 = fma(ax[0], ax[i1], fma(az[0], az[i1], Y2));
                const double d02 = fma(ax[0], ax[i2], fma(az[0], az[i2], Y2));
                const double d12 = fma(ax[i1], ax[i2], fma(az[i1], az[i2], Y2));
                const double D = fma(R[0] * R[i1], R[i2], fma(d01, R[i2], fma(d02, R[i1], d12 * R[0])));
                const double Nf = e.twoA[f] * Y;
                if (f == 0) {
                    re = D;
                    im = Nf;
                } else {
                    const double r2 = fma(re, D, -im * Nf);
                    im = fma(re, Nf, im * D);
                    re = r2;
                }
            }
            om = 2.0 * atan2(im, re);
        } else {
            // Close to the plane the fan split is ill-conditioned where the projection
            // meets the shared diagonal; split at the projection instead: triangle
            // (p0, q_i, q_i+1) per edge, tan(Omega_i / 2) = sign(Y) c_i / (R_i R_j +
            // |Y| (R_i + R_j) + r_i . r_j) with c_i the doubled signed area.
            const double h = fabs(Y);
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int j = (i + 1 == NV) ? 0 : i + 1;
                const double cr = ax[i] * az[j] - az[i] * ax[j];
                const double dij = fma(ax[i], ax[j], fma(az[i], az[j], Y2));
                const double D = fma(R[i], R[j], fma(h, R[i] + R[j], dij));
                om += 2.0 * atan2(cr, D);
            }
            om = (Y > 0.0) ? om : -om;
        }
    }
    phi = sphi - Y * om;
    Ex = sx;
    Ey = om;
    Ez = sz;
}

// Local influence of element e at a global point (Px, Py, Pz); self forces Y = 0.
__device__ __forceinline__ void elem_local_f64(const Elem& e, double Px, double Py, double Pz, bool self,
                                               double& phi, double& lx, double& ly, double& lz) {
    const double dx = Px - e.o[0], dy = Py - e.o[1], dz = Pz - e.o[2];
    const double X = fma(dx, e.ex[0], fma(dy, e.ex[1], dz * e.ex[2]));
    double Y = fma(dx, e.ey[0], fma(dy, e.ey[1], dz * e.ey[2]));
    const double Z = fma(dx, e.ez[0], fma(dy, e.ez[1], dz * e.ez[2]));
    if (self) Y = 0.0;
    if (e.nv == 4)
        poly_f64<4>(e, X, Y, Z, phi, lx, ly, lz);
    else
        poly_f64<3>(e, X, Y, Z, phi, lx, ly, lz);
}

}  // namespace nb
