/*
 * nebem_oracle.c -- plain, slow, FP64 CPU oracle for the neBEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path (paper_2606_24154_gb300/csrc).
 *
 * What it computes (paper section / equation cited per function):
 *   - the potential and field integrals of a uniformly charged flat element
 *       Phi'(P) = int_S dA / |P - r'|,      E'(P) = int_S (P - r') dA / |P - r'|^3
 *     (Sec. 2.1: rectangle with corners (X1,0,Z1),(X2,0,Z2); right/general triangle;
 *     field integral of r-hat / r^2), evaluated in closed form:
 *       * rectangles by the corner antiderivative in the paper's own parametrisation;
 *       * triangles and planar convex quadrilaterals by the boundary (edge)
 *         decomposition of the surface integral, with the solid angle written as a sum
 *         of per-edge arctangent differences;
 *   - periodic images ("virtual copies", Sec. 5 Case 2) of every element,
 *     t = k1*a1 + k2*a2 for k1, k2 in [lo, hi], image index (k1-lo)*m + (k2-lo);
 *   - the collocation influence matrix K (Eq. Matrix) with conductor rows
 *     K_ij = ke * sum_k Phi'(c_i; j + t_k) and dielectric-interface rows
 *     K_ij = ke * sum_k n_i . E'(c_i; j + t_k) + delta_ij (ea + eb) / (2 eps0 (eb - ea));
 *   - LU with partial pivoting (lowest row index on ties) and the triangular solves
 *     (rho = K^-1 phi, Eq. 6, by factorisation instead of an explicit inverse);
 *   - potential and field at points by superposition (Eq. Potential, Eq. Field);
 *   - the direct point-charge sum (Alg. 2) with Plummer softening, self excluded by index;
 *   - one dynamic space-charge update step (Alg. 4) with carriers moved by mu*E*dt.
 *
 * Conventions fixed here where the paper is silent:
 *   - ke = 1 / (4 pi eps0), eps0 = 8.8541878128e-12 F/m (CODATA 2018);
 *   - the normal field on an element's own plane is the principal value (the mean of
 *     the one-sided limits), i.e. the solid-angle term is zero when the normal
 *     coordinate is exactly zero; a self pair (target = own centroid, image 0) takes
 *     the normal coordinate as exactly zero;
 *   - ln(a + R) with a < 0 is evaluated as ln(rho^2 / (R - a)) to avoid cancellation.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math), so that the
 * image translation is one rounded multiply per term and one rounded add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_EPS0 8.8541878128e-12

/* Raw element record: same 128-byte layout as the input records. */
typedef struct {
    int32_t kind; /* 0 rectangle, 1 triangle */
    int32_t bc;   /* 0 conductor, 1 dielectric interface */
    int32_t conductor;
    int32_t reserved;
    double eps_a, eps_b;
    double v[4][3];
} or_input;

/* Element with its local frame: origin o = v0, ex along v0->v1, ey = unit normal
 * (right-hand rule on v0, v1, v2), ez = ey x ex; the element lies in the local y = 0
 * plane with local (x, z) vertex coordinates q[]. */
typedef struct {
    int kind, bc, cond, nv;
    double eps_a, eps_b;
    double o[3], ex[3], ey[3], ez[3];
    double q[4][2];
    double c[3];
    double area;
} or_elem;

double or_ke(void) { return 1.0 / (4.0 * OR_PI * OR_EPS0); }
double or_eps0(void) { return OR_EPS0; }

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Build local frames. Returns 0, or -(1+i) for the first degenerate element i. */
int or_build(const or_input *in, int64_t n, or_elem *out) {
    for (int64_t i = 0; i < n; ++i) {
        const or_input *r = &in[i];
        or_elem *e = &out[i];
        memset(e, 0, sizeof(*e));
        e->kind = r->kind;
        e->bc = r->bc;
        e->cond = r->conductor;
        e->eps_a = r->eps_a;
        e->eps_b = r->eps_b;
        e->nv = (r->kind == 0 || r->kind == 2) ? 4 : 3;
        double e1[3], e2[3], nn[3];
        for (int k = 0; k < 3; ++k) {
            e->o[k] = r->v[0][k];
            e1[k] = r->v[1][k] - r->v[0][k];
            e2[k] = r->v[2][k] - r->v[0][k];
        }
        double l1 = norm3(e1);
        cross3(e1, e2, nn);
        double ln = norm3(nn);
        if (!(l1 > 0.0) || !(ln > 0.0)) return -(int)(1 + i);
        for (int k = 0; k < 3; ++k) {
            e->ex[k] = e1[k] / l1;
            e->ey[k] = nn[k] / ln;
        }
        cross3(e->ey, e->ex, e->ez);
        for (int vtx = 0; vtx < e->nv; ++vtx) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = r->v[vtx][k] - e->o[k];
            e->q[vtx][0] = dot3(d, e->ex);
            e->q[vtx][1] = dot3(d, e->ez);
        }
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int vtx = 0; vtx < e->nv; ++vtx) s += r->v[vtx][k];
            e->c[k] = s / e->nv;
        }
        if (e->kind == 2) {
            /* planar convex quadrilateral: v3 in the plane of v0, v1, v2, every corner
             * turning counter-clockwise in the local (x, z) frame; the centroid is the
             * area centroid (triangles (v0, v1, v2) and (v0, v2, v3) weighted by area) */
            double d3[3], size = 0.0;
            for (int k = 0; k < 3; ++k) d3[k] = r->v[3][k] - r->v[0][k];
            for (int vtx = 1; vtx < 4; ++vtx) {
                double dv[3] = {r->v[vtx][0] - r->v[0][0], r->v[vtx][1] - r->v[0][1], r->v[vtx][2] - r->v[0][2]};
                if (norm3(dv) > size) size = norm3(dv);
            }
            if (fabs(dot3(d3, e->ey)) > 1e-9 * size) return -(int)(1 + i);
            for (int vtx = 0; vtx < 4; ++vtx) {
                const double *a = e->q[vtx], *b = e->q[(vtx + 1) % 4], *c = e->q[(vtx + 2) % 4];
                double turn = (b[0] - a[0]) * (c[1] - b[1]) - (b[1] - a[1]) * (c[0] - b[0]);
                if (!(turn > 0.0)) return -(int)(1 + i);
            }
            double A1 = 0.5 * ((e->q[1][0] - e->q[0][0]) * (e->q[2][1] - e->q[0][1]) -
                               (e->q[1][1] - e->q[0][1]) * (e->q[2][0] - e->q[0][0]));
            double A2 = 0.5 * ((e->q[2][0] - e->q[0][0]) * (e->q[3][1] - e->q[0][1]) -
                               (e->q[2][1] - e->q[0][1]) * (e->q[3][0] - e->q[0][0]));
            for (int k = 0; k < 3; ++k)
                e->c[k] = (A1 * (r->v[0][k] + r->v[1][k] + r->v[2][k]) / 3.0 +
                           A2 * (r->v[0][k] + r->v[2][k] + r->v[3][k]) / 3.0) / (A1 + A2);
            e->area = A1 + A2;
        } else if (e->kind == 0) {
            /* rectangle: v3 - v0 must be perpendicular to v1 - v0 and v2 = v1 + v3 - v0 */
            double e3[3];
            for (int k = 0; k < 3; ++k) e3[k] = r->v[3][k] - r->v[0][k];
            double l3 = norm3(e3);
            if (!(l3 > 0.0)) return -(int)(1 + i);
            if (fabs(dot3(e1, e3)) > 1e-9 * l1 * l3) return -(int)(1 + i);
            e->area = l1 * l3;
        } else {
            e->area = 0.5 * ln;
        }
    }
    return 0;
}

/* int_{a1}^{a2} da / sqrt(a^2 + rho2), a1 <= a2, with R1 = sqrt(a1^2+rho2), R2 likewise. */
static double line_integral(double a1, double a2, double rho2, double R1, double R2) {
    if (a1 >= 0.0) return log((a2 + R2) / (a1 + R1));
    if (a2 <= 0.0) return log((R1 - a1) / (R2 - a2));
    return log((a2 + R2) * (R1 - a1) / rho2);
}

/* ln(a + R) with R = sqrt(a^2 + rho2), rho2 > 0 whenever a < 0 is passed. */
static double log_a_plus_R(double a, double rho2, double R) {
    if (a >= 0.0) return log(a + R);
    return log(rho2 / (R - a));
}

/* Corner antiderivative of the rectangle potential (Sec. 2.1), u = x - X, w = z - Z:
 * F = u ln(w + R) + w ln(u + R) - Y atan(u w / (Y R)); mixed derivative = 1/R. */
static double rect_corner_F(double u, double w, double Y) {
    double R = sqrt(u * u + w * w + Y * Y);
    double t1 = (u == 0.0) ? 0.0 : u * log_a_plus_R(w, u * u + Y * Y, R);
    double t2 = (w == 0.0) ? 0.0 : w * log_a_plus_R(u, w * w + Y * Y, R);
    double t3 = (Y == 0.0) ? 0.0 : Y * atan(u * w / (Y * R));
    return t1 + t2 - t3;
}

/* Rectangle [0,L1] x [0,L2] in the local y = 0 plane; target (X, Y, Z). Local phi, E. */
static void rect_local(double L1, double L2, double X, double Y, double Z, double *phi, double El[3]) {
    double u1 = -X, u2 = L1 - X, w1 = -Z, w2 = L2 - Z;
    *phi = rect_corner_F(u2, w2, Y) - rect_corner_F(u1, w2, Y) - rect_corner_F(u2, w1, Y) +
           rect_corner_F(u1, w1, Y);
    double Y2 = Y * Y;
    double R11 = sqrt(u1 * u1 + w1 * w1 + Y2), R12 = sqrt(u1 * u1 + w2 * w2 + Y2);
    double R21 = sqrt(u2 * u2 + w1 * w1 + Y2), R22 = sqrt(u2 * u2 + w2 * w2 + Y2);
    /* E_x = int int -u/R^3 = [line integral over w at u2] - [same at u1] */
    double Ex = line_integral(w1, w2, u2 * u2 + Y2, R21, R22) - line_integral(w1, w2, u1 * u1 + Y2, R11, R12);
    double Ez = line_integral(u1, u2, w2 * w2 + Y2, R12, R22) - line_integral(u1, u2, w1 * w1 + Y2, R11, R21);
    double Ey = 0.0;
    if (Y != 0.0) {
        Ey = atan(u2 * w2 / (Y * R22)) - atan(u1 * w2 / (Y * R12)) - atan(u2 * w1 / (Y * R21)) +
             atan(u1 * w1 / (Y * R11));
    }
    El[0] = Ex;
    El[1] = Ey;
    El[2] = Ez;
}

/* Planar polygon (counter-clockwise local (x,z) vertices q, nv of them) at target
 * (X, Y, Z): Phi' = sum_i d_i L_i - |Y| Omega, in-plane E' = sum_i m_i L_i,
 * E'_y = sign(Y) Omega, where per edge i: m_i outward unit normal, d_i signed distance
 * from the target's projection to the edge line, L_i = int_edge dl / R, and the solid
 * angle Omega = sum_i [atan(d_i l+ / (rho_i^2 + |Y| R+)) - atan(d_i l- / (rho_i^2 + |Y| R-))]. */
static void poly_local(const double q[][2], int nv, double X, double Y, double Z, double *phi, double El[3]) {
    double h = fabs(Y);
    double sphi = 0.0, ex = 0.0, ez = 0.0, omega = 0.0;
    for (int i = 0; i < nv; ++i) {
        const double *a = q[i], *b = q[(i + 1) % nv];
        double tx = b[0] - a[0], tz = b[1] - a[1];
        double len = sqrt(tx * tx + tz * tz);
        tx /= len;
        tz /= len;
        double mx = tz, mz = -tx; /* outward normal for counter-clockwise order */
        double ax = a[0] - X, az = a[1] - Z, bx = b[0] - X, bz = b[1] - Z;
        double d = ax * mx + az * mz;
        double lm = ax * tx + az * tz;
        double lp = bx * tx + bz * tz;
        double rho2 = d * d + h * h;
        double Rm = sqrt(lm * lm + rho2), Rp = sqrt(lp * lp + rho2);
        double L = line_integral(lm, lp, rho2, Rm, Rp);
        if (d != 0.0) sphi += d * L;
        ex += mx * L;
        ez += mz * L;
        if (h != 0.0 && d != 0.0)
            omega += atan(d * lp / (rho2 + h * Rp)) - atan(d * lm / (rho2 + h * Rm));
    }
    *phi = sphi - h * omega;
    El[0] = ex;
    El[2] = ez;
    El[1] = (Y > 0.0) ? omega : ((Y < 0.0) ? -omega : 0.0);
}

/* Phi' and global E' of element e (unit charge density) at global point P.
 * self != 0 forces the normal coordinate to zero (target = own centroid, image 0). */
void or_influence(const or_elem *e, const double P[3], int self, double *phi, double E[3]) {
    double d[3] = {P[0] - e->o[0], P[1] - e->o[1], P[2] - e->o[2]};
    double X = dot3(d, e->ex), Y = dot3(d, e->ey), Z = dot3(d, e->ez);
    if (self) Y = 0.0;
    double El[3];
    if (e->kind == 0)
        rect_local(e->q[2][0], e->q[2][1], X, Y, Z, phi, El);
    else
        poly_local((const double(*)[2])e->q, e->nv, X, Y, Z, phi, El);
    for (int k = 0; k < 3; ++k) E[k] = El[0] * e->ex[k] + El[1] * e->ey[k] + El[2] * e->ez[k];
}

/* Same, forcing the polygon (edge) formula also for rectangles: used by tests. */
void or_influence_poly(const or_elem *e, const double P[3], int self, double *phi, double E[3]) {
    double d[3] = {P[0] - e->o[0], P[1] - e->o[1], P[2] - e->o[2]};
    double X = dot3(d, e->ex), Y = dot3(d, e->ey), Z = dot3(d, e->ez);
    if (self) Y = 0.0;
    double El[3];
    poly_local((const double(*)[2])e->q, e->nv, X, Y, Z, phi, El);
    for (int k = 0; k < 3; ++k) E[k] = El[0] * e->ex[k] + El[1] * e->ey[k] + El[2] * e->ez[k];
}

/* Vectorised single-element influence at many points (raw record in). */
int or_influence_points(const or_input *rec, const double *P, int64_t n, int poly, double *phi, double *E) {
    or_elem e;
    int rc = or_build(rec, 1, &e);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        if (poly)
            or_influence_poly(&e, P + 3 * i, 0, phi + i, E + 3 * i);
        else
            or_influence(&e, P + 3 * i, 0, phi + i, E + 3 * i);
    }
    return 0;
}

/* Image translation t = k1*a1 + k2*a2 (each product and the sum rounded once). */
void or_image_shift(const double *lattice, int k1, int k2, double t[3]) {
    for (int c = 0; c < 3; ++c) {
        double p1 = (double)k1 * lattice[c];
        double p2 = (double)k2 * lattice[3 + c];
        t[c] = p1 + p2;
    }
}

/* All image translations in index order k = (k1-lo)*m + (k2-lo); returns the count. */
int64_t or_image_table(const double *lattice, int lo, int hi, double *t /* count x 3 */) {
    if (!lattice) {
        t[0] = t[1] = t[2] = 0.0;
        return 1;
    }
    int m = hi - lo + 1;
    for (int k1 = lo; k1 <= hi; ++k1)
        for (int k2 = lo; k2 <= hi; ++k2) or_image_shift(lattice, k1, k2, t + 3 * ((int64_t)(k1 - lo) * m + (k2 - lo)));
    return (int64_t)m * m;
}

static int64_t image_count(const double *lattice, int lo, int hi) {
    return lattice ? (int64_t)(hi - lo + 1) * (hi - lo + 1) : 1;
}

/* Influence matrix (Eq. Matrix), column-major K[i + j*n]. */
int or_fill(const or_input *in, int64_t n, const double *lattice, int lo, int hi, double *K) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    int rc = or_build(in, n, el);
    if (rc) {
        free(el);
        return rc;
    }
    int64_t nimg = image_count(lattice, lo, hi);
    double *tt = (double *)malloc(sizeof(double) * 3 * (size_t)nimg);
    or_image_table(lattice, lo, hi, tt);
    int64_t kzero = lattice ? (int64_t)(0 - lo) * (hi - lo + 1) + (0 - lo) : 0;
    double ke = or_ke();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        const or_elem *ei = &el[i];
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t k = 0; k < nimg; ++k) {
                double P[3] = {ei->c[0] - tt[3 * k], ei->c[1] - tt[3 * k + 1], ei->c[2] - tt[3 * k + 2]};
                double phi, E[3];
                or_influence(&el[j], P, (i == j && k == kzero), &phi, E);
                acc += (ei->bc == 0) ? phi : dot3(ei->ey, E);
            }
            double v = ke * acc;
            if (i == j && ei->bc == 1) v += (ei->eps_a + ei->eps_b) / (2.0 * OR_EPS0 * (ei->eps_b - ei->eps_a));
            K[i + j * n] = v;
        }
    }
    free(tt);
    free(el);
    return 0;
}

/* Selected entries K[rows[e], cols[e]] of the influence matrix (same definition as
 * or_fill), for checks of full-size matrices one entry at a time. */
int or_fill_entries(const or_input *in, int64_t n, const double *lattice, int lo, int hi, const int64_t *rows,
                    const int64_t *cols, int64_t count, double *out) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    int rc = or_build(in, n, el);
    if (rc) {
        free(el);
        return rc;
    }
    int64_t nimg = image_count(lattice, lo, hi);
    double *tt = (double *)malloc(sizeof(double) * 3 * (size_t)nimg);
    or_image_table(lattice, lo, hi, tt);
    int64_t kzero = lattice ? (int64_t)(0 - lo) * (hi - lo + 1) + (0 - lo) : 0;
    double ke = or_ke();
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < count; ++e) {
        int64_t i = rows[e], j = cols[e];
        const or_elem *ei = &el[i];
        double acc = 0.0;
        for (int64_t k = 0; k < nimg; ++k) {
            double P[3] = {ei->c[0] - tt[3 * k], ei->c[1] - tt[3 * k + 1], ei->c[2] - tt[3 * k + 2]};
            double phi, E[3];
            or_influence(&el[j], P, (i == j && k == kzero), &phi, E);
            acc += (ei->bc == 0) ? phi : dot3(ei->ey, E);
        }
        double v = ke * acc;
        if (i == j && ei->bc == 1) v += (ei->eps_a + ei->eps_b) / (2.0 * OR_EPS0 * (ei->eps_b - ei->eps_a));
        out[e] = v;
    }
    free(tt);
    free(el);
    return 0;
}

/* Distance tier of every (point, element, image) pair for the mixed-precision evaluation
 * (a pair classification written out for checks; codes[(p * n + j) * nimg + k]):
 *   0: d >= r0 rho_j,  1: >= ra rho_j,  2: >= rb rho_j,  3: >= rn rho_j,  4: nearer,
 * with rho_j the element's circumradius about its centroid c_j and d the distance from
 * the point to c_j + t_k.  The decision is taken in FP32, as the evaluation takes it: both
 * positions split into two floats (hi = fl(x), lo = fl(x - hi)), each difference
 * (P_hi - C_hi) + (P_lo - C_lo) and d^2 = fma(dx, dx, fma(dy, dy, dz * dz)) rounded in
 * float (this file is compiled without contraction), thresholds fl((r rho)^2). */
int or_pair_tiers(const or_input *in, int64_t n, const double *lattice, int lo, int hi, const double *pts,
                  int64_t npts, const double *ratios, uint8_t *codes) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    int rc = or_build(in, n, el);
    if (rc) {
        free(el);
        return rc;
    }
    int64_t nimg = image_count(lattice, lo, hi);
    double *tt = (double *)malloc(sizeof(double) * 3 * (size_t)nimg);
    or_image_table(lattice, lo, hi, tt);
    float *thr = (float *)malloc(sizeof(float) * 4 * (size_t)(n ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
        double rho = 0.0;
        for (int v = 0; v < el[j].nv; ++v) {
            double d[3] = {in[j].v[v][0] - el[j].c[0], in[j].v[v][1] - el[j].c[1], in[j].v[v][2] - el[j].c[2]};
            rho = fmax(rho, sqrt(dot3(d, d)));
        }
        for (int t = 0; t < 4; ++t) {
            double r = ratios[t] * rho;
            thr[4 * j + t] = (float)(r * r);
        }
    }
    for (int64_t p = 0; p < npts; ++p) {
        float ph[3], pl[3];
        for (int a = 0; a < 3; ++a) {
            ph[a] = (float)pts[3 * p + a];
            pl[a] = (float)(pts[3 * p + a] - (double)ph[a]);
        }
        for (int64_t j = 0; j < n; ++j)
            for (int64_t k = 0; k < nimg; ++k) {
                float ch[3], cl[3], dd[3];
                for (int a = 0; a < 3; ++a) {
                    double C = el[j].c[a] + tt[3 * k + a];
                    ch[a] = (float)C;
                    cl[a] = (float)(C - (double)ch[a]);
                    float u = ph[a] - ch[a];
                    float w = pl[a] - cl[a];
                    dd[a] = u + w;
                }
                float d2 = fmaf(dd[0], dd[0], fmaf(dd[1], dd[1], dd[2] * dd[2]));
                const float *th = thr + 4 * j;
                uint8_t code = (d2 >= th[0]) ? 0 : (d2 >= th[1]) ? 1 : (d2 >= th[2]) ? 2 : (d2 >= th[3]) ? 3 : 4;
                codes[(p * n + j) * nimg + k] = code;
            }
    }
    free(thr);
    free(tt);
    free(el);
    return 0;
}

/* In-place LU with partial pivoting (row of max |a|, lowest index on ties), column-major.
 * piv[k] = row swapped with row k at step k.  Returns 0 or -(1+k) for a zero pivot. */
int or_lu_factor(int64_t n, double *A, int32_t *piv) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = fabs(A[k + k * n]);
        for (int64_t i = k + 1; i < n; ++i) {
            double v = fabs(A[i + k * n]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        piv[k] = (int32_t)p;
        if (best == 0.0) return -(int)(1 + k);
        if (p != k)
            for (int64_t j = 0; j < n; ++j) {
                double s = A[k + j * n];
                A[k + j * n] = A[p + j * n];
                A[p + j * n] = s;
            }
        double d = A[k + k * n];
        for (int64_t i = k + 1; i < n; ++i) A[i + k * n] /= d;
        for (int64_t j = k + 1; j < n; ++j) {
            double ukj = A[k + j * n];
            if (ukj == 0.0) continue;
            for (int64_t i = k + 1; i < n; ++i) A[i + j * n] -= A[i + k * n] * ukj;
        }
    }
    return 0;
}

/* Solve A x = b with the factors from or_lu_factor (b overwritten by x). */
void or_lu_solve(int64_t n, const double *LU, const int32_t *piv, double *b) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = piv[k];
        if (p != k) {
            double s = b[k];
            b[k] = b[p];
            b[p] = s;
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        double bj = b[j];
        for (int64_t i = j + 1; i < n; ++i) b[i] -= LU[i + j * n] * bj;
    }
    for (int64_t j = n - 1; j >= 0; --j) {
        b[j] /= LU[j + j * n];
        double bj = b[j];
        for (int64_t i = 0; i < j; ++i) b[i] -= LU[i + j * n] * bj;
    }
}

/* Right-hand side: conductor rows V(conductor), dielectric rows 0. */
int or_rhs(const or_input *in, int64_t n, const double *voltages, int32_t ncond, double *b) {
    for (int64_t i = 0; i < n; ++i) {
        if (in[i].bc == 0) {
            if (in[i].conductor < 0 || in[i].conductor >= ncond) return -1;
            b[i] = voltages[in[i].conductor];
        } else {
            b[i] = 0.0;
        }
    }
    return 0;
}

/* Potential and field at points (Eq. Potential / Eq. Field): sum over j, then images. */
int or_eval(const or_input *in, int64_t n, const double *sigma, const double *lattice, int lo, int hi,
            const double *pts, int64_t npts, double *phi_out, double *E_out) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    int rc = or_build(in, n, el);
    if (rc) {
        free(el);
        return rc;
    }
    int64_t nimg = image_count(lattice, lo, hi);
    double *tt = (double *)malloc(sizeof(double) * 3 * (size_t)nimg);
    or_image_table(lattice, lo, hi, tt);
    double ke = or_ke();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npts; ++p) {
        double sphi = 0.0, sE[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            double aphi = 0.0, aE[3] = {0.0, 0.0, 0.0};
            for (int64_t k = 0; k < nimg; ++k) {
                double P[3] = {pts[3 * p] - tt[3 * k], pts[3 * p + 1] - tt[3 * k + 1], pts[3 * p + 2] - tt[3 * k + 2]};
                double f, E[3];
                or_influence(&el[j], P, 0, &f, E);
                aphi += f;
                aE[0] += E[0];
                aE[1] += E[1];
                aE[2] += E[2];
            }
            sphi += sigma[j] * aphi;
            sE[0] += sigma[j] * aE[0];
            sE[1] += sigma[j] * aE[1];
            sE[2] += sigma[j] * aE[2];
        }
        if (phi_out) phi_out[p] = ke * sphi;
        if (E_out) {
            E_out[3 * p] = ke * sE[0];
            E_out[3 * p + 1] = ke * sE[1];
            E_out[3 * p + 2] = ke * sE[2];
        }
    }
    free(tt);
    free(el);
    return 0;
}

/* Element centroids and unit normals, for callers that need collocation points. */
int or_centroids(const or_input *in, int64_t n, double *c, double *nrm, double *area) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    int rc = or_build(in, n, el);
    if (rc == 0)
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                if (c) c[3 * i + k] = el[i].c[k];
                if (nrm) nrm[3 * i + k] = el[i].ey[k];
                if (area && k == 0) area[i] = el[i].area;
            }
    free(el);
    return rc;
}

/* Direct space-charge sum (Alg. 2, softened): for each target t,
 *   phi_t = ke sum_{c != self(t)} q_c / sqrt(r^2 + s^2),
 *   E_t   = ke sum_{c != self(t)} q_c (x_t - x_c) / (r^2 + s^2)^{3/2}.
 * self_is_index != 0: target t is source t and is excluded. */
void or_space_charge(const double *src, const double *q, int64_t nsrc, const double *tgt, int64_t ntgt,
                     int self_is_index, double soft, double *phi_out, double *E_out) {
    double ke = or_ke(), s2 = soft * soft;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < ntgt; ++t) {
        double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
        for (int64_t c = 0; c < nsrc; ++c) {
            if (self_is_index && c == t) continue;
            double dx = tgt[3 * t] - src[3 * c], dy = tgt[3 * t + 1] - src[3 * c + 1], dz = tgt[3 * t + 2] - src[3 * c + 2];
            double r2 = dx * dx + dy * dy + dz * dz + s2;
            double ri = 1.0 / sqrt(r2);
            double qr = q[c] * ri;
            double qr3 = qr * ri * ri;
            ph += qr;
            ex += qr3 * dx;
            ey += qr3 * dy;
            ez += qr3 * dz;
        }
        if (phi_out) phi_out[t] = ke * ph;
        if (E_out) {
            E_out[3 * t] = ke * ex;
            E_out[3 * t + 1] = ke * ey;
            E_out[3 * t + 2] = ke * ez;
        }
    }
}

/* Right-hand side with known charges (OptKnCh): conductor rows V - phi_sc(c_i),
 * dielectric rows -n_i . E_sc(c_i). */
int or_rhs_space_charge(const or_input *in, int64_t n, const double *voltages, int32_t ncond, const double *pos,
                        const double *q, int64_t ncar, double soft, double *b) {
    int rc = or_rhs(in, n, voltages, ncond, b);
    if (rc) return rc;
    if (ncar == 0) return 0;
    double *c = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *nr = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *ph = (double *)malloc(sizeof(double) * (size_t)n);
    double *E = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    rc = or_centroids(in, n, c, nr, NULL);
    if (rc == 0) {
        or_space_charge(pos, q, ncar, c, n, 0, soft, ph, E);
        for (int64_t i = 0; i < n; ++i)
            b[i] -= (in[i].bc == 0) ? ph[i] : dot3(nr + 3 * i, E + 3 * i);
    }
    free(c);
    free(nr);
    free(ph);
    free(E);
    return rc;
}

/* One dynamic space-charge step (Alg. 4 with SpChTh = 0 and drift in place of tracking):
 * (1) RHS with the known charges at the collocation points, (2) sigma from the retained
 * LU factors, (3) E at every carrier from all elements (with images) plus all other
 * carriers, (4) x += sign(q) mu E dt.  sigma_out (n) and E_out (ncar x 3) may be NULL. */
int or_dynamic_step(const or_input *in, int64_t n, const double *voltages, int32_t ncond, const double *lattice,
                    int lo, int hi, const double *LU, const int32_t *piv, double *pos, const double *q, int64_t ncar,
                    double soft, double mu, double dt, double *sigma_out, double *E_out) {
    double *b = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *Ee = (double *)malloc(sizeof(double) * 3 * (size_t)(ncar ? ncar : 1));
    double *Es = (double *)malloc(sizeof(double) * 3 * (size_t)(ncar ? ncar : 1));
    int rc = or_rhs_space_charge(in, n, voltages, ncond, pos, q, ncar, soft, b);
    if (rc == 0) {
        or_lu_solve(n, LU, piv, b);
        rc = or_eval(in, n, b, lattice, lo, hi, pos, ncar, NULL, Ee);
    }
    if (rc == 0) {
        or_space_charge(pos, q, ncar, pos, ncar, 1, soft, NULL, Es);
        for (int64_t c = 0; c < ncar; ++c) {
            double sg = (q[c] > 0.0) ? 1.0 : ((q[c] < 0.0) ? -1.0 : 0.0);
            for (int k = 0; k < 3; ++k) {
                double Ek = Ee[3 * c + k] + Es[3 * c + k];
                if (E_out) E_out[3 * c + k] = Ek;
                pos[3 * c + k] += sg * mu * Ek * dt;
            }
        }
        if (sigma_out) memcpy(sigma_out, b, sizeof(double) * (size_t)n);
    }
    free(b);
    free(Ee);
    free(Es);
    return rc;
}

/* ---------------------------------------------------------------------------------
 * Line-charge representation of the known charges (Sec. 4.2, Alg. 3; the LineCh
 * branch of Alg. 4).
 *
 * Alg. 3, kernel 1: every point charge p falls in voxel v = f(p; dx, dy, dz) and adds its
 * charge to that voxel's total; a voxel that receives a point is occupied.  Kernel 2:
 * every occupied voxel yields one line charge (start, stop, lambda).
 * Readings fixed here where the paper is silent:
 *   - the grid is anchored at the minimum corner (xmin, ymin, zmin) of the cloud:
 *     i = floor((x - xmin) / dx), likewise j, k; nx = floor((xmax - xmin) / dx) + 1;
 *     flat voxel index v = (k * ny + j) * nx + i;
 *   - the line runs along z (the drift direction) through the voxel's centre, from its
 *     lower to its upper z face: start = (xmin + (i + 1/2) dx, ymin + (j + 1/2) dy,
 *     zmin + k dz), stop = start + (0, 0, dz), lambda = total charge / dz (C/m);
 *   - lines are listed in increasing voxel index, and a voxel's total is summed over
 *     its points in increasing point index.
 * ------------------------------------------------------------------------------- */

typedef struct {
    int64_t v;
    int64_t i;
} or_vox_pair;

static int vox_pair_cmp(const void *a, const void *b) {
    const or_vox_pair *x = (const or_vox_pair *)a, *y = (const or_vox_pair *)b;
    if (x->v != y->v) return (x->v < y->v) ? -1 : 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* Grid of Alg. 3 for a cloud: lo[3] (minimum corner) and dims[3]; 0, or -1 for bad input
 * or a grid of 4e18 voxels or more. */
int or_voxel_grid(const double *pos, int64_t n, const double d[3], double lo[3], int64_t dims[3]) {
    if (n <= 0) return -1;
    for (int a = 0; a < 3; ++a) {
        if (!(d[a] > 0.0)) return -1;
        double mn = pos[a], mx = pos[a];
        for (int64_t p = 1; p < n; ++p) {
            if (pos[3 * p + a] < mn) mn = pos[3 * p + a];
            if (pos[3 * p + a] > mx) mx = pos[3 * p + a];
        }
        lo[a] = mn;
        double na = floor((mx - mn) / d[a]) + 1.0;
        if (!(na < 4.0e18)) return -1;
        dims[a] = (int64_t)na;
    }
    /* the flat voxel index must fit in 62 bits */
    if ((double)dims[0] * (double)dims[1] * (double)dims[2] >= 4.0e18) return -1;
    return 0;
}

/* Alg. 3.  Returns the number of lines L (all written: start, stop L x 3; lambda L;
 * voxel L, the flat voxel index of each line; each may be NULL), or -1 on bad input.
 * The caller sizes the outputs for n lines (the most there can be). */
int64_t or_voxel_lines(const double *pos, const double *q, int64_t n, const double d[3], double *start,
                       double *stop, double *lambda, int64_t *voxel) {
    double lo[3];
    int64_t dims[3];
    if (or_voxel_grid(pos, n, d, lo, dims)) return -1;
    /* kernel 1: the voxel of every point */
    or_vox_pair *pv = (or_vox_pair *)malloc(sizeof(or_vox_pair) * (size_t)n);
    for (int64_t p = 0; p < n; ++p) {
        int64_t ijk[3];
        for (int a = 0; a < 3; ++a) {
            int64_t c = (int64_t)floor((pos[3 * p + a] - lo[a]) / d[a]);
            ijk[a] = c < dims[a] - 1 ? c : dims[a] - 1;
        }
        pv[p].v = (ijk[2] * dims[1] + ijk[1]) * dims[0] + ijk[0];
        pv[p].i = p;
    }
    /* kernel 2: occupied voxels in increasing index, each summing its points in order */
    qsort(pv, (size_t)n, sizeof(or_vox_pair), vox_pair_cmp);
    int64_t L = 0;
    for (int64_t s = 0; s < n;) {
        int64_t v = pv[s].v, e = s;
        double Q = 0.0;
        while (e < n && pv[e].v == v) Q += q[pv[e++].i];
        int64_t i = v % dims[0], j = (v / dims[0]) % dims[1], k = v / (dims[0] * dims[1]);
        double a[3] = {lo[0] + ((double)i + 0.5) * d[0], lo[1] + ((double)j + 0.5) * d[1], lo[2] + (double)k * d[2]};
        if (start) memcpy(start + 3 * L, a, sizeof a);
        if (stop) {
            stop[3 * L] = a[0];
            stop[3 * L + 1] = a[1];
            stop[3 * L + 2] = a[2] + d[2];
        }
        if (lambda) lambda[L] = Q / d[2];
        if (voxel) voxel[L] = v;
        ++L;
        s = e;
    }
    free(pv);
    return L;
}

/* Potential and field of finite uniform line charges (LineCh), softened like the point
 * charges: for a line from A to B (unit u, length L) and target P, with w = P - A,
 * a = w.u, perpendicular part p = w - a u, rho^2 = |p|^2 + s^2, s1 = -a, s2 = L - a,
 *   phi = ke lambda int_0^L dt / sqrt((a - t)^2 + rho^2)
 *       = ke lambda (asinh(s2 / rho) - asinh(s1 / rho)),
 *   (on the axis with s = 0: ke lambda ln(s2 / s1) before the start, ln(s1 / s2) past the end),
 *   E = -grad phi = ke lambda [ (1/R2 - 1/R1) u + (s2/R2 - s1/R1) p / rho^2 ],
 *   R1,2 = sqrt(s1,2^2 + rho^2).
 * accumulate != 0 adds to phi_out / E_out. */
void or_line_charge(const double *start, const double *stop, const double *lambda, int64_t nl, const double *tgt,
                    int64_t nt, double soft, int accumulate, double *phi_out, double *E_out) {
    double ke = or_ke(), s2s = soft * soft;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) {
        double ph = 0.0, E[3] = {0.0, 0.0, 0.0};
        for (int64_t l = 0; l < nl; ++l) {
            double u[3], w[3], p[3];
            for (int a = 0; a < 3; ++a) u[a] = stop[3 * l + a] - start[3 * l + a];
            double len = norm3(u);
            for (int a = 0; a < 3; ++a) {
                u[a] /= len;
                w[a] = tgt[3 * t + a] - start[3 * l + a];
            }
            double ax = dot3(w, u);
            for (int a = 0; a < 3; ++a) p[a] = w[a] - ax * u[a];
            double rho2 = dot3(p, p) + s2s, rho = sqrt(rho2);
            double s1 = -ax, s2 = len - ax;
            double R1 = sqrt(s1 * s1 + rho2), R2 = sqrt(s2 * s2 + rho2);
            /* asinh(s/rho) = ln(s + R) - ln(rho): for a target on either side of the
             * segment's span the difference is a log ratio (also at rho = 0, on the axis);
             * beside the span rho > 0 and the asinh difference is used directly */
            double I;
            if (s1 >= 0.0)
                I = log((s2 + R2) / (s1 + R1));
            else if (s2 <= 0.0)
                I = log((R1 - s1) / (R2 - s2));
            else
                I = asinh(s2 / rho) - asinh(s1 / rho);
            ph += lambda[l] * I;
            double cu = lambda[l] * (1.0 / R2 - 1.0 / R1);
            double cp = (rho2 > 0.0) ? lambda[l] * (s2 / R2 - s1 / R1) / rho2 : 0.0;
            for (int a = 0; a < 3; ++a) E[a] += cu * u[a] + cp * p[a];
        }
        if (phi_out) phi_out[t] = (accumulate ? phi_out[t] : 0.0) + ke * ph;
        if (E_out)
            for (int a = 0; a < 3; ++a) E_out[3 * t + a] = (accumulate ? E_out[3 * t + a] : 0.0) + ke * E[a];
    }
}

/* Right-hand side with line charges as the known charges: conductor rows
 * V - phi_lines(c_i), dielectric rows -n_i . E_lines(c_i). */
int or_rhs_lines(const or_input *in, int64_t n, const double *voltages, int32_t ncond, const double *start,
                 const double *stop, const double *lambda, int64_t nl, double soft, double *b) {
    int rc = or_rhs(in, n, voltages, ncond, b);
    if (rc || nl == 0) return rc;
    double *c = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *nr = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *ph = (double *)malloc(sizeof(double) * (size_t)n);
    double *E = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    rc = or_centroids(in, n, c, nr, NULL);
    if (rc == 0) {
        or_line_charge(start, stop, lambda, nl, c, n, soft, 0, ph, E);
        for (int64_t i = 0; i < n; ++i) b[i] -= (in[i].bc == 0) ? ph[i] : dot3(nr + 3 * i, E + 3 * i);
    }
    free(c);
    free(nr);
    free(ph);
    free(E);
    return rc;
}

/* One dynamic step with the line representation (Alg. 4, Type == Line, SpChTh = 0):
 * (1) Alg. 3 on the carriers, (2) RHS with the lines, (3) sigma from the retained
 * factors, (4) E at every carrier from the elements (with images) and all lines,
 * (5) x += sign(q) mu E dt.  E_out (ncar x 3) may be NULL. */
int or_dynamic_step_lines(const or_input *in, int64_t n, const double *voltages, int32_t ncond,
                          const double *lattice, int lo, int hi, const double *LU, const int32_t *piv, double *pos,
                          const double *q, int64_t ncar, const double d[3], double soft, double mu, double dt,
                          double *sigma_out, double *E_out) {
    double *st = (double *)malloc(sizeof(double) * 3 * (size_t)ncar);
    double *sp = (double *)malloc(sizeof(double) * 3 * (size_t)ncar);
    double *lam = (double *)malloc(sizeof(double) * (size_t)ncar);
    double *b = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *Ee = (double *)malloc(sizeof(double) * 3 * (size_t)ncar);
    int64_t nl = or_voxel_lines(pos, q, ncar, d, st, sp, lam, NULL);
    int rc = nl < 0 ? -1 : or_rhs_lines(in, n, voltages, ncond, st, sp, lam, nl, soft, b);
    if (rc == 0) {
        or_lu_solve(n, LU, piv, b);
        rc = or_eval(in, n, b, lattice, lo, hi, pos, ncar, NULL, Ee);
    }
    if (rc == 0) {
        or_line_charge(st, sp, lam, nl, pos, ncar, soft, 1, NULL, Ee);
        for (int64_t c = 0; c < ncar; ++c) {
            double sg = (q[c] > 0.0) ? 1.0 : ((q[c] < 0.0) ? -1.0 : 0.0);
            for (int k = 0; k < 3; ++k) {
                if (E_out) E_out[3 * c + k] = Ee[3 * c + k];
                pos[3 * c + k] += sg * mu * Ee[3 * c + k] * dt;
            }
        }
        if (sigma_out) memcpy(sigma_out, b, sizeof(double) * (size_t)n);
    }
    free(st);
    free(sp);
    free(lam);
    free(b);
    free(Ee);
    return rc;
}

/* ---------------------------------------------------------------------------------
 * Adaptive Modelling (Sec. 3.3; PrimAfter in Sec. 5.3.1): far copies of the periodic
 * structure are represented by whole primitives carrying their average charge density.
 * Readings fixed here where the paper is silent:
 *   - a primitive is a flat polygon (rectangle, triangle or convex quadrilateral) that
 *     the elements assigned to it tile; prim_of[j] is the primitive of element j, or -1
 *     when element j belongs to none (it then stands for itself in every copy);
 *   - the average charge density of primitive p is its total charge over its area,
 *     sigma_p = sum_{j in p} sigma_j A_j / A_p;
 *   - copy k = (k1, k2) of the lattice is distant when its ring index max(|k1|, |k2|)
 *     exceeds prim_after; prim_after < 0 means no copy is distant (plain evaluation);
 *   - the point's potential and field are the element sums over the near copies plus
 *     the primitive sums over the distant copies.
 * ------------------------------------------------------------------------------- */
int or_eval_am(const or_input *in, int64_t n, const double *sigma, const double *lattice, int lo, int hi,
               const or_input *prim, int64_t np, const int32_t *prim_of, int prim_after, const double *pts,
               int64_t npts, double *phi_out, double *E_out) {
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(n ? n : 1));
    or_elem *pe = (or_elem *)malloc(sizeof(or_elem) * (size_t)(np ? np : 1));
    double *psig = (double *)calloc((size_t)(np ? np : 1), sizeof(double));
    double *parea = (double *)calloc((size_t)(np ? np : 1), sizeof(double));
    int rc = or_build(in, n, el);
    if (rc == 0 && np > 0) rc = or_build(prim, np, pe) ? -1 : 0;
    for (int64_t j = 0; rc == 0 && j < n; ++j) {
        if (prim_of[j] < -1 || prim_of[j] >= np) rc = -2;
        else if (prim_of[j] >= 0) {
            psig[prim_of[j]] += sigma[j] * el[j].area;
            parea[prim_of[j]] += el[j].area;
        }
    }
    for (int64_t p = 0; rc == 0 && p < np; ++p) {
        if (fabs(parea[p] - pe[p].area) > 1e-9 * pe[p].area) rc = -3; /* elements do not tile it */
        psig[p] /= pe[p].area;
    }
    int64_t nimg = image_count(lattice, lo, hi);
    int m = hi - lo + 1;
    double *tt = (double *)malloc(sizeof(double) * 3 * (size_t)nimg);
    int *far = (int *)malloc(sizeof(int) * (size_t)nimg);
    or_image_table(lattice, lo, hi, tt);
    for (int64_t k = 0; k < nimg; ++k) {
        int k1 = lattice ? (int)(k / m) + lo : 0, k2 = lattice ? (int)(k % m) + lo : 0;
        int ring = abs(k1) > abs(k2) ? abs(k1) : abs(k2);
        far[k] = (prim_after >= 0 && ring > prim_after);
    }
    double ke = or_ke();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < (rc == 0 ? npts : 0); ++p) {
        double sphi = 0.0, sE[3] = {0.0, 0.0, 0.0};
        for (int64_t k = 0; k < nimg; ++k) {
            double P[3] = {pts[3 * p] - tt[3 * k], pts[3 * p + 1] - tt[3 * k + 1], pts[3 * p + 2] - tt[3 * k + 2]};
            double f, E[3];
            for (int64_t j = 0; j < n; ++j) {
                if (far[k] && prim_of[j] >= 0) continue;
                or_influence(&el[j], P, 0, &f, E);
                sphi += sigma[j] * f;
                for (int c = 0; c < 3; ++c) sE[c] += sigma[j] * E[c];
            }
            if (!far[k]) continue;
            for (int64_t q = 0; q < np; ++q) {
                or_influence(&pe[q], P, 0, &f, E);
                sphi += psig[q] * f;
                for (int c = 0; c < 3; ++c) sE[c] += psig[q] * E[c];
            }
        }
        if (phi_out) phi_out[p] = ke * sphi;
        if (E_out)
            for (int c = 0; c < 3; ++c) E_out[3 * p + c] = ke * sE[c];
    }
    free(el);
    free(pe);
    free(psig);
    free(parea);
    free(tt);
    free(far);
    return rc;
}
