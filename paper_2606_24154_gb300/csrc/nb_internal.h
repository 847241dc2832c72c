// nb_internal.h -- library-internal types of libnebem (device element table, image
// table, kernel launch wrappers).  Not part of the public C-ABI (include/nebem.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nebem.h"

namespace nb {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEps0 = 8.8541878128e-12;  // F/m, CODATA 2018
constexpr int kMaxImgAxis = 11;
constexpr int kMaxImg = kMaxImgAxis * kMaxImgAxis;

// Device element record (256 bytes), built on the host in FP64.  The element lies in
// the plane y = 0 of its local frame (origin o = v0, ex along v0->v1, ey = unit normal,
// ez = ey x ex) with counter-clockwise local (x, z) vertices (qx, qz).
struct __align__(16) Elem {
    double o[3], ex[3], ey[3], ez[3];  // frame
    double qx[4], qz[4];                // local vertices (nv = 3 or 4)
    double inv_len[4];                  // 1 / edge length, edge i = vertex i -> i+1
    double twoA[2];                     // doubled areas of the fan triangles (0,1,2), (0,2,3)
    double c[3];                        // centroid (global)
    double rho;                         // circumradius about the centroid
    int32_t nv, bc, cond, flags;
};
static_assert(sizeof(Elem) == 256, "Elem must be 256 bytes");

// FP32 far-field shadow of one element for the mixed evaluation: Gauss nodes for four
// distance tiers, and headers.  Tiers by distance d to the image centroid in element
// circumradii rho:
//   tier 0 (d >= ratio_0 rho):    triangle 4-point degree-3 rule, rectangle 2x2 Gauss-Legendre
//   tier a (d >= ratio_a rho):    triangle 6-point degree-4 rule, rectangle 3x3
//   tier b (d >= ratio_b rho):    triangle collapsed 4x4, rectangle 4x4
//   tier c (d >= ratio_near rho): triangle collapsed 6x6, rectangle 6x6
// (quadrilaterals: the rectangle rules on their bilinear map).  Nodes are stored in pairs
// for the packed FP32x2 arithmetic: pair i of a tier is the two float4
//   (sa.x, sb.x, sa.y, sb.y), (sa.z, sb.z, wa, wb)
// with s = centroid - node and w = weight x area; an odd count is padded with a node of
// weight 0 at the position of the last node.  hdr = squared tier distances (tier 0, a, b,
// near) in m^2; n_a = node pairs of tier a (5 rectangle / quadrilateral, 3 triangle).
constexpr int kNodes0 = 4;
constexpr int kNodesA = 9;
constexpr int kNodesB = 16;
constexpr int kNodesC = 36;
constexpr int kPairs0 = 2;
constexpr int kPairsA = 5;
constexpr int kPairsB = 8;
constexpr int kPairsC = 18;
struct __align__(16) FarNodes {
    float4 f[2 * kPairs0];
    float4 a[2 * kPairsA];
    float4 b[2 * kPairsB];
    float4 c[2 * kPairsC];
    float4 hdr;
    int32_t n_a;
    float wcorr;  // area / (tier 0's FP32 weight total) - 1: applied to sigma (geometry.cpp)
    int32_t pad[2];
};

// Mixed-precision fill (Eq. Matrix with far pairs by Gauss rules in two-float arithmetic).
// Pairs are tiered by the distance d from the collocation point to the image centroid, in
// radii rho of the column element:
//   d >= kFillRatioA rho   tier a: rectangle / quadrilateral 3x3, triangle 6-point rule
//   d >= kFillRatioB rho   tier b: 4x4 / collapsed 4x4
//   d >= kFillRatioC rho   tier c: 6x6 / collapsed 6x6
//   nearer                 FP64 closed form
// The rule truncation errors at these distances (worst over thin rectangles, obtuse and
// sliver triangles and skewed quadrilaterals) stay below ~3e-12 of the pair's value.
// Nodes are kept in the element's local (x, z) frame as offsets s = centroid - node; every
// value is stored as an unevaluated sum of two floats (hi + lo), two nodes per record for
// the packed FP32x2 arithmetic (an odd count is padded with a copy of the last node of
// weight 0):
//   q0 = (2 s_x hi, 2 s_z hi) of nodes (a, b) as (a, b, a, b),  q1 = (|s|^2 hi, w hi),
//   q2 = (2 s_x lo, 2 s_z lo),  q3 = (|s|^2 lo, w lo),   w = weight x area.
constexpr double kFillRatioA = 96.0;
constexpr double kFillRatioB = 32.0;
constexpr double kFillRatioC = 6.0;
constexpr int kFillPairsA = 5;  // capacity (3 used by triangles)
constexpr int kFillPairsB = 8;
constexpr int kFillPairsC = 18;
// tier 0 of the mixed evaluation (2x2 / 4-point rule) in the same two-float form, appended
// for the two-float re-evaluation of eval_acc.cu (the fill does not use it)
constexpr int kFillPairs0 = 2;
constexpr int kFillOffB = 4 * kFillPairsA;
constexpr int kFillOffC = 4 * (kFillPairsA + kFillPairsB);
constexpr int kFillOff0 = 4 * (kFillPairsA + kFillPairsB + kFillPairsC);
constexpr int kFillNodeRec = kFillOff0 + 4 * kFillPairs0;  // float4 per element
// Per element: centroid c and frame (ex, ey, ez) as hi + lo floats; hdr = squared tier
// distances (a, b, c) in m^2 and the tier-a node-pair count.
struct __align__(16) FillEl {
    float4 ch, cl;
    float4 exh, exl, eyh, eyl, ezh, ezl;
    float4 hdr;
};

struct ImageTable {
    int32_t n;
    int32_t k0;  // index of the zero translation
    double t[kMaxImg][3];
};

// Uniform grid over the image centroids for the near-pair search of the mixed
// evaluation: cell (x, y, z) = floor((c - origin) * inv_h), edge h >= 1.01 x the largest
// near radius, so every near pair of a point lies in its cell or the 26 neighbours.
struct NearGrid {
    double origin[3];
    double inv_h;
    int32_t dims[3];
    int32_t pad;
};

// Device-side view of one geometry for the evaluation bodies.
struct GeomView {
    const Elem* el;
    const FarNodes* far;
    const float4* cjk;
    const double* sigma;
    const int32_t* cell_start;
    const int32_t* cell_items;
    int64_t n_el;
    int32_t nimg;
    int32_t tile_el;
    NearGrid grid;
};

GeomView make_view(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma, int64_t n_el,
                   const ImageTable& img, const NearGrid& grid, const int32_t* cell_start, const int32_t* cell_items);

// ------------------------------------------------------------------ launchers (.cu)
// Each returns cudaSuccess or the launch error.
cudaError_t launch_eval_f64(const Elem* el, const double* sigma, int64_t n_el, const ImageTable& img,
                            const double* pts, int64_t npts, double* phi, double* E, cudaStream_t s);
// Scratch of one mixed evaluation of npts points: binning (bin counts, keys, the binned
// order), the FP32 pass's error scales ke * (B_phi, B_E, S_phi, S_E) per point, and the
// list and count of the points the refinement re-evaluates.
struct MixedScratch {
    int32_t* count;  // kBins
    int32_t* key;    // npts
    int32_t* order;  // npts
    float4* bound;   // npts
    int32_t* list;   // npts: points of the first refinement level (phi and E)
    int32_t* list2;  // npts: points of the second level
    int32_t* list_p; // npts: points of the first level, phi only
    int32_t* list_e; // npts: points of the first level, E only
    int32_t* n_list; // 4: the lengths of list, list2, list_p, list_e
};
MixedScratch mixed_scratch(void* base, int64_t npts);
// scratch bytes a mixed evaluation (FP32 pass and refinement) needs for npts points
size_t eval_mixed_scratch_bytes(int64_t npts);
// FP32 pass (binning, far tiers, FP64 near pairs); fills ms.order and ms.bound
cudaError_t launch_eval_mixed(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma,
                              int64_t n_el, const ImageTable& img, const NearGrid& grid, const int32_t* cell_start,
                              const int32_t* cell_items, const double* pts, int64_t npts, double* phi, double* E,
                              const MixedScratch& ms, cudaStream_t s);
// Tables of the two-float evaluation (the mixed fill's): element records, node records,
// tau = t_k . frame, two-float image centroids, and the cell list with the near radius
// kFillRatioC rho.
struct AccView {
    GeomView view;  // the FP32 pass's tables (tier radii, near cell list) for the first level
    const Elem* el;
    const FarNodes* far;
    const FillEl* fe;
    const float4* nodes;
    const float4* tau;
    const float4* cjk;
    const double* sigma;
    int64_t n_el;
    NearGrid grid;
    const int32_t* cell_start;
    const int32_t* cell_items;
};
// Error model of the FP32 pass: estimate = gamma_r |x| + gamma_b B + gamma_s S for x = phi
// and |E| (B, S: the scales in MixedScratch::bound); defaults in eval_acc.cu.
struct ErrModel {
    double gamma_r, gamma_b, gamma_s;
};
ErrModel default_err_model();
// Refinement after launch_eval_mixed: every point whose estimated error (em, from the
// scales in ms.bound) exceeds tol times its |phi| or |E| is re-evaluated in two-float
// arithmetic with FP64 near pairs, in two levels (eval_acc.cu); err (may be NULL, n x 2)
// receives the estimated absolute error of phi and |E| of every point.  sms =
// multiprocessors of the device.
// ev (may be NULL): two events recorded after the first and after the second level.
// part: refine_part_bytes(npts, sms, n_el) bytes of device scratch for the partial sums of
// the point groups that a level splits over element chunks to keep every block busy.
cudaError_t launch_eval_refine(const AccView& A, const ImageTable& img, const double* pts, int64_t npts,
                               double* phi, double* E, double* err, double tol, const ErrModel& em,
                               const MixedScratch& ms, int sms, cudaStream_t s, cudaEvent_t* ev, void* part);
size_t refine_part_bytes(int64_t npts, int sms, int64_t n_el);
cudaError_t launch_pair_tiers(const FarNodes* far, const float4* cjk, int64_t n_el, int nimg, const double* pts,
                              int64_t npts, uint8_t* codes, cudaStream_t s);
cudaError_t launch_image_centroids(const Elem* el, int64_t n, const ImageTable& img, float4* cjk, cudaStream_t s);
cudaError_t launch_fill_f64(const Elem* el, const double* diag, int64_t n, const ImageTable& img, double* K,
                            cudaStream_t s);
// Mixed fill: far pairs (tiers a-c) write K; near pairs (grid of image centroids with
// the near radius kFillRatioC rho) add their FP64 closed forms afterwards.  tau[j][k] =
// t_k . (ex_j, ey_j, ez_j) as (hi, lo) float4 pairs; nodes of kFillNodeRec float4 per element.
cudaError_t launch_fill_mixed(const Elem* el, const FillEl* fe, const float4* nodes, const float4* tau,
                              const float4* cjk, const double* diag, int64_t n, const ImageTable& img,
                              const NearGrid& grid, const int32_t* cell_start, const int32_t* cell_items, double* K,
                              cudaStream_t s);
cudaError_t launch_element_influence(const Elem* el, int64_t n_el, const double* pts, int64_t npts,
                                     double* phi, double* E, cudaStream_t s);

// C[M x N] -= A[M x 64] * B[64 x N] on tcgen05 tensor cores (TF32 x3 split, FP32
// accumulation); *err is set if a bounded wait gave up.  split (may be NULL): device work
// space of tc_split_bytes(M, N, 1) bytes (256-byte aligned) for the pre-split operand tiles
// of the bulk-asynchronous path, taken when ldc % 4 == 0 and C is 16-byte aligned.
cudaError_t tc_update_f32(int64_t M, int64_t N, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                          int64_t ldc, void* split, int* err, cudaStream_t s);
// C[M x N] -= A[M x K] * B[K x N], K <= 256 (a multiple of 64 unless the bulk path runs), in
// one pass over C: the products of the K/64 chunks accumulate in tensor memory.  split:
// tc_split_bytes(M, N, ceil(K / 64)) bytes.  Without the bulk path: K/64 rank-64 updates.
cudaError_t tc_update_f32_k(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                            int64_t ldb, float* C, int64_t ldc, void* split, int* err, cudaStream_t s);
size_t tc_split_bytes(int64_t M, int64_t N, int kc);

// Dense LU (column-major, lda = n).  d_info: two ints (first zero pivot, tensor-core timeout).  Scratch: pivots int32[n], work as documented in lu.cu.
cudaError_t lu_factor_f64(double* A, int64_t n, int32_t* piv, int nb, double* work, int* d_info,
                          cudaStream_t s);
// polls > 0: poll limit of the software waits (the cooperative panel's grid barrier, the
// triangular sweeps' block flags); 0 = their defaults
cudaError_t lu_factor_f32(float* A, int64_t n, int32_t* piv, int nb, float* work, int* d_info,
                          cudaStream_t s, long long polls = 0);
size_t lu_work_elems(int64_t n, int nb);
// bytes of work space lu_factor_f32 takes (lu_work_elems floats, then the split operands of
// the tensor-core updates)
size_t lu_work_bytes_f32(int64_t n, int nb);
// Solves with the factors: perm from lu_make_perm (b'[i] = b[perm[i]] applies the pivot
// swaps), work of lu_solve_work_bytes(n, sizeof(T)) bytes (16-byte aligned).
cudaError_t lu_make_perm(const int32_t* piv, int64_t n, int32_t* perm, cudaStream_t s);
size_t lu_solve_work_bytes(int64_t n, size_t tsize);
cudaError_t lu_solve_f64(const double* LU, int64_t n, const int32_t* perm, double* b, void* work, cudaStream_t s,
                         long long polls = 0);
cudaError_t lu_solve_f32(const float* LU, int64_t n, const int32_t* perm, float* b, void* work, cudaStream_t s,
                         long long polls = 0);
// the solves' give-up flag (nonzero: a block flag wait ran out and the sweep wrote NaN)
// inside their work space
const int* lu_solve_err_flag(const void* work, int64_t n, size_t tsize);
cudaError_t convert_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
// r = b - K x; work of residual_work_bytes(n) bytes
size_t residual_work_bytes(int64_t n);
cudaError_t gemv_residual(const double* K, int64_t n, const double* x, const double* b, double* r, void* work,
                          cudaStream_t s);
cudaError_t ir_update(double* x, const float* d, int64_t n, double* d_norms, cudaStream_t s);
cudaError_t copy_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
cudaError_t launch_gather(const double* a, const int64_t* idx, int64_t n, double* out, cudaStream_t s);
cudaError_t vec_absmax(const double* a, int64_t n, double* out, cudaStream_t s);
// Several right-hand sides (nrhs columns of leading dimension n, solved in place), each
// column with the single solve's arithmetic (bit for bit); work of
// lu_solve_multi_work_bytes(n, sizeof(T)) bytes, its give-up flag at lu_solve_multi_err_flag.
size_t lu_solve_multi_work_bytes(int64_t n, size_t tsize);
const int* lu_solve_multi_err_flag(const void* work, int64_t n, size_t tsize);
cudaError_t lu_solve_multi_f64(const double* LU, int64_t n, const int32_t* perm, double* B, int64_t nrhs, void* work,
                               cudaStream_t s, long long polls);
cudaError_t lu_solve_multi_f32(const float* LU, int64_t n, const int32_t* perm, float* B, int64_t nrhs, void* work,
                               cudaStream_t s, long long polls);
// R = B - K X per column (bit for bit gemv_residual's), work of residual_multi_work_bytes(n)
size_t residual_multi_work_bytes(int64_t n);
cudaError_t gemv_residual_multi(const double* K, int64_t n, const double* X, int64_t nrhs, const double* B, double* R,
                                void* work, cudaStream_t s);
// X_j += D_j for the columns whose bit is set in active (nrhs <= 64); norms: 2 nrhs doubles
// (max |D_j|, max |X_j|)
cudaError_t ir_update_multi(double* X, const float* D, int64_t n, int64_t nrhs, uint64_t active, double* d_norms,
                            cudaStream_t s);

// space charge (spacecharge.cu)
cudaError_t launch_sc_split(const double* pos, const double* q, int64_t n, float4* hq, float4* lo, cudaStream_t s);
cudaError_t launch_sc_eval(int precision, const double* src, const double* q, const float4* hq, const float4* lo,
                           int64_t nsrc, const double* tgt, int64_t ntgt, int exclude_self, double soft,
                           int accumulate, double* phi, double* E, cudaStream_t s);
cudaError_t launch_rhs_sc(const Elem* el, int64_t n, const double* phi, const double* E, double* b, cudaStream_t s);
cudaError_t launch_centroids(const Elem* el, int64_t n, double* c, cudaStream_t s);
cudaError_t launch_drift(double* pos, const double* q, const double* E, int64_t n, double mu_dt, cudaStream_t s);

// line charges (lines.cu): point -> line reduction (Sec. 4.2, Alg. 3) and line-charge sums
// Grid of the reduction and the resulting line count, kept on the device so that a
// dynamic step needs no host round trip.  err != 0: the grid had too many voxels;
// sticky keeps that flag over a sequence of reductions until the host clears it.
struct VoxGrid {
    double lo[3], d[3];
    long long dims[3];
    long long nvox;
    long long nl;
    int err;
    int sticky;
};
// One line charge: start a, unit direction u, length len, density lam (C/m).
struct __align__(16) LineRec {
    double a[3], lam;
    double u[3], len;
};
// FP32 shadow for the mixed sum: midpoint as two floats (mh.xyz + ml.xyz), half length
// (mh.w), density (ml.w), direction (u.xyz).
struct __align__(16) LineF {
    float4 mh, ml, u;
};
// Device work space of one reduction of n points.
struct VoxWork {
    long long* keys;   // pad_len(n) sort keys (voxel * n + point)
    int* flags;        // n segment heads, scanned in place to line indices
    int* bsum;         // scan block sums, scan_blocks(n)
    double* partial;   // 6 per min/max block
    VoxGrid* grid;     // one
    LineRec* lines;    // n (at most one line per point)
    LineF* linesf;     // n
    long long* line_vox;  // n: flat voxel index of every line (ascending)
};
int64_t vox_pad_len(int64_t n);     // sort length: power of two >= max(n, 2048)
int64_t vox_scan_blocks(int64_t n);
constexpr int64_t kVoxMaxPoints = (int64_t)1 << 26;
cudaError_t launch_voxelize(const double* pos, const double* q, int64_t n, const double d[3], const VoxWork& w,
                            cudaStream_t s);
// phi/E at targets from the lines of w.grid->nl (device count); perm (may be NULL) lists
// the targets in the order the threads take them, as perm[t] % perm_div.
cudaError_t launch_line_eval(int precision, const VoxWork& w, const double* tgt, const long long* perm,
                             int64_t perm_div, int64_t nt, double soft, int accumulate, double* phi, double* E,
                             cudaStream_t s);

// Adaptive Modelling (am.cu): average density of every far entry f,
// sbar[f] = sum_{t in [start[f], start[f+1])} sigma[items[t]] * elarea[items[t]] / parea[f],
// summed in list order; and phi += phi2, E += E2 (either may be NULL).
cudaError_t launch_prim_sigma(const int32_t* start, const int32_t* items, const double* elarea, const double* parea,
                              const double* sigma, int64_t nf, double* sbar, cudaStream_t s);
cudaError_t launch_add_fields(double* phi, double* E, const double* phi2, const double* E2, int64_t n,
                              cudaStream_t s);

// FastVolume (fastvol.cu)
cudaError_t launch_grid_nodes(const double* ax, const double* ay, const double* az, int nx, int ny, int nz,
                              double* pts, cudaStream_t s);
cudaError_t launch_fastvol_lookup(const double* ax, const double* ay, const double* az, int nx, int ny, int nz,
                                  const double* vphi, const double* vE, const double* pts, int64_t n, double* phi,
                                  double* E, cudaStream_t s);

// thread-local last error message
void set_error(const std::string& msg);

}  // namespace nb
