// context.h -- the state behind an opaque nebem_ctx (one geometry on one device).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "nb_internal.h"

namespace nb {

// A device allocation (grown on demand).  It owns its memory: freed by release() or when
// the buffer goes out of scope, so an entry point that returns early on an error frees
// its work buffers too.  Not copyable (a copy would free the memory twice).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t ensure(size_t nbytes);
    void release();
    template <typename T>
    T* as() const {
        return static_cast<T*>(ptr);
    }
};

// An element table with an image set, in the form the evaluation kernels take.  The
// pointers are views (the context's own tables, or the own_* buffers).
struct EvalSet {
    int64_t n = 0;
    ImageTable img{};
    NearGrid grid{};
    const Elem* el = nullptr;
    const FarNodes* far = nullptr;
    const double* sigma = nullptr;
    DevBuf own_el, own_far, own_sigma, cjk, cell_start, cell_items;
    void release_all();
};

struct Ctx {
    nebem_options opt{};
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // stage times of the last plain mixed evaluation (FP32 pass, refinement levels 1 and 2)
    cudaEvent_t ev_eval[4] = {nullptr, nullptr, nullptr, nullptr};
    bool eval_timed = false;
    int64_t eval_points_n = 0;
    cudaDeviceProp props{};

    // geometry
    int64_t n = 0;
    ImageTable img{};
    int32_t img_lo = 0, img_hi = 0;  // image index range per lattice axis
    std::vector<Elem> h_el;
    std::vector<int32_t> h_bc, h_cond;
    DevBuf d_el, d_far, d_diag;
    DevBuf d_cjk, d_cell_start, d_cell_items;  // mixed eval: two-float image centroids, near cell list
    NearGrid grid{};

    // boundary conditions and solution
    std::vector<double> voltages;
    bool bc_set = false;
    DevBuf d_sigma;
    bool sigma_valid = false;
    int64_t sigma_version = 0;  // bumped whenever the charge densities or known charges change

    // FastVolume map (node axes and node values), built from sigma_version fv_version
    DevBuf d_fv_ax, d_fv_ay, d_fv_az, d_fv_phi, d_fv_E;
    int32_t fv_dims[3] = {0, 0, 0};
    int64_t fv_version = -1;

    // Adaptive Modelling: element sums over the near copies (am_near), primitive sums with
    // average densities over the distant ones (am_far); CSR lists of the elements (with
    // their areas) whose charge each far entry carries
    bool am_on = false;
    int32_t am_prim_after = -1;
    int64_t am_n_prim = 0;
    EvalSet am_near, am_far;
    DevBuf d_am_start, d_am_items, d_am_elarea, d_am_parea, d_am_tmp;
    int64_t am_sigma_version = -1;

    // mixed fill tables (built on the first mixed fill of a geometry): element records,
    // two-float nodes, tau = t_k . frame, and the cell list for its near radius
    DevBuf d_fill_el, d_fill_nodes, d_fill_tau, d_fill_cell_start, d_fill_cell_items;
    NearGrid fill_grid{};
    bool fill_tables = false;

    // matrix and factors; K_prec = the fill that made K (NEBEM_FP64 or NEBEM_MIXED)
    int K_prec = NEBEM_FP64;
    DevBuf d_K, d_LU64, d_LU32, d_piv64, d_piv32, d_work;
    DevBuf d_perm64, d_perm32, d_swork;  // pivot permutations, solve / residual work space
    bool K_valid = false, fac64_valid = false, fac32_valid = false;
    DevBuf d_b, d_x, d_r, d_r32, d_small;
    // weighting fields: unit right-hand sides, solutions, residuals (n x k), FP32 corrections
    DevBuf d_wB, d_wX, d_wR, d_wR32;

    // evaluation staging (host-pointer variant) and scratch; refine_list = device count of
    // the points the last refined mixed evaluation re-evaluated (inside d_scratch)
    DevBuf d_pts, d_phi, d_E, d_err, d_scratch;
    const int32_t* refine_list = nullptr;
    // error model of the FP32 pass (nebem_set_error_model; default_err_model())
    ErrModel err_model = default_err_model();

    // known-charge set (space charge)
    int64_t n_car = 0;
    double soft = 1e-6;
    int sc_precision = NEBEM_FP64;  // precision of the known-charge RHS term
    DevBuf d_car, d_q, d_car2, d_sc_tgt, d_sc_phi, d_sc_E;
    std::vector<double> h_q;
    // line-charge representation of the known charges (Alg. 3): on when sc_lines
    bool sc_lines = false;
    double voxel[3] = {0.0, 0.0, 0.0};
    DevBuf d_vkeys, d_vflags, d_vbsum, d_vpartial, d_vgrid, d_lines, d_linesf, d_line_vox;

    ~Ctx();
};

int fail(int code, const std::string& msg);
// NEBEM_TOO_LARGE for a count above NEBEM_MAX_COUNT, else 0
int check_count(int64_t n, const char* what);
int cuda_fail(cudaError_t e, const char* where);

// solve.cpp
// K in the given precision; an FP64 matrix also serves a mixed request
int ensure_fill(Ctx* c, int precision, double* ms);
int ensure_factors(Ctx* c, int precision, double* ms);
int build_rhs(Ctx* c);
int solve_with_factors(Ctx* c, int precision, nebem_solve_info* info);
// k weighting-field solutions (unit potential on readout[j], 0 on the other conductors, no
// known charges) into c->d_wX (n x k, column-major) with the retained factors
int weighting_solve(Ctx* c, const int32_t* readout, int k, int precision, nebem_solve_info* info);
// two-float tables of the mixed fill and of the refined evaluation (built on first use)
int ensure_fill_tables(Ctx* c);
// elements only (with images); err (may be NULL, n x 2): per-point error estimates of a
// mixed evaluation (see eval_acc.cu)
int eval_elements(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision, cudaStream_t s,
                  double* err = nullptr);
// one evaluation set (elements or primitives with their images)
int eval_set(Ctx* c, const EvalSet& es, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
             cudaStream_t s);
// am_api.cpp: the adaptive evaluation (near copies by elements, distant ones by primitives)
int eval_adaptive(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision, cudaStream_t s);
// elements + known charges (PFAtPoint)
int eval_points(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision, cudaStream_t s,
                double* err = nullptr);

// spacecharge_api.cpp
int rhs_known_charge(Ctx* c);
int add_known_charge(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
                     cudaStream_t s);
VoxWork vox_work(Ctx* c);

}  // namespace nb
