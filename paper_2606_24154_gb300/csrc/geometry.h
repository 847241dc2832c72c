// geometry.h -- host-side element-table construction (see geometry.cpp).
#pragma once
#include <string>
#include <vector>

#include "nb_internal.h"

namespace nb {

// Build the device record, the interface-row diagonal term and the FP32 far-field nodes
// of one raw element (tier distances in element radii from opt).  Returns NEBEM_OK or an
// error code with a reason in `why`.
int build_element(const nebem_element& r, const nebem_options& opt, Elem& e, double& diag, FarNodes& fn,
                  std::string& why);

// Gauss-Legendre nodes and weights on [0, 1] (m <= 16), by Newton iteration on P_m.
void gauss_legendre01(int m, double* x, double* w);

// Cell list of the image centroids c_j + t_k (entry j * nimg + k) for the near-pair search;
// near radius of element j = ratio_near * rho_j.  Cells in x-fastest order, CSR form.
int build_near_grid(const std::vector<Elem>& el, const ImageTable& img, double ratio_near, NearGrid& grid,
                    std::vector<int32_t>& cell_start, std::vector<int32_t>& cell_items, std::string& why);

// Tables of the mixed fill: per element the FillEl record and kFillNodeRec float4 of
// two-float Gauss nodes (local frame); per (element, image) the two float4 of
// tau = t_k . (ex, ey, ez) (hi, lo).
void build_fill_tables(const std::vector<Elem>& el, const ImageTable& img, std::vector<FillEl>& fe,
                       std::vector<float4>& nodes, std::vector<float4>& tau);

// Image translations t = k1 a1 + k2 a2, index (k1-lo)*m + (k2-lo); lattice NULL -> one
// zero translation.
int build_images(const double* lattice, int lo, int hi, ImageTable& img, std::string& why);

}  // namespace nb
