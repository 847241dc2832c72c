// geometry.h -- host-side element-table construction (see geometry.cpp).
#pragma once
#include <string>

#include "nb_internal.h"

namespace nb {

// Build the device record, the interface-row diagonal term and the FP32 far-field nodes
// of one raw element (tier distances in element radii from opt).  Returns NEBEM_OK or an
// error code with a reason in `why`.
int build_element(const nebem_element& r, const nebem_options& opt, Elem& e, double& diag, FarNodes& fn,
                  std::string& why);

// Gauss-Legendre nodes and weights on [0, 1] (m <= 16), by Newton iteration on P_m.
void gauss_legendre01(int m, double* x, double* w);

// Image translations t = k1 a1 + k2 a2, index (k1-lo)*m + (k2-lo); lattice NULL -> one
// zero translation.
int build_images(const double* lattice, int lo, int hi, ImageTable& img, std::string& why);

}  // namespace nb
