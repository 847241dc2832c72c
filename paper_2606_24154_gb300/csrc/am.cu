// am.cu -- device pieces of Adaptive Modelling (Sec. 3.3): the average charge density of
// every primitive (total charge of its elements over its area, summed in a fixed order)
// and the sum of the near-copy and distant-copy parts of an evaluation.
#include "nb_internal.h"

namespace nb {

namespace {

__global__ void k_prim_sigma(const int32_t* __restrict__ start, const int32_t* __restrict__ items,
                             const double* __restrict__ elarea, const double* __restrict__ parea,
                             const double* __restrict__ sigma, int64_t nf, double* __restrict__ sbar) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double q = 0.0;
    for (int32_t t = start[f]; t < start[f + 1]; ++t) {
        const int32_t j = items[t];
        q += sigma[j] * elarea[j];
    }
    sbar[f] = q / parea[f];
}

__global__ void k_add_fields(double* __restrict__ phi, double* __restrict__ E, const double* __restrict__ phi2,
                             const double* __restrict__ E2, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (phi) phi[i] += phi2[i];
    if (E) {
        E[3 * i] += E2[3 * i];
        E[3 * i + 1] += E2[3 * i + 1];
        E[3 * i + 2] += E2[3 * i + 2];
    }
}

}  // namespace

cudaError_t launch_prim_sigma(const int32_t* start, const int32_t* items, const double* elarea, const double* parea,
                              const double* sigma, int64_t nf, double* sbar, cudaStream_t s) {
    if (nf == 0) return cudaSuccess;
    k_prim_sigma<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(start, items, elarea, parea, sigma, nf, sbar);
    return cudaGetLastError();
}

cudaError_t launch_add_fields(double* phi, double* E, const double* phi2, const double* E2, int64_t n,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_add_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi, E, phi2, E2, n);
    return cudaGetLastError();
}

}  // namespace nb
