// Set-up of the 1-D convolution factors, in float64 on the device.
//
// The paper precomputes the quadrature sums of the 1-D convolutions once and reuses them for
// every pair (the rearranged sum after Eq. discInteg).  With nodal quadrature on the grid the
// precomputed quantity is C_td[a][b] = w_b exp(-theta_t (x_a - x_b)^2), and applied to the
// basis it gives A_td = C_td U_d, the 1-D convolutions of the basis functions in Eq. final.
// mu_t is folded into the mode-3 factor in float64 before any rounding.
#include <cuda_runtime.h>

#include "tx_internal.h"

namespace tx {
namespace {

__global__ void k_conv_factor(const double* __restrict__ x, const double* __restrict__ w,
                              const double* __restrict__ U, const double* __restrict__ theta,
                              const double* __restrict__ mu, int n, int r, int fold_mu,
                              double* __restrict__ A64, float* __restrict__ A32) {
    extern __shared__ double kv[];   // [n]: row a of C_td
    const int a = blockIdx.x, t = blockIdx.y;
    const double th = theta[t];
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const double dx = x[a] - x[b];
        kv[b] = w[b] * exp(-th * dx * dx);
    }
    __syncthreads();
    const double scale = fold_mu ? mu[t] : 1.0;
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s = fma(kv[b], U[(long)b * r + k], s);
        s *= scale;
        const long o = ((long)t * n + a) * r + k;
        A64[o] = s;
        A32[o] = (float)s;
    }
}

}  // namespace

int setup_factor_matrices(tx_ctx* c, cudaStream_t s) {
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d], r = c->r[d];
        const size_t smem = sizeof(double) * n;
        k_conv_factor<<<dim3(n, c->T), 128, smem, s>>>(c->d_x[d], c->d_w[d], c->d_U[d], c->d_theta, c->d_mu, n, r,
                                                        d == 2 ? 1 : 0, c->d_A64[d], c->f_A[d]);
        TX_LAUNCHED();
    }
    return TX_OK;
}

}  // namespace tx
