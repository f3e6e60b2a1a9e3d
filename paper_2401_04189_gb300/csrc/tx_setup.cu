// Set-up of the 1-D convolution factors, in float64 on the device.
//
// The paper precomputes the quadrature sums of the 1-D convolutions once and reuses them for
// every pair (the rearranged sum after Eq. discInteg).  With nodal quadrature on the grid the
// precomputed quantity is C_td[a][b] = w_b exp(-theta_t (x_a - x_b)^2), and applied to the
// basis it gives A_td = C_td U_d, the 1-D convolutions of the basis functions in Eq. final.
// mu_t is folded into the mode-3 factor in float64 before any rounding.
#include <cuda_runtime.h>

#include <cmath>

#include "tx_internal.h"

namespace tx {
namespace {

__global__ void k_conv_factor(const double* __restrict__ x, const double* __restrict__ w,
                              const double* __restrict__ U, const double* __restrict__ theta,
                              const double* __restrict__ mu, int n, int r, int fold_mu,
                              double* __restrict__ A64, float* __restrict__ A32, float* __restrict__ C32) {
    extern __shared__ double kv[];   // [n]: row a of C_td
    const int a = blockIdx.x, t = blockIdx.y;
    const double th = theta[t];
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const double dx = x[a] - x[b];
        kv[b] = w[b] * exp(-th * dx * dx);
    }
    __syncthreads();
    const double scale = fold_mu ? mu[t] : 1.0;
    if (C32)
        for (int b = threadIdx.x; b < n; b += blockDim.x) C32[((long)t * n + a) * n + b] = (float)(scale * kv[b]);
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s = fma(kv[b], U[(long)b * r + k], s);
        s *= scale;
        const long o = ((long)t * n + a) * r + k;
        A64[o] = s;
        A32[o] = (float)s;
    }
}

// Finite-element quadrature (Eqs. quadVal, discInteg): the 1-D field is interpolated by Lagrange
// elements of order p (element e holds nodes p e .. p e + p) and each convolution integral is
// evaluated with q Gauss-Legendre points per element:
//   C_td[a][b] = sum_{e contains b} sum_q J_e w_q N_b(x_q) exp(-theta_t (x_a - x_q)^2)
__global__ void k_conv_factor_fe(const double* __restrict__ x, const double* __restrict__ U,
                                 const double* __restrict__ theta, const double* __restrict__ mu, int n, int r,
                                 int fold_mu, int p, int q, const double* __restrict__ gx, const double* __restrict__ gw,
                                 double* __restrict__ A64, float* __restrict__ A32, float* __restrict__ C32) {
    extern __shared__ double kv[];   // [n]: row a of C_td
    const int a = blockIdx.x, t = blockIdx.y;
    const double th = theta[t], xa = x[a];
    const int nel = (n - 1) / p;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double v = 0.0;
        // the one or two elements that hold node b
        const int e_hi = min(b / p, nel - 1);
        const int e_lo = (b % p == 0 && b > 0) ? b / p - 1 : e_hi;
        for (int e = e_lo; e <= e_hi; ++e) {
            const int k = b - p * e;                     // local node index in element e
            const double* xe = x + p * e;
            const double xl = xe[0], xr = xe[p], half = 0.5 * (xr - xl), mid = 0.5 * (xl + xr);
            for (int g = 0; g < q; ++g) {
                const double xq = mid + half * gx[g];
                double L = 1.0;
                for (int m = 0; m <= p; ++m)
                    if (m != k) L *= (xq - xe[m]) / (xe[k] - xe[m]);
                const double dx = xa - xq;
                v += half * gw[g] * L * exp(-th * dx * dx);
            }
        }
        kv[b] = v;
    }
    __syncthreads();
    const double scale = fold_mu ? mu[t] : 1.0;
    if (C32)
        for (int b = threadIdx.x; b < n; b += blockDim.x) C32[((long)t * n + a) * n + b] = (float)(scale * kv[b]);
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

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on the Legendre polynomial P_q
// (three-term recurrence for P_q and its derivative), started from cos(pi (i - 1/4) / (q + 1/2)).
static void gauss_legendre(int q, double* xg, double* wg) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; ++i) {
        double z = cos(pi * (i + 0.75) / (q + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        xg[i] = z;
        wg[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int setup_factor_matrices_fe(tx_ctx* c, int order, int points, cudaStream_t s, bool with_c) {
    double hx[64], hw[64];
    gauss_legendre(points, hx, hw);
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 2 * points) != cudaSuccess) {
        cudaGetLastError();
        return fail(TX_ERR_OOM, "quadrature points");
    }
    int st = TX_OK;
    if (cudaMemcpy(d, hx, sizeof(double) * points, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + points, hw, sizeof(double) * points, cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(TX_ERR_CUDA, "quadrature points copy");
    for (int dd = 0; dd < 3 && st == TX_OK; ++dd) {
        const int n = c->n[dd], r = c->r[dd];
        k_conv_factor_fe<<<dim3(n, c->T), 128, sizeof(double) * n, s>>>(c->d_x[dd], c->d_U[dd], c->d_theta, c->d_mu, n, r,
                                                                         dd == 2 ? 1 : 0, order, points, d, d + points,
                                                                         c->d_A64[dd], c->f_A[dd],
                                                                         with_c ? c->f_C[dd] : nullptr);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) st = fail(TX_ERR_CUDA, "k_conv_factor_fe launch");
    }
    cudaStreamSynchronize(s);
    cudaFree(d);
    return st;
}

int setup_factor_matrices(tx_ctx* c, cudaStream_t s, bool with_c) {
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d], r = c->r[d];
        const size_t smem = sizeof(double) * n;
        k_conv_factor<<<dim3(n, c->T), 128, smem, s>>>(c->d_x[d], c->d_w[d], c->d_U[d], c->d_theta, c->d_mu, n, r,
                                                        d == 2 ? 1 : 0, c->d_A64[d], c->f_A[d],
                                                        with_c ? c->f_C[d] : nullptr);
        TX_LAUNCHED();
    }
    return TX_OK;
}

}  // namespace tx

namespace tx {

// float32 copies of the convolution matrices C_td (mu_t folded into mode 3), made on first use
// (the per-pair path needs them) with the context's current quadrature
int ensure_conv_matrices(tx_ctx* c, cudaStream_t s) {
    if (c->c_valid) return TX_OK;
    for (int d = 0; d < 3; ++d)
        if (!c->f_C[d]) {
            if (cudaMalloc(&c->f_C[d], sizeof(float) * (size_t)c->T * c->n[d] * c->n[d]) != cudaSuccess) {
                cudaGetLastError();
                c->f_C[d] = nullptr;
                return fail(TX_ERR_OOM, "convolution matrices");
            }
        }
    if (c->quad_order > 0) TX_TRY(setup_factor_matrices_fe(c, c->quad_order, c->quad_points, s, true));
    else TX_TRY(setup_factor_matrices(c, s, true));
    c->c_valid = true;
    return TX_OK;
}

}  // namespace tx
