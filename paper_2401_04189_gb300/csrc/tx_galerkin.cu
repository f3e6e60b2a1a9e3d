// Two-sided (Galerkin) projection of the separable convolution onto the Tucker basis.
//
// The one-sided operator of Eq. final, phi = sum_t mu_t G x_d A_td with G = rho x_d U_d^T, is
// C P with P = (x)_d U_d U_d^T.  Projecting its output as well, with P^* = D^-1 P D (the adjoint
// of P in the inner product weighted by the quadrature weights D), gives
//   phi = P^* C P rho = (sum_t mu_t G x_d B_td) x_d (D_d^-1 U_d),   B_td = U_d^T D_d A_td,
// whose form <sigma, P^* C P rho>_w is symmetric and positive semi-definite, so the exchange
// energy -1/2 sum_ij <G_ij, sum_t mu_t G_ij x_d B_td> is exactly non-positive and is evaluated
// in core space at O(T r^4) per pair.  Everything here runs in float32 on the CUDA cores; the
// projection and the single reconstruction are the float32 path's own kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "tx_paths.h"

namespace tx {
namespace {

// B_td[i][k] = sum_a U_d[a][i] w_d[a] A_td[a][k]  (mu_t is already folded into A_t3), and
// Ut_d[a][k] = U_d[a][k] / w_d[a].  One thread per output element, float64 sums.
__global__ void k_galerkin_operators(const double* __restrict__ U, const double* __restrict__ w,
                                     const double* __restrict__ A64, int n, int r, int T, float* __restrict__ B,
                                     float* __restrict__ Ut) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nb = (long)T * r * r;
    if (e < nb) {
        const int t = (int)(e / ((long)r * r)), i = (int)((e / r) % r), k = (int)(e % r);
        const double* At = A64 + (long)t * n * r;
        double s = 0.0;
        for (int a = 0; a < n; ++a) s = fma(U[(long)a * r + i] * w[a], At[(long)a * r + k], s);
        B[e] = (float)s;
    } else if (e < nb + (long)n * r) {
        const long q = e - nb;
        Ut[q] = (float)(U[q] / w[q / r]);
    }
}

// H[p][e] = sum_t X[p][t][e]
__global__ void k_sum_terms(const float* __restrict__ X, int T, long m, int np, float* __restrict__ H) {
    const long total = (long)np * m;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long p = q / m, e = q % m;
        const float* x = X + (long)p * T * m + e;
        float s = 0.f;
        for (int t = 0; t < T; ++t) s += x[(long)t * m];
        H[q] = s;
    }
}

// epart[p] = ew_p * sum_e G[p][e] H[p][e]   (float64 sum; one block per pair)
__global__ void __launch_bounds__(256) k_core_dot(const PairRec* __restrict__ recs, int p0, const float* __restrict__ G,
                                                  const float* __restrict__ H, long m, double* __restrict__ epart) {
    __shared__ double red[256];
    const int p = blockIdx.x;
    const float* g = G + (long)p * m;
    const float* h = H + (long)p * m;
    double s = 0.0;
    for (long e = threadIdx.x; e < m; e += blockDim.x) s += (double)g[e] * (double)h[e];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) epart[p] = red[0] * (double)recs[p0 + p].ew;
}

}  // namespace

size_t galerkin_operator_floats(const tx_ctx* c) {
    size_t f = 0;
    for (int d = 0; d < 3; ++d) f += (size_t)c->T * c->r[d] * c->r[d] + (size_t)c->n[d] * c->r[d];
    return f;
}

int galerkin_operators(const tx_ctx* c, float* ops, GalerkinOps* g, cudaStream_t s) {
    float* q = ops;
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d], r = c->r[d];
        float* B = q;
        float* Ut = B + (size_t)c->T * r * r;
        q = Ut + (size_t)n * r;
        g->B[d] = B;
        g->Ut[d] = Ut;
        const long total = (long)c->T * r * r + (long)n * r;
        k_galerkin_operators<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(c->d_U[d], c->d_w[d], c->d_A64[d], n, r,
                                                                            c->T, B, Ut);
        TX_LAUNCHED();
    }
    return TX_OK;
}

// H[p] = sum_t G[p] x1 B_t1 x2 B_t2 x3 B_t3, three batched GEMM passes over all terms.  Each pass
// contracts the fastest index of its input and writes the new index slowest, so the layout
// turns [g][b][a] -> [a'][g][b] -> [b'][a'][g] -> [g'][b'][a'] (back to G's own order).
int galerkin_core(const tx_ctx* c, const GalerkinOps& o, const float* G, float* X1, float* X2, float* H, int np,
                  cudaStream_t s) {
    const int r1 = c->r[0], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const long m = (long)r1 * r2 * r3;
    GemmArgs g{};
    g.nb1 = T; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
    // mode 1: X1[p][t][a'][(g,b)] = sum_a B_t1[a'][a] G[p][(g,b)][a]
    g.M = r1; g.N = r3 * r2; g.K = r1;
    g.A = o.B[0]; g.a_m = r1; g.a_k = 1; g.a_b1 = (long)r1 * r1; g.a_b2 = 0;
    g.B = G; g.b_k = 1; g.b_n = r1; g.b_b1 = 0; g.b_b2 = m;
    g.C = X1; g.c_m = (long)r3 * r2; g.c_n = 1; g.c_b1 = m; g.c_b2 = T * m;
    TX_TRY(simt_gemm(g, s));
    // mode 2: X2[p][t][b'][(a',g)] = sum_b B_t2[b'][b] X1[p][t][(a',g)][b]
    g.M = r2; g.N = r1 * r3; g.K = r2;
    g.A = o.B[1]; g.a_m = r2; g.a_k = 1; g.a_b1 = (long)r2 * r2; g.a_b2 = 0;
    g.B = X1; g.b_k = 1; g.b_n = r2; g.b_b1 = m; g.b_b2 = T * m;
    g.C = X2; g.c_m = (long)r1 * r3; g.c_n = 1; g.c_b1 = m; g.c_b2 = T * m;
    TX_TRY(simt_gemm(g, s));
    // mode 3: X1[p][t][g'][(b',a')] = sum_g B_t3[g'][g] X2[p][t][(b',a')][g]   (mu_t inside B_t3)
    g.M = r3; g.N = r2 * r1; g.K = r3;
    g.A = o.B[2]; g.a_m = r3; g.a_k = 1; g.a_b1 = (long)r3 * r3; g.a_b2 = 0;
    g.B = X2; g.b_k = 1; g.b_n = r3; g.b_b1 = m; g.b_b2 = T * m;
    g.C = X1; g.c_m = (long)r2 * r1; g.c_n = 1; g.c_b1 = m; g.c_b2 = T * m;
    TX_TRY(simt_gemm(g, s));
    const long total = np * m;
    const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
    k_sum_terms<<<blocks, 256, 0, s>>>(X1, T, m, np, H);
    TX_LAUNCHED();
    return TX_OK;
}

int galerkin_core_dot(const tx_ctx* c, const PairRec* recs, int p0, const float* G, const float* H, int np,
                      double* epart, cudaStream_t s) {
    const long m = (long)c->r[0] * c->r[1] * c->r[2];
    k_core_dot<<<np, 256, 0, s>>>(recs, p0, G, H, m, epart);
    TX_LAUNCHED();
    return TX_OK;
}

}  // namespace tx
