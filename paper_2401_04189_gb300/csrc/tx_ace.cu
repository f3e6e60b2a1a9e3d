// Adaptively compressed exchange (the paper's "ACE implementation" section, Eqs. eta and ace1),
// built on top of the exchange potentials W_i = K psi_i of the hot path:
//
//   M_ij = <psi_i, W_j>_w                 weighted Gram matrix (float32 products, float64 sums)
//   M_s  = (M + M^T) / 2                  (the paper is silent on the asymmetry a truncated Tucker
//                                          rank leaves; the symmetric part is factorised)
//   -M_s = L L^T                          Cholesky, float64 (M_s is negative definite)
//   xi_k = sum_i (L^-1)_ki W_i            the ACE projection vectors
//   V_ACE f = - sum_k xi_k <xi_k, f>_w    the ACE operator applied to a block
//
// The Gram matrices and the two small-by-large products cost O(N^2 n^3) flops, about 0.1% of the
// N^2 / 2 pair potentials behind W, so they run on the CUDA cores: float32 products summed in
// float64 across the grid (the factorisation needs M to about the accuracy of W).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "tx_internal.h"
#include "tx_paths.h"

namespace tx {
namespace {

constexpr int kGramTile = 16;     // 16 x 16 (i, j) outputs per CTA
constexpr int kGramChunk = 32;    // grid points per shared-memory chunk

// partial[s][i][j] = sum over slice s of the grid of w(x) A_i(x) B_j(x): float32 within a chunk
// of 32 points, float64 across chunks
__global__ void __launch_bounds__(256) k_wgram(const float* __restrict__ A, int na, const float* __restrict__ B, int nb,
                                               const float* __restrict__ w1, const float* __restrict__ w2,
                                               const float* __restrict__ w3, int n1, int n2, int n3, long slice,
                                               double* __restrict__ partial) {
    __shared__ float As[kGramTile][kGramChunk + 1], Bs[kGramTile][kGramChunk + 1], ws[kGramChunk];
    const long N3 = (long)n1 * n2 * n3, N23 = (long)n2 * n3;
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    const int i0 = blockIdx.x * kGramTile, j0 = blockIdx.y * kGramTile;
    const long x0 = (long)blockIdx.z * slice, x1 = min(N3, x0 + slice);
    double acc = 0.0;
    for (long xc = x0; xc < x1; xc += kGramChunk) {
        for (int e = threadIdx.x; e < kGramTile * kGramChunk; e += 256) {
            const int r = e / kGramChunk, k = e - r * kGramChunk;
            const long x = xc + k;
            const bool in = x < x1;
            As[r][k] = (in && i0 + r < na) ? A[(long)(i0 + r) * N3 + x] : 0.f;
            Bs[r][k] = (in && j0 + r < nb) ? B[(long)(j0 + r) * N3 + x] : 0.f;
        }
        if (threadIdx.x < kGramChunk) {
            const long x = xc + threadIdx.x;
            float wv = 0.f;
            if (x < x1) {
                const int a = (int)(x / N23), yz = (int)(x - a * N23), b = yz / n3, c = yz - b * n3;
                wv = w1[a] * w2[b] * w3[c];
            }
            ws[threadIdx.x] = wv;
        }
        __syncthreads();
        float f = 0.f;
#pragma unroll 8
        for (int k = 0; k < kGramChunk; ++k) f += ws[k] * As[ti][k] * Bs[tj][k];
        acc += (double)f;
        __syncthreads();
    }
    const int i = i0 + ti, j = j0 + tj;
    if (i < na && j < nb) partial[((long)blockIdx.z * na + i) * nb + j] = acc;
}

// G[i][j] = sum_s partial[s][i][j] (fixed order), and optionally its transpose in float32 scaled
__global__ void k_gram_reduce(const double* __restrict__ partial, int ns, int na, int nb, double* __restrict__ G,
                              float* __restrict__ GTf, float scale) {
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)na * nb) return;
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += partial[(long)k * na * nb + idx];
    if (G) G[idx] = s;
    if (GTf) {
        const int i = (int)(idx / nb), j = (int)(idx - (long)i * nb);
        GTf[(long)j * na + i] = (float)(scale * s);
    }
}

// One CTA: A = -(M + M^T) / 2 in float64, Cholesky A = L L^T in place (lower triangle), then
// Linv = L^-1 (lower triangular), written in float64 and in float32.  flag[0] = 1 + the first
// pivot that is not positive (M not negative definite), else 0.
__global__ void __launch_bounds__(1024) k_ace_factor(const double* __restrict__ M, int N, double* __restrict__ A,
                                                     double* __restrict__ Linv, float* __restrict__ Linv32, int* flag) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (long e = threadIdx.x; e < (long)N * N; e += blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (long)i * N);
        A[e] = -0.5 * (M[(long)i * N + j] + M[(long)j * N + i]);
    }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        const double d = A[(long)k * N + k];
        if (!(d > 0.0)) {
            if (threadIdx.x == 0) bad = k + 1;
            __syncthreads();
            break;
        }
        const double s = sqrt(d);
        __syncthreads();
        for (int i = k + threadIdx.x; i < N; i += blockDim.x) A[(long)i * N + k] = (i == k) ? s : A[(long)i * N + k] / s;
        __syncthreads();
        // trailing update of the lower triangle: A[i][j] -= L[i][k] L[j][k], k < j <= i
        const long m = N - k - 1, cnt = m * (m + 1) / 2;
        for (long e = threadIdx.x; e < cnt; e += blockDim.x) {
            // e -> (ii, jj) with 0 <= jj <= ii < m
            long ii = (long)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
            while (ii * (ii + 1) / 2 > e) --ii;
            while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
            const long jj = e - ii * (ii + 1) / 2;
            const int i = k + 1 + (int)ii, j = k + 1 + (int)jj;
            A[(long)i * N + j] -= A[(long)i * N + k] * A[(long)j * N + k];
        }
        __syncthreads();
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) flag[0] = bad;
        return;
    }
    // Linv column by column (forward substitution), one thread per column
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        for (int i = 0; i < N; ++i) {
            double v = 0.0;
            if (i >= j) {
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) s -= A[(long)i * N + k] * Linv[(long)k * N + j];
                v = s / A[(long)i * N + i];
            }
            Linv[(long)i * N + j] = v;
            Linv32[(long)i * N + j] = (float)v;
        }
    }
    if (threadIdx.x == 0) flag[0] = 0;
}

constexpr int kMixK = 32;     // output orbitals per CTA
constexpr int kMixI = 32;     // input orbitals per shared-memory tile

// out[k][x] = alpha * sum_i C[k][i] X[i][x]  (C float32 [nk][ni], X float32 [ni][N3])
__global__ void __launch_bounds__(256) k_mix(const float* __restrict__ C, int nk, int ni, const float* __restrict__ X,
                                             long N3, float alpha, float* __restrict__ out) {
    __shared__ float Cs[kMixK][kMixI];
    const long x = blockIdx.x * 256L + threadIdx.x;
    const int k0 = blockIdx.y * kMixK;
    float acc[kMixK];
#pragma unroll
    for (int k = 0; k < kMixK; ++k) acc[k] = 0.f;
    for (int i0 = 0; i0 < ni; i0 += kMixI) {
        __syncthreads();
        for (int e = threadIdx.x; e < kMixK * kMixI; e += 256) {
            const int k = e / kMixI, i = e - k * kMixI;
            Cs[k][i] = (k0 + k < nk && i0 + i < ni) ? C[(long)(k0 + k) * ni + i0 + i] : 0.f;
        }
        __syncthreads();
        if (x < N3) {
            const int iend = min(kMixI, ni - i0);
            for (int i = 0; i < iend; ++i) {
                const float v = X[(long)(i0 + i) * N3 + x];
#pragma unroll
                for (int k = 0; k < kMixK; ++k) acc[k] += Cs[k][i] * v;
            }
        }
    }
    if (x < N3)
#pragma unroll
        for (int k = 0; k < kMixK; ++k)
            if (k0 + k < nk) out[(long)(k0 + k) * N3 + x] = alpha * acc[k];
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// weighted Gram matrix of A (na orbitals) and B (nb orbitals) into G (float64 [na][nb]) and/or
// the scaled float32 transpose GTf [nb][na]; partials in `scratch`
int wgram(const tx_ctx* c, const float* A, int na, const float* B, int nb, double* partial, int ns, double* G,
          float* GTf, float scale, cudaStream_t s) {
    const long N3 = (long)c->n[0] * c->n[1] * c->n[2];
    const long slice = (N3 + ns - 1) / ns;
    dim3 grid((unsigned)((na + kGramTile - 1) / kGramTile), (unsigned)((nb + kGramTile - 1) / kGramTile), (unsigned)ns);
    k_wgram<<<grid, 256, 0, s>>>(A, na, B, nb, c->f_w[0], c->f_w[1], c->f_w[2], c->n[0], c->n[1], c->n[2], slice,
                                 partial);
    TX_LAUNCHED();
    const long cnt = (long)na * nb;
    k_gram_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(partial, ns, na, nb, G, GTf, scale);
    TX_LAUNCHED();
    return TX_OK;
}

int mix(const float* C, int nk, int ni, const float* X, long N3, float alpha, float* out, cudaStream_t s) {
    dim3 grid((unsigned)((N3 + 255) / 256), (unsigned)((nk + kMixK - 1) / kMixK));
    k_mix<<<grid, 256, 0, s>>>(C, nk, ni, X, N3, alpha, out);
    TX_LAUNCHED();
    return TX_OK;
}

// grid slices of the Gram kernel: enough CTAs to fill the GPU a few times over
int gram_slices(long N3, int na, int nb) {
    const long tiles = (long)((na + kGramTile - 1) / kGramTile) * ((nb + kGramTile - 1) / kGramTile);
    const long want = std::max<long>(1, (4L * 152 + tiles - 1) / tiles);
    return (int)std::min<long>(want, std::max<long>(1, N3 / 4096));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_orbitals(const float* p, int n, const char* what) {
    if (n < 1 || !p) return fail(TX_ERR_INVALID_ARG, std::string(what) + " is NULL or empty");
    if (!aligned16(p)) return fail(TX_ERR_ALIGNMENT, std::string(what) + " is not 16-byte aligned");
    return TX_OK;
}

}  // namespace
}  // namespace tx

using namespace tx;

extern "C" int tx_ace_projectors(tx_ctx* c, const float* psi_occ, int n_occ, const float* W, float* xi, double* M,
                                 tx_stream_t stream) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    TX_TRY(check_orbitals(psi_occ, n_occ, "psi_occ"));
    TX_TRY(check_orbitals(W, n_occ, "W"));
    TX_TRY(check_orbitals(xi, n_occ, "xi"));
    if (n_occ > 4096) return fail(TX_ERR_UNSUPPORTED_SHAPE, "ACE construction supports at most 4096 orbitals");
    const long N3 = (long)c->n[0] * c->n[1] * c->n[2];
    {
        const uintptr_t bytes = (uintptr_t)n_occ * N3 * sizeof(float);
        const uintptr_t o = (uintptr_t)xi;
        for (const float* in : {psi_occ, W}) {
            const uintptr_t a = (uintptr_t)in;
            if (o < a + bytes && a < o + bytes) return fail(TX_ERR_INVALID_ARG, "xi overlaps psi_occ or W");
        }
    }
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    const int N = n_occ;
    const int ns = gram_slices(N3, N, N);
    const size_t nn = (size_t)N * N;
    const size_t off_part = 0, off_M = up256(sizeof(double) * ns * nn), off_A = off_M + up256(sizeof(double) * nn),
                 off_Li = off_A + up256(sizeof(double) * nn), off_L32 = off_Li + up256(sizeof(double) * nn),
                 off_flag = off_L32 + up256(sizeof(float) * nn), total = off_flag + 256;
    TX_TRY(ensure_workspace(c, total));
    char* ws = c->ws;
    double* partial = (double*)(ws + off_part);
    double* Mw = M ? M : (double*)(ws + off_M);
    int* flag = (int*)(ws + off_flag);
    TX_TRY_CUDA(cudaMemsetAsync(flag, 0xff, sizeof(int), s));
    TX_TRY(wgram(c, psi_occ, N, W, N, partial, ns, Mw, nullptr, 1.f, s));
    k_ace_factor<<<1, 1024, 0, s>>>(Mw, N, (double*)(ws + off_A), (double*)(ws + off_Li), (float*)(ws + off_L32), flag);
    TX_LAUNCHED();
    TX_TRY(mix((const float*)(ws + off_L32), N, N, W, N3, 1.f, xi, s));
    // the factorisation's outcome decides the status: read it back (the call synchronises)
    int h = -1;
    TX_TRY_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    TX_TRY_CUDA(cudaStreamSynchronize(s));
    if (h != 0)
        return fail(TX_ERR_NOT_DEFINITE, "the symmetric part of M = <psi_i, W_j>_w is not negative definite (pivot " +
                                             std::to_string(h - 1) + "); xi is not valid");
    return TX_OK;
}

extern "C" int tx_ace_apply(tx_ctx* c, const float* xi, int n_xi, const float* psi, int n, float* out,
                            tx_stream_t stream) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    TX_TRY(check_orbitals(xi, n_xi, "xi"));
    TX_TRY(check_orbitals(psi, n, "psi"));
    TX_TRY(check_orbitals(out, n, "out"));
    const long N3 = (long)c->n[0] * c->n[1] * c->n[2];
    {
        const uintptr_t o = (uintptr_t)out, ob = (uintptr_t)n * N3 * sizeof(float);
        const uintptr_t a = (uintptr_t)psi, ab = ob;
        const uintptr_t x = (uintptr_t)xi, xb = (uintptr_t)n_xi * N3 * sizeof(float);
        if ((o < a + ab && a < o + ob) || (o < x + xb && x < o + ob))
            return fail(TX_ERR_INVALID_ARG, "out overlaps psi or xi");
    }
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    const int ns = gram_slices(N3, n_xi, n);
    const size_t off_part = 0, off_C = up256(sizeof(double) * ns * (size_t)n_xi * n),
                 total = off_C + up256(sizeof(float) * (size_t)n_xi * n);
    TX_TRY(ensure_workspace(c, total));
    double* partial = (double*)c->ws;
    float* CT = (float*)(c->ws + off_C);   // CT[a][k] = <xi_k, psi_a>_w
    TX_TRY(wgram(c, xi, n_xi, psi, n, partial, ns, nullptr, CT, 1.f, s));
    // out[a] = - sum_k CT[a][k] xi_k
    return mix(CT, n, n_xi, xi, N3, -1.f, out, s);
}
