// Per-pair Tucker bases (Eq. TuckerDecompField): the paper decomposes every pair density with
// its own sequentially truncated HOSVD.  For each pair of a batch, in float32 on the CUDA cores:
//   rho = psi_a psi_b                                   (k_pair_density)
//   mode 1: S1 = Gram of the mode-1 unfolding of rho    (k_gram), U1 = its r1 leading
//           eigenvectors (k_jacobi_eig), T1 = rho x1 U1^T                        [a][y][z]
//   mode 2: S2 from T1, U2, T2 = T1 x2 U2^T, stored                              [z][b][a]
//   mode 3: S3 from T2, U3, G = T2 x3 U3^T, stored                               [g][b][a]
//   A_td,ij = C_td U_d,ij for every term                (simt_gemm, mu_t inside C_t3)
//   Z = G x1 A_t1,ij for every term, then modes 2 and 3, the sum over t and the Hadamard
//   epilogue with the per-pair operators                (the float32 path's kernels)
// The eigenvectors come from a cyclic Jacobi method with the round-robin ordering, one CTA per
// matrix held in shared memory (n_d <= 160).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "tx_paths.h"

namespace tx {
namespace {

__global__ void __launch_bounds__(256) k_pair_density(const PairRec* __restrict__ recs, int p0, const float* __restrict__ SA,
                                                      const float* __restrict__ SB, long N3, float* __restrict__ rho) {
    const int p = blockIdx.y;
    const PairRec r = recs[p0 + p];
    const float* a = SA + (long)r.ia * N3;
    const float* b = SB + (long)r.ib * N3;
    float* o = rho + (long)p * N3;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < N3; e += (long)gridDim.x * blockDim.x) o[e] = a[e] * b[e];
}

// S[p][b][b'] = sum_{a < A, c < C} T[p][a][b][c] T[p][a][b'][c]   (32 x 32 output tiles)
__global__ void __launch_bounds__(256) k_gram(const float* __restrict__ T, int A, int B, int C, long t_stride,
                                              float* __restrict__ S, long s_stride) {
    __shared__ float t1[32][33], t2[32][33];
    const int p = blockIdx.z, b0 = blockIdx.y * 32, b1 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;     // 8 rows of 4 outputs
    const float* Tp = T + (long)p * t_stride;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int a = 0; a < A; ++a)
        for (int c0 = 0; c0 < C; c0 += 32) {
            for (int e = threadIdx.x; e < 32 * 32; e += 256) {
                const int bb = e / 32, cc = e % 32, c = c0 + cc;
                const long base = (long)a * B * C + c;
                t1[bb][cc] = (b0 + bb < B && c < C) ? Tp[base + (long)(b0 + bb) * C] : 0.f;
                t2[bb][cc] = (b1 + bb < B && c < C) ? Tp[base + (long)(b1 + bb) * C] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int cc = 0; cc < 32; ++cc) {
                const float v = t2[tx][cc];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] = fmaf(t1[ty * 4 + i][cc], v, acc[i]);
            }
            __syncthreads();
        }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = b0 + ty * 4 + i, q = b1 + tx;
        if (r < B && q < B) S[(long)p * s_stride + (long)r * B + q] = acc[i];
    }
}

// Eigenvectors of the symmetric B x B matrix S[p] (destroyed), one CTA per matrix: cyclic
// Jacobi with the round-robin ordering (Bp = B rounded up to even; a padding index is a
// zero row and column whose rotations are skipped), every round's Bp / 2 disjoint rotations
// applied together, rows then columns.  Sweeps stop when the off-diagonal part is below
// 1e-7 of the whole (at most 20).  U[p] [B][r] receives the eigenvectors of the r largest
// eigenvalues, in descending order.
__global__ void __launch_bounds__(512) k_jacobi_eig(float* __restrict__ S, int B, long s_stride, int r,
                                                    float* __restrict__ U, long u_stride) {
    extern __shared__ float sm[];
    const int Bp = (B + 1) & ~1, ld = Bp + 1, half = Bp / 2;
    float* A = sm;                       // [Bp][ld]
    float* V = A + (size_t)Bp * ld;      // [Bp][ld]
    float* cs = V + (size_t)Bp * ld;     // [half] cosines
    float* sn = cs + half;               // [half] sines
    int* pp = (int*)(sn + half);         // [half]
    int* qq = pp + half;                 // [half]
    __shared__ float red[16];
    __shared__ int stop;
    const float* Sp = S + (long)blockIdx.x * s_stride;
    for (int e = threadIdx.x; e < Bp * Bp; e += blockDim.x) {
        const int i = e / Bp, j = e % Bp;
        A[i * ld + j] = (i < B && j < B) ? Sp[(long)i * B + j] : 0.f;
        V[i * ld + j] = i == j ? 1.f : 0.f;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 20; ++sweep) {
        // off-diagonal and total squared norms
        float off = 0.f, tot = 0.f;
        for (int e = threadIdx.x; e < Bp * Bp; e += blockDim.x) {
            const int i = e / Bp, j = e % Bp;
            const float v = A[i * ld + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            tot += __shfl_down_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off;
        __syncthreads();
        if (threadIdx.x == 0) {
            float so = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) so += red[w];
            red[0] = so;
        }
        __syncthreads();
        const float off_all = red[0];
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
        __syncthreads();
        if (threadIdx.x == 0) {
            float st = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) st += red[w];
            stop = (off_all <= 1e-14f * st) ? 1 : 0;
        }
        __syncthreads();
        if (stop) break;
        for (int round = 0; round < Bp - 1; ++round) {
            // pairs of this round (circle method): position 0 fixed, the rest rotate
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                const int i1 = k == 0 ? 0 : 1 + (k - 1 + round) % (Bp - 1);
                const int i2 = 1 + (Bp - 2 - k + round) % (Bp - 1);
                const int p = min(i1, i2), q = max(i1, i2);
                float c = 1.f, s = 0.f;
                const float apq = A[p * ld + q];
                if (q < B && fabsf(apq) > 1e-30f) {
                    const float tau = (A[q * ld + q] - A[p * ld + p]) / (2.f * apq);
                    const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
                    c = rsqrtf(1.f + t * t);
                    s = t * c;
                }
                pp[k] = p;
                qq[k] = q;
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // rows p, q of A: J^T A
            for (int e = threadIdx.x; e < half * Bp; e += blockDim.x) {
                const int k = e / Bp, j = e % Bp, p = pp[k], q = qq[k];
                const float c = cs[k], s = sn[k];
                const float ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and of V: A J, V J
            for (int e = threadIdx.x; e < half * Bp; e += blockDim.x) {
                const int k = e / Bp, i = e % Bp, p = pp[k], q = qq[k];
                const float c = cs[k], s = sn[k];
                const float ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - s * aq;
                A[i * ld + q] = s * ap + c * aq;
                const float vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - s * vq;
                V[i * ld + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    // order by eigenvalue, descending (ties by index), and keep the first r
    float* Up = U + (long)blockIdx.x * u_stride;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const float li = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < B; ++j) {
            const float lj = A[j * ld + j];
            rank += (lj > li || (lj == li && j < i)) ? 1 : 0;
        }
        if (rank < r)
            for (int row = 0; row < B; ++row) Up[(long)row * r + rank] = V[row * ld + i];
    }
}

size_t jacobi_smem(int B) {
    const int Bp = (B + 1) & ~1;
    return sizeof(float) * ((size_t)2 * Bp * (Bp + 1) + Bp) + sizeof(int) * Bp;
}

}  // namespace

// floats per pair of the per-pair path's batch scratch
size_t sthosvd_floats_per_pair(const tx_ctx* c) {
    const size_t n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const size_t nmax = std::max(n1, std::max(n2, n3));
    return n1 * n2 * n3 +                       // rho
           r1 * n2 * n3 +                       // T1
           n3 * r2 * r1 +                       // T2
           r3 * r2 * r1 +                       // G
           nmax * nmax +                        // Gram matrix
           n1 * r1 + n2 * r2 + n3 * r3 +        // U_d
           T * (n1 * r1 + n2 * r2 + n3 * r3) +  // A_td per pair
           T * n1 * r3 * r2;                    // Z
}

int sthosvd_check(const tx_ctx* c) {
    for (int d = 0; d < 3; ++d)
        if (c->n[d] > 160) return fail(TX_ERR_UNSUPPORTED_SHAPE, "per-pair bases: n_d <= 160 (Jacobi in shared memory)");
    if (c->n[2] > 256) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 path supports n3 <= 256");
    return TX_OK;
}

int sthosvd_batch(tx_ctx* c, const CallSpec& cs, const PairRec* recs, int p0, int np, float* scratch, double* epart,
                  cudaStream_t s) {
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const long N3 = (long)n1 * n2 * n3;
    const int nmax = std::max(n1, std::max(n2, n3));
    float* rho = scratch;
    float* T1 = rho + (size_t)np * N3;
    float* T2 = T1 + (size_t)np * r1 * n2 * n3;
    float* G = T2 + (size_t)np * n3 * r2 * r1;
    float* S = G + (size_t)np * r3 * r2 * r1;
    float* U1 = S + (size_t)np * nmax * nmax;
    float* U2 = U1 + (size_t)np * n1 * r1;
    float* U3 = U2 + (size_t)np * n2 * r2;
    float* A1 = U3 + (size_t)np * n3 * r3;
    float* A2 = A1 + (size_t)np * T * n1 * r1;
    float* A3 = A2 + (size_t)np * T * n2 * r2;
    float* Z = A3 + (size_t)np * T * n3 * r3;
    const bool subset = cs.mode == PAIRS_SUBSET;
    FieldArgs f{};
    f.SA = subset ? cs.occ : cs.tgt;
    f.SB = cs.occ;
    f.MUL0 = cs.occ;
    f.MUL1 = cs.occ;
    f.OUT0 = cs.out0;
    f.OUT1 = cs.out0;
    k_pair_density<<<dim3(64, np), 256, 0, s>>>(recs, p0, f.SA, f.SB, N3, rho);
    TX_LAUNCHED();
    const size_t jsm = jacobi_smem(nmax);
    TX_TRY_CUDA(cudaFuncSetAttribute(k_jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm));
    auto gram_eig = [&](const float* Tt, int A, int B, int C, long t_stride, float* U, int r) -> int {
        k_gram<<<dim3((B + 31) / 32, (B + 31) / 32, np), 256, 0, s>>>(Tt, A, B, C, t_stride, S, (long)nmax * nmax);
        TX_LAUNCHED();
        k_jacobi_eig<<<np, 512, jacobi_smem(B), s>>>(S, B, (long)nmax * nmax, r, U, (long)B * r);
        TX_LAUNCHED();
        return TX_OK;
    };
    // ---- mode 1: T1[a][(y,z)] = sum_x U1[x][a] rho[x][(y,z)]
    TX_TRY(gram_eig(rho, 1, n1, n2 * n3, N3, U1, r1));
    {
        GemmArgs g{};
        g.M = r1; g.N = n2 * n3; g.K = n1;
        g.A = U1; g.a_m = 1; g.a_k = r1; g.a_b1 = 0; g.a_b2 = (long)n1 * r1;
        g.B = rho; g.b_k = (long)n2 * n3; g.b_n = 1; g.b_b1 = 0; g.b_b2 = N3;
        g.C = T1; g.c_m = (long)n2 * n3; g.c_n = 1; g.c_b1 = 0; g.c_b2 = (long)r1 * n2 * n3;
        g.nb1 = 1; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
        TX_TRY(simt_gemm(g, s));
    }
    // ---- mode 2: Gram of T1 [a][y][z] over (a, z); T2[z][b][a] = sum_y U2[y][b] T1[a][y][z]
    TX_TRY(gram_eig(T1, r1, n2, n3, (long)r1 * n2 * n3, U2, r2));
    {
        GemmArgs g{};
        g.M = r2; g.N = n3; g.K = n2;
        g.A = U2; g.a_m = 1; g.a_k = r2; g.a_b1 = 0; g.a_b2 = (long)n2 * r2;
        g.B = T1; g.b_k = n3; g.b_n = 1; g.b_b1 = (long)n2 * n3; g.b_b2 = (long)r1 * n2 * n3;
        g.C = T2; g.c_m = r1; g.c_n = (long)r2 * r1; g.c_b1 = 1; g.c_b2 = (long)n3 * r2 * r1;
        g.nb1 = r1; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
        TX_TRY(simt_gemm(g, s));
    }
    // ---- mode 3: Gram of T2 [z][(b,a)]; G[g][(b,a)] = sum_z U3[z][g] T2[z][(b,a)]
    TX_TRY(gram_eig(T2, 1, n3, r2 * r1, (long)n3 * r2 * r1, U3, r3));
    {
        GemmArgs g{};
        g.M = r3; g.N = r2 * r1; g.K = n3;
        g.A = U3; g.a_m = 1; g.a_k = r3; g.a_b1 = 0; g.a_b2 = (long)n3 * r3;
        g.B = T2; g.b_k = (long)r2 * r1; g.b_n = 1; g.b_b1 = 0; g.b_b2 = (long)n3 * r2 * r1;
        g.C = G; g.c_m = (long)r2 * r1; g.c_n = 1; g.c_b1 = 0; g.c_b2 = (long)r3 * r2 * r1;
        g.nb1 = 1; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
        TX_TRY(simt_gemm(g, s));
    }
    // ---- A_td,ij = C_td U_d,ij for every term (mu_t inside C_t3)
    const float* Us[3] = {U1, U2, U3};
    float* As[3] = {A1, A2, A3};
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d], r = c->r[d];
        GemmArgs g{};
        g.M = n; g.N = r; g.K = n;
        g.A = c->f_C[d]; g.a_m = n; g.a_k = 1; g.a_b1 = (long)n * n; g.a_b2 = 0;
        g.B = Us[d]; g.b_k = r; g.b_n = 1; g.b_b1 = 0; g.b_b2 = (long)n * r;
        g.C = As[d]; g.c_m = r; g.c_n = 1; g.c_b1 = (long)n * r; g.c_b2 = (long)T * n * r;
        g.nb1 = T; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
        TX_TRY(simt_gemm(g, s));
    }
    // ---- expansion with the per-pair operators, Hadamard epilogue
    TX_TRY(simt_expand_mode1_pp(c, G, A1, (long)T * n1 * r1, T, Z, np, s));
    return simt_expand_consume(c, recs, p0, np, f, Z, T, A2, A3, EPI_OUT, epart, s, (long)T * n2 * r2,
                               (long)T * n3 * r3);
}

}  // namespace tx
