// Plain float32 CUDA-core kernels: the reference GPU form of the hot path, and the building
// blocks every precision shares (pair tables, energy reductions).
//
// Steps (arXiv 2401.04189, "Convolution operation"):
//   k_project_s2    rho = psi_a psi_b (pointwise on the nodes), then modes 3 and 2 of the
//                   projection onto the shared Tucker basis (Eq. TuckerDecompField)
//   simt_gemm       mode 1 of the projection; mode 1 of the expansion (Eq. final) for all t
//   k_consume       modes 2 and 3 of the expansion, summed over the Gaussian terms t (Eq. final),
//                   then W -= psi_j * phi (Eq. hadam) and the weighted energy sums
//   k_adjoint_r     the transposed chain used by the gradients (no counterpart in the paper)
#include <cuda_runtime.h>

#include "tx_internal.h"

namespace tx {

// ====================================================================================
// strided batched GEMM: C[b1,b2][m][n] = alpha * sum_k A[m][k] B[k][n] (+ C)
// 64x64 tiles, 16-deep K slices through shared memory, 4x4 outputs per thread
// ====================================================================================
namespace {
constexpr int GT = 64;
constexpr int GK = 16;

__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
    const int b = blockIdx.z;
    const int b1 = b % g.nb1, b2 = b / g.nb1;
    const float* A = g.A + b1 * g.a_b1 + b2 * g.a_b2;
    const float* B = g.B + b1 * g.b_b1 + b2 * g.b_b2;
    float* C = g.C + b1 * g.c_b1 + b2 * g.c_b2;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const bool a_kfast = (g.a_k == 1);
    const bool b_nfast = (g.b_n == 1);
    for (int k0 = 0; k0 < g.K; k0 += GK) {
        for (int e = tid; e < GT * GK; e += 256) {
            int mm, kk;
            if (a_kfast) { mm = e / GK; kk = e % GK; } else { kk = e / GT; mm = e % GT; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < g.M && k < g.K) ? A[m * g.a_m + k * g.a_k] : 0.f;
        }
        for (int e = tid; e < GT * GK; e += 256) {
            int nn, kk;
            if (b_nfast) { kk = e / GT; nn = e % GT; } else { nn = e / GK; kk = e % GK; }
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < g.N && k < g.K) ? B[k * g.b_k + n * g.b_n] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tn + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tm + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tn + 16 * j;
            if (n >= g.N) continue;
            float* dst = C + m * g.c_m + n * g.c_n;
            const float v = g.alpha * acc[i][j];
            *dst = g.accumulate ? (*dst + v) : v;
        }
    }
}

struct Dims {
    int n1, n2, n3, r1, r2, r3;
};

Dims dims_of(const tx_ctx* c) {
    return Dims{c->n[0], c->n[1], c->n[2], c->r[0], c->r[1], c->r[2]};
}

// ====================================================================================
// pair tables
// ====================================================================================
__global__ void k_build_pairs(PairRec* recs, int mode, int role, int n_occ, int n_tgt, int k0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tgt) return;
    long q = (mode == PAIRS_GENERAL) ? (long)i * n_occ : (long)i * n_occ - (long)i * (i - 1) / 2;
    const int g = k0 + i;
    for (int j = 0; j < n_occ; ++j) {
        if (mode == PAIRS_SUBSET && j >= k0 && j < g) continue;   // counted in an earlier row
        PairRec r;
        r.ia = (mode == PAIRS_SUBSET) ? g : i;
        r.ib = j;
        const bool partner = (mode == PAIRS_SUBSET) && j > g && j < k0 + n_tgt;
        if (role == ROLE_APPLY) {
            r.o0 = i; r.m0 = j; r.o1 = partner ? j - k0 : -1; r.m1 = g;
        } else if (role == ROLE_VJP_FWD) {
            r.o0 = j; r.m0 = i; r.o1 = -1; r.m1 = -1;
        } else {
            r.o0 = i; r.m0 = j; r.o1 = j; r.m1 = i;
        }
        r.ew = (mode == PAIRS_SUBSET) ? (j == g ? 1.f : 2.f) : 1.f;
        r.pad = 0;
        recs[q++] = r;
    }
}

// ====================================================================================
// projection, modes 3 and 2, with the pair-density producer fused in
// ====================================================================================
constexpr int PYC = 8;   // y rows of rho staged per step

__global__ void __launch_bounds__(256) k_project_s2(Dims d, const PairRec* __restrict__ recs, int p0,
                                                    const float* __restrict__ SA, const float* __restrict__ SB,
                                                    const float* __restrict__ U2, const float* __restrict__ U3,
                                                    const float* __restrict__ w1, const float* __restrict__ w2,
                                                    const float* __restrict__ w3, int flags,
                                                    float* __restrict__ S2) {
    extern __shared__ float sm[];
    float* U3s = sm;                       // [n3][r3]
    float* S1 = U3s + d.n3 * d.r3;         // [n2][r3]
    float* rc = S1 + d.n2 * d.r3;          // [PYC][n3]
    const int x = blockIdx.x, pl = blockIdx.y;
    const PairRec rec = recs[p0 + pl];
    const long N3 = (long)d.n1 * d.n2 * d.n3;
    const float* a = SA + rec.ia * N3 + (long)x * d.n2 * d.n3;
    const float* b = SB + rec.ib * N3 + (long)x * d.n2 * d.n3;
    const int tid = threadIdx.x;
    for (int e = tid; e < d.n3 * d.r3; e += 256) U3s[e] = U3[e];
    const float wx = (flags & PROD_MULW) ? w1[x] : 1.f;
    for (int y0 = 0; y0 < d.n2; y0 += PYC) {
        __syncthreads();
        for (int e = tid; e < PYC * d.n3; e += 256) {
            const int yy = e / d.n3, z = e % d.n3, y = y0 + yy;
            float v = 0.f;
            if (y < d.n2) {
                v = a[y * d.n3 + z] * b[y * d.n3 + z];
                if (flags & PROD_MULW) v *= wx * w2[y] * w3[z];
            }
            rc[e] = v;
        }
        __syncthreads();
        for (int o = tid; o < PYC * d.r3; o += 256) {
            const int yy = o / d.r3, gg = o % d.r3;
            if (y0 + yy >= d.n2) continue;
            float s = 0.f;
            for (int z = 0; z < d.n3; ++z) s = fmaf(rc[yy * d.n3 + z], U3s[z * d.r3 + gg], s);
            S1[(y0 + yy) * d.r3 + gg] = s;
        }
    }
    __syncthreads();
    float* out = S2 + ((long)pl * d.n1 + x) * d.r3 * d.r2;
    for (int o = tid; o < d.r3 * d.r2; o += 256) {
        const int gg = o / d.r2, bb = o % d.r2;
        float s = 0.f;
        for (int y = 0; y < d.n2; ++y) s = fmaf(U2[y * d.r2 + bb], S1[y * d.r3 + gg], s);
        out[o] = s;
    }
}

// ====================================================================================
// expansion consumer: for each term t, Y_t = Z_t x2 M2_t (for a 32-row y tile of one x
// slice), then phi += Y_t x3 M3_t; epilogue Hadamard-accumulate and energy sums
// ====================================================================================
constexpr int CYT = 32;   // y rows per block
constexpr int CZC = 8;    // z columns per thread (n3 <= 256)

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(256) k_consume(Dims d, const PairRec* __restrict__ recs, int p0,
                                                 const float* __restrict__ Z, int nt,
                                                 const float* __restrict__ M2, const float* __restrict__ M3,
                                                 const float* __restrict__ SA, const float* __restrict__ SB,
                                                 const float* __restrict__ MUL0, const float* __restrict__ MUL1,
                                                 float* __restrict__ OUT0, float* __restrict__ OUT1,
                                                 const float* __restrict__ w1, const float* __restrict__ w2,
                                                 const float* __restrict__ w3, int flags,
                                                 double* __restrict__ epart, long m2_ps, long m3_ps) {
    extern __shared__ float sm[];
    const int ldz = d.r2 + 1;
    const int ld3 = (d.r3 % 2 == 0) ? d.r3 + 1 : d.r3;
    float* Zs = sm;                          // [r3][ldz]
    float* Ys = Zs + d.r3 * ldz;             // [CYT][r3 + 1]
    float* A3s = Ys + CYT * (d.r3 + 1);      // [n3][ld3]
    __shared__ double red[8];
    const int y0 = blockIdx.x * CYT, x = blockIdx.y, pl = blockIdx.z;
    const PairRec rec = recs[p0 + pl];
    const int tid = threadIdx.x, ty = tid >> 5, tz = tid & 31;
    float acc[4][CZC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < CZC; ++c) acc[i][c] = 0.f;
    const long zslice = (long)d.r3 * d.r2;
    for (int t = 0; t < nt; ++t) {
        const float* zt = Z + (((long)pl * nt + t) * d.n1 + x) * zslice;
        const float* m2 = M2 + pl * m2_ps + (long)t * d.n2 * d.r2;
        const float* m3 = M3 + pl * m3_ps + (long)t * d.n3 * d.r3;
        __syncthreads();
        for (int e = tid; e < d.r3 * d.r2; e += 256) Zs[(e / d.r2) * ldz + e % d.r2] = zt[e];
        for (int e = tid; e < d.n3 * d.r3; e += 256) A3s[(e / d.r3) * ld3 + e % d.r3] = m3[e];
        __syncthreads();
        for (int o = tid; o < CYT * d.r3; o += 256) {
            const int yy = o / d.r3, gg = o % d.r3, y = y0 + yy;
            float s = 0.f;
            if (y < d.n2)
                for (int bb = 0; bb < d.r2; ++bb) s = fmaf(m2[y * d.r2 + bb], Zs[gg * ldz + bb], s);
            Ys[yy * (d.r3 + 1) + gg] = s;
        }
        __syncthreads();
        for (int gg = 0; gg < d.r3; ++gg) {
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ys[(ty * 4 + i) * (d.r3 + 1) + gg];
#pragma unroll
            for (int c = 0; c < CZC; ++c) {
                const int z = tz + 32 * c;
                const float bv = (z < d.n3) ? A3s[z * ld3 + gg] : 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][c] = fmaf(a[i], bv, acc[i][c]);
            }
        }
    }
    // epilogue
    const long N3 = (long)d.n1 * d.n2 * d.n3;
    double e = 0.0;
    const float wx = w1[x];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int y = y0 + ty * 4 + i;
        if (y >= d.n2) continue;
        const float wxy = wx * w2[y];
#pragma unroll
        for (int c = 0; c < CZC; ++c) {
            const int z = tz + 32 * c;
            if (z >= d.n3) continue;
            const long idx = ((long)x * d.n2 + y) * d.n3 + z;
            const float phi = acc[i][c];
            const float wv = wxy * w3[z];
            const float f = (flags & EPI_MULW) ? phi * wv : phi;
            if (flags & EPI_OUT) {
                if (rec.o0 >= 0 && OUT0) atomicAdd(OUT0 + rec.o0 * N3 + idx, -MUL0[rec.m0 * N3 + idx] * f);
                if (rec.o1 >= 0 && OUT1) atomicAdd(OUT1 + rec.o1 * N3 + idx, -MUL1[rec.m1 * N3 + idx] * f);
            }
            if (flags & EPI_ENERGY)
                e += (double)wv * (double)SA[rec.ia * N3 + idx] * (double)SB[rec.ib * N3 + idx] * (double)phi;
        }
    }
    if (flags & EPI_ENERGY) {
        const double s = block_sum(e * rec.ew, red);
        if (tid == 0) epart[(long)pl * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// ====================================================================================
// adjoint chain, modes 3 and 2 for every term: R_t[x][g][b] = sum_{y,z} M2_t[y][b] M3_t[z][g] q[x][y][z]
// ====================================================================================
__global__ void __launch_bounds__(256) k_adjoint_r(Dims d, const PairRec* __restrict__ recs, int p0, int nt,
                                                   const float* __restrict__ M2, const float* __restrict__ M3,
                                                   const float* __restrict__ SA, const float* __restrict__ SB,
                                                   const float* __restrict__ w1, const float* __restrict__ w2,
                                                   const float* __restrict__ w3, int flags,
                                                   float* __restrict__ R) {
    extern __shared__ float sm[];
    float* q = sm;                     // [n2][n3]
    float* Q = q + d.n2 * d.n3;        // [n2][r3]
    const int x = blockIdx.x, pl = blockIdx.y;
    const PairRec rec = recs[p0 + pl];
    const long N3 = (long)d.n1 * d.n2 * d.n3;
    const float* a = SA + rec.ia * N3 + (long)x * d.n2 * d.n3;
    const float* b = SB + rec.ib * N3 + (long)x * d.n2 * d.n3;
    const int tid = threadIdx.x;
    const float wx = (flags & PROD_MULW) ? w1[x] : 1.f;
    for (int e = tid; e < d.n2 * d.n3; e += 256) {
        float v = a[e] * b[e];
        if (flags & PROD_MULW) v *= wx * w2[e / d.n3] * w3[e % d.n3];
        q[e] = v;
    }
    for (int t = 0; t < nt; ++t) {
        const float* m2 = M2 + (long)t * d.n2 * d.r2;
        const float* m3 = M3 + (long)t * d.n3 * d.r3;
        __syncthreads();
        for (int o = tid; o < d.n2 * d.r3; o += 256) {
            const int y = o / d.r3, gg = o % d.r3;
            float s = 0.f;
            for (int z = 0; z < d.n3; ++z) s = fmaf(q[y * d.n3 + z], m3[z * d.r3 + gg], s);
            Q[o] = s;
        }
        __syncthreads();
        float* out = R + (((long)pl * nt + t) * d.n1 + x) * d.r3 * d.r2;
        for (int o = tid; o < d.r3 * d.r2; o += 256) {
            const int gg = o / d.r2, bb = o % d.r2;
            float s = 0.f;
            for (int y = 0; y < d.n2; ++y) s = fmaf(m2[y * d.r2 + bb], Q[y * d.r3 + gg], s);
            out[o] = s;
        }
    }
}

// ====================================================================================
// float64 energy reductions in a fixed order
// ====================================================================================
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ src, long count, double* dst) {
    __shared__ double red[8];
    double s = 0.0;
    for (long i = threadIdx.x; i < count; i += 256) s += src[i];
    const double tot = block_sum(s, red);
    if (threadIdx.x == 0) *dst = tot;
}

__global__ void k_finalize(const double* __restrict__ batches, int nb, double scale, double* e_dev) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += batches[i];
    *e_dev = scale * s;
}

// partial[b] = sum over block b's share of the flat index (i, x, y, z) of w(x, y, z) a[i] b[i]:
// float32 within groups of 32 products, float64 across groups and threads
__global__ void __launch_bounds__(256) k_weighted_dot(const float* __restrict__ A, const float* __restrict__ B,
                                                      const float* __restrict__ w1, const float* __restrict__ w2,
                                                      const float* __restrict__ w3, int n1, int n2, int n3, long total,
                                                      double* partial) {
    __shared__ double red[8];
    const long N23 = (long)n2 * n3, N3 = (long)n1 * N23;
    const long stride = (long)gridDim.x * 256;
    double s = 0.0;
    float f = 0.f;
    int cnt = 0;
    for (long i = blockIdx.x * 256L + threadIdx.x; i < total; i += stride) {
        const long r = i % N3;
        const int x = (int)(r / N23), yz = (int)(r - x * N23), y = yz / n3, z = yz - y * n3;
        f += w1[x] * w2[y] * w3[z] * A[i] * B[i];
        if (++cnt == 32) {
            s += (double)f;
            f = 0.f;
            cnt = 0;
        }
    }
    s += (double)f;
    const double tot = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

int smem_attr(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return fail(TX_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    return TX_OK;
}
}  // namespace

// ====================================================================================
// host wrappers
// ====================================================================================
int simt_gemm(const GemmArgs& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return TX_OK;
    dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, g.nb1 * g.nb2);
    const int ps = prof_begin("gemm", s);
    k_gemm<<<grid, 256, 0, s>>>(g);
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

long pair_count(int mode, int n_occ, int n_tgt) {
    if (mode == PAIRS_GENERAL) return (long)n_occ * n_tgt;
    return (long)n_tgt * n_occ - (long)n_tgt * (n_tgt - 1) / 2;
}

int build_pairs(PairRec* d_recs, int mode, int role, int n_occ, int n_tgt, int k0, cudaStream_t s) {
    k_build_pairs<<<(n_tgt + 127) / 128, 128, 0, s>>>(d_recs, mode, role, n_occ, n_tgt, k0);
    TX_LAUNCHED();
    return TX_OK;
}

int simt_project_s2(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f, int flags,
                    float* S2, cudaStream_t s) {
    const Dims d = dims_of(c);
    const size_t smem = sizeof(float) * ((size_t)d.n3 * d.r3 + (size_t)d.n2 * d.r3 + (size_t)PYC * d.n3);
    TX_TRY(smem_attr((const void*)k_project_s2, smem));
    const int ps = prof_begin("project", s);
    k_project_s2<<<dim3(d.n1, np), 256, smem, s>>>(d, recs, p0, f.SA, f.SB, c->f_U[1], c->f_U[2], c->f_w[0],
                                                    c->f_w[1], c->f_w[2], flags, S2);
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

int simt_expand_consume_blocks(const tx_ctx* c) {
    return ((c->n[1] + CYT - 1) / CYT) * c->n[0];
}

int simt_expand_consume(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f, const float* Z,
                        int nterms, const float* M2, const float* M3, int flags, double* epart, cudaStream_t s,
                        long m2_ps, long m3_ps) {
    const Dims d = dims_of(c);
    if (d.n3 > 32 * CZC) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 path supports n3 <= 256");
    const int ld3 = (d.r3 % 2 == 0) ? d.r3 + 1 : d.r3;
    const size_t smem = sizeof(float) * ((size_t)d.r3 * (d.r2 + 1) + (size_t)CYT * (d.r3 + 1) + (size_t)d.n3 * ld3);
    TX_TRY(smem_attr((const void*)k_consume, smem));
    dim3 grid((d.n2 + CYT - 1) / CYT, d.n1, np);
    const int ps = prof_begin("consume", s);
    k_consume<<<grid, 256, smem, s>>>(d, recs, p0, Z, nterms, M2, M3, f.SA, f.SB, f.MUL0, f.MUL1, f.OUT0, f.OUT1,
                                      c->f_w[0], c->f_w[1], c->f_w[2], flags, epart, m2_ps, m3_ps);
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

int simt_adjoint_r(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f, int flags, float* R,
                   cudaStream_t s) {
    const Dims d = dims_of(c);
    const size_t smem = sizeof(float) * ((size_t)d.n2 * d.n3 + (size_t)d.n2 * d.r3);
    if (smem > 220 * 1024) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 adjoint needs n2*(n3+r3) <= 56K");
    TX_TRY(smem_attr((const void*)k_adjoint_r, smem));
    const int ps = prof_begin("adjoint", s);
    k_adjoint_r<<<dim3(d.n1, np), 256, smem, s>>>(d, recs, p0, c->T, c->f_A[1], c->f_A[2], f.SA, f.SB, c->f_w[0],
                                                   c->f_w[1], c->f_w[2], flags, R);
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

int reduce_energy_batch(const double* epart, long count, double* dst, cudaStream_t s) {
    k_reduce<<<1, 256, 0, s>>>(epart, count, dst);
    TX_LAUNCHED();
    return TX_OK;
}

int weighted_dot(const tx_ctx* c, const float* A, const float* B, int count, double* partial, int nblocks, double scale,
                 double* e_dev, cudaStream_t s) {
    const long total = (long)count * c->n[0] * c->n[1] * c->n[2];
    k_weighted_dot<<<nblocks, 256, 0, s>>>(A, B, c->f_w[0], c->f_w[1], c->f_w[2], c->n[0], c->n[1], c->n[2], total,
                                           partial);
    TX_LAUNCHED();
    k_reduce<<<1, 256, 0, s>>>(partial, nblocks, partial + nblocks);
    TX_LAUNCHED();
    return finalize_energy(partial + nblocks, 1, scale, e_dev, s);
}

int finalize_energy(const double* batches, int nb, double scale, double* e_dev, cudaStream_t s) {
    k_finalize<<<1, 1, 0, s>>>(batches, nb, scale, e_dev);
    TX_LAUNCHED();
    return TX_OK;
}

}  // namespace tx
