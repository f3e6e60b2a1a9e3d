// Tensor-core path: operand preparation and the per-batch sequence of the forward hot path.
//
//   projection (Eq. TuckerDecompField, shared basis)
//     S1[p][g][x][y] = sum_z rho_p[x][y][z] U3[z][g]        tc_project_mode3 (rho fused in)
//     S2[p][g][b][x] = sum_y S1[p][g][x][y] U2[y][b]        tc_gemm
//     G[p][g][b][a]  = sum_x S2[p][g][b][x] U1[x][a]        tc_gemm
//   expansion (Eq. final)
//     Z[p][t][x][g][b] = sum_a A_t1[x][a] G[p][g][b][a]     tc_gemm, every term t at once
//     modes 2 and 3, the sum over t and the Hadamard/energy epilogue (Eq. hadam): tc_consume
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "tx_paths.h"
#include "tx_tc_common.cuh"
#include "tx_tc_ops.h"

namespace tx {

bool tc_consume_supported(const tx_ctx* c, bool tf32, bool split, std::string* why);

namespace {

// dst[r][c] (row stride ld) = operand(src[r * srs + c * scs]) for r < rows, c < cols
__global__ void k_static_operand(const double* __restrict__ src, long rows, int cols, long srs, long scs, int ld,
                                 int tf32, int split, void* dst, size_t lo_elems) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const long r = i / cols, c = i - r * cols;
    const double v = src[r * srs + c * scs];
    const long o = r * ld + c;
    if (tf32) {
        const float h = tc::tf32_hi((float)v);
        ((float*)dst)[o] = h;
        if (split) ((float*)dst)[o + lo_elems] = tc::tf32_hi((float)(v - (double)h));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
        ((__nv_bfloat16*)dst)[o] = h;
        if (split) ((__nv_bfloat16*)dst)[o + lo_elems] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    }
}

// Self-test of the bounded device wait: one warp holds TMEM columns (when asked) and waits on an
// mbarrier that nothing ever completes.  The wait gives up after the context's limit, records
// the timeout in the error block, and the warp frees its TMEM and returns: the same unwinding
// every pipeline kernel of this library goes through when one of its waits gives up.
__global__ void __launch_bounds__(32, 1) k_wait_selftest(int* err, int hold_tmem) {
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_barrier_init();
    }
    __syncwarp();
    if (hold_tmem) {
        tc::tmem_alloc(&tbase, 32);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncwarp();
    tc::tc_fence_after();
    const bool ok = tc::mbar_wait(&bar, 0, err, 90);   // phase 0 never completes
    (void)__all_sync(0xffffffffu, ok);
    tc::tc_fence_before();
    __syncwarp();
    if (hold_tmem) tc::tmem_dealloc(tbase, 32);
}

// Z of the split precisions: the float32 first-mode product Zf[p][t][x][g][b] (b < r2) rounded
// into the expansion's operand layout Z[p][t][(x, g)][ld_b] as hi + lo parts (lo after the
// batch's hi part), with the b padding zero
__global__ void k_split_z(const float* __restrict__ Zf, long rows, int r2, int ld_b, int tf32, void* Z, size_t lo_elems) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= rows * ld_b) return;
    const long row = i / ld_b;
    const int b = (int)(i - row * ld_b);
    const float v = b < r2 ? Zf[row * r2 + b] : 0.f;
    if (tf32) {
        const float h = tc::tf32_hi(v);
        ((float*)Z)[i] = h;
        ((float*)Z)[i + lo_elems] = tc::tf32_hi(v - h);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        ((__nv_bfloat16*)Z)[i] = h;
        ((__nv_bfloat16*)Z)[i + lo_elems] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

}  // namespace

int tc_wait_selftest(tx_ctx* c, int hold_tmem, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(c->d_err, hold_tmem ? 1 : 0);
    TX_LAUNCHED();
    return TX_OK;
}

TcScratch tc_scratch(const tx_ctx* c) {
    TcScratch s;
    const size_t n1 = c->n[0], n2 = c->n[1], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2];
    s.ld_y = pad8((int)n2);
    s.ld_x = pad8((int)n1);
    const int eb = (c->prec == TX_PREC_TF32 || c->prec == TX_PREC_TF32X3) ? 4 : 2;
    s.ld_a = ldk((int)r1, eb);     // G and Z rows are read by TMA along K: whole 32-byte sectors
    s.ld_b = ldk((int)r2, eb);
    s.s1 = r3 * n1 * s.ld_y;
    s.s2 = r3 * s.ld_b * s.ld_x;
    s.g = r3 * s.ld_b * s.ld_a;
    s.z = (size_t)c->T * n1 * r3 * s.ld_b;
    return s;
}

bool tc_supported(const tx_ctx* c, std::string* why) {
    const bool tf32 = c->prec == TX_PREC_TF32 || c->prec == TX_PREC_TF32X3;
    const bool split = c->prec == TX_PREC_TF32X3 || c->prec == TX_PREC_BF16X3;
    if (c->n[2] % 4) {
        if (why) *why = "tensor-core precisions need n3 % 4 == 0 (16-byte orbital rows for TMA)";
        return false;
    }
    if (c->r[2] > 256) {
        if (why) *why = "tensor-core precisions need r3 <= 256";
        return false;
    }
    if ((long)c->T * c->n[0] > (1L << 30)) {
        if (why) *why = "T * n1 too large";
        return false;
    }
    return tc_consume_supported(c, tf32, split, why);
}

void tc_release(tx_ctx* c) {
    if (!c->tc) return;
    bump_gen(c);
    cudaFree(c->tc->buf);
    if (c->tc->img) cudaFree(c->tc->img);
    delete c->tc;
    c->tc = nullptr;
}

int tc_prepare(tx_ctx* c, cudaStream_t s) {
    tc_release(c);
    bump_gen(c);
    TcOperands* op = new TcOperands();
    op->prec = c->prec;
    op->tf32 = c->prec == TX_PREC_TF32 || c->prec == TX_PREC_TF32X3;
    op->split = c->prec == TX_PREC_TF32X3 || c->prec == TX_PREC_BF16X3;
    op->esize = op->tf32 ? 4 : 2;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2], T = c->T;
    // every static operand row is K padded with zeros to a whole number of 32-byte sectors
    const int eb = op->esize;
    const size_t e_u3 = (size_t)r3 * ldk(n3, eb), e_u2 = (size_t)r2 * ldk(n2, eb), e_u1 = (size_t)r1 * ldk(n1, eb);
    const size_t e_a1 = (size_t)T * n1 * ldk(r1, eb), e_a2 = (size_t)T * n2 * ldk(r2, eb);
    const size_t e_a3 = (size_t)T * n3 * ldk(r3, eb), e_a3f = (size_t)T * n3 * pad8(r3);
    const size_t e_a3t = (size_t)T * r3 * ldk(n3, eb), e_a2t = (size_t)T * r2 * ldk(n2, eb);
    auto al = [](size_t e) { return (e + 127) & ~(size_t)127; };   // 256-byte aligned pieces
    const size_t tot = al(e_u3) + al(e_u2) + al(e_u1) + al(e_a1) + al(e_a2) + al(e_a3) + al(e_a3t) + al(e_a2t);
    // bf16 single pass: the stage-3 B operand also in float32 (TF32), after everything else
    const bool a3f_extra = !op->split && !op->tf32;
    const size_t bytes = tot * op->esize * (op->split ? 2 : 1) + (a3f_extra ? al(e_a3f) * 4 : 0);
    if (cudaMalloc(&op->buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete op;
        return fail(TX_ERR_OOM, "tensor-core operand copies");
    }
    c->tc = op;
    TX_TRY_CUDA(cudaMemsetAsync(op->buf, 0, bytes, s));
    char* p = op->buf;
    auto take = [&](size_t e) {
        void* r = p;
        p += al(e) * op->esize;
        return r;
    };
    op->st.U3T = take(e_u3);
    op->st.U2T = take(e_u2);
    op->st.U1T = take(e_u1);
    op->st.A1s = take(e_a1);
    op->st.A2 = take(e_a2);
    op->st.A3 = take(e_a3);
    op->st.A3T = take(e_a3t);
    op->st.A2T = take(e_a2t);
    op->st.off_lo = tot * op->esize;
    op->st.A3f = a3f_extra ? (void*)(op->buf + tot * op->esize) : (op->split ? nullptr : op->st.A3);
    const size_t lo = tot;   // element offset of every lo copy
    auto conv = [&](const double* src, long rows, int cols, long srs, long scs, int ld, void* dst) -> int {
        const long n = rows * cols;
        k_static_operand<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, rows, cols, srs, scs, ld, op->tf32 ? 1 : 0,
                                                                    op->split ? 1 : 0, dst, lo);
        TX_LAUNCHED();
        return TX_OK;
    };
    // U_d^T: rows r_d, K = n_d  (U_d is [n_d][r_d])
    TX_TRY(conv(c->d_U[2], r3, n3, 1, r3, ldk(n3, eb), op->st.U3T));
    TX_TRY(conv(c->d_U[1], r2, n2, 1, r2, ldk(n2, eb), op->st.U2T));
    TX_TRY(conv(c->d_U[0], r1, n1, 1, r1, ldk(n1, eb), op->st.U1T));
    // A_td: [T][n_d][r_d] -> rows (t, x), K = r_d
    TX_TRY(conv(c->d_A64[0], (long)T * n1, r1, r1, 1, ldk(r1, eb), op->st.A1s));
    TX_TRY(conv(c->d_A64[1], (long)T * n2, r2, r2, 1, ldk(r2, eb), op->st.A2));
    TX_TRY(conv(c->d_A64[2], (long)T * n3, r3, r3, 1, ldk(r3, eb), op->st.A3));
    // the adjoint's transposed operators, one term at a time: rows gamma (beta), K = z (y)
    for (int t = 0; t < T; ++t) {
        TX_TRY(conv(c->d_A64[2] + (size_t)t * n3 * r3, r3, n3, 1, r3, ldk(n3, eb),
                    (char*)op->st.A3T + (size_t)t * r3 * ldk(n3, eb) * op->esize));
        TX_TRY(conv(c->d_A64[1] + (size_t)t * n2 * r2, r2, n2, 1, r2, ldk(n2, eb),
                    (char*)op->st.A2T + (size_t)t * r2 * ldk(n2, eb) * op->esize));
    }
    if (a3f_extra) {
        const long n = (long)T * n3 * r3;
        k_static_operand<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->d_A64[2], (long)T * n3, r3, r3, 1, pad8(r3), 1, 0,
                                                                    op->st.A3f, 0);
        TX_LAUNCHED();
    }
    if (!op->split) TX_TRY(tc_build_operand_image(c, s));
    return TX_OK;
}

// float32 scratch of the split precisions' projection and first expansion mode (elements per pair)
struct SplitF32 {
    size_t s2, g, z;
};
static SplitF32 split_f32(const tx_ctx* c) {
    const size_t n1 = c->n[0], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2];
    return SplitF32{n1 * r3 * r2, r3 * r2 * r1, (size_t)c->T * n1 * r3 * r2};
}

size_t tc_adjoint_bytes_per_pair(const tx_ctx* c);

size_t tc_batch_bytes_per_pair(const tx_ctx* c, int kind) {
    const TcScratch sc = tc_scratch(c);
    const TcOperands* op = c->tc;
    size_t fwd;
    if (op->split) {
        const SplitF32 f = split_f32(c);
        fwd = (f.s2 + f.g + f.z) * sizeof(float) + sc.z * op->esize * 2 + 1024;
    } else {
        fwd = (sc.s1 + sc.s2 + sc.g + sc.z) * op->esize + 1024;
    }
    if (kind == CALL_GRAD || kind == CALL_VJP) return std::max(fwd, tc_adjoint_bytes_per_pair(c));
    return fwd;
}

// G[p][(g,b)][a] = sum_x S2[p][x][(g,b)] U1[x][a]  (float32, mode 1 of the projection)
static int f32_mode1_project(const tx_ctx* c, const float* S2, float* G, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2];
    GemmArgs g{};
    g.M = rr; g.N = r1; g.K = n1;
    g.A = S2; g.a_m = 1; g.a_k = rr; g.a_b2 = (long)n1 * rr;
    g.B = c->f_U[0]; g.b_k = r1; g.b_n = 1;
    g.C = G; g.c_m = r1; g.c_n = 1; g.c_b2 = (long)rr * r1;
    g.nb1 = 1; g.nb2 = np; g.alpha = 1.f;
    return simt_gemm(g, s);
}

// Zf[p][t][x][(g,b)] = sum_a A_t1[x][a] G[p][(g,b)][a]  (float32, mode 1 of the expansion, every term)
static int f32_mode1_expand(const tx_ctx* c, const float* G, float* Z, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2], T = c->T;
    GemmArgs g{};
    g.M = n1; g.N = rr; g.K = r1;
    g.A = c->f_A[0]; g.a_m = r1; g.a_k = 1; g.a_b1 = (long)n1 * r1;
    g.B = G; g.b_k = 1; g.b_n = r1; g.b_b2 = (long)rr * r1;
    g.C = Z; g.c_m = rr; g.c_n = 1; g.c_b1 = (long)n1 * rr; g.c_b2 = (long)T * n1 * rr;
    g.nb1 = T; g.nb2 = np; g.alpha = 1.f;
    return simt_gemm(g, s);
}

long tc_epart_per_pair(const tx_ctx* c) { return tc_consume_blocks(c); }

// The forward hot path of one pair batch (Eq. final, Eq. hadam): pair densities SA[ia] * SB[ib]
// projected onto the core, expanded over every Gaussian term, and out0[o0] -= mul0[m0] * phi,
// out1[o1] -= mul1[m1] * phi (and the energy sums) in the expansion's epilogue.
static int tc_forward(tx_ctx* c, const BatchBuffers& b, const PairRec* recs, const float* SA, int nA, const float* SB,
                      int nB, const float* MUL0, const float* MUL1, float* OUT0, float* OUT1, const OrbCounts& cnt,
                      int flags, bool subset, cudaStream_t s) {
    const TcOperands* op = c->tc;
    const TcScratch sc = tc_scratch(c);
    const int np = b.np;
    const int eb = op->esize;
    const int n1 = c->n[0], n2 = c->n[1], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2], T = c->T;
    if (op->split) {
        // Split precisions: the projection onto the core and the first expansion mode run in
        // float32 on the CUDA cores (13% of the flops on the Pt-shaped block), so that the core
        // and Z carry full float32 precision into the hi + lo split; modes 2 and 3 and the sum
        // over terms run on the tensor cores (tc_consume).
        const SplitF32 f = split_f32(c);
        float* S2f = (float*)b.scratch;
        float* Gf = S2f + (size_t)np * f.s2;
        float* Zf = Gf + (size_t)np * f.g;
        char* Z = (char*)(Zf + (size_t)np * f.z);
        Z = (char*)(((uintptr_t)Z + 255) & ~(uintptr_t)255);
        FieldArgs fa{};
        fa.SA = SA;
        fa.SB = SB;
        TX_TRY(simt_project_s2(c, recs, b.p0, np, fa, 0, S2f, s));
        TX_TRY(f32_mode1_project(c, S2f, Gf, np, s));
        TX_TRY(f32_mode1_expand(c, Gf, Zf, np, s));
        const long rows = (long)np * T * n1 * r3;
        const long nz = rows * sc.ld_b;
        k_split_z<<<(unsigned)((nz + 255) / 256), 256, 0, s>>>(Zf, rows, r2, sc.ld_b, op->tf32 ? 1 : 0, Z,
                                                              (size_t)np * sc.z);
        TX_LAUNCHED();
        return tc_consume(c, recs, b.p0, np, Z, SA, SB, MUL0, MUL1, OUT0, OUT1, cnt, flags, b.epart, s, subset);
    }
    char* S1 = b.scratch;
    char* S2 = S1 + (size_t)np * sc.s1 * eb;
    char* G = S2 + (size_t)np * sc.s2 * eb;
    char* Z = G + (size_t)np * sc.g * eb;
    const int out_type = op->tf32 ? TC_OUT_F32 : TC_OUT_BF16;

    // 1. S1 = rho x3 U3^T (rho = psi_a psi_b formed in the kernel)
    TX_TRY(tc_project_mode3(c, recs, b.p0, np, SA, nA, SB, nB, 0, S1, s));

    // 2. S2[p][g][b][x] = sum_y S1[p][(g,x)][y] U2T[b][y], b < ld_b: the columns past r2 read
    //    rows of U2^T past its end (zero-filled), so the b padding is exact zeros and stays zero
    //    through G and Z (whose rows TMA reads along b in whole 32-byte sectors)
    {
        TcOperand A{S1, nullptr, (uint64_t)n2, (uint64_t)r3 * n1, (uint64_t)np, (uint64_t)sc.ld_y, sc.s1};
        TcOperand B{op->st.U2T, nullptr, (uint64_t)ldk(n2, eb), (uint64_t)r2, 1, (uint64_t)ldk(n2, eb), 0};
        TcGemmArgs g{};
        g.M = r3 * n1; g.N = sc.ld_b; g.K = n2; g.nb1 = np; g.nb2 = 1;
        g.a_z1 = 1;
        g.C = S2; g.rdiv = n1; g.c_mh = (long)sc.ld_b * sc.ld_x; g.c_m = 1; g.c_n = sc.ld_x; g.c_b1 = (long)sc.s2;
        g.c_type = out_type; g.alpha = 1.f; g.err = c->d_err;
        TX_TRY(tc_gemm_launch(A, B, g, op->tf32, false, "tc_proj2", s));
    }
    // 3. G[p][(g,b)][a] = sum_x S2[p][(g,b)][x] U1T[a][x]  (rows (g, b < ld_b), a < ld_a: the
    //    columns past r1 read rows of U1^T past its end, so G's a padding is zeros too)
    {
        TcOperand A{S2, nullptr, (uint64_t)n1, (uint64_t)r3 * sc.ld_b, (uint64_t)np, (uint64_t)sc.ld_x, sc.s2};
        TcOperand B{op->st.U1T, nullptr, (uint64_t)ldk(n1, eb), (uint64_t)r1, 1, (uint64_t)ldk(n1, eb), 0};
        TcGemmArgs g{};
        g.M = r3 * sc.ld_b; g.N = sc.ld_a; g.K = n1; g.nb1 = np; g.nb2 = 1;
        g.a_z1 = 1;
        g.C = G; g.c_m = sc.ld_a; g.c_n = 1; g.c_b1 = (long)sc.g;
        g.c_type = out_type; g.alpha = 1.f; g.err = c->d_err;
        TX_TRY(tc_gemm_launch(A, B, g, op->tf32, false, "tc_proj1", s));
    }
    // 4. Z[p][(t,x)][(g,b)] = sum_a A1s[(t,x)][a] G[p][(g,b)][a]  (b < ld_b, padding included)
    {
        TcOperand A{op->st.A1s, nullptr, (uint64_t)ldk(r1, eb), (uint64_t)T * n1, 1, (uint64_t)ldk(r1, eb), 0};
        TcOperand B{G, nullptr, (uint64_t)sc.ld_a, (uint64_t)r3 * sc.ld_b, (uint64_t)np, (uint64_t)sc.ld_a, sc.g};
        TcGemmArgs g{};
        g.M = T * n1; g.N = r3 * sc.ld_b; g.K = r1; g.nb1 = np; g.nb2 = 1;
        g.b_z1 = 1;
        g.C = Z; g.c_m = (long)r3 * sc.ld_b; g.c_n = 1; g.c_b1 = (long)sc.z;
        g.c_type = out_type; g.alpha = 1.f; g.err = c->d_err;
        TX_TRY(tc_rows_launch(A, B, g, op->tf32, false, "tc_zprod", s));
    }
    // 5. modes 2 and 3 for every term, phi accumulated in TMEM, Hadamard / energy epilogue
    return tc_consume(c, recs, b.p0, np, Z, SA, SB, MUL0, MUL1, OUT0, OUT1, cnt, flags, b.epart, s, subset);
}

// float32 scratch of the adjoint (elements per pair): R [T][n1][r3 r2], H [r3 r2][r1], Z [n1][r3 r2]
struct AdjF32 {
    size_t r, h, z;
};
static AdjF32 adj_f32(const tx_ctx* c) {
    const size_t n1 = c->n[0], r1 = c->r[0], rr = (size_t)c->r[1] * c->r[2];
    return AdjF32{(size_t)c->T * n1 * rr, rr * r1, n1 * rr};
}

// The adjoint of one pair batch (derived; the paper has no gradient): with L = sum_t mu_t
// (x)_d A_td U_d^T, zeta_p = L^T y_p = (x)_d U_d [sum_t mu_t y_p x1 A_t1^T x2 A_t2^T x3 A_t3^T] for the
// pair products y_p = SA[ia] * SB[ib] (* w), then fo.OUT0[o0] -= fo.MUL0[m0] * zeta and
// fo.OUT1[o1] -= fo.MUL1[m1] * zeta.  Modes 3 and 2 of every term (2 n^3 r + 2 n^2 r^2 flops per
// term, the adjoint's dominant work) run on the tensor cores; the sum over terms and x of mode 1
// and the single-term expansion with U run in float32 on the CUDA cores (as the split forms'
// projection does, so that the split forms keep float32 accuracy there).
static int tc_adjoint(tx_ctx* c, const BatchBuffers& b, const PairRec* recs, const float* SA, int nA, const float* SB,
                      int nB, int pflags, const FieldArgs& fo, cudaStream_t s) {
    const TcOperands* op = c->tc;
    const TcScratch sc = tc_scratch(c);
    const int np = b.np;
    const int eb = op->esize, mult = op->split ? 2 : 1;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const long rr = (long)r2 * r3;
    const AdjF32 f = adj_f32(c);
    char* S1 = b.scratch;
    float* R = (float*)(((uintptr_t)(S1 + (size_t)np * sc.s1 * eb * mult) + 255) & ~(uintptr_t)255);
    float* H = R + (size_t)np * f.r;
    float* Z = H + (size_t)np * f.h;
    const int out_type = op->tf32 ? (op->split ? TC_OUT_F32_SPLIT : TC_OUT_F32) : (op->split ? TC_OUT_BF16_SPLIT : TC_OUT_BF16);
    (void)out_type;
    for (int t = 0; t < T; ++t) {
        // S1[p][g][x][y] = sum_z y_p[x][y][z] (mu_t A_t3)[z][g]
        const char* a3t = (const char*)op->st.A3T + (size_t)t * r3 * ldk(n3, eb) * eb;
        TX_TRY(tc_project_mode3(c, recs, b.p0, np, SA, nA, SB, nB, pflags, S1, s, a3t));
        // R[p][t][x][g][b] = sum_y S1[p][(g,x)][y] A_t2[y][b]   (float32)
        const char* a2t = (const char*)op->st.A2T + (size_t)t * r2 * ldk(n2, eb) * eb;
        TcOperand A{S1, op->split ? S1 + (size_t)np * sc.s1 * eb : nullptr, (uint64_t)n2, (uint64_t)r3 * n1, (uint64_t)np,
                    (uint64_t)sc.ld_y, sc.s1};
        TcOperand B{a2t, op->split ? a2t + op->st.off_lo : nullptr, (uint64_t)ldk(n2, eb), (uint64_t)r2, 1,
                    (uint64_t)ldk(n2, eb), 0};
        TcGemmArgs g{};
        g.M = r3 * n1; g.N = r2; g.K = n2; g.nb1 = np; g.nb2 = 1;
        g.a_z1 = 1;
        g.C = R + (size_t)t * n1 * rr; g.rdiv = n1; g.c_mh = r2; g.c_m = rr; g.c_n = 1; g.c_b1 = (long)f.r;
        g.c_type = TC_OUT_F32; g.alpha = 1.f; g.err = c->d_err;
        TX_TRY(tc_gemm_launch(A, B, g, op->tf32, op->split, "tc_adj2", s));
    }
    TX_TRY(simt_adjoint_mode1(c, R, H, np, s));                  // H = sum_{t,x} R A_t1
    TX_TRY(simt_expand_mode1(c, H, c->f_U[0], 1, Z, np, s));     // Z = U1 H
    return simt_expand_consume(c, recs, b.p0, np, fo, Z, 1, c->f_U[1], c->f_U[2], EPI_OUT, b.epart, s);
}

size_t tc_adjoint_bytes_per_pair(const tx_ctx* c) {
    const TcScratch sc = tc_scratch(c);
    const TcOperands* op = c->tc;
    const AdjF32 f = adj_f32(c);
    return sc.s1 * op->esize * (op->split ? 2 : 1) + (f.r + f.h + f.z) * sizeof(float) + 1024;
}

int tc_run_batch(tx_ctx* c, const CallSpec& cs, const BatchBuffers& b, cudaStream_t s) {
    const bool subset = cs.mode == PAIRS_SUBSET;
    switch (cs.kind) {
        case CALL_APPLY:
        case CALL_ENERGY: {
            const float* SA = subset ? cs.occ : cs.tgt;
            const int nA = subset ? cs.n_occ : cs.n_tgt;
            int flags = (cs.kind == CALL_APPLY) ? EPI_OUT : 0;
            if (cs.kind == CALL_ENERGY || cs.e_dev) flags |= EPI_ENERGY;
            // OUT rows: the call's targets (apply only; the energy call writes no W); symmetric
            // pairs: rec.ia == rec.m1 and rec.ib == rec.m0, so the energy factors are the multipliers
            const int nout = cs.out0 ? cs.n_tgt : 0;
            const OrbCounts cnt{nA, cs.n_occ, cs.n_occ, cs.n_occ, nout, nout};
            return tc_forward(c, b, b.recs, SA, nA, cs.occ, cs.n_occ, cs.occ, cs.occ, cs.out0, cs.out0, cnt, flags, subset,
                              s);
        }
        case CALL_GRAD: {
            // dE/dpsi_k = w * W_k - sum_j psi_j * L^T(w * rho_kj): the forward pipeline with the
            // weights folded into the epilogue, then the adjoint of the weighted pair densities
            const int n = cs.n_occ;
            const OrbCounts cnt{n, n, n, n, n, n};
            const int flags = EPI_OUT | EPI_MULW | (cs.e_dev ? EPI_ENERGY : 0);
            TX_TRY(tc_forward(c, b, b.recs, cs.occ, n, cs.occ, n, cs.occ, cs.occ, cs.out0, cs.out0, cnt, flags, true, s));
            FieldArgs fo{};
            fo.MUL0 = cs.occ;
            fo.MUL1 = cs.occ;
            fo.OUT0 = cs.out0;
            fo.OUT1 = cs.out0;
            return tc_adjoint(c, b, b.recs, cs.occ, n, cs.occ, n, PROD_MULW, fo, s);
        }
        case CALL_VJP: {
            if (cs.out0) {
                // grad_occ_j -= cot_k * phi_kj
                const OrbCounts cnt{cs.n_tgt, cs.n_occ, cs.n_tgt, 0, cs.n_occ, 0};
                TX_TRY(tc_forward(c, b, b.recs, cs.tgt, cs.n_tgt, cs.occ, cs.n_occ, cs.cot, nullptr, cs.out0, nullptr, cnt,
                                  EPI_OUT, false, s));
            }
            // zeta_kj = L^T(cot_k psi_j): grad_tgt_k -= psi_j zeta, grad_occ_j -= psi_tgt_k zeta
            FieldArgs fo{};
            fo.MUL0 = cs.occ;
            fo.OUT0 = cs.out1;
            fo.MUL1 = cs.tgt;
            fo.OUT1 = cs.out0;
            return tc_adjoint(c, b, b.recs2, cs.cot, cs.n_tgt, cs.occ, cs.n_occ, 0, fo, s);
        }
    }
    return fail(TX_ERR_INVALID_ARG, "unknown call kind");
}

}  // namespace tx
