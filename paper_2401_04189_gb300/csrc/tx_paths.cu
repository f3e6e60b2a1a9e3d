// Per-call plan: pair table, pair batches that fit the workspace, and the sequence of steps
// for apply / energy / gradient / VJP.  The float32 path is written out here; the tensor-core
// precisions hand each pair batch to tc_run_batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "tx_paths.h"

namespace tx {
namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct SimtLayout {
    size_t s2, g, z;   // floats per pair
};

SimtLayout simt_layout(const tx_ctx* c) {
    const size_t n1 = c->n[0], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2];
    SimtLayout L;
    L.s2 = n1 * r3 * r2;
    L.g = r3 * r2 * r1;
    L.z = (size_t)c->T * n1 * r3 * r2;
    return L;
}

// G[p][(g,b)][a] = sum_x S2[p][x][(g,b)] M1[x][a]   (mode 1 of the projection; M1 = U1)
int gemm_mode1_project(const tx_ctx* c, const float* S2, const float* M1, float* G, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2];
    GemmArgs g{};
    g.M = rr; g.N = r1; g.K = n1;
    g.A = S2; g.a_m = 1; g.a_k = rr; g.a_b1 = 0; g.a_b2 = (long)n1 * rr;
    g.B = M1; g.b_k = r1; g.b_n = 1; g.b_b1 = 0; g.b_b2 = 0;
    g.C = G; g.c_m = r1; g.c_n = 1; g.c_b1 = 0; g.c_b2 = (long)rr * r1;
    g.nb1 = 1; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
    return simt_gemm(g, s);
}

// H[p][(g,b)][a] = sum_{t,x} R[p][t][x][(g,b)] A_t1[x][a]   (mode 1 of the adjoint, summed over t)
int gemm_mode1_adjoint(const tx_ctx* c, const float* R, float* H, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2], T = c->T;
    GemmArgs g{};
    g.M = rr; g.N = r1; g.K = T * n1;
    g.A = R; g.a_m = 1; g.a_k = rr; g.a_b1 = 0; g.a_b2 = (long)T * n1 * rr;
    g.B = c->f_A[0]; g.b_k = r1; g.b_n = 1; g.b_b1 = 0; g.b_b2 = 0;
    g.C = H; g.c_m = r1; g.c_n = 1; g.c_b1 = 0; g.c_b2 = (long)rr * r1;
    g.nb1 = 1; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
    return simt_gemm(g, s);
}

// Z[p][t][x][(g,b)] = sum_a M1_t[x][a] G[p][(g,b)][a]   (mode 1 of the expansion, every term;
// M1 per pair when m1_ps > 0)
int gemm_mode1_expand(const tx_ctx* c, const float* G, const float* M1, int nt, float* Z, int np, cudaStream_t s,
                      long m1_ps = 0) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2];
    GemmArgs g{};
    g.M = n1; g.N = rr; g.K = r1;
    g.A = M1; g.a_m = r1; g.a_k = 1; g.a_b1 = (long)n1 * r1; g.a_b2 = m1_ps;
    g.B = G; g.b_k = 1; g.b_n = r1; g.b_b1 = 0; g.b_b2 = (long)rr * r1;
    g.C = Z; g.c_m = rr; g.c_n = 1; g.c_b1 = (long)n1 * rr; g.c_b2 = (long)nt * n1 * rr;
    g.nb1 = nt; g.nb2 = np; g.alpha = 1.f; g.accumulate = 0;
    return simt_gemm(g, s);
}

int simt_batch(tx_ctx* c, const CallSpec& cs, const PairRec* recs, const PairRec* recs2, int p0, int np,
               float* S2, float* G, float* Z, double* epart, cudaStream_t s) {
    const bool subset = cs.mode == PAIRS_SUBSET;
    FieldArgs f{};
    switch (cs.kind) {
        case CALL_APPLY:
        case CALL_ENERGY:
        case CALL_GRAD: {
            f.SA = subset ? cs.occ : cs.tgt;
            f.SB = cs.occ;
            f.MUL0 = cs.occ;
            f.MUL1 = cs.occ;
            f.OUT0 = cs.out0;
            f.OUT1 = cs.out0;
            TX_TRY(simt_project_s2(c, recs, p0, np, f, 0, S2, s));
            TX_TRY(gemm_mode1_project(c, S2, c->f_U[0], G, np, s));
            TX_TRY(gemm_mode1_expand(c, G, c->f_A[0], c->T, Z, np, s));
            int flags = 0;
            if (cs.kind == CALL_APPLY) flags = EPI_OUT | (cs.e_dev ? EPI_ENERGY : 0);
            if (cs.kind == CALL_ENERGY) flags = EPI_ENERGY;
            if (cs.kind == CALL_GRAD) flags = EPI_OUT | EPI_MULW | (cs.e_dev ? EPI_ENERGY : 0);
            TX_TRY(simt_expand_consume(c, recs, p0, np, f, Z, c->T, c->f_A[1], c->f_A[2], flags, epart, s));
            if (cs.kind == CALL_GRAD) {
                // second term: - sum_j psi_j * L^T(w rho_kj)
                TX_TRY(simt_adjoint_r(c, recs, p0, np, f, PROD_MULW, Z, s));
                TX_TRY(gemm_mode1_adjoint(c, Z, G, np, s));
                TX_TRY(gemm_mode1_expand(c, G, c->f_U[0], 1, Z, np, s));
                TX_TRY(simt_expand_consume(c, recs, p0, np, f, Z, 1, c->f_U[1], c->f_U[2], EPI_OUT, epart, s));
            }
            return TX_OK;
        }
        case CALL_VJP: {
            if (cs.out0) {
                // grad_occ_j -= cot_k * phi_kj
                f.SA = cs.tgt; f.SB = cs.occ;
                f.MUL0 = cs.cot; f.OUT0 = cs.out0;
                f.MUL1 = nullptr; f.OUT1 = nullptr;
                TX_TRY(simt_project_s2(c, recs, p0, np, f, 0, S2, s));
                TX_TRY(gemm_mode1_project(c, S2, c->f_U[0], G, np, s));
                TX_TRY(gemm_mode1_expand(c, G, c->f_A[0], c->T, Z, np, s));
                TX_TRY(simt_expand_consume(c, recs, p0, np, f, Z, c->T, c->f_A[1], c->f_A[2], EPI_OUT, epart, s));
            }
            // zeta_kj = L^T(cot_k psi_j): grad_tgt_k -= psi_j zeta, grad_occ_j -= psi_tgt_k zeta
            FieldArgs f2{};
            f2.SA = cs.cot; f2.SB = cs.occ;
            f2.MUL0 = cs.occ; f2.OUT0 = cs.out1;
            f2.MUL1 = cs.tgt; f2.OUT1 = cs.out0;
            TX_TRY(simt_adjoint_r(c, recs2, p0, np, f2, 0, Z, s));
            TX_TRY(gemm_mode1_adjoint(c, Z, G, np, s));
            TX_TRY(gemm_mode1_expand(c, G, c->f_U[0], 1, Z, np, s));
            TX_TRY(simt_expand_consume(c, recs2, p0, np, f2, Z, 1, c->f_U[1], c->f_U[2], EPI_OUT, epart, s));
            return TX_OK;
        }
    }
    return fail(TX_ERR_INVALID_ARG, "unknown call kind");
}

// One pair batch with the two-sided projection: the float32 projection, the core-space
// convolution, then either the core-space energy or one reconstruction with D^-1 U and the
// Hadamard epilogue.
int galerkin_batch(tx_ctx* c, const CallSpec& cs, const GalerkinOps& o, const PairRec* recs, int p0, int np,
                   float* S2, float* G, float* H, float* X1, float* X2, double* epart, cudaStream_t s) {
    const bool subset = cs.mode == PAIRS_SUBSET;
    FieldArgs f{};
    f.SA = subset ? cs.occ : cs.tgt;
    f.SB = cs.occ;
    f.MUL0 = cs.occ;
    f.MUL1 = cs.occ;
    f.OUT0 = cs.out0;
    f.OUT1 = cs.out0;
    TX_TRY(simt_project_s2(c, recs, p0, np, f, 0, S2, s));
    TX_TRY(gemm_mode1_project(c, S2, c->f_U[0], G, np, s));
    TX_TRY(galerkin_core(c, o, G, X1, X2, H, np, s));
    if (cs.kind == CALL_ENERGY) return galerkin_core_dot(c, recs, p0, G, H, np, epart, s);
    float* Z = S2;   // [np][1][n1][r3 r2]: the size of S2
    TX_TRY(gemm_mode1_expand(c, H, o.Ut[0], 1, Z, np, s));
    return simt_expand_consume(c, recs, p0, np, f, Z, 1, o.Ut[1], o.Ut[2], EPI_OUT, epart, s);
}

}  // namespace

int simt_adjoint_mode1(const tx_ctx* c, const float* R, float* H, int np, cudaStream_t s) {
    return gemm_mode1_adjoint(c, R, H, np, s);
}
int simt_expand_mode1(const tx_ctx* c, const float* G, const float* M1, int nt, float* Z, int np, cudaStream_t s) {
    return gemm_mode1_expand(c, G, M1, nt, Z, np, s);
}
int simt_expand_mode1_pp(const tx_ctx* c, const float* G, const float* M1, long m1_pair_stride, int nt, float* Z,
                         int np, cudaStream_t s) {
    return gemm_mode1_expand(c, G, M1, nt, Z, np, s, m1_pair_stride);
}

int run_call(tx_ctx* c, const CallSpec& cs, cudaStream_t s) {
    const long N3 = (long)c->n[0] * c->n[1] * c->n[2];
    const long P = pair_count(cs.mode, cs.n_occ, cs.n_tgt);
    // every call kind of a tensor-core precision runs the tensor-core kernels (the adjoint's
    // first-mode sum over the terms and its single-term expansion run in float32)
    // (the two-sided projection runs in float32 on the CUDA cores in every precision)
    const bool gk = cs.galerkin != 0;
    const bool pp = cs.per_pair != 0;
    const bool tc = c->prec != TX_PREC_FP32 && !gk && !pp;
    const int ntables = cs.kind == CALL_VJP ? 2 : 1;
    const size_t recs_bytes = align_up(sizeof(PairRec) * (size_t)P, 256) * ntables;
    const size_t prefix = gk ? align_up(sizeof(float) * galerkin_operator_floats(c), 256) : 0;
    size_t per_pair;
    long epp;
    SimtLayout L = simt_layout(c);
    if (pp) {
        TX_TRY(sthosvd_check(c));
        per_pair = sizeof(float) * sthosvd_floats_per_pair(c);
        epp = simt_expand_consume_blocks(c);
    } else if (gk) {
        per_pair = sizeof(float) * (L.s2 + 2 * L.g + 2 * (size_t)c->T * L.g);
        epp = cs.kind == CALL_ENERGY ? 1 : simt_expand_consume_blocks(c);
    } else if (tc) {
        per_pair = tc_batch_bytes_per_pair(c, cs.kind);
        epp = tc_epart_per_pair(c);
    } else {
        per_pair = sizeof(float) * (L.s2 + L.g + L.z);
        epp = simt_expand_consume_blocks(c);
    }
    per_pair += sizeof(double) * epp;
    size_t avail = c->ws_limit > recs_bytes + prefix + 4096 ? c->ws_limit - recs_bytes - prefix - 4096 : 0;
    long Pb = std::max<long>(1, std::min<long>(P, (long)(avail / per_pair)));
    Pb = std::min<long>(Pb, 65535 / std::max(1, c->T));   // grid.z of the per-term GEMMs is T * pairs
    const long nb = (P + Pb - 1) / Pb;
    const size_t batch_bytes = align_up((size_t)Pb * per_pair, 256) + 4096;
    TX_TRY(ensure_workspace(c, recs_bytes + prefix + batch_bytes));
    TX_TRY(ensure_ebatch(c, (int)nb));
    char* base = c->ws;
    PairRec* recs = (PairRec*)base;
    PairRec* recs2 = ntables == 2 ? (PairRec*)(base + recs_bytes / 2) : nullptr;
    char* scratch = base + recs_bytes + prefix;
    GalerkinOps gops{};
    if (gk) TX_TRY(galerkin_operators(c, (float*)(base + recs_bytes), &gops, s));
    if (pp) TX_TRY(ensure_conv_matrices(c, s));

    // zero the outputs that are accumulated into
    if (cs.kind == CALL_APPLY) TX_TRY_CUDA(cudaMemsetAsync(cs.out0, 0, sizeof(float) * N3 * cs.n_tgt, s));
    if (cs.kind == CALL_GRAD) TX_TRY_CUDA(cudaMemsetAsync(cs.out0, 0, sizeof(float) * N3 * cs.n_occ, s));
    if (cs.kind == CALL_VJP) {
        if (cs.out0) TX_TRY_CUDA(cudaMemsetAsync(cs.out0, 0, sizeof(float) * N3 * cs.n_occ, s));
        if (cs.out1) TX_TRY_CUDA(cudaMemsetAsync(cs.out1, 0, sizeof(float) * N3 * cs.n_tgt, s));
    }
    if (cs.kind == CALL_VJP) {
        TX_TRY(build_pairs(recs, PAIRS_GENERAL, ROLE_VJP_FWD, cs.n_occ, cs.n_tgt, 0, s));
        TX_TRY(build_pairs(recs2, PAIRS_GENERAL, ROLE_VJP_ADJ, cs.n_occ, cs.n_tgt, 0, s));
    } else {
        TX_TRY(build_pairs(recs, cs.mode, ROLE_APPLY, cs.n_occ, cs.n_tgt, cs.k0, s));
    }
    const bool energy = (cs.kind == CALL_ENERGY) || (!gk && !pp && (cs.kind == CALL_GRAD || cs.kind == CALL_APPLY) && cs.e_dev);
    for (long b = 0; b < nb; ++b) {
        const int p0 = (int)(b * Pb);
        const int np = (int)std::min<long>(Pb, P - p0);
        double* epart = (double*)(scratch + align_up((size_t)Pb * (per_pair - sizeof(double) * epp), 256));
        if (pp) {
            TX_TRY(sthosvd_batch(c, cs, recs, p0, np, (float*)scratch, epart, s));
        } else if (gk) {
            float* S2 = (float*)scratch;
            float* G = S2 + (size_t)Pb * L.s2;
            float* H = G + (size_t)Pb * L.g;
            float* X1 = H + (size_t)Pb * L.g;
            float* X2 = X1 + (size_t)Pb * c->T * L.g;
            TX_TRY(galerkin_batch(c, cs, gops, recs, p0, np, S2, G, H, X1, X2, epart, s));
        } else if (tc) {
            BatchBuffers bb{recs, recs2, p0, np, scratch, epart};
            TX_TRY(tc_run_batch(c, cs, bb, s));
        } else {
            float* S2 = (float*)scratch;
            float* G = S2 + (size_t)Pb * L.s2;
            float* Z = G + (size_t)Pb * L.g;
            TX_TRY(simt_batch(c, cs, recs, recs2, p0, np, S2, G, Z, epart, s));
        }
        if (energy) TX_TRY(reduce_energy_batch(epart, (long)np * epp, c->d_ebatch + b, s));
    }
    if (energy) TX_TRY(finalize_energy(c->d_ebatch, (int)nb, -0.5, cs.e_dev, s));
    return TX_OK;
}

}  // namespace tx
