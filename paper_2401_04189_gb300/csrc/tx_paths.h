// Per-call plan shared by the float32 and tensor-core paths.
#pragma once

#include "tx_internal.h"

namespace tx {

enum CallKind { CALL_APPLY = 0, CALL_ENERGY = 1, CALL_GRAD = 2, CALL_VJP = 3 };

struct CallSpec {
    int kind = CALL_APPLY;
    int mode = PAIRS_SUBSET;     // PairMode
    int k0 = 0;                  // first target inside the occupied block (PAIRS_SUBSET)
    int n_occ = 0, n_tgt = 0;
    const float* occ = nullptr;
    const float* tgt = nullptr;
    const float* cot = nullptr;  // cotangent of the apply output (CALL_VJP)
    float* out0 = nullptr;       // apply: K psi_tgt; grad: dE/dpsi; vjp: grad_occ
    float* out1 = nullptr;       // vjp: grad_tgt
    double* e_dev = nullptr;
    int galerkin = 0;            // CALL_APPLY / CALL_ENERGY with the two-sided projection
    int per_pair = 0;            // CALL_APPLY with per-pair Tucker bases (sequentially truncated HOSVD)
};

// per-pair Tucker bases (tx_sthosvd.cu)
size_t sthosvd_floats_per_pair(const tx_ctx* c);
int sthosvd_check(const tx_ctx* c);
int sthosvd_batch(tx_ctx* c, const CallSpec& cs, const PairRec* recs, int p0, int np, float* scratch, double* epart,
                  cudaStream_t s);
// Z[p][t][x][(g,b)] = sum_a M1_p[t][x][a] G[p][(g,b)][a] with per-pair operators (stride per pair)
int simt_expand_mode1_pp(const tx_ctx* c, const float* G, const float* M1, long m1_pair_stride, int nt, float* Z,
                         int np, cudaStream_t s);

// two-sided (Galerkin) projection (tx_galerkin.cu): B_td = U_d^T D_d A_td and D_d^-1 U_d
struct GalerkinOps {
    const float* B[3];           // [T][r_d][r_d], mu_t folded into mode 3
    const float* Ut[3];          // [n_d][r_d]
};
size_t galerkin_operator_floats(const tx_ctx* c);
int galerkin_operators(const tx_ctx* c, float* ops, GalerkinOps* g, cudaStream_t s);
// H[p] = sum_t G[p] x_d B_td (X1, X2: [np][T][r1 r2 r3] scratch)
int galerkin_core(const tx_ctx* c, const GalerkinOps& o, const float* G, float* X1, float* X2, float* H, int np,
                  cudaStream_t s);
// epart[p] = ew_p <G_p, H_p>
int galerkin_core_dot(const tx_ctx* c, const PairRec* recs, int p0, const float* G, const float* H, int np,
                      double* epart, cudaStream_t s);

int run_call(tx_ctx* c, const CallSpec& cs, cudaStream_t s);
int ensure_workspace(tx_ctx* c, size_t bytes);
int ensure_ebatch(tx_ctx* c, int nb);

// tensor-core implementation of one pair batch of a call (tx_tc.cu)
struct BatchBuffers {
    const PairRec* recs;      // the call's pair table
    const PairRec* recs2;     // second table (VJP adjoint pass) or null
    int p0, np;               // pair range of this batch
    char* scratch;            // per-batch scratch
    double* epart;            // energy partials of this batch
};
size_t tc_batch_bytes_per_pair(const tx_ctx* c, int kind);
// float32 building blocks shared with the tensor-core adjoint (tx_paths.cu):
// H[p][(g,b)][a] = sum_{t,x} R[p][t][x][(g,b)] A_t1[x][a]
int simt_adjoint_mode1(const tx_ctx* c, const float* R, float* H, int np, cudaStream_t s);
// Z[p][t][x][(g,b)] = sum_a M1_t[x][a] G[p][(g,b)][a]  (nt terms of M1 = [nt][n1][r1])
int simt_expand_mode1(const tx_ctx* c, const float* G, const float* M1, int nt, float* Z, int np, cudaStream_t s);
long tc_epart_per_pair(const tx_ctx* c);
int tc_run_batch(tx_ctx* c, const CallSpec& cs, const BatchBuffers& b, cudaStream_t s);

}  // namespace tx
