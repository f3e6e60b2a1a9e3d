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
};

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
