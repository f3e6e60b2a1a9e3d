// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tuxc.h"   // the public C ABI (include/ is on the include path)

namespace tx {

// ------------------------------------------------------------------------------------
// error reporting (thread-local message, no exceptions across the ABI)
// ------------------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
void count_launch(int k = 1);

// opt-in per-kernel timing (tx_profile_*): returns a slot or -1 when profiling is off
int prof_begin(const char* name, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);

#define TX_TRY_CUDA(call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::tx::fail(TX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TX_TRY(expr)                      \
    do {                                  \
        int s_ = (expr);                  \
        if (s_ != TX_OK) return s_;       \
    } while (0)

// launch bookkeeping: every kernel launch goes through this so a failed launch is caught
#define TX_LAUNCHED()                                                                  \
    do {                                                                               \
        ::tx::count_launch();                                                          \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess)                                                         \
            return ::tx::fail(TX_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------------------------
// pair records: rho = SA[ia] * SB[ib]; out0[o0] -= MUL0[m0] * field; out1[o1] -= MUL1[m1] * field
// (an index < 0 skips that output); ew = energy weight of the pair (1 diagonal, 2 off-diagonal)
// ------------------------------------------------------------------------------------
struct PairRec {
    int ia, ib;
    int o0, m0;
    int o1, m1;
    float ew;
    int pad;
};

// how a pair table is laid out (see build_pairs)
enum PairMode { PAIRS_SUBSET = 0, PAIRS_GENERAL = 1 };
// which indices the outputs use
enum PairRole {
    ROLE_APPLY = 0,      // o0 = target row, m0 = occ j; o1 = partner target (symmetric reuse), m1 = target orbital
    ROLE_VJP_FWD = 1,    // o0 = j (grad_occ), m0 = k (grad_out); no o1
    ROLE_VJP_ADJ = 2     // o0 = k (grad_tgt), m0 = j (occ); o1 = j (grad_occ), m1 = k (tgt)
};

// ------------------------------------------------------------------------------------
// epilogue / producer flags
// ------------------------------------------------------------------------------------
enum : int {
    EPI_MULW = 1,        // multiply the field by the quadrature weight w(x) before the Hadamard product
    EPI_ENERGY = 2,      // accumulate ew * sum_x w * SA * SB * field into the energy partials
    EPI_OUT = 4,         // perform the Hadamard-accumulate into out0 / out1
    PROD_MULW = 8        // multiply the pair density by w(x) (adjoint producer)
};

// ------------------------------------------------------------------------------------
// the context
// ------------------------------------------------------------------------------------
struct TcOperands;   // tensor-core operand copies (tx_tc.cu)

}  // namespace tx

struct tx_ctx {
    uint32_t magic;
    int device;
    int n[3], r[3], T, prec;
    // float64 inputs on the device
    double* d_x[3];
    double* d_w[3];
    double* d_U[3];
    double* d_theta;
    double* d_mu;
    double* d_A64[3];    // [T][n_d][r_d]; mu_t folded into mode 3
    // float32 copies
    float* f_U[3];       // [n_d][r_d]
    float* f_A[3];       // [T][n_d][r_d]; mu_t folded into mode 3
    float* f_w[3];       // [n_d]
    float* f_C[3];       // [T][n_d][n_d] convolution matrices, mu_t folded into mode 3 (per-pair path; lazy)
    bool c_valid;        // f_C matches the current quadrature
    int quad_order, quad_points;   // 0 = nodal quadrature; else finite elements (tx_set_quadrature)
    // tensor-core operands (null for TX_PREC_FP32)
    tx::TcOperands* tc;
    // workspace
    char* ws;
    size_t ws_bytes;
    size_t ws_limit;
    int* d_err;          // device error word (bounded waits)
    double* d_ebatch;    // per-batch energy partial sums
    int ebatch_cap;
    cudaStream_t last_stream;
    int tile_bx, tile_nstage;   // forced expansion tile plan (0 = built-in choice)
    int acc_chunk;              // split precisions: Gaussian terms per phi accumulation chunk (0 = default)
    int consume_form;           // single-pass expansion: 0 = automatic (persistent where it applies), 1 = one CTA per item
    uint64_t gen;               // bumped whenever a device buffer a captured launch may use is freed or replaced
};

namespace tx {

constexpr uint32_t kMagic = 0x54554331u;

// Device error block of a context (int words): [0] code of the first bounded wait that gave up
// (1 = time limit), [1] where, [2] number of best-effort drains that gave up, [4..5] the wait
// limit in ns as a 64-bit value (0 = the built-in 2 s).
constexpr int kErrWords = 8;

// Liveness and buffer generation of contexts: a captured batch graph holds raw device
// pointers of its contexts, so replaying it is refused once any of them was freed or replaced.
void ctx_register(tx_ctx* c);
void ctx_unregister(const tx_ctx* c);
void bump_gen(tx_ctx* c);
// current generation of a live context; 0 if the context was destroyed (or never existed)
uint64_t ctx_generation(const tx_ctx* c);

// Makes a context's device current for the duration of one entry point and restores the
// caller's device on every return path.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    int use(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return fail(TX_ERR_CUDA, "cudaGetDevice failed");
        if (prev != dev) {
            if (cudaSetDevice(dev) != cudaSuccess) return fail(TX_ERR_CUDA, "cudaSetDevice failed");
            switched = true;
        }
        return TX_OK;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

// ------------------------------------------------------------------------------------
// SIMT (float32 CUDA-core) building blocks -- tx_simt.cu
// ------------------------------------------------------------------------------------
struct GemmArgs {
    int M, N, K;
    const float* A; long a_m, a_k, a_b1, a_b2;
    const float* B; long b_k, b_n, b_b1, b_b2;
    float* C; long c_m, c_n, c_b1, c_b2;
    int nb1, nb2;
    float alpha;
    int accumulate;
};
int simt_gemm(const GemmArgs& g, cudaStream_t s);

struct FieldArgs {          // orbital-space arrays of one call
    const float* SA; const float* SB;          // producer sources
    const float* MUL0; const float* MUL1;      // epilogue multipliers
    float* OUT0; float* OUT1;                  // epilogue outputs
};

int build_pairs(PairRec* d_recs, int mode, int role, int n_occ, int n_tgt, int k0, cudaStream_t s);
long pair_count(int mode, int n_occ, int n_tgt);

// forward projection: ws_S2[p][x][g][b] = sum_{y,z} U2[y][b] U3[z][g] rho_p[x][y][z]
int simt_project_s2(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f,
                    int flags, float* S2, cudaStream_t s);
// expansion consumer: modes 2 and 3 for every term, Hadamard epilogue, energy partials
int simt_expand_consume(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f,
                        const float* Z, int nterms, const float* M2, const float* M3, int flags,
                        double* epart, cudaStream_t s, long m2_ps = 0, long m3_ps = 0);
int simt_expand_consume_blocks(const tx_ctx* c);
// adjoint stage: R[p][t][x][g][b] = sum_{y,z} A_t2[y][b] A_t3[z][g] (prod)[x][y][z]
int simt_adjoint_r(const tx_ctx* c, const PairRec* recs, int p0, int np, const FieldArgs& f,
                   int flags, float* R, cudaStream_t s);
// energy reductions
int reduce_energy_batch(const double* epart, long count, double* dst, cudaStream_t s);
int finalize_energy(const double* batches, int nb, double scale, double* e_dev, cudaStream_t s);
// e_dev = scale * sum_i sum_x w(x) A_i(x) B_i(x) over `count` orbitals, reduced in a fixed order
// through partial[0 .. nblocks] (nblocks + 1 doubles of device scratch)
int weighted_dot(const tx_ctx* c, const float* A, const float* B, int count, double* partial, int nblocks, double scale,
                 double* e_dev, cudaStream_t s);

// setup -- tx_setup.cu (with_c: also write the float32 convolution matrices f_C)
int setup_factor_matrices(tx_ctx* c, cudaStream_t s, bool with_c = false);
// the same with finite-element quadrature (Lagrange elements of `order`, `points` Gauss points)
int setup_factor_matrices_fe(tx_ctx* c, int order, int points, cudaStream_t s, bool with_c = false);
// f_C allocated and filled for the context's current quadrature
int ensure_conv_matrices(tx_ctx* c, cudaStream_t s);

// tensor-core path -- tx_tc.cu
int tc_prepare(tx_ctx* c, cudaStream_t s);
int tc_wait_selftest(tx_ctx* c, int hold_tmem, cudaStream_t s);
void tc_release(tx_ctx* c);
bool tc_supported(const tx_ctx* c, std::string* why);

}  // namespace tx
