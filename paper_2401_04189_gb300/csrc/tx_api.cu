// The C ABI: argument validation, context and workspace management, and the per-call
// dispatch of the hot path (pair tables, pair batches, projection, expansion, epilogues).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "tx_internal.h"
#include "tx_paths.h"

namespace tx {

static thread_local std::string g_err;
static thread_local uint64_t g_launches = 0;

void set_error(const std::string& m) { g_err = m; }
int fail(int status, const std::string& m) {
    g_err = m;
    return status;
}
void count_launch(int k) { g_launches += (uint64_t)k; }

// ---- opt-in per-kernel timing --------------------------------------------------------
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
static thread_local bool g_prof_on = false;
static thread_local std::vector<ProfRec> g_prof;
static thread_local size_t g_prof_used = 0;

int prof_begin(const char* name, cudaStream_t s) {
    if (!g_prof_on) return -1;
    if (g_prof_used == g_prof.size()) {
        ProfRec r;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        g_prof.push_back(r);
    }
    ProfRec& r = g_prof[g_prof_used];
    r.name = name;
    if (cudaEventRecord(r.a, s) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int)g_prof_used++;
}

void prof_end(int slot, cudaStream_t s) {
    if (slot < 0) return;
    if (cudaEventRecord(g_prof[slot].b, s) != cudaSuccess) cudaGetLastError();
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int check_ctx(const tx_ctx* c) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    return TX_OK;
}

// ---- context registry (liveness and buffer generation) ---------------------------------
static std::mutex g_ctx_mu;
static std::unordered_map<const tx_ctx*, uint64_t> g_ctx_gen;
static uint64_t g_gen_counter = 0;

void ctx_register(tx_ctx* c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    c->gen = ++g_gen_counter;
    g_ctx_gen[c] = c->gen;
}
void ctx_unregister(const tx_ctx* c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    g_ctx_gen.erase(c);
}
void bump_gen(tx_ctx* c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    c->gen = ++g_gen_counter;
    auto it = g_ctx_gen.find(c);
    if (it != g_ctx_gen.end()) it->second = c->gen;
}
uint64_t ctx_generation(const tx_ctx* c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    auto it = g_ctx_gen.find(c);
    return it == g_ctx_gen.end() ? 0 : it->second;
}

int ensure_workspace(tx_ctx* c, size_t bytes) {
    if (bytes <= c->ws_bytes) return TX_OK;
    bump_gen(c);
    if (c->ws) {
        cudaError_t e = cudaFree(c->ws);   // synchronises the device
        c->ws = nullptr;
        c->ws_bytes = 0;
        if (e != cudaSuccess) return fail(TX_ERR_CUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&c->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->ws = nullptr;
        return fail(TX_ERR_OOM, "workspace of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    c->ws_bytes = bytes;
    return TX_OK;
}

int ensure_ebatch(tx_ctx* c, int nb) {
    if (nb <= c->ebatch_cap) return TX_OK;
    bump_gen(c);
    if (c->d_ebatch) cudaFree(c->d_ebatch);
    c->d_ebatch = nullptr;
    int cap = std::max(nb, 64);
    cudaError_t e = cudaMalloc(&c->d_ebatch, sizeof(double) * cap);
    if (e != cudaSuccess) return fail(TX_ERR_OOM, "energy batch buffer");
    c->ebatch_cap = cap;
    return TX_OK;
}

}  // namespace tx

using namespace tx;

// ======================================================================================
// set-up / destroy
// ======================================================================================
static int validate_setup(const int n[3], const double* const x[3], const double* const w[3], const int r[3],
                          const double* const U[3], int T, const double* th, const double* mu, int prec) {
    if (!n || !r) return fail(TX_ERR_INVALID_ARG, "n and r must not be NULL");
    if (prec < TX_PREC_FP32 || prec > TX_PREC_BF16X3) return fail(TX_ERR_UNSUPPORTED_PRECISION, "unknown precision");
    if (T < 1) return fail(TX_ERR_INVALID_ARG, "T must be >= 1");
    if (!th || !mu) return fail(TX_ERR_INVALID_ARG, "gauss_exponents / gauss_weights must not be NULL");
    for (int t = 0; t < T; ++t) {
        if (!std::isfinite(th[t]) || th[t] <= 0) return fail(TX_ERR_INVALID_ARG, "gauss_exponents must be finite and > 0");
        if (!std::isfinite(mu[t]) || mu[t] <= 0) return fail(TX_ERR_INVALID_ARG, "gauss_weights must be finite and > 0");
    }
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 2 || n[d] > 4096) return fail(TX_ERR_SHAPE, "grid sizes must be in [2, 4096]");
        if (r[d] < 1 || r[d] > n[d]) return fail(TX_ERR_SHAPE, "ranks must satisfy 1 <= r_d <= n_d");
        if (!x[d] || !w[d] || !U[d]) return fail(TX_ERR_INVALID_ARG, "grid, weight and basis arrays must not be NULL");
        for (int a = 0; a < n[d]; ++a) {
            if (!std::isfinite(x[d][a])) return fail(TX_ERR_INVALID_ARG, "node coordinates must be finite");
            if (!std::isfinite(w[d][a]) || w[d][a] <= 0) return fail(TX_ERR_INVALID_ARG, "weights must be finite and > 0");
        }
        const int nd = n[d], rd = r[d];
        for (long i = 0; i < (long)nd * rd; ++i)
            if (!std::isfinite(U[d][i])) return fail(TX_ERR_INVALID_ARG, "basis entries must be finite");
        for (int a = 0; a < rd; ++a)
            for (int b = a; b < rd; ++b) {
                double s = 0.0;
                for (int k = 0; k < nd; ++k) s += U[d][(long)k * rd + a] * U[d][(long)k * rd + b];
                if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-10)
                    return fail(TX_ERR_NOT_ORTHONORMAL, "U_" + std::to_string(d + 1) + "^T U_" + std::to_string(d + 1) +
                                                            " differs from I by more than 1e-10");
            }
    }
    return TX_OK;
}

static void free_ctx(tx_ctx* c) {
    if (!c) return;
    ctx_unregister(c);
    for (int d = 0; d < 3; ++d) {
        cudaFree(c->d_x[d]);
        cudaFree(c->d_w[d]);
        cudaFree(c->d_U[d]);
        cudaFree(c->d_A64[d]);
        cudaFree(c->f_U[d]);
        cudaFree(c->f_A[d]);
        cudaFree(c->f_w[d]);
        cudaFree(c->f_C[d]);
    }
    cudaFree(c->d_theta);
    cudaFree(c->d_mu);
    cudaFree(c->ws);
    cudaFree(c->d_err);
    cudaFree(c->d_ebatch);
    tc_release(c);
    c->magic = 0;
    delete c;
}

template <typename T>
static int dalloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(TX_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return TX_OK;
}

extern "C" int tx_tucker_setup(tx_ctx** out, const int n[3], const double* x1, const double* x2, const double* x3,
                               const double* w1, const double* w2, const double* w3, const int r[3],
                               const double* U1, const double* U2, const double* U3, int T,
                               const double* gauss_exponents, const double* gauss_weights, int precision,
                               tx_stream_t stream) {
    if (!out) return fail(TX_ERR_INVALID_ARG, "ctx output pointer is NULL");
    *out = nullptr;
    const double* xs[3] = {x1, x2, x3};
    const double* ws[3] = {w1, w2, w3};
    const double* Us[3] = {U1, U2, U3};
    TX_TRY(validate_setup(n, xs, ws, r, Us, T, gauss_exponents, gauss_weights, precision));
    cudaStream_t s = (cudaStream_t)stream;
    tx_ctx* c = new tx_ctx();
    std::memset(c, 0, sizeof(*c));
    c->magic = kMagic;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(TX_ERR_CUDA, "no CUDA device");
    }
    ctx_register(c);
    c->T = T;
    c->prec = TX_PREC_FP32;
    c->ws_limit = (size_t)2 << 30;
    for (int d = 0; d < 3; ++d) {
        c->n[d] = n[d];
        c->r[d] = r[d];
    }
    int st = TX_OK;
#define SETUP_TRY(e)            \
    do {                        \
        st = (e);               \
        if (st != TX_OK) {      \
            free_ctx(c);        \
            return st;          \
        }                       \
    } while (0)
    for (int d = 0; d < 3; ++d) {
        const size_t nd = n[d], rd = r[d];
        SETUP_TRY(dalloc(&c->d_x[d], nd));
        SETUP_TRY(dalloc(&c->d_w[d], nd));
        SETUP_TRY(dalloc(&c->d_U[d], nd * rd));
        SETUP_TRY(dalloc(&c->d_A64[d], (size_t)T * nd * rd));
        SETUP_TRY(dalloc(&c->f_U[d], nd * rd));
        SETUP_TRY(dalloc(&c->f_A[d], (size_t)T * nd * rd));
        SETUP_TRY(dalloc(&c->f_w[d], nd));
        // host float32 copies are made synchronously (the host arrays may be freed on return)
        std::vector<float> fu(nd * rd), fw(nd);
        for (size_t i = 0; i < nd * rd; ++i) fu[i] = (float)Us[d][i];
        for (size_t i = 0; i < nd; ++i) fw[i] = (float)ws[d][i];
        if (cudaMemcpy(c->d_x[d], xs[d], sizeof(double) * nd, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_w[d], ws[d], sizeof(double) * nd, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_U[d], Us[d], sizeof(double) * nd * rd, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->f_U[d], fu.data(), sizeof(float) * nd * rd, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->f_w[d], fw.data(), sizeof(float) * nd, cudaMemcpyHostToDevice) != cudaSuccess)
            SETUP_TRY(fail(TX_ERR_CUDA, "set-up copy failed"));
    }
    SETUP_TRY(dalloc(&c->d_theta, T));
    SETUP_TRY(dalloc(&c->d_mu, T));
    SETUP_TRY(dalloc(&c->d_err, kErrWords));
    if (cudaMemcpy(c->d_theta, gauss_exponents, sizeof(double) * T, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_mu, gauss_weights, sizeof(double) * T, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int) * kErrWords) != cudaSuccess)
        SETUP_TRY(fail(TX_ERR_CUDA, "set-up copy failed"));
    SETUP_TRY(setup_factor_matrices(c, s));
    SETUP_TRY(tx_set_precision(c, precision, stream));
#undef SETUP_TRY
    c->last_stream = s;
    *out = c;
    return TX_OK;
}

extern "C" int tx_set_precision(tx_ctx* c, int precision, tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    if (precision < TX_PREC_FP32 || precision > TX_PREC_BF16X3)
        return fail(TX_ERR_UNSUPPORTED_PRECISION, "unknown precision");
    if (precision == TX_PREC_FP32) {
        if (c->n[2] > 256) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 path supports n3 <= 256");
        c->prec = precision;
        return TX_OK;
    }
    std::string why;
    int old = c->prec;
    c->prec = precision;
    if (!tc_supported(c, &why)) {
        c->prec = old;
        return fail(TX_ERR_UNSUPPORTED_SHAPE, why);
    }
    int st = tc_prepare(c, (cudaStream_t)stream);
    if (st != TX_OK) c->prec = old;
    return st;
}

extern "C" void tx_destroy(tx_ctx* c) {
    if (!c || c->magic != kMagic) return;
    DeviceGuard dg;
    if (dg.use(c->device) != TX_OK) return;
    cudaDeviceSynchronize();
    free_ctx(c);
}

extern "C" size_t tx_workspace_bytes(const tx_ctx* c) { return (c && c->magic == kMagic) ? c->ws_bytes : 0; }

extern "C" int tx_set_workspace_limit(tx_ctx* c, size_t bytes) {
    TX_TRY(check_ctx(c));
    if (bytes < ((size_t)1 << 20)) return fail(TX_ERR_INVALID_ARG, "workspace limit must be at least 1 MiB");
    c->ws_limit = bytes;
    return TX_OK;
}

extern "C" int tx_check_device_error(tx_ctx* c) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    int h[4] = {0, 0, 0, 0};
    TX_TRY_CUDA(cudaStreamSynchronize(c->last_stream));
    TX_TRY_CUDA(cudaMemcpy(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost));
    TX_TRY_CUDA(cudaMemset(c->d_err, 0, sizeof(h)));   // words 4..5 (the wait limit) are kept
    if (h[0] != 0)
        return fail(TX_ERR_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(h[0]) + ", where " +
                                        std::to_string(h[1]) + "; drains that gave up: " + std::to_string(h[2]) + ")");
    if (h[2] != 0)
        return fail(TX_ERR_TIMEOUT, "a best-effort drain of in-flight copies gave up " + std::to_string(h[2]) + " time(s)");
    return TX_OK;
}

extern "C" int tx_set_wait_limit(tx_ctx* c, uint64_t ns) {
    TX_TRY(check_ctx(c));
    if (ns != 0 && (ns < 1000ull || ns > 60000000000ull))
        return fail(TX_ERR_INVALID_ARG, "wait limit must be 0 (default 2 s) or between 1 us and 60 s");
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY_CUDA(cudaStreamSynchronize(c->last_stream));
    TX_TRY_CUDA(cudaMemcpy(c->d_err + 4, &ns, sizeof(ns), cudaMemcpyHostToDevice));
    return TX_OK;
}

extern "C" int tx_selftest_wait(tx_ctx* c, int hold_tmem, tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    return tc_wait_selftest(c, hold_tmem, s);
}

extern "C" const char* tx_status_string(int s) {
    switch (s) {
        case TX_OK: return "TX_OK";
        case TX_ERR_INVALID_ARG: return "TX_ERR_INVALID_ARG";
        case TX_ERR_SHAPE: return "TX_ERR_SHAPE";
        case TX_ERR_NOT_ORTHONORMAL: return "TX_ERR_NOT_ORTHONORMAL";
        case TX_ERR_UNSUPPORTED_PRECISION: return "TX_ERR_UNSUPPORTED_PRECISION";
        case TX_ERR_CUDA: return "TX_ERR_CUDA";
        case TX_ERR_OOM: return "TX_ERR_OOM";
        case TX_ERR_TIMEOUT: return "TX_ERR_TIMEOUT";
        case TX_ERR_NOT_SETUP: return "TX_ERR_NOT_SETUP";
        case TX_ERR_UNSUPPORTED_SHAPE: return "TX_ERR_UNSUPPORTED_SHAPE";
        case TX_ERR_ALIGNMENT: return "TX_ERR_ALIGNMENT";
        case TX_ERR_NOT_DEFINITE: return "TX_ERR_NOT_DEFINITE";
        default: return "TX_ERR_UNKNOWN";
    }
}

extern "C" const char* tx_last_error_message(void) { return g_err.c_str(); }
extern "C" uint64_t tx_launch_count(void) { return g_launches; }
extern "C" void tx_profile_enable(int enable) { g_prof_on = enable != 0; }
extern "C" void tx_profile_reset(void) { g_prof_used = 0; }
extern "C" int tx_profile_read(const char* name, int* launches, double* total_ms) {
    if (!name || !launches || !total_ms) return fail(TX_ERR_INVALID_ARG, "NULL argument");
    int n = 0;
    double ms = 0.0;
    for (size_t i = 0; i < g_prof_used; ++i) {
        if (g_prof[i].name != name) continue;
        TX_TRY_CUDA(cudaEventSynchronize(g_prof[i].b));
        float t = 0.f;
        TX_TRY_CUDA(cudaEventElapsedTime(&t, g_prof[i].a, g_prof[i].b));
        ms += t;
        ++n;
    }
    *launches = n;
    *total_ms = ms;
    return TX_OK;
}
extern "C" void tx_reset_launch_count(void) { g_launches = 0; }

// ======================================================================================
// per-call dispatch
// ======================================================================================
static int check_block(const float* p, int count, const char* what) {
    if (count < 0) return fail(TX_ERR_INVALID_ARG, std::string(what) + ": negative orbital count");
    if (count > 0 && !p) return fail(TX_ERR_INVALID_ARG, std::string(what) + " is NULL");
    if (p && !aligned16(p)) return fail(TX_ERR_ALIGNMENT, std::string(what) + " is not 16-byte aligned");
    return TX_OK;
}

// an output block must share no memory with an input block (orbital blocks of n3 = N3 floats)
static int check_no_alias(const tx_ctx* c, const float* out, int n_out, const float* in, int n_in, const char* what) {
    if (!out || !in || n_out <= 0 || n_in <= 0) return TX_OK;
    const uintptr_t N3b = (uintptr_t)c->n[0] * c->n[1] * c->n[2] * sizeof(float);
    const uintptr_t o0 = (uintptr_t)out, o1 = o0 + N3b * (uintptr_t)n_out;
    const uintptr_t i0 = (uintptr_t)in, i1 = i0 + N3b * (uintptr_t)n_in;
    if (o0 < i1 && i0 < o1) return fail(TX_ERR_INVALID_ARG, std::string(what) + ": an output overlaps an input");
    return TX_OK;
}

// decides how the targets relate to the occupied block
static void classify_targets(const tx_ctx* c, const float* occ, int n_occ, const float* tgt, int n_tgt, int* mode,
                             int* k0) {
    const long N3 = (long)c->n[0] * c->n[1] * c->n[2];
    *mode = PAIRS_GENERAL;
    *k0 = 0;
    if (!tgt) {
        *mode = PAIRS_SUBSET;
        return;
    }
    const ptrdiff_t diff = tgt - occ;
    if (diff >= 0 && diff % N3 == 0) {
        const long k = diff / N3;
        if (k + n_tgt <= n_occ) {
            *mode = PAIRS_SUBSET;
            *k0 = (int)k;
        }
    }
}

static int exchange_apply(tx_ctx* c, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt, float* out,
                          tx_stream_t stream, int galerkin, int per_pair = 0) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi_occ, n_occ, "psi_occ"));
    if (!psi_tgt) n_tgt = n_occ;
    else TX_TRY(check_block(psi_tgt, n_tgt, "psi_tgt"));
    TX_TRY(check_block(out, n_tgt, "out"));
    if (!out && n_tgt > 0) return fail(TX_ERR_INVALID_ARG, "out is NULL");
    if (n_occ < 1) return fail(TX_ERR_INVALID_ARG, "n_occ must be >= 1");
    TX_TRY(check_no_alias(c, out, n_tgt, psi_occ, n_occ, "out / psi_occ"));
    TX_TRY(check_no_alias(c, out, n_tgt, psi_tgt, n_tgt, "out / psi_tgt"));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    if (n_tgt == 0) return TX_OK;
    int mode, k0;
    classify_targets(c, psi_occ, n_occ, psi_tgt, n_tgt, &mode, &k0);
    CallSpec cs;
    cs.kind = CALL_APPLY;
    cs.mode = mode;
    cs.k0 = k0;
    cs.n_occ = n_occ;
    cs.n_tgt = n_tgt;
    cs.occ = psi_occ;
    cs.tgt = psi_tgt ? psi_tgt : psi_occ;
    cs.out0 = out;
    cs.galerkin = galerkin;
    cs.per_pair = per_pair;
    return run_call(c, cs, s);
}

extern "C" int tx_exchange_apply_sthosvd(tx_ctx* c, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                                         float* out, tx_stream_t stream) {
    return exchange_apply(c, psi_occ, n_occ, psi_tgt, n_tgt, out, stream, 0, 1);
}

extern "C" int tx_exchange_apply(tx_ctx* c, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                                 float* out, tx_stream_t stream) {
    return exchange_apply(c, psi_occ, n_occ, psi_tgt, n_tgt, out, stream, 0);
}

extern "C" int tx_exchange_apply_galerkin(tx_ctx* c, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                                          float* out, tx_stream_t stream) {
    return exchange_apply(c, psi_occ, n_occ, psi_tgt, n_tgt, out, stream, 1);
}

extern "C" int tx_exchange_apply_energy(tx_ctx* c, const float* psi_occ, int n_occ, float* out, double* e_dev,
                                        tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi_occ, n_occ, "psi_occ"));
    TX_TRY(check_block(out, n_occ, "out"));
    if (n_occ < 1) return fail(TX_ERR_INVALID_ARG, "n_occ must be >= 1");
    if (!out || !e_dev) return fail(TX_ERR_INVALID_ARG, "out and e_dev must not be NULL");
    TX_TRY(check_no_alias(c, out, n_occ, psi_occ, n_occ, "out / psi_occ"));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    CallSpec cs;
    cs.kind = CALL_APPLY;
    cs.mode = PAIRS_SUBSET;
    cs.n_occ = n_occ;
    cs.n_tgt = n_occ;
    cs.occ = cs.tgt = psi_occ;
    cs.out0 = out;
    cs.e_dev = e_dev;
    return run_call(c, cs, s);
}

static int exchange_energy(tx_ctx* c, const float* psi_occ, int n_occ, double* e_dev, tx_stream_t stream,
                           int galerkin) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi_occ, n_occ, "psi_occ"));
    if (n_occ < 1) return fail(TX_ERR_INVALID_ARG, "n_occ must be >= 1");
    if (!e_dev) return fail(TX_ERR_INVALID_ARG, "e_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    CallSpec cs;
    cs.kind = CALL_ENERGY;
    cs.mode = PAIRS_SUBSET;
    cs.n_occ = n_occ;
    cs.n_tgt = n_occ;
    cs.occ = cs.tgt = psi_occ;
    cs.e_dev = e_dev;
    cs.galerkin = galerkin;
    return run_call(c, cs, s);
}

extern "C" int tx_exchange_energy(tx_ctx* c, const float* psi_occ, int n_occ, double* e_dev, tx_stream_t stream) {
    return exchange_energy(c, psi_occ, n_occ, e_dev, stream, 0);
}

extern "C" int tx_exchange_energy_galerkin(tx_ctx* c, const float* psi_occ, int n_occ, double* e_dev,
                                           tx_stream_t stream) {
    return exchange_energy(c, psi_occ, n_occ, e_dev, stream, 1);
}

extern "C" int tx_exchange_energy_grad(tx_ctx* c, const float* psi_occ, int n_occ, float* grad, double* e_dev,
                                       tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi_occ, n_occ, "psi_occ"));
    TX_TRY(check_block(grad, n_occ, "grad"));
    if (n_occ < 1) return fail(TX_ERR_INVALID_ARG, "n_occ must be >= 1");
    if (!grad) return fail(TX_ERR_INVALID_ARG, "grad is NULL");
    TX_TRY(check_no_alias(c, grad, n_occ, psi_occ, n_occ, "grad / psi_occ"));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    CallSpec cs;
    cs.kind = CALL_GRAD;
    cs.mode = PAIRS_SUBSET;
    cs.n_occ = n_occ;
    cs.n_tgt = n_occ;
    cs.occ = cs.tgt = psi_occ;
    cs.out0 = grad;
    cs.e_dev = e_dev;
    return run_call(c, cs, s);
}

extern "C" int tx_exchange_apply_vjp(tx_ctx* c, const float* psi_occ, int n_occ, const float* psi_tgt, int n_tgt,
                                     const float* grad_out, float* grad_occ, float* grad_tgt, tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi_occ, n_occ, "psi_occ"));
    if (!psi_tgt) return fail(TX_ERR_INVALID_ARG, "psi_tgt must be a separate target block");
    TX_TRY(check_block(psi_tgt, n_tgt, "psi_tgt"));
    TX_TRY(check_block(grad_out, n_tgt, "grad_out"));
    TX_TRY(check_block(grad_occ, grad_occ ? n_occ : 0, "grad_occ"));
    TX_TRY(check_block(grad_tgt, grad_tgt ? n_tgt : 0, "grad_tgt"));
    if (n_occ < 1 || n_tgt < 1) return fail(TX_ERR_INVALID_ARG, "n_occ and n_tgt must be >= 1");
    if (!grad_out) return fail(TX_ERR_INVALID_ARG, "grad_out is NULL");
    const float* ins[3] = {psi_occ, psi_tgt, grad_out};
    const int n_ins[3] = {n_occ, n_tgt, n_tgt};
    for (int k = 0; k < 3; ++k) {
        TX_TRY(check_no_alias(c, grad_occ, n_occ, ins[k], n_ins[k], "grad_occ"));
        TX_TRY(check_no_alias(c, grad_tgt, n_tgt, ins[k], n_ins[k], "grad_tgt"));
    }
    TX_TRY(check_no_alias(c, grad_occ, n_occ, grad_tgt, n_tgt, "grad_occ / grad_tgt"));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    CallSpec cs;
    cs.kind = CALL_VJP;
    cs.mode = PAIRS_GENERAL;
    cs.n_occ = n_occ;
    cs.n_tgt = n_tgt;
    cs.occ = psi_occ;
    cs.tgt = psi_tgt;
    cs.cot = grad_out;
    cs.out0 = grad_occ;
    cs.out1 = grad_tgt;
    return run_call(c, cs, s);
}

extern "C" int tx_exchange_energy_from_w(tx_ctx* c, const float* psi, const float* W, int n, double* e_dev,
                                         tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    TX_TRY(check_block(psi, n, "psi"));
    TX_TRY(check_block(W, n, "W"));
    if (n < 0) return fail(TX_ERR_INVALID_ARG, "n must be >= 0");
    if (!e_dev) return fail(TX_ERR_INVALID_ARG, "e_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    if (n == 0) {
        TX_TRY_CUDA(cudaMemsetAsync(e_dev, 0, sizeof(double), s));
        return TX_OK;
    }
    const long total = (long)n * c->n[0] * c->n[1] * c->n[2];
    const int nblocks = (int)std::max<long>(1, std::min<long>(1024, (total + 8191) / 8192));
    TX_TRY(ensure_ebatch(c, nblocks + 1));
    return weighted_dot(c, psi, W, n, c->d_ebatch, nblocks, 0.5, e_dev, s);
}

extern "C" int tx_set_quadrature(tx_ctx* c, int order, int points, tx_stream_t stream) {
    TX_TRY(check_ctx(c));
    if (order < 0 || order > 8) return fail(TX_ERR_INVALID_ARG, "element order must be 0 (nodal) .. 8");
    if (order > 0 && (points < 1 || points > 64)) return fail(TX_ERR_INVALID_ARG, "points must be 1 .. 64");
    for (int d = 0; order > 0 && d < 3; ++d)
        if ((c->n[d] - 1) % order)
            return fail(TX_ERR_SHAPE, "n_" + std::to_string(d + 1) + " - 1 is not a multiple of the element order");
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    TX_TRY_CUDA(cudaStreamSynchronize(c->last_stream));
    c->last_stream = s;
    if (order == 0) TX_TRY(setup_factor_matrices(c, s));
    else TX_TRY(setup_factor_matrices_fe(c, order, points, s));
    c->quad_order = order;
    c->quad_points = order > 0 ? points : 0;
    c->c_valid = false;
    // the operand copies of the tensor-core precisions are rebuilt from the new A_td
    if (c->prec != TX_PREC_FP32) TX_TRY(tc_prepare(c, s));
    return TX_OK;
}
