// Allocation-free variant of the float32 apply path.
//
// Some callers cannot let a library call cudaMalloc: applications that hand all device memory
// to their own arena or pool allocator, and latency-sensitive loops in which the implicit
// device-wide synchronisation of cudaMalloc / cudaFree is not acceptable.  For them,
// tx_exchange_apply_static keeps every piece of scratch the float32 kernels need (the pair
// table and the per-batch projection / expansion intermediates) in one fixed array in the
// library's own device memory, and allocates nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "tx_internal.h"
#include "tx_paths.h"

namespace tx {

// 32 MiB, reserved on every device where the library's module is loaded, until process exit
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code `g_static_scratch` names
// a host-side stand-in, never a device address, so the address is looked up once per device
// (with that device current) and cached.
int static_scratch(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TX_ERR_CUDA, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(TX_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return TX_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// G[p][(g,b)][a] = sum_x S2[p][x][(g,b)] U1[x][a]  (mode 1 of the projection)
int simt_mode1_project(const tx_ctx* c, const float* S2, float* G, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2];
    GemmArgs q{};
    q.M = rr; q.N = r1; q.K = n1;
    q.A = S2; q.a_m = 1; q.a_k = rr; q.a_b2 = (long)n1 * rr;
    q.B = c->f_U[0]; q.b_k = r1; q.b_n = 1;
    q.C = G; q.c_m = r1; q.c_n = 1; q.c_b2 = (long)rr * r1;
    q.nb1 = 1; q.nb2 = np; q.alpha = 1.f;
    return simt_gemm(q, s);
}

// Z[p][t][x][(g,b)] = sum_a M1_t[x][a] G[p][(g,b)][a]  (mode 1 of the expansion, every term)
int simt_mode1_expand(const tx_ctx* c, const float* G, const float* M1, int nt, float* Z, int np, cudaStream_t s) {
    const int n1 = c->n[0], r1 = c->r[0], rr = c->r[1] * c->r[2];
    GemmArgs q{};
    q.M = n1; q.N = rr; q.K = r1;
    q.A = M1; q.a_m = r1; q.a_k = 1; q.a_b1 = (long)n1 * r1;
    q.B = G; q.b_k = 1; q.b_n = r1; q.b_b2 = (long)rr * r1;
    q.C = Z; q.c_m = rr; q.c_n = 1; q.c_b1 = (long)n1 * rr; q.c_b2 = (long)nt * n1 * rr;
    q.nb1 = nt; q.nb2 = np; q.alpha = 1.f;
    return simt_gemm(q, s);
}

}  // namespace
}  // namespace tx

using namespace tx;

// K psi_occ with float32 kernels, all scratch in the fixed array (see include/tuxc.h).
extern "C" int tx_exchange_apply_static(tx_ctx* c, const float* psi_occ, int n_occ, float* out, tx_stream_t stream) {
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    if (!psi_occ || !out || n_occ < 1) return fail(TX_ERR_INVALID_ARG, "psi_occ / out NULL or n_occ < 1");
    if (((uintptr_t)psi_occ | (uintptr_t)out) & 15u) return fail(TX_ERR_ALIGNMENT, "arrays must be 16-byte aligned");
    if (c->n[2] > 256) return fail(TX_ERR_UNSUPPORTED_SHAPE, "float32 kernels need n3 <= 256");
    {
        const uintptr_t bytes = (uintptr_t)n_occ * c->n[0] * c->n[1] * c->n[2] * sizeof(float);
        const uintptr_t a = (uintptr_t)psi_occ, b = (uintptr_t)out;
        if (a < b + bytes && b < a + bytes) return fail(TX_ERR_INVALID_ARG, "out overlaps psi_occ");
    }
    DeviceGuard dg;   // the caller's current device is restored on return
    TX_TRY(dg.use(c->device));
    void* base = nullptr;
    TX_TRY(static_scratch(c->device, &base));
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;

    // sizes: pair table, then per-pair float32 intermediates of the expansion path
    const long P = pair_count(PAIRS_SUBSET, n_occ, n_occ);
    const size_t recs_bytes = up256(sizeof(PairRec) * (size_t)P);
    const size_t n1 = c->n[0], r1 = c->r[0], r2 = c->r[1], r3 = c->r[2];
    const size_t s2 = n1 * r3 * r2, g = r3 * r2 * r1, z = (size_t)c->T * n1 * r3 * r2;
    const size_t per_pair = sizeof(float) * (s2 + g + z);
    if (recs_bytes + per_pair + 4096 > kStaticScratchBytes)
        return fail(TX_ERR_UNSUPPORTED_SHAPE,
                    "tx_exchange_apply_static needs " + std::to_string(recs_bytes + per_pair + 4096) +
                        " bytes of scratch for one pair; its fixed array holds " + std::to_string(kStaticScratchBytes));
    long Pb = (long)((kStaticScratchBytes - recs_bytes - 4096) / per_pair);
    Pb = std::min<long>(std::min<long>(Pb, P), 65535 / std::max(1, c->T));
    PairRec* recs = (PairRec*)base;
    float* S2 = (float*)((char*)base + recs_bytes);
    float* G = S2 + (size_t)Pb * s2;
    float* Z = G + (size_t)Pb * g;

    // nothing in the array is read before this call writes it: the pair table is rebuilt and
    // every intermediate is produced before it is consumed
    TX_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * n1 * c->n[1] * c->n[2] * n_occ, s));
    TX_TRY(build_pairs(recs, PAIRS_SUBSET, ROLE_APPLY, n_occ, n_occ, 0, s));
    FieldArgs f{};
    f.SA = psi_occ;
    f.SB = psi_occ;
    f.MUL0 = psi_occ;
    f.MUL1 = psi_occ;
    f.OUT0 = out;
    f.OUT1 = out;
    for (long p0 = 0; p0 < P; p0 += Pb) {
        const int np = (int)std::min<long>(Pb, P - p0);
        TX_TRY(simt_project_s2(c, recs, (int)p0, np, f, 0, S2, s));
        TX_TRY(simt_mode1_project(c, S2, G, np, s));
        TX_TRY(simt_mode1_expand(c, G, c->f_A[0], c->T, Z, np, s));
        TX_TRY(simt_expand_consume(c, recs, (int)p0, np, f, Z, c->T, c->f_A[1], c->f_A[2], EPI_OUT, nullptr, s));
    }
    return TX_OK;
}
