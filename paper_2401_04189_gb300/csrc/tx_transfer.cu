// Transfer of orbitals between an unstructured finite-element basis and the structured grid of
// a context (section "Transfer of wavefunctions", Eq. interpolate).
//
// Unstructured -> structured: every structured node a lies in one unstructured cell c (the
// first cell in the list whose box contains it), and
//     psi_s[i][a] = sum_b N_ab psi_u[conn[c][b]][i],
// N_ab the value at a of cell c's tensor-product Lagrange shape function of local node b.  The
// map (the structured nodes of each cell and their N rows) is computed once on the host and
// stored; the transfer is one batched per-cell product over all orbitals: a CTA stages the
// cell's orbital rows (orbital index fastest, as an FE code stores them) in shared memory and
// writes the cell's structured nodes orbital by orbital, neighbouring threads on neighbouring
// nodes.
//
// Structured -> unstructured: every unstructured node b lies in one element of the structured
// mesh (tensor product of 1-D Lagrange elements of order ps on the grid nodes), and
//     psi_u[b][i] = sum_l M_bl psi_s[i][e_b + off(l)],
// M_bl the element's shape function of local node l at b.  A CTA computes a tile of 32 nodes x
// 32 orbitals (lanes on nodes, so each lane reads its own element), then writes the tile with
// the orbital index fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "tx_internal.h"

struct tx_transfer {
    uint32_t magic;
    int device;
    int n[3];
    int n_nodes, n_cells, pu, ps;
    long n_map;                // structured nodes (every one is mapped to a cell)
    int max_cell;              // most structured nodes in one cell
    int* d_cell_start;         // [n_cells + 1] offsets into snode / N
    int* d_snode;              // [n_map] flat structured index of each mapped node, grouped by cell
    float* d_N;                // [n_map][(pu + 1)^3]
    int* d_conn;               // [n_cells][(pu + 1)^3]
    int* d_ebase;              // [n_nodes] flat structured index of local node 0 of b's element
    float* d_M;                // [n_nodes][(ps + 1)^3]
};

using namespace tx;

namespace {

constexpr uint32_t kTransferMagic = 0x54555446u;
constexpr int kChunk = 32;     // orbitals per pass

// One CTA per (cell, block of kUNodes of its structured nodes): the cell's orbital rows
// (kUChunk orbitals at a time) are staged in shared memory; each thread takes one structured
// node, keeps its N row in registers and writes that node for every orbital of the chunk
// (neighbouring threads on neighbouring nodes, so each orbital's writes are runs along z).
// Splitting the large cells over several CTAs keeps all SMs busy when coarse and refined cells
// hold very different numbers of nodes.
constexpr int kUChunk = 128;
constexpr int kUNodes = 256;

template <int NB>
__global__ void __launch_bounds__(256) k_u_to_s(const int* __restrict__ cell_start, const int* __restrict__ snode,
                                                const float* __restrict__ N, const int* __restrict__ conn,
                                                const float* __restrict__ psi_u, int n_orb, long n3,
                                                float* __restrict__ psi_s) {
    extern __shared__ __align__(16) float v[];   // [NB][kUChunk]
    const int c = blockIdx.x;
    const int kc = cell_start[c], kb = blockIdx.y * kUNodes;
    const int k0 = kc + kb, m = min(kUNodes, cell_start[c + 1] - k0);
    if (m <= 0) return;
    for (int i0 = 0; i0 < n_orb; i0 += kUChunk) {
        const int ni = min(kUChunk, n_orb - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < NB * kUChunk; e += blockDim.x) {
            const int b = e / kUChunk, ii = e % kUChunk;
            v[e] = ii < ni ? psi_u[(long)conn[(long)c * NB + b] * n_orb + i0 + ii] : 0.f;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            float w[NB];
            const float* Nk = N + (long)(k0 + k) * NB;
#pragma unroll
            for (int b = 0; b < NB; ++b) w[b] = __ldg(Nk + b);
            float* dst = psi_s + (long)i0 * n3 + snode[k0 + k];
            // four orbitals per pass: one 16-byte shared-memory broadcast feeds four FMAs (the
            // staged chunk is zero beyond ni, so the reads stay inside it; the stores are guarded)
            for (int ii = 0; ii < ni; ii += 4) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const float4 q = *reinterpret_cast<const float4*>(v + b * kUChunk + ii);
                    s0 = fmaf(w[b], q.x, s0);
                    s1 = fmaf(w[b], q.y, s1);
                    s2 = fmaf(w[b], q.z, s2);
                    s3 = fmaf(w[b], q.w, s3);
                }
                dst[(long)ii * n3] = s0;
                if (ii + 1 < ni) dst[(long)(ii + 1) * n3] = s1;
                if (ii + 2 < ni) dst[(long)(ii + 2) * n3] = s2;
                if (ii + 3 < ni) dst[(long)(ii + 3) * n3] = s3;
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_s_to_u(const int* __restrict__ ebase, const float* __restrict__ M,
                                                const float* __restrict__ psi_s, int n_orb, int n_nodes, int n2, int n3,
                                                long N3, float* __restrict__ psi_u) {
    constexpr int NS = (P + 1) * (P + 1) * (P + 1);
    __shared__ float tile[32][kChunk + 1];
    const int b0 = blockIdx.x * 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = b0 + lane;
    const bool ok = b < n_nodes;
    const int eb = ok ? ebase[b] : 0;
    float w[NS];
#pragma unroll
    for (int l = 0; l < NS; ++l) w[l] = ok ? M[(long)b * NS + l] : 0.f;
    for (int i0 = 0; i0 < n_orb; i0 += kChunk) {
        const int ni = min(kChunk, n_orb - i0);
        for (int ii = warp; ii < kChunk; ii += 8) {
            float s = 0.f;
            if (ok && ii < ni) {
                const float* src = psi_s + (long)(i0 + ii) * N3 + eb;
#pragma unroll
                for (int lx = 0; lx <= P; ++lx)
#pragma unroll
                    for (int ly = 0; ly <= P; ++ly)
#pragma unroll
                        for (int lz = 0; lz <= P; ++lz)
                            s = fmaf(w[(lx * (P + 1) + ly) * (P + 1) + lz], __ldg(src + ((long)lx * n2 + ly) * n3 + lz), s);
            }
            tile[lane][ii] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * kChunk; e += blockDim.x) {
            const int r = e / kChunk, ii = e % kChunk;
            if (b0 + r < n_nodes && ii < ni) psi_u[(long)(b0 + r) * n_orb + i0 + ii] = tile[r][ii];
        }
        __syncthreads();
    }
}

// 1-D Lagrange basis values at x of the nodes nd[0..p]
void lagrange(const double* nd, int p, double x, double* out) {
    for (int k = 0; k <= p; ++k) {
        double v = 1.0;
        for (int m = 0; m <= p; ++m)
            if (m != k) v *= (x - nd[m]) / (nd[k] - nd[m]);
        out[k] = v;
    }
}

void transfer_free(tx_transfer* t) {
    if (!t) return;
    cudaFree(t->d_cell_start);
    cudaFree(t->d_snode);
    cudaFree(t->d_N);
    cudaFree(t->d_conn);
    cudaFree(t->d_ebase);
    cudaFree(t->d_M);
    t->magic = 0;
    delete t;
}

template <typename T>
int upload(T** dst, const std::vector<T>& v, const char* what) {
    *dst = nullptr;
    if (v.empty()) return TX_OK;
    if (cudaMalloc(dst, sizeof(T) * v.size()) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return fail(TX_ERR_OOM, std::string("transfer map: ") + what);
    }
    if (cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(TX_ERR_CUDA, std::string("transfer map copy: ") + what);
    return TX_OK;
}

int check_transfer(const tx_transfer* t) {
    if (!t || t->magic != kTransferMagic) return fail(TX_ERR_NOT_SETUP, "transfer is NULL or was destroyed");
    return TX_OK;
}

}  // namespace

extern "C" int tx_transfer_create(tx_transfer** out, tx_ctx* c, int order_s, const double* X, int n_nodes,
                                  const int* conn, int n_cells, int order_u) {
    if (!out) return fail(TX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!c || c->magic != kMagic) return fail(TX_ERR_NOT_SETUP, "context is NULL or was destroyed");
    if (order_u < 1 || order_u > 3 || order_s < 1 || order_s > 3)
        return fail(TX_ERR_INVALID_ARG, "element orders must be 1, 2 or 3");
    if (!X || !conn || n_nodes < 1 || n_cells < 1) return fail(TX_ERR_INVALID_ARG, "empty or NULL mesh");
    for (int d = 0; d < 3; ++d)
        if ((c->n[d] - 1) % order_s)
            return fail(TX_ERR_SHAPE, "n_" + std::to_string(d + 1) + " - 1 is not a multiple of the structured order");
    const int pu = order_u, nb = (pu + 1) * (pu + 1) * (pu + 1);
    const int ps = order_s, ns = (ps + 1) * (ps + 1) * (ps + 1);
    for (long q = 0; q < (long)n_cells * nb; ++q)
        if (conn[q] < 0 || conn[q] >= n_nodes) return fail(TX_ERR_INVALID_ARG, "cell node index out of range");
    DeviceGuard dg;
    TX_TRY(dg.use(c->device));
    // the structured grid's nodes
    std::vector<double> xs[3];
    for (int d = 0; d < 3; ++d) {
        xs[d].resize(c->n[d]);
        TX_TRY_CUDA(cudaMemcpy(xs[d].data(), c->d_x[d], sizeof(double) * c->n[d], cudaMemcpyDeviceToHost));
    }
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2];
    const long N3 = (long)n1 * n2 * n3;
    // ---- unstructured -> structured: structured nodes of each cell, first cell wins ----
    std::vector<char> done(N3, 0);
    std::vector<int> cell_start(n_cells + 1, 0), snode;
    std::vector<float> Nv;
    std::vector<double> ax[3];
    for (int d = 0; d < 3; ++d) ax[d].resize(pu + 1);
    double L[3][4];
    for (int cc = 0; cc < n_cells; ++cc) {
        cell_start[cc] = (int)snode.size();
        const int* cn = conn + (long)cc * nb;
        for (int l = 0; l <= pu; ++l) {
            ax[0][l] = X[3L * cn[(l * (pu + 1)) * (pu + 1)] + 0];
            ax[1][l] = X[3L * cn[l * (pu + 1)] + 1];
            ax[2][l] = X[3L * cn[l] + 2];
        }
        int lo[3], hi[3];
        bool empty = false;
        for (int d = 0; d < 3; ++d) {
            const double a = *std::min_element(ax[d].begin(), ax[d].end());
            const double bnd = *std::max_element(ax[d].begin(), ax[d].end());
            const double tol = 1e-9 * (bnd - a);
            lo[d] = (int)(std::lower_bound(xs[d].begin(), xs[d].end(), a - tol) - xs[d].begin());
            hi[d] = (int)(std::upper_bound(xs[d].begin(), xs[d].end(), bnd + tol) - xs[d].begin()) - 1;
            if (hi[d] < lo[d]) empty = true;
        }
        if (empty) continue;
        for (int i = lo[0]; i <= hi[0]; ++i)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int k = lo[2]; k <= hi[2]; ++k) {
                    const long a = ((long)i * n2 + j) * n3 + k;
                    if (done[a]) continue;
                    done[a] = 1;
                    snode.push_back((int)a);
                    lagrange(ax[0].data(), pu, xs[0][i], L[0]);
                    lagrange(ax[1].data(), pu, xs[1][j], L[1]);
                    lagrange(ax[2].data(), pu, xs[2][k], L[2]);
                    for (int lx = 0; lx <= pu; ++lx)
                        for (int ly = 0; ly <= pu; ++ly)
                            for (int lz = 0; lz <= pu; ++lz) Nv.push_back((float)(L[0][lx] * L[1][ly] * L[2][lz]));
                }
    }
    cell_start[n_cells] = (int)snode.size();
    if ((long)snode.size() != N3) return fail(TX_ERR_SHAPE, "the unstructured mesh does not cover every structured node");
    // ---- structured -> unstructured: the structured element of each unstructured node ----
    std::vector<int> ebase(n_nodes);
    std::vector<float> Mv((size_t)n_nodes * ns);
    for (int b = 0; b < n_nodes; ++b) {
        int e[3];
        for (int d = 0; d < 3; ++d) {
            const int nel = (c->n[d] - 1) / ps;
            int k = 0;
            while (k < nel - 1 && X[3L * b + d] > xs[d][(size_t)ps * (k + 1)]) ++k;
            e[d] = k;
            lagrange(&xs[d][(size_t)ps * k], ps, X[3L * b + d], L[d]);
        }
        ebase[b] = (int)((((long)ps * e[0]) * n2 + (long)ps * e[1]) * n3 + (long)ps * e[2]);
        int l = 0;
        for (int lx = 0; lx <= ps; ++lx)
            for (int ly = 0; ly <= ps; ++ly)
                for (int lz = 0; lz <= ps; ++lz) Mv[(size_t)b * ns + l++] = (float)(L[0][lx] * L[1][ly] * L[2][lz]);
    }
    tx_transfer* t = new tx_transfer{};
    t->magic = kTransferMagic;
    t->device = c->device;
    for (int d = 0; d < 3; ++d) t->n[d] = c->n[d];
    t->n_nodes = n_nodes;
    t->n_cells = n_cells;
    t->pu = pu;
    t->ps = ps;
    t->n_map = (long)snode.size();
    t->max_cell = 0;
    for (int cc = 0; cc < n_cells; ++cc) t->max_cell = std::max(t->max_cell, cell_start[cc + 1] - cell_start[cc]);
    std::vector<int> connv(conn, conn + (long)n_cells * nb);
    int st = upload(&t->d_cell_start, cell_start, "cell offsets");
    if (st == TX_OK) st = upload(&t->d_snode, snode, "structured nodes");
    if (st == TX_OK) st = upload(&t->d_N, Nv, "shape values");
    if (st == TX_OK) st = upload(&t->d_conn, connv, "cells");
    if (st == TX_OK) st = upload(&t->d_ebase, ebase, "elements");
    if (st == TX_OK) st = upload(&t->d_M, Mv, "structured shape values");
    if (st != TX_OK) {
        transfer_free(t);
        return st;
    }
    *out = t;
    return TX_OK;
}

extern "C" int tx_transfer_u_to_s(tx_transfer* t, const float* psi_u, int n_orb, float* psi_s, tx_stream_t stream) {
    TX_TRY(check_transfer(t));
    if (n_orb < 0) return fail(TX_ERR_INVALID_ARG, "n_orb must be >= 0");
    if (n_orb == 0) return TX_OK;
    if (!psi_u || !psi_s) return fail(TX_ERR_INVALID_ARG, "psi_u and psi_s must not be NULL");
    DeviceGuard dg;
    TX_TRY(dg.use(t->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long N3 = (long)t->n[0] * t->n[1] * t->n[2];
    const size_t sm1 = sizeof(float) * 8 * kUChunk, sm2 = sizeof(float) * 27 * kUChunk, sm3 = sizeof(float) * 64 * kUChunk;
    const dim3 grid((unsigned)t->n_cells, (unsigned)std::max(1, (t->max_cell + kUNodes - 1) / kUNodes));
    switch (t->pu) {
        case 1: k_u_to_s<8><<<grid, 256, sm1, s>>>(t->d_cell_start, t->d_snode, t->d_N, t->d_conn, psi_u, n_orb, N3, psi_s); break;
        case 2: k_u_to_s<27><<<grid, 256, sm2, s>>>(t->d_cell_start, t->d_snode, t->d_N, t->d_conn, psi_u, n_orb, N3, psi_s); break;
        default: k_u_to_s<64><<<grid, 256, sm3, s>>>(t->d_cell_start, t->d_snode, t->d_N, t->d_conn, psi_u, n_orb, N3, psi_s); break;
    }
    TX_LAUNCHED();
    return TX_OK;
}

extern "C" int tx_transfer_s_to_u(tx_transfer* t, const float* psi_s, int n_orb, float* psi_u, tx_stream_t stream) {
    TX_TRY(check_transfer(t));
    if (n_orb < 0) return fail(TX_ERR_INVALID_ARG, "n_orb must be >= 0");
    if (n_orb == 0) return TX_OK;
    if (!psi_u || !psi_s) return fail(TX_ERR_INVALID_ARG, "psi_u and psi_s must not be NULL");
    DeviceGuard dg;
    TX_TRY(dg.use(t->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long N3 = (long)t->n[0] * t->n[1] * t->n[2];
    const unsigned grid = (unsigned)((t->n_nodes + 31) / 32);
    switch (t->ps) {
        case 1: k_s_to_u<1><<<grid, 256, 0, s>>>(t->d_ebase, t->d_M, psi_s, n_orb, t->n_nodes, t->n[1], t->n[2], N3, psi_u); break;
        case 2: k_s_to_u<2><<<grid, 256, 0, s>>>(t->d_ebase, t->d_M, psi_s, n_orb, t->n_nodes, t->n[1], t->n[2], N3, psi_u); break;
        default: k_s_to_u<3><<<grid, 256, 0, s>>>(t->d_ebase, t->d_M, psi_s, n_orb, t->n_nodes, t->n[1], t->n[2], N3, psi_u); break;
    }
    TX_LAUNCHED();
    return TX_OK;
}

extern "C" long tx_transfer_map_bytes(const tx_transfer* t) {
    if (!t || t->magic != kTransferMagic) return 0;
    const long nb = (long)(t->pu + 1) * (t->pu + 1) * (t->pu + 1), ns = (long)(t->ps + 1) * (t->ps + 1) * (t->ps + 1);
    return 4L * (t->n_cells + 1) + 4L * t->n_map * (1 + nb) + 4L * t->n_cells * nb + 4L * t->n_nodes * (1 + ns);
}

extern "C" void tx_transfer_destroy(tx_transfer* t) {
    if (!t || t->magic != kTransferMagic) return;
    DeviceGuard dg;
    if (dg.use(t->device) != TX_OK) return;
    transfer_free(t);
}
