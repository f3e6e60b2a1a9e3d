// Generic batched tensor-core GEMM on tcgen05: D[b][m][n] = alpha * sum_k A[b][m][k] B[b][n][k]
// with A and B K-major in global memory, loaded by TMA (128-byte swizzle) through a multi-
// stage mbarrier pipeline, accumulated in TMEM by one issuing thread, and written back by
// four epilogue warps with arbitrary output strides (float32 or bf16, optionally split into
// hi + lo parts for the 3-pass precisions).
//
// Used for the small mode products of the hot path: the second and third modes of the
// projection onto the Tucker core, the first mode of the expansion for every Gaussian term
// (Eq. final) and the first mode of the adjoint.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "tx_internal.h"
#include "tx_tc.h"
#include "tx_tc_common.cuh"

namespace tx {
namespace tcg {

using namespace tx::tc;

constexpr int kMaxStages = 4;
constexpr int kBM = 128;

// 16-byte store of VE consecutive outputs (8 bf16 or 4 float), hi and, for split types, lo
__device__ __forceinline__ void store_vec(const TcGemmArgs& g, long o, const float* v) {
    if (g.c_type == TC_OUT_F32 || g.c_type == TC_OUT_F32_SPLIT) {
        float h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) h[e] = g.c_type == TC_OUT_F32 ? v[e] : tf32_hi(v[e]);
        *(float4*)((float*)g.C + o) = make_float4(h[0], h[1], h[2], h[3]);
        if (g.c_type == TC_OUT_F32_SPLIT)
            *(float4*)((float*)g.C + o + g.c_lo) = make_float4(tf32_hi(v[0] - h[0]), tf32_hi(v[1] - h[1]),
                                                               tf32_hi(v[2] - h[2]), tf32_hi(v[3] - h[3]));
    } else {
        uint32_t w[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            w[e] = *(const uint32_t*)&hv;
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
            l[e] = *(const uint32_t*)&lv;
        }
        *(uint4*)((__nv_bfloat16*)g.C + o) = make_uint4(w[0], w[1], w[2], w[3]);
        if (g.c_type == TC_OUT_BF16_SPLIT) *(uint4*)((__nv_bfloat16*)g.C + o + g.c_lo) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

__device__ __forceinline__ void store_out(const TcGemmArgs& g, long o, float v) {
    if (g.c_type == TC_OUT_F32) {
        ((float*)g.C)[o] = v;
    } else if (g.c_type == TC_OUT_BF16) {
        ((__nv_bfloat16*)g.C)[o] = __float2bfloat16_rn(v);
    } else if (g.c_type == TC_OUT_F32_SPLIT) {
        const float hi = tf32_hi(v);
        ((float*)g.C)[o] = hi;
        ((float*)g.C)[o + g.c_lo] = tf32_hi(v - hi);
    } else {   // TC_OUT_BF16_SPLIT
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        ((__nv_bfloat16*)g.C)[o] = hi;
        ((__nv_bfloat16*)g.C)[o + g.c_lo] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
              const __grid_constant__ CUtensorMap mAlo, const __grid_constant__ CUtensorMap mBlo, TcGemmArgs g) {
    constexpr int kAtomK = TF32 ? 32 : 64;      // elements per 128-byte row
    constexpr int kMmaK = TF32 ? 8 : 16;        // K per instruction (32 bytes)
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
    __shared__ uint32_t tmem_base;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int BN = g.BN;
    const uint32_t a_bytes = kBM * 128, b_bytes = (uint32_t)BN * 128;
    const uint32_t stage_bytes = (SPLIT ? 2 : 1) * (a_bytes + b_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z, b1 = b % g.nb1, b2 = b / g.nb1;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int nk = (g.K + kAtomK - 1) / kAtomK;
    const int kStages = g.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        fence_barrier_init();
    }
    if (warp == 2) {
        tmem_alloc(&tmem_base, g.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        const int arow = m0 + b1 * g.a_row1 + b2 * g.a_row2, az = b1 * g.a_z1 + b2 * g.a_z2;
        const int brow = n0 + b1 * g.b_row1 + b2 * g.b_row2, bz = b1 * g.b_z1 + b2 * g.b_z2;
        bool ok = true;
        int issued = 0;
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&empty_bar[s], ((kb / kStages) & 1) ^ 1, g.err, 11)) { ok = false; break; }
            issued = kb + 1;
            uint8_t* st = smem + s * stage_bytes;
            mbar_arrive_expect_tx(&full_bar[s], stage_bytes);
            tma_load_3d(st, &mA, &full_bar[s], kb * kAtomK, arow, az);
            tma_load_3d(st + a_bytes, &mB, &full_bar[s], kb * kAtomK, brow, bz);
            if constexpr (SPLIT) {
                tma_load_3d(st + a_bytes + b_bytes, &mAlo, &full_bar[s], kb * kAtomK, arow, az);
                tma_load_3d(st + 2 * a_bytes + b_bytes, &mBlo, &full_bar[s], kb * kAtomK, brow, bz);
            }
        }
        // do not leave the kernel with copies in flight
        if (!ok)
            for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
                mbar_drain(&full_bar[kb % kStages], (kb / kStages) & 1, g.err);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = TF32 ? idesc_tf32(kBM, BN) : idesc_bf16(kBM, BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&full_bar[s], (kb / kStages) & 1, g.err, 13)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(smem + s * stage_bytes);
            const uint32_t b_addr = a_addr + a_bytes;
            const int krem = g.K - kb * kAtomK;
            const int nsteps = (min(krem, kAtomK) + kMmaK - 1) / kMmaK;
            // descriptors advance by adds (32 bytes per K step = 2 in the address / 16 field)
            // (each lo copy sits a_bytes + b_bytes after its hi copy)
            uint64_t ad = sdesc_sw128(a_addr), bd = sdesc_sw128(b_addr);
            const uint64_t lo = (uint64_t)((a_bytes + b_bytes) >> 4);
            // K atom kb accumulates into accumulator kb % nacc: the tensor core rounds its float32
            // accumulator at every MMA, so split precisions spread K over several accumulators
            // and the epilogue adds them in float32
            const uint32_t dacc = tmem + (uint32_t)((kb % g.nacc) * BN);
            for (int k = 0; k < nsteps; ++k) {
                mma_ss<TF32>(dacc, ad, bd, idesc, (kb >= g.nacc || k > 0) ? 1u : 0u);
                if constexpr (SPLIT) {
                    mma_ss<TF32>(dacc, ad, bd + lo, idesc, 1u);
                    mma_ss<TF32>(dacc, ad + lo, bd, idesc, 1u);
                }
                ad += 2;
                bd += 2;
            }
            mma_commit(&empty_bar[s]);
        }
        (void)ok;
        mma_commit(&done_bar);
    }
    __syncwarp();

    // ---------------- epilogue: 4 warps, one TMEM lane (= output row) per thread ----------------
    const bool ok = mbar_wait_idle(&done_bar, 0, g.err, 14);
    tc_fence_after();
    const int nacc_used = min(g.nacc, nk);     // accumulators that received a K atom
    const long boff = (long)b1 * g.c_b1 + (long)b2 * g.c_b2;
    auto row_off = [&](int m) { return boff + (long)(m / g.rdiv) * g.c_mh + (long)(m % g.rdiv) * g.c_m; };
    auto col_off = [&](int n) { return (long)(n / g.cdiv) * g.c_nh + (long)(n % g.cdiv) * g.c_n; };
    if (ok && g.c_m == 1) {
        // consecutive rows are adjacent in memory: lanes (= consecutive rows) already coalesce
        const int m = m0 + warp * 32 + lane;
        const long base = row_off(m);
        int nq = n0 / g.cdiv, nr = n0 % g.cdiv;     // column split tracked incrementally
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            for (int ac = 1; ac < nacc_used; ++ac) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ac * BN + c0), r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(r[j]);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = n0 + c0 + j;
                if (m < g.M && n < g.N)
                    store_out(g, base + (long)nq * g.c_nh + (long)nr * g.c_n, g.alpha * v[j]);
                if (++nr == g.cdiv) {
                    nr = 0;
                    ++nq;
                }
            }
        }
    } else if (ok) {
        // columns are (mostly) contiguous: stage 32 rows x 64 columns per warp in the idle
        // pipeline buffers, then write each row segment with the whole warp
        float* stg = (float*)(smem + warp * (32 * 65 * 4));
        // row offsets of this warp's 32 rows: one division each, shared through a shuffle
        const int mrow = m0 + warp * 32 + lane;
        const long my_row = row_off(mrow);
        for (int cb = 0; cb < BN; cb += 64) {
            const int nck = min(64, BN - cb) / 16;
            uint32_t r[4][16];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nck) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb + 16 * c), r[c]);
            tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nck)
#pragma unroll
                    for (int j = 0; j < 16; ++j) stg[lane * 65 + 16 * c + j] = __uint_as_float(r[c][j]);
            for (int ac = 1; ac < nacc_used; ++ac) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c < nck)
                        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ac * BN + cb + 16 * c), r[c]);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c < nck)
#pragma unroll
                        for (int j = 0; j < 16; ++j) stg[lane * 65 + 16 * c + j] += __uint_as_float(r[c][j]);
            }
            __syncwarp();
            if (g.vec) {
                // contiguous 16-byte aligned rows: each lane stores one vector of one row
                const int VE = (g.c_type == TC_OUT_F32 || g.c_type == TC_OUT_F32_SPLIT) ? 4 : 8;
                const int lpr = 64 / VE, rpp = 32 / lpr;            // lanes per row, rows per pass
                const int sub = lane / lpr, cv = (lane % lpr) * VE;
                for (int rr0 = 0; rr0 < 32; rr0 += rpp) {
                    const int rr = rr0 + sub;
                    const long base = __shfl_sync(0xffffffffu, my_row, rr);
                    const int n = n0 + cb + cv;
                    if (m0 + warp * 32 + rr < g.M && cb + cv < BN && n < g.N) {
                        float v[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] = e < VE ? g.alpha * stg[rr * 65 + cv + e] : 0.f;
                        store_vec(g, base + n, v);
                    }
                }
                __syncwarp();
                continue;
            }
            // this lane's two columns: offsets computed once per chunk
            const int cc0 = lane, cc1 = 32 + lane;
            const int n_0 = n0 + cb + cc0, n_1 = n0 + cb + cc1;
            const bool v0 = cb + cc0 < BN && n_0 < g.N, v1 = cb + cc1 < BN && n_1 < g.N;
            const long co0 = v0 ? col_off(n_0) : 0, co1 = v1 ? col_off(n_1) : 0;
            for (int rr = 0; rr < 32; ++rr) {
                const long base = __shfl_sync(0xffffffffu, my_row, rr);
                if (m0 + warp * 32 + rr >= g.M) break;
                if (v0) store_out(g, base + co0, g.alpha * stg[rr * 65 + cc0]);
                if (v1) store_out(g, base + co1, g.alpha * stg[rr * 65 + cc1]);

            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tmem_dealloc(tmem, g.tmem_cols);
}

}  // namespace tcg

// ======================================================================================
// host side
// ======================================================================================
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

int make_map(CUtensorMap* m, const void* base, int elem_bytes, uint64_t k_extent, uint64_t rows, uint64_t depth,
             uint64_t row_stride_elems, uint64_t depth_stride_elems, uint32_t box_k, uint32_t box_rows) {
    return make_map_sw(m, base, elem_bytes, k_extent, rows, depth, row_stride_elems, depth_stride_elems, box_k, box_rows,
                       CU_TENSOR_MAP_SWIZZLE_128B);
}

int make_map_sw(CUtensorMap* m, const void* base, int elem_bytes, uint64_t k_extent, uint64_t rows, uint64_t depth,
                uint64_t row_stride_elems, uint64_t depth_stride_elems, uint32_t box_k, uint32_t box_rows,
                CUtensorMapSwizzle swizzle) {
    auto fn = encode_fn();
    if (!fn) return fail(TX_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (((uintptr_t)base & 15) || (row_stride_elems * elem_bytes) % 16 || (depth_stride_elems * elem_bytes) % 16)
        return fail(TX_ERR_ALIGNMENT, "tensor map base / strides must be 16-byte multiples");
    cuuint64_t dims[3] = {k_extent, rows, depth};
    cuuint64_t strides[2] = {row_stride_elems * elem_bytes, depth_stride_elems * elem_bytes};
    if (depth <= 1) strides[1] = strides[0] * rows;
    if (strides[1] == 0) strides[1] = 16;
    cuuint32_t box[3] = {box_k, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(TX_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
    return TX_OK;
}

int make_map_f32_plain(CUtensorMap* m, const void* base, uint64_t k_extent, uint64_t rows, uint64_t depth,
                       uint32_t box_k, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return fail(TX_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (((uintptr_t)base & 15) || (k_extent * 4) % 16)
        return fail(TX_ERR_UNSUPPORTED_SHAPE, "tensor-core path needs n3 % 4 == 0 and 16-byte aligned orbitals");
    cuuint64_t dims[3] = {k_extent, rows, depth < 1 ? 1 : depth};
    cuuint64_t strides[2] = {k_extent * 4, k_extent * 4 * rows};
    cuuint32_t box[3] = {box_k, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(TX_ERR_CUDA, "cuTensorMapEncodeTiled (float32 plain) failed (code " + std::to_string((int)r) + ")");
    return TX_OK;
}

static uint32_t tmem_cols_for(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

int tc_gemm_launch(const TcOperand& A, const TcOperand& B, TcGemmArgs g, bool tf32, bool split, const char* prof,
                   cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return TX_OK;
    if (g.rdiv <= 0) {
        g.rdiv = 1 << 30;
        g.c_mh = 0;
    }
    if (g.cdiv <= 0) {
        g.cdiv = 1 << 30;
        g.c_nh = 0;
    }
    if (g.BN <= 0) {
        g.BN = 16;
        while (g.BN < g.N && g.BN < 128) g.BN += 16;   // <= 128 keeps several CTAs per SM
    }
    if (g.BN % 16 || g.BN > 256) return fail(TX_ERR_INVALID_ARG, "tc_gemm: BN must be a multiple of 16 <= 256");
    size_t stage = (size_t)(split ? 2 : 1) * (128 * 128 + (size_t)g.BN * 128);
    const size_t budget = 225 * 1024;
    while (g.BN > 16 && 2 * stage + 1024 > budget) {   // keep at least two stages in flight
        g.BN -= 16;
        stage = (size_t)(split ? 2 : 1) * (128 * 128 + (size_t)g.BN * 128);
    }
    const int nk_atoms = (g.K + (tf32 ? 32 : 64) - 1) / (tf32 ? 32 : 64);
    // split precisions: up to 4 accumulators along K (TMEM permitting), summed in float32
    g.nacc = split ? std::max(1, std::min({nk_atoms, 4, 512 / g.BN})) : 1;
    g.tmem_cols = tmem_cols_for(g.nacc * g.BN);
    {
        // vector stores: contiguous columns, no column split, every row start and the lo copy
        // 16-byte aligned, whole vectors
        const long ve = (g.c_type == TC_OUT_F32 || g.c_type == TC_OUT_F32_SPLIT) ? 4 : 8;
        g.vec = g.c_n == 1 && g.cdiv >= g.N && g.c_m != 1 && ((uintptr_t)g.C % 16) == 0 && g.c_m % ve == 0 &&
                g.c_mh % ve == 0 && g.c_b1 % ve == 0 && g.c_b2 % ve == 0 && g.c_lo % ve == 0 && g.N % ve == 0;
    }
    g.stages = (int)std::min<size_t>({(size_t)tcg::kMaxStages, (budget - 1024) / stage, (size_t)nk_atoms});
    // the epilogue stages 4 warps x 32 rows x 65 floats in the (then idle) pipeline buffers
    const size_t smem = std::max(stage * g.stages, (size_t)4 * 32 * 65 * 4) + 1024;
    const int eb = tf32 ? 4 : 2;
    const uint32_t atom_k = 128 / eb;
    CUtensorMap mA, mB, mAlo, mBlo;
    TX_TRY(make_map(&mA, A.hi, eb, A.k_extent, A.rows, A.depth, A.row_stride, A.depth_stride, atom_k, 128));
    TX_TRY(make_map(&mB, B.hi, eb, B.k_extent, B.rows, B.depth, B.row_stride, B.depth_stride, atom_k, g.BN));
    if (split) {
        TX_TRY(make_map(&mAlo, A.lo, eb, A.k_extent, A.rows, A.depth, A.row_stride, A.depth_stride, atom_k, 128));
        TX_TRY(make_map(&mBlo, B.lo, eb, B.k_extent, B.rows, B.depth, B.row_stride, B.depth_stride, atom_k, g.BN));
    } else {
        mAlo = mA;
        mBlo = mB;
    }
    dim3 grid((g.N + g.BN - 1) / g.BN, (g.M + 127) / 128, g.nb1 * g.nb2);
    if (grid.z > 65535) return fail(TX_ERR_INVALID_ARG, "tc_gemm: too many batches in one launch");
    const int ps = prof_begin(prof ? prof : "tc_gemm", s);
#define TCG_LAUNCH(TF, SP)                                                                                       \
    do {                                                                                                         \
        auto fn = tcg::k_tc_gemm<TF, SP>;                                                                        \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                        \
        fn<<<grid, 128, smem, s>>>(mA, mB, mAlo, mBlo, g);                                                       \
    } while (0)
    if (tf32) {
        if (split) TCG_LAUNCH(true, true); else TCG_LAUNCH(true, false);
    } else {
        if (split) TCG_LAUNCH(false, true); else TCG_LAUNCH(false, false);
    }
#undef TCG_LAUNCH
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

// ======================================================================================
// Row-streaming form for GEMMs with a short K (at most two 128-byte atoms), many row tiles and
// contiguous output rows: one CTA per (column tile, batch, row-tile stride) keeps its B tile in
// shared memory and walks its row tiles with two A stages, two TMEM accumulators and TMA
// stores of the output, so that the loads, the MMAs and the output of consecutive row tiles
// overlap and the output leaves as whole 128-byte lines.  Used for the expansion's first mode
// (T * n1 rows against one pair's core), a store stream of T n r^2 operand values per pair.
// ======================================================================================
namespace tcg {

constexpr int kRowsThreads = 192;   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t kStgBuf = 32 * 128;   // one staged 32-row x 128-byte output box


template <bool TF32>
__global__ void __launch_bounds__(kRowsThreads, 1)
    k_tc_rows(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
              const __grid_constant__ CUtensorMap mC, TcGemmArgs g) {
    constexpr int kAtomK = TF32 ? 32 : 64;      // elements per 128-byte row
    constexpr int kMmaK = TF32 ? 8 : 16;        // K per instruction (32 bytes)
    constexpr int CE = TF32 ? 32 : 64;          // output elements per 128-byte staged row
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bbar, afull[2], aempty[2], accfull[2], accfree[2];
    __shared__ uint32_t tmem_base;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int BN = g.BN;
    const int nk = (g.K + kAtomK - 1) / kAtomK;
    const uint32_t a_atom = kBM * 128, b_atom = (uint32_t)BN * 128;
    uint8_t* sB = smem;                                                  // [nk][BN][128 B]
    uint8_t* sA = smem + ((nk * b_atom + 1023) & ~1023u);                 // [2][nk][128][128 B]
    uint8_t* sC = sA + 2 * nk * a_atom;                                   // [4 warps][2][32][128 B]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, b1 = blockIdx.y;
    const int mtiles = (g.M + kBM - 1) / kBM;
    const int ntile = blockIdx.z < mtiles ? (mtiles - 1 - (int)blockIdx.z) / (int)gridDim.z + 1 : 0;
    auto m0_of = [&](int j) { return ((int)blockIdx.z + j * (int)gridDim.z) * kBM; };

    if (threadIdx.x == 0) {
        mbar_init(&bbar, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&afull[i], 1);
            mbar_init(&aempty[i], 1);
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], 4);
        }
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base, g.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer: B once, then A per row tile ----------------
        const int brow = n0 + b1 * g.b_row1, bz = b1 * g.b_z1;
        const int arow = b1 * g.a_row1, az = b1 * g.a_z1;
        mbar_arrive_expect_tx_w(&bbar, (uint32_t)nk * b_atom);
        for (int kb = 0; kb < nk; ++kb) tma_load_3d_w(sB + kb * b_atom, &mB, &bbar, kb * kAtomK, brow, bz);
        int s = 0, issued = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int j = 0; j < ntile; ++j) {
            ok = __all_sync(0xffffffffu, mbar_wait(&aempty[s], ph ^ 1, g.err, 15));
            if (!ok) break;
            issued = j + 1;
            mbar_arrive_expect_tx_w(&afull[s], (uint32_t)nk * a_atom);
            for (int kb = 0; kb < nk; ++kb)
                tma_load_3d_w(sA + (s * nk + kb) * a_atom, &mA, &afull[s], kb * kAtomK, arow + m0_of(j), az);
            if (++s == 2) { s = 0; ph ^= 1; }
        }
        // do not leave the kernel with copies in flight
        mbar_drain(&bbar, 0, g.err);
        if (!ok)
            for (int j = (issued > 2 ? issued - 2 : 0); j < issued; ++j) mbar_drain(&afull[j & 1], (j >> 1) & 1, g.err);
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = TF32 ? idesc_tf32(kBM, BN) : idesc_bf16(kBM, BN);
        bool ok = __all_sync(0xffffffffu, mbar_wait(&bbar, 0, g.err, 16));
        const uint64_t bd0 = sdesc_sw128(smem_u32(sB));
        int s = 0;
        uint32_t ph = 0;
        for (int j = 0; j < ntile && ok; ++j) {
            bool w = mbar_wait(&afull[s], ph, g.err, 17);
            // accumulator s was last read by the epilogue for row tile j - 2
            if (w && j >= 2) w = mbar_wait(&accfree[s], ph ^ 1, g.err, 18);
            if (!__all_sync(0xffffffffu, w)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(s * BN);
            const uint64_t ad0 = sdesc_sw128(smem_u32(sA + s * nk * a_atom));
            for (int kb = 0; kb < nk; ++kb) {
                const int steps = (min(g.K - kb * kAtomK, kAtomK) + kMmaK - 1) / kMmaK;
                const uint64_t ad = ad0 + (uint64_t)(kb * (a_atom >> 4)), bd = bd0 + (uint64_t)(kb * (b_atom >> 4));
                for (int k = 0; k < steps; ++k)
                    mma_ss_w<TF32>(d, ad + 2u * k, bd + 2u * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit_w(&aempty[s]);
            mma_commit_w(&accfull[s]);
            if (++s == 2) { s = 0; ph ^= 1; }
        }
    } else {
        // ---------------- epilogue: warps 2-5, TMEM lane quadrant = warp % 4 ----------------
        // Each warp stages its 32 rows x 128 bytes per chunk in the 128-byte swizzle (16-byte
        // piece q of row r at ((q ^ (r & 7)) * 16), conflict-free) and lane 0 stores the box
        // with TMA; two staging buffers alternate, the older store must have read its buffer.
        const int q4 = warp & 3;
        uint8_t* stg = sC + (warp - 2) * 2 * kStgBuf;
        int s = 0, buf = 0;
        uint32_t ph = 0;
        for (int j = 0; j < ntile; ++j) {
            if (!__all_sync(0xffffffffu, mbar_wait(&accfull[s], ph, g.err, 19))) break;
            tc_fence_after();
            const int mrow = m0_of(j) + q4 * 32;
            for (int c0 = 0; c0 < BN; c0 += CE) {
                if (lane == 0) bulk_wait_read1();
                __syncwarp();
                uint8_t* sb = stg + buf * kStgBuf + lane * 128;
#pragma unroll
                for (int u = 0; u < CE / 16; ++u) {
                    uint32_t r[16];
                    tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(s * BN + c0 + 16 * u), r);
                    tmem_ld_wait();
                    if constexpr (TF32) {
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int pc = 4 * u + h;
                            *(uint4*)(sb + ((pc ^ (lane & 7)) << 4)) =
                                make_uint4(__float_as_uint(g.alpha * __uint_as_float(r[4 * h])),
                                           __float_as_uint(g.alpha * __uint_as_float(r[4 * h + 1])),
                                           __float_as_uint(g.alpha * __uint_as_float(r[4 * h + 2])),
                                           __float_as_uint(g.alpha * __uint_as_float(r[4 * h + 3])));
                        }
                    } else {
                        uint32_t w[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const __nv_bfloat162 hv = __floats2bfloat162_rn(g.alpha * __uint_as_float(r[2 * e]),
                                                                            g.alpha * __uint_as_float(r[2 * e + 1]));
                            w[e] = *(const uint32_t*)&hv;
                        }
                        *(uint4*)(sb + (((2 * u) ^ (lane & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
                        *(uint4*)(sb + (((2 * u + 1) ^ (lane & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tma_store_3d(&mC, stg + buf * kStgBuf, n0 + c0, mrow, b1);
                    bulk_commit();
                }
                buf ^= 1;
            }
            // this warp's TMEM reads of accumulator s are complete: release it to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accfree[s]);
            if (++s == 2) { s = 0; ph ^= 1; }
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, g.tmem_cols);
}

}  // namespace tcg

// Whether tc_rows_launch can run this product (else tc_gemm_launch)
static bool rows_form_fits(const TcGemmArgs& g, bool tf32, bool split) {
    const int eb = tf32 ? 4 : 2;
    const int atom = tf32 ? 32 : 64;
    return !split && (g.c_type == (tf32 ? TC_OUT_F32 : TC_OUT_BF16)) && g.K <= 2 * atom && g.nb2 == 1 && g.c_n == 1 &&
           g.rdiv <= 0 && g.cdiv <= 0 && g.N >= 128 && g.c_m >= g.N && ((uintptr_t)g.C % 16) == 0 &&
           (g.c_m * eb) % 16 == 0 && (g.c_b1 * eb) % 16 == 0 && g.nb1 <= 65535;
}

int tc_rows_launch(const TcOperand& A, const TcOperand& B, TcGemmArgs g, bool tf32, bool split, const char* prof,
                   cudaStream_t s) {
    if (!rows_form_fits(g, tf32, split)) return tc_gemm_launch(A, B, g, tf32, split, prof, s);
    if (g.M <= 0) return TX_OK;
    const int eb = tf32 ? 4 : 2;
    const uint32_t atom_k = 128 / eb;
    const int nk = (g.K + (int)atom_k - 1) / (int)atom_k;
    g.BN = 128;
    g.nacc = 1;
    g.tmem_cols = tmem_cols_for(2 * g.BN);
    const size_t smem = (((size_t)nk * g.BN * 128 + 1023) & ~(size_t)1023) + 2 * (size_t)nk * 128 * 128 +
                        4 * 2 * tcg::kStgBuf + 1024;
    CUtensorMap mA, mB, mC;
    TX_TRY(make_map(&mA, A.hi, eb, A.k_extent, A.rows, A.depth, A.row_stride, A.depth_stride, atom_k, 128));
    TX_TRY(make_map(&mB, B.hi, eb, B.k_extent, B.rows, B.depth, B.row_stride, B.depth_stride, atom_k, g.BN));
    // output [nb1][M][N] with row stride c_m and batch stride c_b1; 32-row x 128-byte boxes
    TX_TRY(make_map(&mC, g.C, eb, (uint64_t)g.N, (uint64_t)g.M, (uint64_t)g.nb1, (uint64_t)g.c_m, (uint64_t)g.c_b1,
                    atom_k, 32));
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int mtiles = (g.M + 127) / 128;
    const long base = (long)((g.N + g.BN - 1) / g.BN) * g.nb1;
    // enough CTAs for about three per SM; each walks mtiles / gz row tiles
    const int gz = (int)std::max<long>(1, std::min<long>(mtiles, (3L * nsm + base - 1) / base));
    dim3 grid((unsigned)((g.N + g.BN - 1) / g.BN), (unsigned)g.nb1, (unsigned)gz);
    const int ps = prof_begin(prof ? prof : "tc_gemm", s);
    if (tf32) {
        cudaFuncSetAttribute(tcg::k_tc_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tcg::k_tc_rows<true><<<grid, tcg::kRowsThreads, smem, s>>>(mA, mB, mC, g);
    } else {
        cudaFuncSetAttribute(tcg::k_tc_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tcg::k_tc_rows<false><<<grid, tcg::kRowsThreads, smem, s>>>(mA, mB, mC, g);
    }
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

// ---- self-test of the building block ---------------------------------------------------
namespace {
__global__ void k_split_f32(const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo, long n) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i], h = tc::tf32_hi(v);
    hi[i] = h;
    lo[i] = v - h;
}
__global__ void k_split_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                             long n) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}
}  // namespace

}  // namespace tx

using namespace tx;

// D[b][m][n] = sum_k A[b][m][k] B[b][n][k], A [batch][M][K], B [batch][N][K] float32 row-major
// (K a multiple of 8), D float32; the operands are rounded to the precision's operand type.
extern "C" int tx_selftest_gemm(int precision, int batch, int M, int N, int K, const float* A, const float* B,
                                float* D, tx_stream_t stream) {
    if (!A || !B || !D || batch < 1 || M < 1 || N < 1 || K < 1 || K % 8)
        return fail(TX_ERR_INVALID_ARG, "selftest_gemm: bad arguments");
    if (precision == TX_PREC_FP32) return fail(TX_ERR_UNSUPPORTED_PRECISION, "selftest_gemm: tensor precisions only");
    cudaStream_t s = (cudaStream_t)stream;
    const bool tf32 = precision == TX_PREC_TF32 || precision == TX_PREC_TF32X3;
    const bool split = precision == TX_PREC_TF32X3 || precision == TX_PREC_BF16X3;
    const int eb = tf32 ? 4 : 2;
    const long na = (long)batch * M * K, nbb = (long)batch * N * K;
    char* buf = nullptr;
    TX_TRY_CUDA(cudaMalloc(&buf, (size_t)eb * 2 * (na + nbb) + 256));
    char* ahi = buf;
    char* alo = ahi + eb * na;
    char* bhi = alo + eb * na;
    char* blo = bhi + eb * nbb;
    if (tf32) {
        k_split_f32<<<(na + 255) / 256, 256, 0, s>>>(A, (float*)ahi, (float*)alo, na);
        k_split_f32<<<(nbb + 255) / 256, 256, 0, s>>>(B, (float*)bhi, (float*)blo, nbb);
    } else {
        k_split_bf16<<<(na + 255) / 256, 256, 0, s>>>(A, (__nv_bfloat16*)ahi, (__nv_bfloat16*)alo, na);
        k_split_bf16<<<(nbb + 255) / 256, 256, 0, s>>>(B, (__nv_bfloat16*)bhi, (__nv_bfloat16*)blo, nbb);
    }
    TcOperand oa{ahi, alo, (uint64_t)K, (uint64_t)M, (uint64_t)batch, (uint64_t)K, (uint64_t)M * K};
    TcOperand ob{bhi, blo, (uint64_t)K, (uint64_t)N, (uint64_t)batch, (uint64_t)K, (uint64_t)N * K};
    TcGemmArgs g{};
    g.M = M; g.N = N; g.K = K; g.nb1 = batch; g.nb2 = 1;
    g.a_z1 = 1; g.b_z1 = 1;
    g.C = D; g.c_m = N; g.c_n = 1; g.c_b1 = (long)M * N; g.c_type = TC_OUT_F32; g.alpha = 1.f;
    static int* d_err = nullptr;
    if (!d_err) TX_TRY_CUDA(cudaMalloc(&d_err, kErrWords * sizeof(int)));
    TX_TRY_CUDA(cudaMemsetAsync(d_err, 0, kErrWords * sizeof(int), s));
    g.err = d_err;
    int st = tc_gemm_launch(oa, ob, g, tf32, split, "selftest", s);
    cudaStreamSynchronize(s);
    int h[2] = {0, 0};
    cudaMemcpy(h, d_err, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (st != TX_OK) return st;
    if (h[0]) return fail(TX_ERR_TIMEOUT, "selftest_gemm: device wait gave up at site " + std::to_string(h[1]));
    TX_TRY_CUDA(cudaGetLastError());
    return TX_OK;
}
