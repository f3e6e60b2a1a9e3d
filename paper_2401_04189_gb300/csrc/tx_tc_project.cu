// Projection onto the shared Tucker basis, first contraction (mode 3), on tcgen05 with the
// pair-density producer fused in (the pair product of the "Convolution operation" section,
// then Eq. TuckerDecompField with a shared basis):
//
//   S1[p][gamma][x][y] = sum_z rho_p[x][y][z] U3[z][gamma],   rho_p = psi_a * psi_b (* w)
//
// One CTA owns 128 consecutive (x, y) rows of one pair.  TMA brings the float32 orbital tiles
// of both factors into shared memory (double-buffered); four warps form rho in registers,
// round it to the operand type and write it in the 128-byte swizzled K-major layout; one
// thread issues the MMAs against U3^T; the accumulator lives in TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include <string>

#include "tx_tc_common.cuh"
#include "tx_tc_ops.h"

namespace tx {
namespace tcp {

using namespace tx::tc;

struct ProjArgs {
    int n1, n2, n3, r3, ld_y;
    int N3p;                 // r3 rounded up to 16 (MMA N)
    int p0;
    const PairRec* recs;
    const float* w1;
    const float* w2;
    const float* w3;
    int flags;
    void* S1;                // [pair][r3][n1][ld_y]
    size_t s1_pair;          // elements per pair
    size_t s1_lo;            // element offset of the lo part
    uint32_t tmem_cols;
    int nacc;                // accumulators along K (split precisions), summed in float32
    int* err;
};

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(128, 1)
    k_project3(const __grid_constant__ CUtensorMap mPsiA, const __grid_constant__ CUtensorMap mPsiB,
               const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mUlo, ProjArgs a) {
    constexpr int ZB = TF32 ? 32 : 64;          // z per 128-byte operand row
    constexpr int kMmaK = TF32 ? 8 : 16;
    constexpr uint32_t PSI_BYTES = 128 * ZB * 4; // one float32 orbital tile
    constexpr uint32_t RHO_BYTES = 128 * 128;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[2], rho_free[2], done_bar, u_bar;
    __shared__ uint32_t tmem_base;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)a.N3p * 128;
    const int nk = (a.n3 + ZB - 1) / ZB;
    // layout: [rho hi x2][rho lo x2][U3^T hi, every K atom][U3^T lo][psiA x2][psiB x2]
    // U3^T is loaded once and stays: the MMAs read it asynchronously, so it must not share a
    // buffer with the orbital tiles that are refilled while earlier MMAs may still run.
    uint8_t* rho = smem;
    uint8_t* rho_lo = rho + 2 * RHO_BYTES;
    uint8_t* bt = rho + (SPLIT ? 4 : 2) * RHO_BYTES;
    uint8_t* bt_lo = bt + nk * B_BYTES;
    uint8_t* psa = bt + (SPLIT ? 2 : 1) * nk * B_BYTES;
    uint8_t* psb = psa + 2 * PSI_BYTES;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128, pl = blockIdx.y;
    const PairRec rec = a.recs[a.p0 + pl];
    const uint32_t stage_tx = 2 * PSI_BYTES;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&rho_free[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&u_bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, a.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    auto issue_load = [&](int kb) {
        const int s = kb & 1;
        mbar_arrive_expect_tx(&full_bar[s], stage_tx);
        tma_load_3d(psa + s * PSI_BYTES, &mPsiA, &full_bar[s], kb * ZB, m0, rec.ia);
        tma_load_3d(psb + s * PSI_BYTES, &mPsiB, &full_bar[s], kb * ZB, m0, rec.ib);
    };
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&u_bar, (SPLIT ? 2 : 1) * nk * B_BYTES);
        for (int kb = 0; kb < nk; ++kb) {
            tma_load_3d(bt + kb * B_BYTES, &mU, &u_bar, kb * ZB, 0, 0);
            if constexpr (SPLIT) tma_load_3d(bt_lo + kb * B_BYTES, &mUlo, &u_bar, kb * ZB, 0, 0);
        }
        issue_load(0);
        if (nk > 1) issue_load(1);
    }

    bool ok = true;
    int issued = nk > 1 ? 2 : 1;
    const uint32_t idesc = TF32 ? idesc_tf32(128, a.N3p) : idesc_bf16(128, a.N3p);
    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb & 1;
        bool good = mbar_wait(&full_bar[s], (kb >> 1) & 1, a.err, 21);
        if (good && kb >= 2) good = mbar_wait(&rho_free[s], ((kb - 2) >> 1) & 1, a.err, 22);
        if (good && kb == 0) good = mbar_wait(&u_bar, 0, a.err, 25);
        if (good) {
            // rho = psi_a * psi_b (* w) -> operand tile (128-byte swizzle)
            const float* A = (const float*)(psa + s * PSI_BYTES);
            const float* B = (const float*)(psb + s * PSI_BYTES);
            uint8_t* R = rho + s * RHO_BYTES;
            uint8_t* Rl = rho_lo + s * RHO_BYTES;
            for (int r = warp; r < 128; r += 4) {
                float wr = 1.f;
                if (a.flags & PROD_MULW) {
                    const int m = m0 + r;
                    const int x = m / a.n2, y = m - x * a.n2;
                    wr = (x < a.n1) ? a.w1[x] * a.w2[y] : 0.f;
                }
                if constexpr (TF32) {
                    const int zc = kb * ZB + lane;
                    float v = A[r * ZB + lane] * B[r * ZB + lane];
                    if (a.flags & PROD_MULW) v *= wr * (zc < a.n3 ? a.w3[zc] : 0.f);
                    const float h = tf32_hi(v);
                    const uint32_t off = sw128_offset(r, 4 * lane);
                    *(float*)(R + off) = h;
                    if constexpr (SPLIT) *(float*)(Rl + off) = tf32_hi(v - h);
                } else {
                    const float2 va = *(const float2*)(A + r * ZB + 2 * lane);
                    const float2 vb = *(const float2*)(B + r * ZB + 2 * lane);
                    float v0 = va.x * vb.x, v1 = va.y * vb.y;
                    if (a.flags & PROD_MULW) {
                        const int zc = kb * ZB + 2 * lane;
                        v0 *= wr * (zc < a.n3 ? a.w3[zc] : 0.f);
                        v1 *= wr * (zc + 1 < a.n3 ? a.w3[zc + 1] : 0.f);
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    const uint32_t off = sw128_offset(r, 4 * lane);
                    *(__nv_bfloat162*)(R + off) = h;
                    if constexpr (SPLIT) {
                        const float2 hf = __bfloat1622float2(h);
                        *(__nv_bfloat162*)(Rl + off) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
                    }
                }
            }
        }
        fence_async_smem();
        ok = __syncthreads_and(good) != 0;      // block-uniform: everyone stops together
        if (!ok) break;
        if (threadIdx.x == 0) {
            if (kb + 2 < nk) {                   // buffer s is no longer read
                issue_load(kb + 2);
                ++issued;
            }
            tc_fence_after();
            const uint32_t ra = smem_u32(rho + s * RHO_BYTES), rl = smem_u32(rho_lo + s * RHO_BYTES);
            const uint32_t ba = smem_u32(bt + kb * B_BYTES), bl = smem_u32(bt_lo + kb * B_BYTES);
            const int nsteps = (min(a.n3 - kb * ZB, ZB) + kMmaK - 1) / kMmaK;
            // descriptors advance by adds (32 bytes per K step = 2 in the address / 16 field)
            uint64_t ad = sdesc_sw128(ra), bd = sdesc_sw128(ba), al = sdesc_sw128(rl), bdl = sdesc_sw128(bl);
            // K chunk kb accumulates into accumulator kb % nacc (added in float32 by the epilogue)
            const uint32_t dacc = tmem + (uint32_t)((kb % a.nacc) * a.N3p);
            for (int k = 0; k < nsteps; ++k) {
                mma_ss<TF32>(dacc, ad, bd, idesc, (kb >= a.nacc || k > 0) ? 1u : 0u);
                if constexpr (SPLIT) {
                    mma_ss<TF32>(dacc, ad, bdl, idesc, 1u);
                    mma_ss<TF32>(dacc, al, bd, idesc, 1u);
                }
                ad += 2;
                bd += 2;
                al += 2;
                bdl += 2;
            }
            mma_commit(&rho_free[s]);
            if (kb == nk - 1) mma_commit(&done_bar);
        }
    }
    if (!ok && threadIdx.x == 0) {
        mma_commit(&done_bar);
        // do not exit with copies in flight: wait (bounded) for every issued stage
        for (int kb = (issued > 2 ? issued - 2 : 0); kb < issued; ++kb) mbar_drain(&full_bar[kb & 1], (kb >> 1) & 1, a.err);
        mbar_drain(&u_bar, 0, a.err);
    }
    __syncwarp();
    // epilogue: S1[p][gamma][x][y]
    const bool ok2 = mbar_wait(&done_bar, 0, a.err, 23);
    tc_fence_after();
    if (ok2 && ok) {
        const int m = m0 + warp * 32 + lane;
        const int x = m / a.n2, y = m - x * a.n2;
        const bool valid = x < a.n1;
        const size_t base = (size_t)pl * a.s1_pair + (size_t)x * a.ld_y + y;
        const size_t gstride = (size_t)a.n1 * a.ld_y;
        const int nacc_used = min(a.nacc, nk);
        for (int c0 = 0; c0 < a.N3p; c0 += 16) {
            uint32_t r[16];
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = __uint_as_float(r[j]);
            for (int ac = 1; ac < nacc_used; ++ac) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ac * a.N3p + c0), r);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(r[j]);
            }
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int g = c0 + j;
                if (g >= a.r3) break;
                const float v = acc[j];
                const size_t o = base + (size_t)g * gstride;
                if constexpr (TF32) {
                    const float h = tf32_hi(v);
                    ((float*)a.S1)[o] = h;
                    if constexpr (SPLIT) ((float*)a.S1)[o + a.s1_lo] = tf32_hi(v - h);
                } else {
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    ((__nv_bfloat16*)a.S1)[o] = h;
                    if constexpr (SPLIT) ((__nv_bfloat16*)a.S1)[o + a.s1_lo] = __float2bfloat16_rn(v - __bfloat162float(h));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}


// Persistent, pipelined form for the single-pass precisions.  Work items are (pair, 128-row
// tile) in pair-major order; each CTA walks items blockIdx.x, blockIdx.x + gridDim.x, ... with
// U3^T resident and every stage in flight at once: warp 0 streams the orbital tiles through a
// two-stage ring, warps 2-5 form rho into a two-buffer operand ring, warp 1 issues the MMAs
// into two TMEM accumulators, and warps 6-9 write S1 from the accumulator of the previous
// tile.  The one-CTA-per-tile form above runs load, product, MMA and store one after another.
constexpr int kP3Threads = 320;

template <bool TF32>
__global__ void __launch_bounds__(kP3Threads, 1)
    k_project3p(const __grid_constant__ CUtensorMap mPsiA, const __grid_constant__ CUtensorMap mPsiB,
                const __grid_constant__ CUtensorMap mU, ProjArgs a, int nitems, int mtiles) {
    constexpr int ZB = TF32 ? 32 : 64;          // z per 128-byte operand row
    constexpr int kMmaK = TF32 ? 8 : 16;
    constexpr uint32_t PSI_BYTES = 128 * ZB * 4; // one float32 orbital tile
    constexpr uint32_t RHO_BYTES = 128 * 128;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t u_bar, pfull[2], pempty[2], rfull[2], rfree[2], accfull[2], accfree[2];
    __shared__ uint32_t tmem_base;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)a.N3p * 128;
    const int nk = (a.n3 + ZB - 1) / ZB;
    // layout: [U3^T, every K atom][rho x2][psiA, psiB] x2
    uint8_t* bt = smem;
    uint8_t* rho = bt + ((nk * B_BYTES + 1023) & ~1023u);
    uint8_t* psi = rho + 2 * RHO_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's items: blockIdx.x + j * gridDim.x
    const int nmine = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto item = [&](int j, int& pl, int& m0) {
        const int it = (int)blockIdx.x + j * (int)gridDim.x;
        pl = it / mtiles;
        m0 = (it - pl * mtiles) * 128;
    };

    if (threadIdx.x == 0) {
        mbar_init(&u_bar, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&pfull[i], 1);
            mbar_init(&pempty[i], 4);
            mbar_init(&rfull[i], 4);
            mbar_init(&rfree[i], 1);
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], 4);
        }
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base, a.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer: U3^T once, then both orbital tiles per (item, atom) ----------------
        mbar_arrive_expect_tx_w(&u_bar, (uint32_t)nk * B_BYTES);
        for (int kb = 0; kb < nk; ++kb) tma_load_3d_w(bt + kb * B_BYTES, &mU, &u_bar, kb * ZB, 0, 0);
        int s = 0, issued = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int j = 0; j < nmine && ok; ++j) {
            int pl, m0;
            item(j, pl, m0);
            const PairRec rec = a.recs[a.p0 + pl];
            for (int kb = 0; kb < nk; ++kb) {
                ok = __all_sync(0xffffffffu, mbar_wait(&pempty[s], ph ^ 1, a.err, 26));
                if (!ok) break;
                ++issued;
                mbar_arrive_expect_tx_w(&pfull[s], 2 * PSI_BYTES);
                tma_load_3d_w(psi + s * 2 * PSI_BYTES, &mPsiA, &pfull[s], kb * ZB, m0, rec.ia);
                tma_load_3d_w(psi + s * 2 * PSI_BYTES + PSI_BYTES, &mPsiB, &pfull[s], kb * ZB, m0, rec.ib);
                if (++s == 2) { s = 0; ph ^= 1; }
            }
        }
        // do not leave the kernel with copies in flight
        mbar_drain(&u_bar, 0, a.err);
        if (!ok)
            for (int q = (issued > 2 ? issued - 2 : 0); q < issued; ++q) mbar_drain(&pfull[q & 1], (q >> 1) & 1, a.err);
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = TF32 ? idesc_tf32(128, a.N3p) : idesc_bf16(128, a.N3p);
        bool ok = __all_sync(0xffffffffu, mbar_wait(&u_bar, 0, a.err, 27));
        int r = 0, ab = 0;
        uint32_t rph = 0, aph = 0;
        for (int j = 0; j < nmine && ok; ++j) {
            // accumulator ab was last read by the epilogue of item j - 2
            if (j >= 2) ok = __all_sync(0xffffffffu, mbar_wait(&accfree[ab], aph ^ 1, a.err, 28));
            const uint32_t d = tmem + (uint32_t)(ab * a.N3p);
            for (int kb = 0; kb < nk && ok; ++kb) {
                ok = __all_sync(0xffffffffu, mbar_wait(&rfull[r], rph, a.err, 29));
                if (!ok) break;
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(smem_u32(rho + r * RHO_BYTES)), bd = sdesc_sw128(smem_u32(bt + kb * B_BYTES));
                const int nsteps = (min(a.n3 - kb * ZB, ZB) + kMmaK - 1) / kMmaK;
                for (int k = 0; k < nsteps; ++k) mma_ss_w<TF32>(d, ad + 2u * k, bd + 2u * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                mma_commit_w(&rfree[r]);
                if (++r == 2) { r = 0; rph ^= 1; }
            }
            if (!ok) break;
            mma_commit_w(&accfull[ab]);
            if (++ab == 2) { ab = 0; aph ^= 1; }
        }
    } else if (warp < 6) {
        // ---------------- rho = psi_a * psi_b (* w) -> operand ring (128-byte swizzle) ----------------
        const int wq = warp - 2;
        int s = 0, r = 0;
        uint32_t ph = 0, rph = 0;
        int q = 0;
        bool ok = true;
        for (int j = 0; j < nmine && ok; ++j) {
            int pl, m0;
            item(j, pl, m0);
            for (int kb = 0; kb < nk; ++kb, ++q) {
                bool w = mbar_wait(&pfull[s], ph, a.err, 30);
                if (w && q >= 2) w = mbar_wait(&rfree[r], rph ^ 1, a.err, 32);
                ok = __all_sync(0xffffffffu, w);
                if (!ok) break;
                const float* A = (const float*)(psi + s * 2 * PSI_BYTES);
                const float* B = (const float*)(psi + s * 2 * PSI_BYTES + PSI_BYTES);
                uint8_t* R = rho + r * RHO_BYTES;
                for (int rr = wq; rr < 128; rr += 4) {
                    float wr = 1.f;
                    if (a.flags & PROD_MULW) {
                        const int m = m0 + rr;
                        const int x = m / a.n2, y = m - x * a.n2;
                        wr = (x < a.n1) ? a.w1[x] * a.w2[y] : 0.f;
                    }
                    if constexpr (TF32) {
                        const int zc = kb * ZB + lane;
                        float v = A[rr * ZB + lane] * B[rr * ZB + lane];
                        if (a.flags & PROD_MULW) v *= wr * (zc < a.n3 ? a.w3[zc] : 0.f);
                        *(float*)(R + sw128_offset(rr, 4 * lane)) = tf32_hi(v);
                    } else {
                        const float2 va = *(const float2*)(A + rr * ZB + 2 * lane);
                        const float2 vb = *(const float2*)(B + rr * ZB + 2 * lane);
                        float v0 = va.x * vb.x, v1 = va.y * vb.y;
                        if (a.flags & PROD_MULW) {
                            const int zc = kb * ZB + 2 * lane;
                            v0 *= wr * (zc < a.n3 ? a.w3[zc] : 0.f);
                            v1 *= wr * (zc + 1 < a.n3 ? a.w3[zc + 1] : 0.f);
                        }
                        *(__nv_bfloat162*)(R + sw128_offset(rr, 4 * lane)) = __floats2bfloat162_rn(v0, v1);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&pempty[s]);
                    mbar_arrive(&rfull[r]);
                }
                if (++s == 2) { s = 0; ph ^= 1; }
                if (++r == 2) { r = 0; rph ^= 1; }
            }
        }
    } else {
        // ---------------- epilogue: S1[p][gamma][x][y], TMEM lane quadrant = warp % 4 ----------------
        const int q4 = warp & 3;
        int ab = 0;
        uint32_t aph = 0;
        for (int j = 0; j < nmine; ++j) {
            if (!__all_sync(0xffffffffu, mbar_wait(&accfull[ab], aph, a.err, 33))) break;
            tc_fence_after();
            int pl, m0;
            item(j, pl, m0);
            const int m = m0 + q4 * 32 + lane;
            const int x = m / a.n2, y = m - x * a.n2;
            const bool valid = x < a.n1;
            const size_t base = (size_t)pl * a.s1_pair + (size_t)x * a.ld_y + y;
            const size_t gstride = (size_t)a.n1 * a.ld_y;
            for (int c0 = 0; c0 < a.N3p; c0 += 16) {
                uint32_t rv[16];
                tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ab * a.N3p + c0), rv);
                tmem_ld_wait();
                if (!valid) continue;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int g = c0 + jj;
                    if (g >= a.r3) break;
                    const float v = __uint_as_float(rv[jj]);
                    const size_t o = base + (size_t)g * gstride;
                    if constexpr (TF32) ((float*)a.S1)[o] = tf32_hi(v);
                    else ((__nv_bfloat16*)a.S1)[o] = __float2bfloat16_rn(v);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accfree[ab]);
            if (++ab == 2) { ab = 0; aph ^= 1; }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace tcp

int tc_project_mode3(const tx_ctx* c, const PairRec* recs, int p0, int np, const float* SA, int nA, const float* SB,
                     int nB, int flags, void* S1, cudaStream_t s, const void* Bhi) {
    const TcOperands* op = c->tc;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r3 = c->r[2];
    const TcScratch sc = tc_scratch(c);
    tcp::ProjArgs a{};
    a.n1 = n1; a.n2 = n2; a.n3 = n3; a.r3 = r3; a.ld_y = sc.ld_y;
    a.N3p = pad16(r3);
    a.p0 = p0; a.recs = recs;
    a.w1 = c->f_w[0]; a.w2 = c->f_w[1]; a.w3 = c->f_w[2];
    a.flags = flags;
    a.S1 = S1;
    a.s1_pair = sc.s1;
    a.s1_lo = (size_t)np * sc.s1;          // lo part follows the batch's hi part
    {
        const int nk = (n3 + (op->tf32 ? 32 : 64) - 1) / (op->tf32 ? 32 : 64);
        a.nacc = op->split ? std::max(1, std::min({nk, 4, 512 / a.N3p})) : 1;
        const int cols = a.nacc * a.N3p;
        a.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
    }
    a.err = c->d_err;
    if (a.N3p > 256) return fail(TX_ERR_UNSUPPORTED_SHAPE, "tensor-core projection needs r3 <= 256");
    const int ZB = op->tf32 ? 32 : 64;
    const long nrows = (long)n1 * n2;
    CUtensorMap mA, mB, mU, mUlo;
    // psi as [orbital][n1*n2 rows][n3] float32, boxes of 128 rows x ZB z (no swizzle)
    TX_TRY(make_map_f32_plain(&mA, SA, (uint64_t)n3, (uint64_t)nrows, (uint64_t)nA, (uint32_t)ZB, 128));
    TX_TRY(make_map_f32_plain(&mB, SB, (uint64_t)n3, (uint64_t)nrows, (uint64_t)nB, (uint32_t)ZB, 128));
    const int eb = op->esize;
    const void* Bop = Bhi ? Bhi : op->st.U3T;
    TX_TRY(make_map(&mU, Bop, eb, ldk(n3, eb), r3, 1, ldk(n3, eb), 0, (uint32_t)ZB, (uint32_t)a.N3p));
    if (op->split)
        TX_TRY(make_map(&mUlo, (const char*)Bop + op->st.off_lo, eb, ldk(n3, eb), r3, 1, ldk(n3, eb), 0, (uint32_t)ZB,
                        (uint32_t)a.N3p));
    else
        mUlo = mU;
    const size_t psi_bytes = (size_t)128 * ZB * 4, rho_bytes = 128 * 128, b_bytes = (size_t)a.N3p * 128;
    const int nk = (n3 + ZB - 1) / ZB;
    if (!op->split) {
        // persistent pipelined form: one CTA per SM walks the (pair, row tile) items
        a.nacc = 1;
        const int cols = 2 * a.N3p;
        a.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
        const size_t smem_p = ((nk * b_bytes + 1023) & ~(size_t)1023) + 2 * rho_bytes + 4 * psi_bytes + 1024;
        if (smem_p > 227 * 1024) return fail(TX_ERR_UNSUPPORTED_SHAPE, "projection tile does not fit shared memory");
        const int mtiles = (int)((nrows + 127) / 128);
        const long nitems = (long)mtiles * np;
        if (nitems > (1L << 30)) return fail(TX_ERR_INVALID_ARG, "projection: too many row tiles in one launch");
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const unsigned gx = (unsigned)std::min<long>(nitems, nsm);
        const int ps = prof_begin("tc_project", s);
        if (op->tf32) {
            cudaFuncSetAttribute(tcp::k_project3p<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
            tcp::k_project3p<true><<<gx, tcp::kP3Threads, smem_p, s>>>(mA, mB, mU, a, (int)nitems, mtiles);
        } else {
            cudaFuncSetAttribute(tcp::k_project3p<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
            tcp::k_project3p<false><<<gx, tcp::kP3Threads, smem_p, s>>>(mA, mB, mU, a, (int)nitems, mtiles);
        }
        prof_end(ps, s);
        TX_LAUNCHED();
        return TX_OK;
    }
    const size_t smem = (op->split ? 4 : 2) * rho_bytes + (op->split ? 2 : 1) * nk * b_bytes + 4 * psi_bytes + 1024;
    if (smem > 227 * 1024) return fail(TX_ERR_UNSUPPORTED_SHAPE, "projection tile does not fit shared memory");
    dim3 grid((unsigned)((nrows + 127) / 128), (unsigned)np);
    const int ps = prof_begin("tc_project", s);
#define LAUNCH(TF, SP)                                                                                \
    do {                                                                                              \
        auto fn = tcp::k_project3<TF, SP>;                                                            \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
        fn<<<grid, 128, smem, s>>>(mA, mB, mU, mUlo, a);                                              \
    } while (0)
    if (op->tf32) {
        if (op->split) LAUNCH(true, true); else LAUNCH(true, false);
    } else {
        if (op->split) LAUNCH(false, true); else LAUNCH(false, false);
    }
#undef LAUNCH
    prof_end(ps, s);
    TX_LAUNCHED();
    return TX_OK;
}

}  // namespace tx
