// Expansion of one pair potential on a slab of x planes, on tcgen05 (Eq. final), fused with the
// Hadamard product and the sum over j (Eq. hadam) and the weighted energy sums:
//
//   for every Gaussian term t (the K loop of the final contraction):
//     Y_t^T[(x,g)][y] = sum_b Z_t[(x,g)][b] A_t2[y][b]              stage 2 -> TMEM
//     phi[(x,y)][z]  += sum_g Y_t[(x,y)][g] (mu_t A_t3)[z][g]        stage 3 -> TMEM (all t)
//   out0[o0] -= mul0[m0] * phi,  out1[o1] -= mul1[m1] * phi,  energy += ew * w * psi_a psi_b phi
//
// Z_t = G x1 A_t1 comes from the first-mode GEMM.  Y_t is produced transposed (rows (x, g)) so
// the stage-2 MMA has no x-alignment constraint; eight converter warps read it from TMEM,
// round it to the operand type and write it as the K-major stage-3 operand (rows (x, y)) in
// the 128-byte swizzled layout.  phi stays in TMEM across every term and is read once by the
// epilogue.  Warp roles: 0-7 converters + epilogue, 8 TMA producer + TMEM owner, 9 MMA issuer.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "tx_tc_common.cuh"
#include "tx_tc_ops.h"

namespace tx {
namespace tcc {

using namespace tx::tc;

struct ConsumeArgs {
    int n1, n2, n3, r2, r3, nt;
    int bx, R, R2, nT2, nT3, n2p, n3p, nk2, nk3;
    int nbox2, box_rows2, nstage;
    uint32_t a2_bytes, b2_bytes, b3_bytes, a3_bytes, stage_bytes, stage_tx;
    uint32_t tmem_cols, y_cols;
    uint32_t stg_off;          // byte offset of the epilogue staging area (8 warps x 32 x 68 floats)
    int p0;
    const PairRec* recs;
    const float* SA;
    const float* SB;
    const float* MUL0;
    const float* MUL1;
    float* OUT0;
    float* OUT1;
    const float* w1;
    const float* w2;
    const float* w3;
    int flags;
    int emul;                  // 1: SA == MUL1 and SB == MUL0 at the same orbital indices (symmetric pairs)
    double* epart;
    int* err;
};

constexpr int kThreads = 320;

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_consume(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mZlo,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mA2lo,
              const __grid_constant__ CUtensorMap mA3, const __grid_constant__ CUtensorMap mA3lo, ConsumeArgs a) {
    constexpr int AK = TF32 ? 32 : 64;       // K elements per 128-byte row
    constexpr int MK = TF32 ? 8 : 16;        // K per MMA instruction
    constexpr int ES = TF32 ? 4 : 2;         // operand element bytes
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[2], empty_bar[2], a3full[2], a3free[2], yfull, yfree, phidone;
    __shared__ uint32_t tmem_base;
    __shared__ double red[10];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slab = blockIdx.x, pl = blockIdx.y;
    const int x0 = slab * a.bx;
    const PairRec rec = a.recs[a.p0 + pl];
    const int NS = a.nstage;
    // Gaussian terms are accumulated from the largest exponent down (theta ascends with t):
    // the narrow, local terms contribute least, and adding small terms first limits the
    // rounding of the tensor core's float32 accumulator
    auto term_of = [&](int t) { return a.nt - 1 - t; };

    // stage layout: [A2 (Z tile)][B2 (A_t2)][B3 (A_t3)][A3 (stage-3 operand)], each hi then lo
    auto A2s = [&](int s) { return smem + s * a.stage_bytes; };
    auto B2s = [&](int s) { return A2s(s) + (SPLIT ? 2 : 1) * a.a2_bytes; };
    auto B3s = [&](int s) { return B2s(s) + (SPLIT ? 2 : 1) * a.b2_bytes; };
    auto A3s = [&](int s) { return B3s(s) + (SPLIT ? 2 : 1) * a.b3_bytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&a3full[s], 8);
            mbar_init(&a3free[s], 1);
        }
        mbar_init(&yfull, 1);
        mbar_init(&yfree, 8);
        mbar_init(&phidone, 1);
        fence_barrier_init();
    }
    // the stage-3 operand: padded K columns and unused rows must hold finite values
    for (int s = 0; s < NS; ++s) {
        uint4* p = (uint4*)A3s(s);
        const int n16 = (SPLIT ? 2 : 1) * a.a3_bytes / 16;
        for (int i = threadIdx.x; i < n16; i += kThreads) p[i] = make_uint4(0, 0, 0, 0);
    }
    fence_async_smem();
    if (warp == 8) {
        tmem_alloc(&tmem_base, a.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tY = tmem, tPhi = tmem + a.y_cols;

    if (warp == 8) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int t = 0; t < a.nt && ok; ++t) {
                const int s = t % NS;
                if (!mbar_wait(&empty_bar[s], ((t / NS) & 1) ^ 1, a.err, 31)) { ok = false; break; }
                issued = t + 1;
                // start the HBM reads of later Z tiles early (into L2 only): terms 1-3 at the
                // start, then three terms ahead
                for (int ahead = (t == 0 ? 1 : 3); ahead <= 3; ++ahead)
                    if (t + ahead < a.nt)
                        for (int k = 0; k < a.nk2; ++k)
                            tma_prefetch_l2_3d(&mZ, k * AK, x0 * a.r3, pl * a.nt + term_of(t + ahead));
                mbar_arrive_expect_tx(&full_bar[s], a.stage_tx);
                const int tt = term_of(t);
                const int zdep = pl * a.nt + tt;
                for (int k = 0; k < a.nk2; ++k)
                    for (int bb = 0; bb < a.nbox2; ++bb) {
                        const uint32_t off = k * a.nT2 * 16384u + bb * a.box_rows2 * 128u;
                        tma_load_3d(A2s(s) + off, &mZ, &full_bar[s], k * AK, x0 * a.r3 + bb * a.box_rows2, zdep);
                        if constexpr (SPLIT)
                            tma_load_3d(A2s(s) + a.a2_bytes + off, &mZlo, &full_bar[s], k * AK,
                                        x0 * a.r3 + bb * a.box_rows2, zdep);
                    }
                for (int k = 0; k < a.nk2; ++k) {
                    tma_load_3d(B2s(s) + k * a.n2p * 128u, &mA2, &full_bar[s], k * AK, 0, tt);
                    if constexpr (SPLIT)
                        tma_load_3d(B2s(s) + a.b2_bytes + k * a.n2p * 128u, &mA2lo, &full_bar[s], k * AK, 0, tt);
                }
                for (int k = 0; k < a.nk3; ++k) {
                    tma_load_3d(B3s(s) + k * a.n3p * 128u, &mA3, &full_bar[s], k * AK, 0, tt);
                    if constexpr (SPLIT)
                        tma_load_3d(B3s(s) + a.b3_bytes + k * a.n3p * 128u, &mA3lo, &full_bar[s], k * AK, 0, tt);
                }
            }
            if (!ok)
                for (int t = (issued > NS ? issued - NS : 0); t < issued; ++t)
                    mbar_drain(&full_bar[t % NS], (t / NS) & 1);
        }
    } else if (warp == 9) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            const uint32_t id2 = TF32 ? idesc_tf32(128, a.n2p) : idesc_bf16(128, a.n2p);
            const uint32_t id3 = TF32 ? idesc_tf32(128, a.n3p) : idesc_bf16(128, a.n3p);
            const int st2 = (a.r2 + MK - 1) / MK, st3 = (a.r3 + MK - 1) / MK;
            bool ok = true;
            auto stage3 = [&](int t) -> bool {
                const int s = t % NS;
                if (!mbar_wait(&a3full[s], (t / NS) & 1, a.err, 34)) return false;
                tc_fence_after();
                const uint32_t a3 = smem_u32(A3s(s)), b3 = smem_u32(B3s(s));
                for (int j = 0; j < a.nT3; ++j)
                    for (int k = 0; k < st3; ++k) {
                        const int atom = k * MK / AK, kin = (k * MK) % AK;
                        const uint32_t ao = atom * a.nT3 * 16384u + j * 16384u + kin * ES;
                        const uint32_t bo = atom * a.n3p * 128u + kin * ES;
                        const uint64_t ad = sdesc_sw128(a3 + ao), bd = sdesc_sw128(b3 + bo);
                        const uint32_t acc = (t > 0 || k > 0) ? 1u : 0u;
                        mma_ss<TF32>(tPhi + j * a.n3p, ad, bd, id3, acc);
                        if constexpr (SPLIT) {
                            mma_ss<TF32>(tPhi + j * a.n3p, ad, sdesc_sw128(b3 + a.b3_bytes + bo), id3, 1u);
                            mma_ss<TF32>(tPhi + j * a.n3p, sdesc_sw128(a3 + a.a3_bytes + ao), bd, id3, 1u);
                        }
                    }
                mma_commit(&a3free[s]);
                mma_commit(&empty_bar[s]);
                return true;
            };
            for (int t = 0; t < a.nt && ok; ++t) {
                const int s = t % NS;
                // one stage: term t-1 must finish (and free the buffer) before term t can load
                if (NS == 1 && t > 0 && !stage3(t - 1)) { ok = false; break; }
                if (!mbar_wait(&full_bar[s], (t / NS) & 1, a.err, 32)) { ok = false; break; }
                if (t > 0 && !mbar_wait(&yfree, (t - 1) & 1, a.err, 33)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a2 = smem_u32(A2s(s)), b2 = smem_u32(B2s(s));
                for (int i = 0; i < a.nT2; ++i)
                    for (int k = 0; k < st2; ++k) {
                        const int atom = k * MK / AK, kin = (k * MK) % AK;
                        const uint32_t ao = atom * a.nT2 * 16384u + i * 16384u + kin * ES;
                        const uint32_t bo = atom * a.n2p * 128u + kin * ES;
                        const uint64_t ad = sdesc_sw128(a2 + ao), bd = sdesc_sw128(b2 + bo);
                        mma_ss<TF32>(tY + i * a.n2p, ad, bd, id2, k > 0 ? 1u : 0u);
                        if constexpr (SPLIT) {
                            mma_ss<TF32>(tY + i * a.n2p, ad, sdesc_sw128(b2 + a.b2_bytes + bo), id2, 1u);
                            mma_ss<TF32>(tY + i * a.n2p, sdesc_sw128(a2 + a.a2_bytes + ao), bd, id2, 1u);
                        }
                    }
                mma_commit(&yfull);
                // two stages: stage 3 of term t-1 runs while the converters work on term t
                if (NS == 2 && t > 0 && !stage3(t - 1)) { ok = false; break; }
            }
            if (ok) ok = stage3(a.nt - 1);
            mma_commit(&phidone);
        }
    } else {
        // ------------------------------ converters (warps 0-7) ------------------------------
        const int q = warp & 3, h = warp >> 2;
        const int half2 = ((a.n2p / 16 + 1) / 2) * 16;       // y columns per half, multiple of 16
        const int c2lo = h * half2, c2hi = min(a.n2p, c2lo + half2);
        bool ok = true;
        for (int t = 0; t < a.nt && ok; ++t) {
            const int s = t % NS;
            if (!mbar_wait(&yfull, t & 1, a.err, 35)) { ok = false; break; }
            if (t >= NS && !mbar_wait(&a3free[s], ((t - NS) / NS) & 1, a.err, 36)) { ok = false; break; }
            tc_fence_after();
            uint8_t* a3 = A3s(s);
            // r3 even: lanes 2k and 2k+1 hold (x, g) and (x, g+1) of the same x, so after one
            // shuffle each lane stores a packed pair (g, g+1) for every other y
            const bool pack = (a.r3 & 1) == 0;
            const bool fast = pack && (a.n2 % 16) == 0;
            for (int i = 0; i < a.nT2; ++i) {
                const int m2 = i * 128 + q * 32 + lane;
                const bool valid = m2 < a.R2;
                const int xl = m2 / a.r3, g = m2 - xl * a.r3;
                const int g0 = g & ~1;                       // first column of the packed pair
                const int atom = g / AK, gin = (g % AK) * ES, gin0 = (g0 % AK) * ES;
                const bool odd = lane & 1;
                if (fast) {
                    // 16-row groups of the stage-3 operand start on multiples of 16 (n2 % 16 == 0),
                    // so the swizzled offsets of this lane's rows (2k + odd within each 8-row
                    // group) are fixed: four of them, computed once per tile.
                    const uint32_t cch = (uint32_t)gin0 >> 4, cin = (uint32_t)gin0 & 15u;
                    uint32_t xo[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t rw = 2u * k + (odd ? 1u : 0u);
                        xo[k] = rw * 128u + (((cch ^ rw) & 7u) << 4) + cin;
                    }
                    uint8_t* tile_a3 = a3 + atom * a.nT3 * 16384u;
                    for (int cb = c2lo; cb < c2hi; cb += 64) {
                        const int nck = min(64, c2hi - cb) / 16;
                        uint32_t r[4][16];
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (c < nck) tmem_ld16(tY + ((uint32_t)(q * 32) << 16) + i * a.n2p + cb + 16 * c, r[c]);
                        tmem_ld_wait();
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (c >= nck) break;
                            const int m30 = xl * a.n2 + cb + 16 * c;               // multiple of 16
                            uint8_t* base = tile_a3 + (m30 >> 7) * 16384u + (m30 & 127) * 128u;
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                const float v0 = __uint_as_float(r[c][j]), v1 = __uint_as_float(r[c][j + 1]);
                                const float other = __shfl_xor_sync(0xffffffffu, odd ? v0 : v1, 1);
                                const float lo_g = odd ? other : v0, hi_g = odd ? v1 : other;
                                uint8_t* dst = base + ((j >> 3) << 10) + xo[(j >> 1) & 3];
                                if (valid) {
                                    if constexpr (TF32) {
                                        const float h0 = tf32_hi(lo_g), h1 = tf32_hi(hi_g);
                                        *(float2*)dst = make_float2(h0, h1);
                                        if constexpr (SPLIT)
                                            *(float2*)(dst + a.a3_bytes) = make_float2(tf32_hi(lo_g - h0), tf32_hi(hi_g - h1));
                                    } else {
                                        const __nv_bfloat162 hv = __floats2bfloat162_rn(lo_g, hi_g);
                                        *(__nv_bfloat162*)dst = hv;
                                        if constexpr (SPLIT) {
                                            const float2 hf = __bfloat1622float2(hv);
                                            *(__nv_bfloat162*)(dst + a.a3_bytes) =
                                                __floats2bfloat162_rn(lo_g - hf.x, hi_g - hf.y);
                                        }
                                    }
                                }
                            }
                        }
                    }
                    continue;
                }
                for (int cb = c2lo; cb < c2hi; cb += 64) {
                    const int nck = min(64, c2hi - cb) / 16;
                    uint32_t r[4][16];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < nck) tmem_ld16(tY + ((uint32_t)(q * 32) << 16) + i * a.n2p + cb + 16 * c, r[c]);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (c >= nck) break;
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            const int y = cb + 16 * c + j;
                            const float v0 = __uint_as_float(r[c][j]), v1 = __uint_as_float(r[c][j + 1]);
                            if (pack) {
                                // even lane keeps column y, odd lane keeps y + 1
                                const float mine = odd ? v0 : v1;             // what the partner needs
                                const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                                const int yy = odd ? y + 1 : y;
                                const float lo_g = odd ? other : v0;          // value at column g0
                                const float hi_g = odd ? v1 : other;          // value at column g0 + 1
                                if (!valid || yy >= a.n2) continue;
                                const int m3 = xl * a.n2 + yy;
                                const uint32_t off = atom * a.nT3 * 16384u + (m3 >> 7) * 16384u +
                                                     sw128_offset(m3 & 127, gin0);
                                if constexpr (TF32) {
                                    const float h0 = tf32_hi(lo_g), h1 = tf32_hi(hi_g);
                                    *(float2*)(a3 + off) = make_float2(h0, h1);
                                    if constexpr (SPLIT)
                                        *(float2*)(a3 + a.a3_bytes + off) =
                                            make_float2(tf32_hi(lo_g - h0), tf32_hi(hi_g - h1));
                                } else {
                                    const __nv_bfloat162 hv = __floats2bfloat162_rn(lo_g, hi_g);
                                    *(__nv_bfloat162*)(a3 + off) = hv;
                                    if constexpr (SPLIT) {
                                        const float2 hf = __bfloat1622float2(hv);
                                        *(__nv_bfloat162*)(a3 + a.a3_bytes + off) =
                                            __floats2bfloat162_rn(lo_g - hf.x, hi_g - hf.y);
                                    }
                                }
                            } else {
                                if (!valid) continue;
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const int yy = y + u;
                                    if (yy >= a.n2) break;
                                    const float v = u ? v1 : v0;
                                    const int m3 = xl * a.n2 + yy;
                                    const uint32_t off = atom * a.nT3 * 16384u + (m3 >> 7) * 16384u +
                                                         sw128_offset(m3 & 127, gin);
                                    if constexpr (TF32) {
                                        const float hv = tf32_hi(v);
                                        *(float*)(a3 + off) = hv;
                                        if constexpr (SPLIT) *(float*)(a3 + a.a3_bytes + off) = tf32_hi(v - hv);
                                    } else {
                                        const __nv_bfloat16 hv = __float2bfloat16_rn(v);
                                        *(__nv_bfloat16*)(a3 + off) = hv;
                                        if constexpr (SPLIT)
                                            *(__nv_bfloat16*)(a3 + a.a3_bytes + off) =
                                                __float2bfloat16_rn(v - __bfloat162float(hv));
                                    }
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&yfree);
                mbar_arrive(&a3full[s]);
            }
        }
        // ------------------------------ epilogue ------------------------------
        double e = 0.0;
        if (ok && mbar_wait(&phidone, 0, a.err, 37) && *(volatile int*)a.err == 0) {
            tc_fence_after();
            const long N3 = (long)a.n1 * a.n2 * a.n3;
            const float* mul0 = a.MUL0 ? a.MUL0 + (long)rec.m0 * N3 : nullptr;
            const float* mul1 = a.MUL1 ? a.MUL1 + (long)rec.m1 * N3 : nullptr;
            float* out0 = (a.OUT0 && rec.o0 >= 0) ? a.OUT0 + (long)rec.o0 * N3 : nullptr;
            float* out1 = (a.OUT1 && rec.o1 >= 0) ? a.OUT1 + (long)rec.o1 * N3 : nullptr;
            const float* sa = a.SA + (long)rec.ia * N3;
            const float* sb = a.SB + (long)rec.ib * N3;
            // Each warp stages its quadrant's 32 rows x 64 columns of phi in shared memory (the
            // pipeline buffers are idle now), then walks the rows with consecutive z across lanes:
            // psi reads are coalesced and W is updated with 8-byte vector reductions.  The two
            // warps of a quadrant split the rows (even / odd).
            float* stg = (float*)(smem + a.stg_off) + warp * (32 * 68);
            for (int jt = 0; jt < a.nT3; ++jt) {
                for (int cb = 0; cb < a.n3p; cb += 64) {
                    const int nck = min(64, a.n3p - cb) / 16;
                    uint32_t r[4][16];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < nck) tmem_ld16(tPhi + ((uint32_t)(q * 32) << 16) + jt * a.n3p + cb + 16 * c, r[c]);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < nck)
#pragma unroll
                            for (int j = 0; j < 16; j += 4)
                                *(float4*)(stg + lane * 68 + 16 * c + j) =
                                    make_float4(__uint_as_float(r[c][j]), __uint_as_float(r[c][j + 1]),
                                                __uint_as_float(r[c][j + 2]), __uint_as_float(r[c][j + 3]));
                    __syncwarp();
                    // lanes 0-15 take row rr, lanes 16-31 row rr + 1; four consecutive z per lane
                    const int sub = lane >> 4, z = cb + 4 * (lane & 15);
                    for (int rp = 2 * h; rp < 32; rp += 4) {
                        const int rr = rp + sub;
                        const int m3 = jt * 128 + q * 32 + rr;
                        const int xl = m3 / a.n2, y = m3 - xl * a.n2, x = x0 + xl;
                        if (m3 >= a.R || x >= a.n1 || z >= a.n3) continue;
                        const long idx = ((long)x * a.n2 + y) * a.n3 + z;   // multiple of 4: n3 % 4 == 0
                        const float4 phi = *(const float4*)(stg + rr * 68 + 4 * (lane & 15));
                        const float wxy = a.w1[x] * a.w2[y];
                        const float4 w3 = *(const float4*)(a.w3 + z);
                        const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
                        float4 f = phi;
                        if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
                        // with symmetric pairs the energy factors (psi_a, psi_b) are the two
                        // multipliers themselves: each orbital value is read once
                        const bool en = (a.flags & EPI_ENERGY) != 0;
                        const bool o0 = (a.flags & EPI_OUT) && out0, o1 = (a.flags & EPI_OUT) && out1;
                        float4 m0 = make_float4(0.f, 0.f, 0.f, 0.f), m1 = m0;
                        if (o0 || (en && a.emul)) m0 = *(const float4*)(mul0 + idx);
                        if (o1 || (en && a.emul)) m1 = *(const float4*)(mul1 + idx);
                        if (o0) atomicAdd((float4*)(out0 + idx), make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w));
                        if (o1) atomicAdd((float4*)(out1 + idx), make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w));
                        if (en) {
                            const float4 va = a.emul ? m1 : *(const float4*)(sa + idx);
                            const float4 vb = a.emul ? m0 : *(const float4*)(sb + idx);
                            e += (double)wv.x * va.x * vb.x * phi.x + (double)wv.y * va.y * vb.y * phi.y +
                                 (double)wv.z * va.z * vb.z * phi.z + (double)wv.w * va.w * vb.w * phi.w;
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (a.flags & EPI_ENERGY) {
            for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
            if (lane == 0) red[warp] = e * rec.ew;
        }
    }
    tc_fence_before();
    __syncthreads();
    if ((a.flags & EPI_ENERGY) && threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        a.epart[(long)pl * gridDim.x + slab] = s;
    }
    if (warp == 8) tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace tcc

// ======================================================================================
// host side: tile plan and launch
// ======================================================================================
struct ConsumePlan {
    int bx, nT2, nT3, n2p, n3p, nk2, nk3, nstage, nbox2, box_rows2;
    uint32_t a2, b2, b3, a3, stage, tmem_cols, y_cols, stg_off;
    size_t smem;
};

static bool plan_for(const tx_ctx* c, bool tf32, bool split, int bx, int nstage, ConsumePlan* p) {
    const int AK = tf32 ? 32 : 64;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2];
    if (bx < 1 || bx > n1) return false;
    p->bx = bx;
    p->n2p = pad16(n2);
    p->n3p = pad16(n3);
    if (p->n2p > 256 || p->n3p > 256) return false;
    const int R2 = bx * r3, R = bx * n2;
    p->nT2 = (R2 + 127) / 128;
    p->nT3 = (R + 127) / 128;
    p->nk2 = (r2 + AK - 1) / AK;
    p->nk3 = (r3 + AK - 1) / AK;
    if (R2 > 256) return false;                 // one TMA box per K atom fills the stage-2 tile
    p->box_rows2 = R2;
    p->nbox2 = 1;
    p->y_cols = (uint32_t)(p->nT2 * p->n2p);
    const uint32_t cols = p->y_cols + (uint32_t)(p->nT3 * p->n3p);
    if (cols > 512) return false;
    p->tmem_cols = 32;
    while (p->tmem_cols < cols) p->tmem_cols <<= 1;
    p->a2 = (uint32_t)(p->nk2 * p->nT2 * 16384);
    p->b2 = (uint32_t)(p->nk2 * p->n2p * 128);
    p->b3 = (uint32_t)(p->nk3 * p->n3p * 128);
    p->a3 = (uint32_t)(p->nk3 * p->nT3 * 16384);
    p->stage = (split ? 2 : 1) * (p->a2 + p->b2 + p->b3 + p->a3);
    p->nstage = nstage;
    p->stg_off = 0;                                    // staging reuses the idle pipeline buffers
    const size_t stg = (size_t)8 * 32 * 68 * 4;
    p->smem = std::max((size_t)p->stage * nstage, stg) + 1024;
    return p->smem <= 226 * 1024;
}

static bool choose_plan(const tx_ctx* c, bool tf32, bool split, ConsumePlan* best) {
    if (c->tile_bx > 0 && plan_for(c, tf32, split, c->tile_bx, c->tile_nstage, best)) return true;
    // prefer two stages, then the slab with the least padding per useful row
    double best_score = -1;
    for (int ns = 2; ns >= 1; --ns)
        for (int bx = 1; bx <= 16; ++bx) {
            ConsumePlan p;
            if (!plan_for(c, tf32, split, bx, ns, &p)) continue;
            const double use3 = (double)(bx * c->n[1]) / (p.nT3 * 128.0);
            const double use2 = (double)(bx * c->r[2]) / (p.nT2 * 128.0);
            const double score = (ns == 2 ? 1.0 : 0.6) * (0.7 * use3 + 0.3 * use2) * (1.0 + 0.02 * bx);
            if (score > best_score) {
                best_score = score;
                *best = p;
            }
        }
    return best_score > 0;
}

// every (bx, nstage) that fits, for the autotuner; returns the count written (<= cap)
int tc_feasible_plans(const tx_ctx* c, int* bx, int* ns, int cap) {
    const TcOperands* op = c->tc;
    if (!op) return 0;
    int k = 0;
    for (int s = 2; s >= 1; --s)
        for (int b = 1; b <= 16 && k < cap; ++b) {
            ConsumePlan p;
            if (plan_for(c, op->tf32, op->split, b, s, &p)) {
                bx[k] = b;
                ns[k] = s;
                ++k;
            }
        }
    return k;
}

// the plan the next launch will use
bool tc_current_plan(const tx_ctx* c, int* bx, int* ns) {
    const TcOperands* op = c->tc;
    ConsumePlan p;
    if (!op || !choose_plan(c, op->tf32, op->split, &p)) return false;
    *bx = p.bx;
    *ns = p.nstage;
    return true;
}

bool tc_plan_fits(const tx_ctx* c, int bx, int ns) {
    const TcOperands* op = c->tc;
    ConsumePlan p;
    return op && plan_for(c, op->tf32, op->split, bx, ns, &p);
}

bool tc_consume_supported(const tx_ctx* c, bool tf32, bool split, std::string* why) {
    ConsumePlan p;
    if (!choose_plan(c, tf32, split, &p)) {
        if (why) *why = "no expansion tile plan fits shared memory and TMEM for this (n, r) and precision";
        return false;
    }
    return true;
}

long tc_consume_blocks(const tx_ctx* c) {
    ConsumePlan p;
    const TcOperands* op = c->tc;
    if (!op || !choose_plan(c, op->tf32, op->split, &p)) return 1;
    return (c->n[0] + p.bx - 1) / p.bx;
}

int tc_consume(const tx_ctx* c, const PairRec* recs, int p0, int np, const void* Z, const float* SA, const float* SB,
               const float* MUL0, const float* MUL1, float* OUT0, float* OUT1, int flags, double* epart,
               cudaStream_t s, bool emul) {
    const TcOperands* op = c->tc;
    ConsumePlan p;
    if (!choose_plan(c, op->tf32, op->split, &p)) return fail(TX_ERR_UNSUPPORTED_SHAPE, "no expansion tile plan");
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const TcScratch sc = tc_scratch(c);
    tcc::ConsumeArgs a{};
    a.n1 = n1; a.n2 = n2; a.n3 = n3; a.r2 = r2; a.r3 = r3; a.nt = T;
    a.bx = p.bx; a.R = p.bx * n2; a.R2 = p.bx * r3; a.nT2 = p.nT2; a.nT3 = p.nT3; a.n2p = p.n2p; a.n3p = p.n3p;
    a.nk2 = p.nk2; a.nk3 = p.nk3; a.nbox2 = p.nbox2; a.box_rows2 = p.box_rows2; a.nstage = p.nstage;
    a.a2_bytes = p.a2; a.b2_bytes = p.b2; a.b3_bytes = p.b3; a.a3_bytes = p.a3; a.stage_bytes = p.stage;
    a.stage_tx = (op->split ? 2 : 1) * (uint32_t)(p.nk2 * p.nbox2 * p.box_rows2 * 128 + p.b2 + p.b3);
    a.tmem_cols = p.tmem_cols; a.y_cols = p.y_cols; a.stg_off = p.stg_off;
    a.p0 = p0; a.recs = recs;
    a.SA = SA; a.SB = SB; a.MUL0 = MUL0; a.MUL1 = MUL1; a.OUT0 = OUT0; a.OUT1 = OUT1;
    a.w1 = c->f_w[0]; a.w2 = c->f_w[1]; a.w3 = c->f_w[2];
    a.flags = flags; a.epart = epart; a.err = c->d_err;
    a.emul = (SA == MUL1 && SB == MUL0 && emul) ? 1 : 0;
    const int eb = op->esize;
    const uint32_t AK = op->tf32 ? 32 : 64;
    // Z of this batch: [pair][t][(x, g) rows][ld_b]; lo part after the batch's hi part
    const size_t zlo = (size_t)np * sc.z * eb;
    CUtensorMap mZ, mZlo, mA2, mA2lo, mA3, mA3lo;
    TX_TRY(make_map(&mZ, Z, eb, r2, (uint64_t)n1 * r3, (uint64_t)np * T, sc.ld_b, (uint64_t)n1 * r3 * sc.ld_b, AK,
                    (uint32_t)p.box_rows2));
    TX_TRY(make_map(&mA2, op->st.A2, eb, r2, n2, T, pad8(r2), (uint64_t)n2 * pad8(r2), AK, (uint32_t)p.n2p));
    TX_TRY(make_map(&mA3, op->st.A3, eb, r3, n3, T, pad8(r3), (uint64_t)n3 * pad8(r3), AK, (uint32_t)p.n3p));
    if (op->split) {
        TX_TRY(make_map(&mZlo, (const char*)Z + zlo, eb, r2, (uint64_t)n1 * r3, (uint64_t)np * T, sc.ld_b,
                        (uint64_t)n1 * r3 * sc.ld_b, AK, (uint32_t)p.box_rows2));
        TX_TRY(make_map(&mA2lo, (const char*)op->st.A2 + op->st.off_lo, eb, r2, n2, T, pad8(r2),
                        (uint64_t)n2 * pad8(r2), AK, (uint32_t)p.n2p));
        TX_TRY(make_map(&mA3lo, (const char*)op->st.A3 + op->st.off_lo, eb, r3, n3, T, pad8(r3),
                        (uint64_t)n3 * pad8(r3), AK, (uint32_t)p.n3p));
    } else {
        mZlo = mZ;
        mA2lo = mA2;
        mA3lo = mA3;
    }
    dim3 grid((unsigned)((n1 + p.bx - 1) / p.bx), (unsigned)np);
    const int ps = prof_begin("tc_consume", s);
#define LAUNCH(TF, SP)                                                                                       \
    do {                                                                                                     \
        auto fn = tcc::k_consume<TF, SP>;                                                                    \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);                  \
        fn<<<grid, tcc::kThreads, p.smem, s>>>(mZ, mZlo, mA2, mA2lo, mA3, mA3lo, a);                          \
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
