// Expansion of one pair potential on a slab of x planes, on tcgen05 (Eq. final), fused with the
// Hadamard product and the sum over j (Eq. hadam) and the weighted energy sums:
//
//   for every Gaussian term t (the K loop of the final contraction):
//     Y_t,x[y][g]    = sum_b A_t2[y][b] Z_t[(x,g)][b]     one stage-2 MMA per x plane -> TMEM
//     phi[(x,y)][z] += sum_g Y_t[(x,y)][g] (mu_t A_t3)[z][g]        stage 3 -> TMEM (all t)
//   out0[o0] -= mul0[m0] * phi,  out1[o1] -= mul1[m1] * phi,  energy += ew * w * psi_a psi_b phi
//
// Z_t = G x1 A_t1 comes from the first-mode GEMM.  Three kernels:
//  - k_consume (the split precisions, below): stage 2 puts y on the TMEM lanes and g on the
//    columns, so each converter lane already holds one row (x, y) of the K-major stage-3
//    operand: it splits the row into hi and lo and writes them with 16-byte stores.  Each x
//    plane has its own TMEM columns and its own full / free barriers, so the MMA of plane p for
//    the next term starts as soon as plane p has been converted.  Operand tiles use the 32-byte
//    swizzle: one sub-tile of `rows x 32 bytes` per MMA K-step, so K is padded only to the
//    K-step.  Warp roles: 0-7 converters + epilogue, 8 TMA producer + TMEM owner, 9 MMA issuer.
//  - k_consume_ts (single-pass precisions): stage 3 reads Y straight from TMEM; one CTA per
//    (pair, slab) work item (described at its definition).
//  - k_consume_tp: the same loop, persistent over the work items, with the epilogue of one item
//    overlapping the main loop of the next (described at its definition).
// phi stays in TMEM across the terms it accumulates and is read once by the epilogue.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "tx_tc_common.cuh"
#include "tx_tc_ops.h"

namespace tx {
namespace tcc {

using namespace tx::tc;

constexpr int kMaxLoad = 6;
constexpr int kMaxPlanes = 16;
constexpr int kMaxYBuf = 4;        // stage-2 output buffers in TMEM (single-pass kernel)

__host__ __device__ constexpr int pad16c(int v) { return (v + 15) & ~15; }

struct ConsumeArgs {
    int n1, n2, n3, r2, r3, nt;
    int bx, R, nY, Nz, npc, nT3, n2p, n3p, ks2, ks3, nq, gs, ycol_tile, ns3;
    int nload, na3, nyb;
    int chunk;                 // split kernel: Gaussian terms per TMEM accumulation chunk
    uint32_t ya_rows, z_rows;                          // rows of the stage-2 A tile (A_t2) and B tile (Z)
    uint32_t ya_bytes, z_bytes, b3_bytes, a3_bytes;    // one hi copy of each operand tile
    uint32_t load_bytes, stage_tx, a3_off;             // load stage stride, bytes per stage, A3 buffers
    int nload3;                                        // single-pass kernel: stage-3 ring stages
    uint32_t load3_bytes;                              // single-pass kernel: stage-3 ring stride
    uint32_t tmem_cols, y_cols;
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
    // single-pass kernel: per-term operator image, and the batch's Z for L2 prefetches
    const uint8_t* img;
    uint32_t img_stride;       // bytes per term of img: ya_bytes + b3_bytes
    const uint8_t* zsrc;
    uint32_t z_plane;          // bytes of one x plane of one term of Z
    int zone;                  // 1: the slab's Z planes load as one box (gs == r3, bx * r3 <= 256 rows)
    // persistent single-pass kernel: work items (pair, slab), slabs per pair, epilogue region
    int nitems, nslab;
    int nyi;                   // persistent kernel: work items per slab (1, or one per y tile of 128 rows)
    // persistent kernel, y tiles packed: the last y tile of a plane holds tail_rows rows, so the
    // tails of tailp consecutive planes share one 128-row item (plane p in rows p * tail_r8 ..);
    // its stage-2 A operand is, per plane, a window of the operator image at win_off + p * ya_bytes
    // holding A_t2's last rows at those rows and zeros elsewhere.  0: every y tile its own item.
    int tailp, tail_r8, tail_rows;
    int per_pair;              // persistent kernel: work items per pair
    uint32_t win_off;
    uint32_t img_ya_rows;      // rows per K atom of the A_t2 tile in the operator image (packed
                               // items keep only 128 rows per atom in shared memory: ya_rows)
    int nys;                   // bf16 persistent kernel: Y operand tiles in shared memory
    uint32_t ys_off, ys_bytes, ys_tile;   // ... their offset, stride per buffer, stride per tile
    uint32_t epi_off;
    // split kernel, y/z items: each CTA covers one 128-row y tile (of nyi per plane) and one part
    // of nzi of the z columns (n3p of them) of one plane; 0: the CTA covers its whole slab
    int yz, nzi;
    // converter kernel: the stage-3 B operand (mu_t A_t3) has a ring of its own after the
    // [A_t2][Z] stages, so that stage 2 releases its stage as soon as its MMAs have run
    uint32_t loadB_bytes, b_off, stageB_tx;
    int nloadB;
};

constexpr int kThreads = 320;
constexpr int kMaxLoadB = 2;       // converter kernel: stages of the stage-3 operand ring
constexpr int kThreadsTs = 352;   // single-pass kernel: one more producer warp (10)
constexpr int kThreadsTp = 384;   // persistent single-pass kernel: a separate stage-3 warp (11)
// epilogue shared memory (reuses the pipeline buffers): phi staging, 8 warps x 32 rows x 68
// floats, then per warp two blocks of orbital values, 8 row pairs x 2 multipliers x 32 lanes
constexpr uint32_t kStgBytes = 8u * 32u * 68u * 4u;
constexpr uint32_t kEpiBytes = kStgBytes + 8u * 2u * 8u * 2u * 32u * 16u;

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// byte offset of (row, byte-in-row) in a 32-byte-swizzled sub-tile (rows 4-7 of every 8-row
// group have their two 16-byte halves swapped)
__device__ __forceinline__ uint32_t sw32_offset(uint32_t row, uint32_t byte_in_row) {
    return row * 32u + (byte_in_row ^ (((row >> 2) & 1u) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *(const uint32_t*)&v;
}

// One 16-byte chunk of a stage-3 operand row: 8 bf16 or 4 tf32 values v[0..]; `lo` receives
// the rounding residuals for the split precisions.
template <bool TF32, bool SPLIT>
__device__ __forceinline__ void convert_chunk(const float* v, uint4& hi, uint4& lo) {
    if constexpr (TF32) {
        float h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) h[e] = tf32_hi(v[e]);
        hi = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
        if constexpr (SPLIT)
            lo = make_uint4(__float_as_uint(tf32_hi(v[0] - h[0])), __float_as_uint(tf32_hi(v[1] - h[1])),
                            __float_as_uint(tf32_hi(v[2] - h[2])), __float_as_uint(tf32_hi(v[3] - h[3])));
    } else {
        uint32_t w[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            w[e] = *(const uint32_t*)&hv;
            if constexpr (SPLIT) {
                const float2 hf = __bfloat1622float2(hv);
                l[e] = pack_bf16(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
            }
        }
        hi = make_uint4(w[0], w[1], w[2], w[3]);
        if constexpr (SPLIT) lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Epilogue of one (pair, slab of x planes): phi, nTiles M-tiles of 128 rows x n3p columns in
// TMEM, goes into the outputs (out -= mul * phi) and the weighted energy sum of this thread.
// rows(jt, r, x, y) gives the grid point (x, y) of row r of tile jt and whether it exists.
template <typename Rows>
__device__ __forceinline__ double consume_epilogue(const ConsumeArgs& a, const PairRec& rec, uint8_t* smem,
                                                   uint32_t tPhi, int nTiles, int warp, int lane, Rows rows,
                                                   int z0 = 0) {
    const int q = warp & 3, h = warp >> 2;
    double e = 0.0;
    const long N3 = (long)a.n1 * a.n2 * a.n3;
    const float* mul0 = a.MUL0 ? a.MUL0 + (long)rec.m0 * N3 : nullptr;
    const float* mul1 = a.MUL1 ? a.MUL1 + (long)rec.m1 * N3 : nullptr;
    float* out0 = (a.OUT0 && rec.o0 >= 0) ? a.OUT0 + (long)rec.o0 * N3 : nullptr;
    float* out1 = (a.OUT1 && rec.o1 >= 0) ? a.OUT1 + (long)rec.o1 * N3 : nullptr;
    const float* sa = a.SA + (long)rec.ia * N3;
    const float* sb = a.SB + (long)rec.ib * N3;
    const bool en = (a.flags & EPI_ENERGY) != 0;
    const bool o0 = (a.flags & EPI_OUT) && out0, o1 = (a.flags & EPI_OUT) && out1;
    // with symmetric pairs the energy factors (psi_a, psi_b) are the two multipliers
    // themselves: each orbital value is read once
    const bool need0 = o0 || (en && a.emul), need1 = o1 || (en && a.emul);
    // Each warp stages its quadrant's 32 rows x 64 columns of phi in shared memory (the
    // pipeline buffers are idle now), then walks the rows with consecutive z across lanes:
    // psi reads are coalesced and W is updated with 16-byte vector reductions.  The two
    // warps of a quadrant split the row pairs.  The orbital values of the next block are
    // copied to shared memory (cp.async) while the current block is processed, so their
    // HBM latency is hidden.
    float* stg = (float*)smem + warp * (32 * 68);
    float4* lbuf = (float4*)(smem + kStgBytes) + warp * (2 * 8 * 2 * 32);   // [buf][it][m][lane]
    const int sub = lane >> 4;
    const int ncb = (a.n3p + 63) / 64, nblk = nTiles * ncb;
    // row, grid offset and validity of iteration `it` of block `blk` for this lane (phi column
    // zl of the item is grid column z = z0 + zl)
    auto locate = [&](int blk, int it, int& x, int& y, int& z, int& idx) -> bool {
        const int jt = blk / ncb, cb = (blk - jt * ncb) * 64;
        const int zl = cb + 4 * (lane & 15);
        z = z0 + zl;
        if (!rows(jt, q * 32 + 2 * h + 4 * it + sub, x, y) || z >= a.n3 || zl >= a.n3p) return false;
        idx = (x * a.n2 + y) * a.n3 + z;       // < 256^3; a multiple of 4 (n3 % 4 == 0)
        return true;
    };
    auto prefetch = [&](int blk) {
        float4* d = lbuf + (blk & 1) * (8 * 2 * 32) + lane;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            int x, y, z, idx;
            if (!locate(blk, it, x, y, z, idx)) continue;
            if (need0) cp_async16(d + (2 * it) * 32, mul0 + idx);
            if (need1) cp_async16(d + (2 * it + 1) * 32, mul1 + idx);
        }
        cp_async_commit();
    };
    prefetch(0);
    for (int blk = 0; blk < nblk; ++blk) {
        const int jt = blk / ncb, cb = (blk - jt * ncb) * 64;
        if (blk + 1 < nblk) prefetch(blk + 1);
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
        if (blk + 1 < nblk) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncwarp();
        const float4* lb = lbuf + (blk & 1) * (8 * 2 * 32) + lane;
        // The energy terms of a block (at most 32 per thread) are summed in float32 and the block
        // sum is added in float64: this GPU runs float64 arithmetic at a small fraction of the
        // float32 rate, and a float64 multiply-add per grid point used to dominate this loop.
        float eb = 0.f;
        // lanes 0-15 take row rr, lanes 16-31 row rr + 1; four consecutive z per lane
#pragma unroll 2
        for (int it = 0; it < 8; ++it) {
            int x, y, z, idx;
            if (!locate(blk, it, x, y, z, idx)) continue;
            const int rr = 2 * h + 4 * it + sub;
            const float4 phi = *(const float4*)(stg + rr * 68 + 4 * (lane & 15));
            const float wxy = a.w1[x] * a.w2[y];
            const float4 w3 = *(const float4*)(a.w3 + z);
            const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
            float4 f = phi;
            if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
            const float4 m0 = need0 ? lb[(2 * it) * 32] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 m1 = need1 ? lb[(2 * it + 1) * 32] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (o0) atomicAdd((float4*)(out0 + idx), make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w));
            if (o1) atomicAdd((float4*)(out1 + idx), make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w));
            if (en) {
                const float4 va = a.emul ? m1 : *(const float4*)(sa + idx);
                const float4 vb = a.emul ? m0 : *(const float4*)(sb + idx);
                eb += wv.x * va.x * vb.x * phi.x + wv.y * va.y * vb.y * phi.y + wv.z * va.z * vb.z * phi.z +
                      wv.w * va.w * vb.w * phi.w;
            }
        }
        e += (double)eb;
        __syncwarp();
    }
    return e;
}

// Orbital and output arrays of the single-pass epilogue as TMA tensors: [orbital * n1 + x][y][z]
// float32, boxes of 32 z x 32 y, 128-byte swizzle.  Maps of absent arrays are never used.
struct EpiMaps {
    CUtensorMap m0, m1, sa, sb, o0, o1;
};
constexpr uint32_t kEpiBox = 32 * 32 * 4;   // one 32 x 32 float32 box
constexpr uint32_t kEpiWarpBytes = 6 * kEpiBox;   // six box slots per epilogue warp
constexpr int kEpiSets = 3;

// Epilogue of the single-pass kernel, on the copy engine.  Work units are (tile jt, 32-column
// z chunk): tile jt holds plane x0 + jt / nY, y rows (jt % nY) * 128 + lane.  The two warps of a
// TMEM lane quadrant take alternate units.  Per unit a warp loads the orbital boxes its outputs
// and energy need (TMA, 128-byte swizzle), each lane combines its own row of phi (tcgen05.ld)
// with them, writes -psi * phi in place, and lane 0 adds the boxes into W with TMA reductions:
// no per-element atomics.  The slots form a ring of up to three units, so the loads of the
// next units are in flight while one is combined.
__device__ __forceinline__ double consume_epilogue_tma(const ConsumeArgs& a, const EpiMaps& em, const PairRec& rec,
                                                       uint8_t* smem, uint64_t* ebar, uint32_t tPhi, int x0, int warp,
                                                       int lane) {
    const int q = warp & 3, h = warp >> 2;
    const bool en = (a.flags & EPI_ENERGY) != 0;
    const bool o0 = (a.flags & EPI_OUT) && a.OUT0 && rec.o0 >= 0, o1 = (a.flags & EPI_OUT) && a.OUT1 && rec.o1 >= 0;
    const bool need0 = o0 || (en && a.emul), need1 = o1 || (en && a.emul), needab = en && !a.emul;
    // box slots of a unit: m0, m1, then sa, sb (only those needed)
    const int k0 = 0, k1 = need0 ? 1 : 0, ka = k1 + (need1 ? 1 : 0), kb = ka + 1;
    const int nbox = ka + (needab ? 2 : 0);
    const int nsets = nbox == 0 ? 1 : min(kEpiSets, 6 / nbox);
    uint8_t* wbuf = smem + warp * kEpiWarpBytes;
    auto slot = [&](int set, int k) { return wbuf + (set * nbox + k) * kEpiBox; };
    const int nch = (a.n3 + 31) / 32, nunits = a.nT3 * nch;
    double e = 0.0;
    if (nbox == 0) return e;
    // this warp's units: h, h + 2, ...
    const int nmine = nunits > h ? (nunits - 1 - h) / 2 + 1 : 0;
    auto unit = [&](int i, int& x, int& y0, int& zc, int& jt) {
        const int u = h + 2 * i;
        jt = u / nch;
        zc = (u - jt * nch) * 32;
        const int p = jt / a.nY;
        x = x0 + p;
        y0 = (jt - p * a.nY) * 128 + q * 32;
        return x < a.n1 && y0 < a.n2;
    };
    bool pending[kEpiSets] = {false, false, false};   // a set's loads issued and not yet waited for
    auto issue = [&](int i) {
        int x, y0, zc, jt;
        if (!unit(i, x, y0, zc, jt)) return;
        const int set = i % nsets;
        pending[set] = true;
        if (lane != 0) return;
        mbar_arrive_expect_tx(&ebar[set], (uint32_t)nbox * kEpiBox);
        if (need0) tma_load_3d(slot(set, k0), &em.m0, &ebar[set], zc, y0, rec.m0 * a.n1 + x);
        if (need1) tma_load_3d(slot(set, k1), &em.m1, &ebar[set], zc, y0, rec.m1 * a.n1 + x);
        if (needab) {
            tma_load_3d(slot(set, ka), &em.sa, &ebar[set], zc, y0, rec.ia * a.n1 + x);
            tma_load_3d(slot(set, kb), &em.sb, &ebar[set], zc, y0, rec.ib * a.n1 + x);
        }
    };
    uint32_t use[kEpiSets] = {0u, 0u, 0u};
    for (int i = 0; i < nsets - 1 && i < nmine; ++i) issue(i);
    for (int i = 0; i < nmine; ++i) {
        const int set = i % nsets;
        int x, y0, zc, jt;
        const bool valid = unit(i, x, y0, zc, jt);
        if (i + nsets - 1 < nmine) {
            // set (i - 1) % nsets was last read by the reductions of unit i - 1
            if (i > 0) {
                if (lane == 0) bulk_wait_read0();
                __syncwarp();
            }
            issue(i + nsets - 1);
        }
        if (!valid) continue;
        // phi of this lane's row, 32 z (only the columns of this tile)
        uint32_t r[32];
        const uint32_t ta = tPhi + ((uint32_t)(q * 32) << 16) + (uint32_t)(jt * a.n3p + zc);
        tmem_ld16(ta, *(uint32_t(*)[16])&r[0]);
        if (zc + 16 < a.n3p) tmem_ld16(ta + 16, *(uint32_t(*)[16])&r[16]);
        const int y = y0 + lane;
        const bool rowin = y < a.n2;
        const float wxy = rowin ? a.w1[x] * a.w2[y] : 0.f;
        tmem_ld_wait();
        if (!mbar_wait(&ebar[set], use[set] & 1, a.err, 49)) break;
        pending[set] = false;
        ++use[set];
        float eb = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int z = zc + 4 * c;
            const uint32_t off = (uint32_t)lane * 128u + ((uint32_t)(c ^ (lane & 7)) << 4);
            float4 phi = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                     __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
            if (zc + 16 >= a.n3p && c >= 4) phi = make_float4(0.f, 0.f, 0.f, 0.f);   // columns past the tile
            const float4 w3 = (rowin && z < a.n3) ? *(const float4*)(a.w3 + z) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
            float4 f = phi;
            if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
            const float4 m0 = need0 ? *(const float4*)(slot(set, k0) + off) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 m1 = need1 ? *(const float4*)(slot(set, k1) + off) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (o0) *(float4*)(slot(set, k0) + off) = make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w);
            if (o1) *(float4*)(slot(set, k1) + off) = make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w);
            if (en && rowin && z < a.n3) {
                const float4 va = a.emul ? m1 : *(const float4*)(slot(set, ka) + off);
                const float4 vb = a.emul ? m0 : *(const float4*)(slot(set, kb) + off);
                eb += wv.x * va.x * vb.x * phi.x + wv.y * va.y * vb.y * phi.y + wv.z * va.z * vb.z * phi.z +
                      wv.w * va.w * vb.w * phi.w;
            }
        }
        e += (double)eb;
        if (o0 || o1) {
            // rows past n2 and columns past n3 lie outside the tensors: the reductions skip them
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (o0) tma_reduce_add_3d(&em.o0, slot(set, k0), zc, y0, rec.o0 * a.n1 + x);
                if (o1) tma_reduce_add_3d(&em.o1, slot(set, k1), zc, y0, rec.o1 * a.n1 + x);
                bulk_commit();
            }
        }
        __syncwarp();
    }
    // never leave with a load in flight (error path)
    for (int set = 0; set < kEpiSets; ++set)
        if (pending[set]) mbar_drain(&ebar[set], use[set] & 1, a.err);
    if (lane == 0) bulk_wait_all();
    __syncwarp();
    return e;
}

// Split precisions: phi of one accumulation chunk (main = hi*hi products, cross = hi*lo + lo*hi
// products, each in its own TMEM columns) is added in float32 into this thread's share of the
// register accumulator `mst`.  Thread (quadrant q, half h) owns TMEM lanes 32q..32q+31 and the
// 16-column groups g = h, h + 2, ... of the nT3 * n3p concatenated phi columns (group g, local
// index g / 2, values mst[16 * (g / 2) + j]).
template <int MG>
__device__ __forceinline__ void fold_chunk(uint32_t tPhi, uint32_t tPhiC, int q, int h, int ngroups, float (&mst)[MG * 16]) {
#pragma unroll
    for (int gi = 0; gi < MG; ++gi) {
        const int g = h + 2 * gi;
        if (g >= ngroups) break;
        uint32_t rm[16], rc[16];
        const uint32_t off = ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * g);
        tmem_ld16(tPhi + off, rm);
        tmem_ld16(tPhiC + off, rc);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) mst[16 * gi + j] += __uint_as_float(rm[j]) + __uint_as_float(rc[j]);
    }
}
// ... and written back into the main phi columns for the epilogue
template <int MG>
__device__ __forceinline__ void store_master(uint32_t tPhi, int q, int h, int ngroups, const float (&mst)[MG * 16]) {
#pragma unroll
    for (int gi = 0; gi < MG; ++gi) {
        const int g = h + 2 * gi;
        if (g >= ngroups) break;
        uint32_t r[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(mst[16 * gi + j]);
        tmem_st16(tPhi + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * g), r);
    }
    tmem_st_wait();
}

// Register share of the split precisions' phi accumulator: at most 4 groups of 16 columns per
// thread, i.e. nT3 * n3p <= 128 (the plan enforces it)
constexpr int kMasterGroups = 4;

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_consume(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mZlo,
              const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mA2lo,
              const __grid_constant__ CUtensorMap mA3, const __grid_constant__ CUtensorMap mA3lo, ConsumeArgs a) {
    constexpr int MK = TF32 ? 8 : 16;        // K per MMA instruction (32 bytes)
    constexpr int ES = TF32 ? 4 : 2;         // operand element bytes
    constexpr int CV = 16 / ES;              // values per 16-byte chunk
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kMaxLoad], empty_bar[kMaxLoad], a3full[2], a3free[2], phidone;
    __shared__ uint64_t fullB[kMaxLoadB], emptyB[kMaxLoadB];
    __shared__ uint64_t yfull, yfree, chunkdone, phifree;
    __shared__ uint32_t tmem_base;
    __shared__ double red[8];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // with y/z items (one plane per slab) blockIdx.x = (slab * nyi + iy) * nzi + iz: rows
    // y0 .. y0 + 127 of the plane and the columns z0 .. z0 + n3p - 1
    const int nyz = a.yz ? a.nyi * a.nzi : 1;
    const int slab = (int)blockIdx.x / nyz, iyz = (int)blockIdx.x - slab * nyz, pl = blockIdx.y;
    const int y0 = a.yz ? (iyz / a.nzi) * 128 : 0, z0 = a.yz ? (iyz % a.nzi) * a.n3p : 0;
    const int x0 = slab * a.bx;
    const PairRec rec = a.recs[a.p0 + pl];
    const int NL = a.nload, NA = a.na3, BX = a.bx;
    // Split precisions: the tensor core rounds its float32 accumulator after every MMA, toward
    // zero, so the error of a long accumulation grows with its length.  The hi*hi products and
    // the cross products (hi*lo + lo*hi, 2^-11 smaller) go to separate accumulators, and phi is
    // accumulated on the tensor core over chunks of C terms only (default 1): after each chunk
    // the converter warps add both accumulators into a float32 register accumulator (round to
    // nearest) and the tensor core restarts.  Single-pass precisions accumulate every term.
    const int C = SPLIT ? (a.chunk > 0 ? a.chunk : 1) : a.nt;
    // Gaussian terms in the order of the exponential sum (theta ascending: wide terms first)
    auto term_of = [&](int t) { return t; };

    // load stage s: [A_t2 tile][Z tile], each hi then lo; stage-3 stage sb: [A_t3 tile] hi then lo;
    // then the NA converted stage-3 operands
    const int NB = a.nloadB;
    auto YAs = [&](int s) { return smem + s * a.load_bytes; };
    auto Zs = [&](int s) { return YAs(s) + (SPLIT ? 2 : 1) * a.ya_bytes; };
    auto B3s = [&](int sb) { return smem + a.b_off + sb * a.loadB_bytes; };
    auto A3s = [&](int b) { return smem + a.a3_off + b * (SPLIT ? 2 : 1) * a.a3_bytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxLoad; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a3full[b], 8);
            mbar_init(&a3free[b], 1);
        }
        for (int b = 0; b < kMaxLoadB; ++b) {
            mbar_init(&fullB[b], 1);
            mbar_init(&emptyB[b], 1);
        }
        mbar_init(&yfull, 1);
        mbar_init(&yfree, 2 * a.nq);
        mbar_init(&phidone, 1);
        mbar_init(&chunkdone, 1);
        mbar_init(&phifree, 8);
        fence_barrier_init();
    }
    // the stage-3 operand: rows past the slab's last (x, y) are never written and must be finite
    {
        uint4* p = (uint4*)A3s(0);
        const int n16 = NA * (SPLIT ? 2 : 1) * a.a3_bytes / 16;
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
    // TMEM: [Y][phi] for the single-pass precisions; [Y][Y cross][phi][phi cross] for the split ones
    const uint32_t phi_cols = (uint32_t)(a.nT3 * a.n3p);
    const uint32_t tY = tmem, tYc = tmem + a.y_cols;
    const uint32_t tPhi = tmem + (SPLIT ? 2u : 1u) * a.y_cols, tPhiC = tPhi + phi_cols;
    const uint32_t ya_sub = a.ya_rows * 32u;                  // one K-step sub-tile of each operand
    const uint32_t z_sub = a.z_rows * 32u;
    const uint32_t a3_sub = (uint32_t)a.nT3 * 128u * 32u;

    if (warp == 8) {
        // ------------------------------ TMA producers ------------------------------
        // lane 0: the [A_t2][Z] ring; lane 1: the [mu_t A_t3] ring (each waits on its own ring)
        if (lane == 1) {
            int issued = 0;
            for (int t = 0; t < a.nt; ++t) {
                const int sb = t % NB;
                if (!mbar_wait(&emptyB[sb], ((t / NB) & 1) ^ 1, a.err, 39)) break;
                issued = t + 1;
                mbar_arrive_expect_tx(&fullB[sb], a.stageB_tx);
                const int tt = term_of(t);
                for (int k = 0; k < a.ks3; ++k) {
                    tma_load_3d(B3s(sb) + k * a.n3p * 32u, &mA3, &fullB[sb], k * MK, z0, tt);
                    if constexpr (SPLIT)
                        tma_load_3d(B3s(sb) + a.b3_bytes + k * a.n3p * 32u, &mA3lo, &fullB[sb], k * MK, z0, tt);
                }
            }
            if (issued < a.nt)
                for (int t = (issued > NB ? issued - NB : 0); t < issued; ++t)
                    mbar_drain(&fullB[t % NB], (t / NB) & 1, a.err);
        }
        if (lane == 0) {
            int issued = 0;
            bool ok = true;
            for (int t = 0; t < a.nt && ok; ++t) {
                const int s = t % NL;
                if (!mbar_wait(&empty_bar[s], ((t / NL) & 1) ^ 1, a.err, 31)) { ok = false; break; }
                issued = t + 1;
                // start the HBM reads of later Z tiles early (into L2 only)
                for (int ahead = (t == 0 ? 1 : NL + 1); ahead <= NL + 1; ++ahead)
                    if (t + ahead < a.nt)
                        for (int p = 0; p < BX; ++p)
                            for (int k = 0; k < a.ks2; ++k)
                                tma_prefetch_l2_3d(&mZ, k * MK, (x0 + p) * a.r3, pl * a.nt + term_of(t + ahead));
                mbar_arrive_expect_tx(&full_bar[s], a.stage_tx);
                const int tt = term_of(t);
                const int zdep = pl * a.nt + tt;
                for (int k = 0; k < a.ks2; ++k) {
                    tma_load_3d(YAs(s) + k * ya_sub, &mA2, &full_bar[s], k * MK, y0, tt);
                    if constexpr (SPLIT) tma_load_3d(YAs(s) + a.ya_bytes + k * ya_sub, &mA2lo, &full_bar[s], k * MK, y0, tt);
                    // plane p's rows start at row p * Nz (a multiple of 16) of the Z tile
                    for (int p = 0; p < BX; ++p) {
                        const uint32_t off = k * z_sub + (uint32_t)(p * a.Nz) * 32u;
                        tma_load_3d(Zs(s) + off, &mZ, &full_bar[s], k * MK, (x0 + p) * a.r3, zdep);
                        if constexpr (SPLIT)
                            tma_load_3d(Zs(s) + a.z_bytes + off, &mZlo, &full_bar[s], k * MK, (x0 + p) * a.r3, zdep);
                    }
                }
            }
            if (!ok)
                for (int t = (issued > NL ? issued - NL : 0); t < issued; ++t)
                    mbar_drain(&full_bar[t % NL], (t / NL) & 1, a.err);
        }
    } else if (warp == 9) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            const uint32_t id3 = TF32 ? idesc_tf32(128, a.n3p) : idesc_bf16(128, a.n3p);
            // Event-driven issue: stage 2 of term t2 as soon as its load stage has landed and the
            // converters have released Y; stage 3 of term t3 as soon as its operand is converted
            // (and, at the start of an accumulation chunk, the previous chunk has been folded).
            // All planes of a term go in one MMA per K step (N = planes x Nz, in chunks of <= 256).
            // Descriptors are built once and advanced by adds.
            const uint64_t d0 = sdesc_sw32(0);
            const uint64_t ya_step = ya_sub >> 4, z_step = z_sub >> 4, b3_step = (uint32_t)a.n3p * 2u;
            const uint64_t a3_step = a3_sub >> 4, ya_lo = a.ya_bytes >> 4, z_lo = a.z_bytes >> 4;
            const uint64_t b3_lo = a.b3_bytes >> 4, a3_lo = a.a3_bytes >> 4;
            auto stage2 = [&](int t) {
                const int s = t % NL;
                const uint64_t ya = d0 + (smem_u32(YAs(s)) >> 4), zb = d0 + (smem_u32(Zs(s)) >> 4);
                for (int i = 0; i < a.nY; ++i)
                    for (int p0 = 0; p0 < BX; p0 += a.npc) {
                        const int N = min(a.npc, BX - p0) * a.Nz;
                        const uint32_t id2 = TF32 ? idesc_tf32(128, N) : idesc_bf16(128, N);
                        const uint32_t col = (uint32_t)((i * BX + p0) * a.Nz);
                        uint64_t ad = ya + (uint32_t)i * 256u, bd = zb + (uint32_t)(p0 * a.Nz) * 2u;
                        for (int k = 0; k < a.ks2; ++k) {
                            mma_ss<TF32>(tY + col, ad, bd, id2, k > 0 ? 1u : 0u);
                            if constexpr (SPLIT) {
                                mma_ss<TF32>(tYc + col, ad, bd + z_lo, id2, k > 0 ? 1u : 0u);
                                mma_ss<TF32>(tYc + col, ad + ya_lo, bd, id2, 1u);
                            }
                            ad += ya_step;
                            bd += z_step;
                        }
                    }
                mma_commit(&yfull);
                mma_commit(&empty_bar[s]);          // the [A_t2][Z] stage is free once these have run
            };
            auto stage3 = [&](int t) {
                const int sb = t % NB, b = t % NA;
                const uint64_t a3 = d0 + (smem_u32(A3s(b)) >> 4), b3 = d0 + (smem_u32(B3s(sb)) >> 4);
                const bool first = (t % C) == 0;
                for (int j = 0; j < a.nT3; ++j) {
                    uint64_t ad = a3 + (uint32_t)j * 256u, bd = b3;
                    for (int k = 0; k < a.ks3; ++k) {
                        const uint32_t acc = (!first || k > 0) ? 1u : 0u;
                        mma_ss<TF32>(tPhi + j * a.n3p, ad, bd, id3, acc);
                        if constexpr (SPLIT) {
                            mma_ss<TF32>(tPhiC + j * a.n3p, ad, bd + b3_lo, id3, acc);
                            mma_ss<TF32>(tPhiC + j * a.n3p, ad + a3_lo, bd, id3, 1u);
                        }
                        ad += a3_step;
                        bd += b3_step;
                    }
                }
                mma_commit(&a3free[b]);
                mma_commit(&emptyB[sb]);
            };
            bool ok = true, fresh = true;
            int t2 = 0, t3 = 0;
            uint32_t idle = 0;
            uint64_t since = 0;
            while (t3 < a.nt) {
                bool prog = false;
                if (t2 < a.nt && mbar_try_wait(&full_bar[t2 % NL], (t2 / NL) & 1) &&
                    (t2 == 0 || mbar_try_wait(&yfree, (t2 - 1) & 1))) {
                    tc_fence_after();
                    stage2(t2);
                    ++t2;
                    prog = true;
                }
                // a new accumulation chunk starts once the previous one has been folded out of TMEM
                if (t3 < t2 && mbar_try_wait(&a3full[t3 % NA], (t3 / NA) & 1) &&
                    mbar_try_wait(&fullB[t3 % NB], (t3 / NB) & 1) &&
                    (t3 % C != 0 || t3 == 0 || mbar_try_wait(&phifree, (t3 / C - 1) & 1))) {
                    tc_fence_after();
                    stage3(t3);
                    if constexpr (SPLIT)
                        if ((t3 + 1) % C == 0 || t3 + 1 == a.nt) mma_commit(&chunkdone);
                    ++t3;
                    prog = true;
                }
                if (prog) {
                    fresh = true;
                    idle = 0;
                } else if ((++idle & 63) == 0) {
                    if (*(volatile int*)a.err != 0) { ok = false; break; }
                    const uint64_t now = globaltimer();
                    if (fresh) {
                        since = now;
                        fresh = false;
                    } else if (now - since > wait_limit_ns(a.err)) {
                        if (atomicCAS(a.err, 0, 1) == 0) atomicExch(a.err + 1, 32);
                        ok = false;
                        break;
                    }
                }
            }
            mma_commit(&phidone);
            // on the error path nobody else waits: keep the CTA (and its TMEM) until the MMAs
            // already issued have finished
            if (!ok) mbar_drain(&phidone, 0, a.err);
        }
    } else {
        // ------------------------------ converters (warps 0-7) ------------------------------
        // warp (q, h) converts the TMEM lanes 32q..32q+31 (y) of the planes p = h, h + 2, ...
        const int q = warp & 3, h = warp >> 2;
        const bool active = q < a.nq;
        bool ok = true;
        double e = 0.0;
        auto rows_of = [&](int jt, int r, int& x, int& y) {
            const int m3 = jt * 128 + r;
            if (a.yz) {                      // one plane, rows y0 .. y0 + 127
                y = y0 + m3;
                x = x0;
                return m3 < 128 && y < a.n2 && x < a.n1;
            }
            const int xl = m3 / a.n2;
            y = m3 - xl * a.n2;
            x = x0 + xl;
            return m3 < a.R && x < a.n1;
        };
        const int ngroups = (int)phi_cols / 16;
        float mst[kMasterGroups * 16];
#pragma unroll
        for (int j = 0; j < kMasterGroups * 16; ++j) mst[j] = 0.f;
        for (int t = 0; t < a.nt && ok; ++t) {
            const int b = t % NA;
            if (t >= NA && !mbar_wait(&a3free[b], ((t - NA) / NA) & 1, a.err, 36)) { ok = false; break; }
            uint8_t* a3 = A3s(b);
            if (active) {
                if (!mbar_wait(&yfull, t & 1, a.err, 35)) { ok = false; break; }
                tc_fence_after();
                for (int p = h; p < BX; p += 2) {
                    for (int i = 0; i < a.nY; ++i) {
                        const int y = i * 128 + q * 32 + lane;
                        const bool valid = y0 + y < a.n2;
                        const uint32_t m3 = (uint32_t)(a.yz ? y : p * a.n2 + y);
                        const uint32_t col = tY + ((uint32_t)(q * 32) << 16) + (uint32_t)((i * BX + p) * a.Nz);
                        for (int g0 = 0; g0 < a.r3; g0 += 64) {
                            const int nck = min(4, (min(a.Nz, g0 + 64) - g0) / 16);
                            uint32_t r[4][16];
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if (c < nck) tmem_ld16(col + g0 + 16 * c, r[c]);
                            tmem_ld_wait();
                            if constexpr (SPLIT) {
                                // Y = main + cross accumulator
#pragma unroll
                                for (int c = 0; c < 4; ++c)
                                    if (c < nck) {
                                        uint32_t rc[16];
                                        tmem_ld16(col + a.y_cols + g0 + 16 * c, rc);
                                        tmem_ld_wait();
#pragma unroll
                                        for (int j = 0; j < 16; ++j)
                                            r[c][j] = __float_as_uint(__uint_as_float(r[c][j]) + __uint_as_float(rc[j]));
                                    }
                            }
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                if (c >= nck) break;
#pragma unroll
                                for (int u = 0; u < 16 / CV; ++u) {
                                    const int g = g0 + 16 * c + CV * u;          // first column of the chunk
                                    if (!valid || g >= a.r3) continue;
                                    float v[CV];
#pragma unroll
                                    for (int e = 0; e < CV; ++e)
                                        v[e] = (g + e < a.r3) ? __uint_as_float(r[c][CV * u + e]) : 0.f;
                                    uint4 hi, lo;
                                    convert_chunk<TF32, SPLIT>(v, hi, lo);
                                    const uint32_t ks = (uint32_t)(g / MK), bin = (uint32_t)((g % MK) * ES);
                                    uint8_t* dst = a3 + ks * a3_sub + sw32_offset(m3, bin);
                                    *(uint4*)dst = hi;
                                    if constexpr (SPLIT) *(uint4*)(dst + a.a3_bytes) = lo;
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&yfree);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a3full[b]);
            if constexpr (SPLIT) {
                // end of an accumulation chunk: fold phi into the register accumulator and let
                // the tensor core restart
                if ((t + 1) % C == 0 || t + 1 == a.nt) {
                    if (!mbar_wait(&chunkdone, (t / C) & 1, a.err, 38)) { ok = false; break; }
                    tc_fence_after();
                    fold_chunk<kMasterGroups>(tPhi, tPhiC, q, h, ngroups, mst);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&phifree);
                }
            }
        }
        // ------------------------------ epilogue ------------------------------
        if (ok && mbar_wait_idle(&phidone, 0, a.err, 37) && *(volatile int*)a.err == 0) {
            tc_fence_after();
            if constexpr (SPLIT) {
                // the register accumulator goes back into the main phi columns for the epilogue,
                // which every converter warp reads for its whole lane quadrant
                store_master<kMasterGroups>(tPhi, q, h, ngroups, mst);
                tc_fence_before();
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
            tc_fence_after();
            e += consume_epilogue(a, rec, smem, tPhi, a.nT3, warp, lane, rows_of, z0);
        } else {
            asm volatile("bar.sync 1, 256;" ::: "memory");   // the eight warps meet here on every path
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
        a.epart[(long)pl * gridDim.x + blockIdx.x] = s;
    }
    if (warp == 8) tmem_dealloc(tmem, a.tmem_cols);
}

// MMA issue sequences of the single-pass kernel.  Every descriptor of a sequence is a per-term
// base plus an immediate and the K steps are unrolled at compile time: a runtime loop or a
// dispatch around the instructions costs the issuing warp more per MMA than the tensor pipe
// needs to run one of these tiles.  The kernel is instantiated for the common step counts
// (KS > 0); other ranks take the dispatch below (KS == 0).
//   stage 2: KS K steps of one 128 x N tile; A (A_t2) and B (Z) K-major, 128-byte swizzle,
//            atoms of 4 K steps `a16` / `b16` descriptor units apart
//   stage 3: KS = 4 * na + kt K steps; A = Y from TMEM (8 columns per step), B = mu_t A_t3:
//            na full 128-byte-swizzled atoms `atom16` apart, then kt 32-byte-swizzled K steps
//            `tail16` apart
template <bool TF32, int KS>
__device__ __forceinline__ void s2_mmas_k(uint32_t d, uint64_t ad, uint64_t bd, uint32_t a16, uint32_t b16, uint32_t id,
                                          uint32_t acc0) {
#pragma unroll
    for (int k = 0; k < KS; ++k)
        mma_ss_w<TF32>(d, ad + (uint32_t)(k >> 2) * a16 + (uint32_t)(k & 3) * 2u,
                       bd + (uint32_t)(k >> 2) * b16 + (uint32_t)(k & 3) * 2u, id, k > 0 ? 1u : acc0);
}
template <bool TF32, int KS>
__device__ __forceinline__ void s2_mmas(int ks, uint32_t d, uint64_t ad, uint64_t bd, uint32_t a16, uint32_t b16,
                                        uint32_t id, uint32_t acc0 = 0u) {
    if constexpr (KS > 0) {
        s2_mmas_k<TF32, KS>(d, ad, bd, a16, b16, id, acc0);
    } else {
        switch (ks) {
            case 1: s2_mmas_k<TF32, 1>(d, ad, bd, a16, b16, id, acc0); break;
            case 2: s2_mmas_k<TF32, 2>(d, ad, bd, a16, b16, id, acc0); break;
            case 3: s2_mmas_k<TF32, 3>(d, ad, bd, a16, b16, id, acc0); break;
            case 4: s2_mmas_k<TF32, 4>(d, ad, bd, a16, b16, id, acc0); break;
            case 5: s2_mmas_k<TF32, 5>(d, ad, bd, a16, b16, id, acc0); break;
            case 6: s2_mmas_k<TF32, 6>(d, ad, bd, a16, b16, id, acc0); break;
            case 8: s2_mmas_k<TF32, 8>(d, ad, bd, a16, b16, id, acc0); break;
            default:
                for (int k = 0; k < ks; ++k)
                    mma_ss_w<TF32>(d, ad + (uint32_t)(k >> 2) * a16 + (uint32_t)(k & 3) * 2u,
                                   bd + (uint32_t)(k >> 2) * b16 + (uint32_t)(k & 3) * 2u, id, k > 0 ? 1u : acc0);
        }
    }
}
template <int KS>
__device__ __forceinline__ void s3_mmas_k(uint32_t d, uint32_t aT, uint64_t b3, uint64_t b3t, uint32_t atom16,
                                          uint32_t tail16, uint32_t id, uint32_t acc0) {
    constexpr int NF = (KS / 4) * 4;   // K steps in full 128-byte atoms; the rest is the 32-byte tail
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const uint64_t bd = k < NF ? b3 + (uint32_t)(k >> 2) * atom16 + (uint32_t)(k & 3) * 2u
                                   : b3t + (uint32_t)(k - NF) * tail16;
        mma_ts_tf32_w(d, aT + 8u * k, bd, id, k > 0 ? 1u : acc0);
    }
}
// stage 3 of the bf16-in-TMEM form: A = Y rounded to bf16 in TMEM (8 columns per K step of 16),
// B = mu_t A_t3 in bf16, 128-byte swizzled K-major atoms of 4 K steps
template <int KS>
__device__ __forceinline__ void s3b_mmas(int ks, uint32_t d, uint32_t aT, uint64_t b3, uint32_t atom16, uint32_t id,
                                         uint32_t acc0) {
    const int n = KS > 0 ? KS : ks;
#pragma unroll
    for (int k = 0; k < n; ++k)
        mma_ts_bf16_w(d, aT + 8u * k, b3 + (uint32_t)(k >> 2) * atom16 + (uint32_t)(k & 3) * 2u, id, k > 0 ? 1u : acc0);
}
template <int KS>
__device__ __forceinline__ void s3_mmas(int ks, uint32_t d, uint32_t aT, uint64_t b3, uint64_t b3t, uint32_t atom16,
                                        uint32_t tail16, uint32_t id, uint32_t acc0) {
    if constexpr (KS > 0) {
        s3_mmas_k<KS>(d, aT, b3, b3t, atom16, tail16, id, acc0);
    } else {
        switch (ks) {
            case 1: s3_mmas_k<1>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 2: s3_mmas_k<2>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 3: s3_mmas_k<3>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 4: s3_mmas_k<4>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 5: s3_mmas_k<5>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 6: s3_mmas_k<6>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 7: s3_mmas_k<7>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            case 8: s3_mmas_k<8>(d, aT, b3, b3t, atom16, tail16, id, acc0); break;
            default: {
                const int nf = (ks / 4) * 4;
                for (int k = 0; k < ks; ++k) {
                    const uint64_t bd = k < nf ? b3 + (uint32_t)(k >> 2) * atom16 + (uint32_t)(k & 3) * 2u
                                               : b3t + (uint32_t)(k - nf) * tail16;
                    mma_ts_tf32_w(d, aT + 8u * k, bd, id, k > 0 ? 1u : acc0);
                }
            }
        }
    }
}

// Variant for the single-pass precisions: stage 3 runs as kind::tf32 with its A operand read
// straight from TMEM.  Stage 2 leaves Y_t,x[y][g] in TMEM with y on the lanes and g on the
// columns, which is exactly the K-major layout of an A operand whose rows are the y of one x
// plane; so stage 3 is one 128-row MMA tile per plane, and no warp touches Y.
//
// Schedule.  Warp 9 issues stage 2 of every term into nyb rotating Y buffers; warps 0..ns3-1
// issue stage 3, one x plane each, as soon as the term's stage 2 has finished, and then run
// the epilogue with warps 1..7.  A warp needs more time to issue a tcgen05.mma than the tensor
// pipe needs to run one of these small tiles, so the stage-3 streams are issued in parallel.
//
// Loads.  Operand tiles use the 128-byte swizzle.  The stage-2 operands (A_t2 tile and the
// slab's Z planes) and the stage-3 operand (mu_t A_t3) travel in two separate rings of load
// stages, each with its own producer warp (8 and 10): a stage-2 stage is free again as soon
// as stage 2 of its term has run, so the Z reads from HBM start several terms ahead instead
// of waiting for the slower stage-3 release.  A_t2 and mu_t A_t3 arrive as plain bulk copies
// of a per-context image (k_operand_image below); each Z plane is one TMA box.
template <bool S2TF32, int KS2, int KS3>
__global__ void __launch_bounds__(kThreadsTs, 1)
    k_consume_ts(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ EpiMaps em, ConsumeArgs a) {
    constexpr int AK2 = S2TF32 ? 32 : 64;    // stage-2 elements per 128-byte atom (4 MMA K steps)
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kMaxLoad], empty_bar[kMaxLoad], full3[kMaxLoad], empty3[kMaxLoad];
    __shared__ uint64_t s2bar[kMaxYBuf], ybar[kMaxYBuf], phidone, s2fin, ebar[8][kEpiSets];
    __shared__ uint32_t tmem_base;
    __shared__ double red[8];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slab = blockIdx.x, pl = blockIdx.y;
    const int x0 = slab * a.bx;
    const PairRec rec = a.recs[a.p0 + pl];
    const int NL = a.nload, NL3 = a.nload3, NYB = a.nyb, BX = a.bx;
    auto term_of = [&](int t) { return t; };     // theta ascending, as in the split-precision kernel

    // stage-2 ring, stage s: [A_t2 tile][Z tile]; stage-3 ring, stage s: [mu_t A_t3 tile (tf32)];
    // every tile [atom][rows][128 bytes] (the A_t3 K tail: [rows][32 bytes])
    auto YAs = [&](int s) { return smem + s * a.load_bytes; };
    auto Zs = [&](int s) { return YAs(s) + a.ya_bytes; };
    auto B3s = [&](int s) { return smem + a.a3_off + s * a.load3_bytes; };

    if (threadIdx.x == 0) {
        // stage-2 stages are released by the stage-2 warp, stage-3 stages, Y buffers and phi by
        // each of the ns3 plane warps
        for (int s = 0; s < kMaxLoad; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&full3[s], 1);
            mbar_init(&empty3[s], a.ns3);
        }
        for (int b = 0; b < kMaxYBuf; ++b) {
            mbar_init(&s2bar[b], 1);
            mbar_init(&ybar[b], a.ns3);
        }
        mbar_init(&phidone, a.ns3);
        mbar_init(&s2fin, 1);
        for (int w = 0; w < 8; ++w)
            for (int k = 0; k < kEpiSets; ++k) mbar_init(&ebar[w][k], 1);
        fence_barrier_init();
    }
    // Z tile rows that no copy writes (rows r3..gs-1 of each plane, the tail up to the MMA's N)
    // feed Y columns that stage 3 multiplies by zeros: they must hold finite values
    for (int s = 0; s < NL; ++s) {
        uint4* z = (uint4*)Zs(s);
        for (int i = threadIdx.x; i < (int)(a.z_bytes / 16); i += kThreadsTs) z[i] = make_uint4(0, 0, 0, 0);
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
    const uint32_t tPhi = tmem + (uint32_t)NYB * a.y_cols;
    const uint32_t ya_atom = a.ya_rows * 128u, z_atom = a.z_rows * 128u, b3_atom = (uint32_t)a.n3p * 128u;
    // mu_t A_t3: na3f full 128-byte atoms (32 K each), then the K tail in 32-byte rows (so that
    // no row is mostly zero fill)
    const int na3f = a.ks3 / 4;

    // The producer and MMA roles run on whole warps with uniform control flow; one elected lane
    // issues each TMA / tcgen05 instruction (see the _w helpers).
    if (warp == 8) {
        // ------------------------- stage-2 producer: A_t2 and Z -------------------------
        const int na2 = (a.ks2 + 3) / 4;   // 128-byte atoms along K
        int issued = 0, s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int t = 0; t < a.nt && ok; ++t) {
            ok = mbar_wait(&empty_bar[s], ph ^ 1, a.err, 41);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            issued = t + 1;
            mbar_arrive_expect_tx_w(&full_bar[s], a.stage_tx);
            const int tt = term_of(t);
            const int zdep = pl * a.nt + tt;
            bulk_load_w(YAs(s), a.img + (size_t)tt * a.img_stride, a.ya_bytes, &full_bar[s]);
            if (a.zone) {
                // planes packed back to back (gs == r3): one box of bx * r3 rows per K atom
                tma_load_3d_w(Zs(s), &mZ, &full_bar[s], 0, x0 * a.r3, zdep);
                for (int k = 1; k < na2; ++k)
                    tma_load_3d_w(Zs(s) + k * z_atom, &mZ, &full_bar[s], k * AK2, x0 * a.r3, zdep);
            } else {
                for (int k = 0; k < na2; ++k)
                    // plane p's rows start at row p * gs (a multiple of 8) of the Z tile
                    for (int p = 0; p < BX; ++p)
                        tma_load_3d_w(Zs(s) + k * z_atom + (uint32_t)(p * a.gs) * 128u, &mZ, &full_bar[s], k * AK2,
                                      (x0 + p) * a.r3, zdep);
            }
            if (++s == NL) { s = 0; ph ^= 1; }
        }
        if (!ok)
            for (int t = (issued > NL ? issued - NL : 0); t < issued; ++t) mbar_drain(&full_bar[t % NL], (t / NL) & 1, a.err);
    } else if (warp == 10) {
        // ------------------- stage-3 producer: mu_t A_t3, and the Z prefetches -------------------
        // The slab's planes of one term are contiguous in Z: one L2 prefetch per term, issued
        // here (this warp runs a few terms behind stage 2, so nl + 2 terms ahead of its own
        // position is ahead of the stage-2 loads) to keep the stage-2 producer's issue short.
        const int nplanes = min(BX, a.n1 - x0);
        const uint32_t zbytes = (uint32_t)nplanes * a.z_plane;
        const uint8_t* zslab = a.zsrc + ((size_t)pl * a.nt * a.n1 + x0) * a.z_plane;
        const size_t zterm = (size_t)a.n1 * a.z_plane;
        int issued = 0, s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int t = 1; t <= NL + 2 && t < a.nt; ++t) bulk_prefetch_l2_w(zslab + (size_t)term_of(t) * zterm, zbytes);
        for (int t = 0; t < a.nt && ok; ++t) {
            ok = mbar_wait(&empty3[s], ph ^ 1, a.err, 46);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            issued = t + 1;
            mbar_arrive_expect_tx_w(&full3[s], a.b3_bytes);
            bulk_load_w(B3s(s), a.img + (size_t)term_of(t) * a.img_stride + a.ya_bytes, a.b3_bytes, &full3[s]);
            if (t > 0 && t + NL + 2 < a.nt) bulk_prefetch_l2_w(zslab + (size_t)term_of(t + NL + 2) * zterm, zbytes);
            if (++s == NL3) { s = 0; ph ^= 1; }
        }
        if (!ok)
            for (int t = (issued > NL3 ? issued - NL3 : 0); t < issued; ++t) mbar_drain(&full3[t % NL3], (t / NL3) & 1, a.err);
    } else if (warp == 9) {
        // ------------------------------ stage-2 MMA issuer ------------------------------
        // descriptors are built once and advanced by adds: +32 bytes (2 units of the
        // address / 16 field) per K step inside a 128-byte atom, one atom stride every 4 steps
        //
        // Ring positions advance by counters, not t % n: a runtime division per barrier index
        // sits on this warp's critical path every term.  The common tile (y tile 0, the first
        // chunk of planes) is issued outside any runtime loop; other tiles follow in a loop.
        const uint64_t d0 = sdesc_sw128(0);
        const int n0 = pad16c(min(a.npc, BX) * a.gs);
        const uint32_t id0 = S2TF32 ? idesc_tf32(128, n0) : idesc_bf16(128, n0);
        const bool more = a.nY > 1 || a.npc < BX;
        int s = 0, yb = 0;
        uint32_t ph = 0, yph = 0;
        bool ok = true;
        for (int t = 0; t < a.nt && ok; ++t) {
            bool w = mbar_wait(&full_bar[s], ph, a.err, 42);
            // Y buffer yb was last read by stage 3 of term t - nyb
            if (w && t >= NYB) w = mbar_wait(&ybar[yb], yph ^ 1, a.err, 43);
            if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
            tc_fence_after();
            const uint64_t ya = d0 + (smem_u32(YAs(s)) >> 4), zb = d0 + (smem_u32(Zs(s)) >> 4);
            const uint32_t tY = tmem + (uint32_t)yb * a.y_cols;
            s2_mmas<S2TF32, KS2>(a.ks2, tY, ya, zb, ya_atom >> 4, z_atom >> 4, id0);
            if (more)
                for (int i = 0; i < a.nY; ++i)
                    for (int p0 = (i == 0 ? a.npc : 0); p0 < BX; p0 += a.npc) {
                        const int N = pad16c(min(a.npc, BX - p0) * a.gs);
                        const uint32_t id2 = S2TF32 ? idesc_tf32(128, N) : idesc_bf16(128, N);
                        const uint32_t d = tY + (uint32_t)(i * a.ycol_tile + p0 * a.gs);
                        s2_mmas<S2TF32, KS2>(a.ks2, d, ya + (uint32_t)i * 1024u, zb + (uint32_t)(p0 * a.gs) * 8u,
                                          ya_atom >> 4, z_atom >> 4, id2);
                    }
            mma_commit_w(&s2bar[yb]);
            mma_commit_w(&empty_bar[s]);
            if (++s == NL) { s = 0; ph ^= 1; }
            if (++yb == NYB) { yb = 0; yph ^= 1; }
        }
        // the CTA must not release TMEM while these MMAs run
        mma_commit_w(&s2fin);
        mbar_drain(&s2fin, 0, a.err);
    } else {
        // ---------------- stage-3 MMA issuers (warps 0..nS3-1), then the epilogue ----------------
        // Issuing one tcgen05.mma costs a warp more time than the tensor pipe needs to run it at
        // these sizes, so stage 3 is issued by one warp per x plane in parallel (each plane
        // accumulates into its own TMEM columns) while warp 9 issues stage 2.
        double e = 0.0;
        bool ok = true;
        if (warp < a.ns3) {
            // ring counters and a loop-free common case, as in the stage-2 issuer: this warp's
            // first plane (warp < ns3 <= bx), y tile 0; further planes / y tiles in a loop
            const uint32_t id3 = idesc_tf32(128, a.n3p);
            const uint64_t d0 = sdesc_sw128(0);
            const uint32_t dP = tPhi + (uint32_t)(warp * a.nY * a.n3p), aP = (uint32_t)(warp * a.gs);
            const bool more = a.nY > 1 || BX > a.ns3;
            int s = 0, yb = 0;
            uint32_t ph = 0, yph = 0;
            for (int t = 0; t < a.nt && ok; ++t) {
                bool w = mbar_wait(&s2bar[yb], yph, a.err, 44);
                if (w) w = mbar_wait(&full3[s], ph, a.err, 48);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                tc_fence_after();
                const uint64_t b3 = d0 + (smem_u32(B3s(s)) >> 4);
                const uint64_t b3t = sdesc_sw32(0) + (smem_u32(B3s(s) + na3f * b3_atom) >> 4);
                const uint32_t tY = tmem + (uint32_t)yb * a.y_cols;
                const uint32_t acc0 = t > 0 ? 1u : 0u;
                s3_mmas<KS3>(a.ks3, dP, tY + aP, b3, b3t, b3_atom >> 4, (uint32_t)a.n3p * 2u, id3, acc0);
                if (more)
                    for (int p = warp; p < BX; p += a.ns3)
                        for (int i = (p == warp ? 1 : 0); i < a.nY; ++i) {
                            const uint32_t aT = tY + (uint32_t)(i * a.ycol_tile + p * a.gs);
                            const uint32_t d = tPhi + (uint32_t)((p * a.nY + i) * a.n3p);
                            s3_mmas<KS3>(a.ks3, d, aT, b3, b3t, b3_atom >> 4, (uint32_t)a.n3p * 2u, id3, acc0);
                        }
                mma_commit_w(&ybar[yb]);
                mma_commit_w(&empty3[s]);
                if (++s == NL3) { s = 0; ph ^= 1; }
                if (++yb == NYB) { yb = 0; yph ^= 1; }
            }
            mma_commit_w(&phidone);
        }
        if (ok && mbar_wait_idle(&phidone, 0, a.err, 45) && *(volatile int*)a.err == 0) {
            tc_fence_after();
            e = consume_epilogue_tma(a, em, rec, smem, ebar[warp], tPhi, x0, warp, lane);
        } else if (warp < a.ns3) {
            mbar_drain(&phidone, 0, a.err);
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

// Persistent form of the single-pass kernel.  One CTA per SM walks the work items (pair, slab)
// blockIdx.x, blockIdx.x + gridDim.x, ...; the two load rings and the MMAs run across item
// boundaries without a break, and the epilogue of item k overlaps the main loop of item k + 1:
// as soon as the last stage-3 MMA of item k has run, the epilogue warps copy phi from TMEM into
// registers (each lane one row of one tile, at most 96 columns) and release the accumulator,
// then combine it with the orbital boxes and reduce into W through the copy engine while the
// next item accumulates.  Warp roles: 0-7 epilogue, 8 stage-2 producer, 9 stage-2 MMAs, 10
// stage-3 producer and Z prefetches, 11 stage-3 MMAs of every plane.  Used when every epilogue
// warp holds at most one tile (bx <= 2, bx * nY <= 2) and n3p <= 96.
constexpr int kTpMaxZ = 96;                           // phi registers per epilogue lane
constexpr int kThreadsTpB = 512;                      // bf16-in-TMEM form: warps 4-7 and 12-15 convert, 0-3 epilogue
constexpr int kThreadsTpD = 448;                      // dual-issuer form: second stage-2 and stage-3 MMA warps (12, 13)
constexpr uint32_t kTpEpiBytes = 0;                   // the epilogue reads the orbitals directly

template <bool S2TF32, int KS2, int KS3, bool BF3 = false, bool DUAL = false>
__global__ void __launch_bounds__(BF3 ? kThreadsTpB : (DUAL ? kThreadsTpD : kThreadsTp), 1)
    k_consume_tp(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ EpiMaps em, ConsumeArgs a) {
    static_assert(!(BF3 && DUAL), "one form at a time");
    constexpr int AK2 = S2TF32 ? 32 : 64;    // stage-2 elements per 128-byte atom (4 MMA K steps)
    constexpr int NTHR = BF3 ? kThreadsTpB : (DUAL ? kThreadsTpD : kThreadsTp);
    constexpr bool PHI2 = BF3 || DUAL;       // phi double-buffered in TMEM, read by the epilogue in place
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kMaxLoad], empty_bar[kMaxLoad], full3[kMaxLoad], empty3[kMaxLoad];
    __shared__ uint64_t s2bar[kMaxYBuf], ybar[kMaxYBuf], phidone, phifree, s3fin[2], ebar[8];
    __shared__ uint64_t cvtbar[kMaxYBuf];      // BF3: Y of the buffer converted to bf16
    __shared__ uint64_t phid[2], phif[2];      // BF3, DUAL: phi buffer b complete / read by the epilogue
    __shared__ uint64_t tok[2];                // DUAL: stage-3 MMAs of the even (0) / odd (1) terms issued
    __shared__ uint64_t tok2[2];               // DUAL: stage-2 operands of the even / odd terms arrived
    __shared__ uint64_t fin2[2];               // DUAL: final commits of MMA warps 12 and 13
    __shared__ uint32_t tmem_base;
    __shared__ double red[2][8];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NL = a.nload, NL3 = a.nload3, NYB = a.nyb, BX = a.bx, NT = a.nt;
    const int nmine = (int)blockIdx.x < a.nitems ? (a.nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // item it = ((pair * nslab) + slab) * nyi + iy: with nyi > 1 an item covers one 128-row y
    // tile (iy) of its slab's planes (a.nY is then 1), so that phi and the Y buffers of grids
    // with more than 128 rows per plane fit TMEM.  With packed tails (a.tailp > 0, one plane per
    // slab) a pair's items are its planes' full y tiles (slab, iy < nyi - 1), then its tail items
    // (iy = nyi - 1, slab = index of the group of tailp planes).  Either way it = pair * per_pair
    // + the item's index inside the pair.
    auto item_of = [&](int k, int& pl, int& slab, int& iy) {
        const int it = (int)blockIdx.x + k * (int)gridDim.x;
        if (a.tailp) {
            pl = it / a.per_pair;
            const int j = it - pl * a.per_pair, ym = a.nyi - 1, nm = a.nslab * ym;
            if (j < nm) {
                slab = j / ym;
                iy = j - slab * ym;
            } else {
                slab = j - nm;
                iy = ym;
            }
            return;
        }
        const int ps = it / a.nyi;
        iy = it - ps * a.nyi;
        pl = ps / a.nslab;
        slab = ps - pl * a.nslab;
    };
    auto is_tail = [&](int iy) { return a.tailp > 0 && iy == a.nyi - 1; };
    auto YAs = [&](int s) { return smem + s * a.load_bytes; };
    auto Zs = [&](int s) { return YAs(s) + a.ya_bytes; };
    auto B3s = [&](int s) { return smem + a.a3_off + s * a.load3_bytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxLoad; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&full3[s], 1);
            mbar_init(&empty3[s], 1);
        }
        for (int b = 0; b < kMaxYBuf; ++b) {
            mbar_init(&s2bar[b], 1);
            mbar_init(&ybar[b], 1);
            mbar_init(&cvtbar[b], 4);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&phid[b], DUAL ? 2 : 1);
            mbar_init(&phif[b], DUAL ? 8 : 4);
            mbar_init(&tok[b], 1);
            mbar_init(&tok2[b], 1);
            mbar_init(&fin2[b], 1);
        }
        mbar_init(&phidone, 1);
        mbar_init(&phifree, 8);
        mbar_init(&s3fin[0], 1);
        mbar_init(&s3fin[1], 1);
        for (int w = 0; w < 8; ++w) mbar_init(&ebar[w], 1);
        fence_barrier_init();
    }
    // Z tile rows that no copy writes feed Y columns that stage 3 multiplies by zeros
    for (int s = 0; s < NL; ++s) {
        uint4* z = (uint4*)Zs(s);
        for (int i = threadIdx.x; i < (int)(a.z_bytes / 16); i += NTHR) z[i] = make_uint4(0, 0, 0, 0);
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
    const uint32_t tPhi = tmem + (uint32_t)NYB * a.y_cols;
    const uint32_t phi_cols = (uint32_t)(a.nT3 * a.n3p);      // BF3, DUAL: phi is double-buffered
    const uint32_t ya_atom = a.ya_rows * 128u, z_atom = a.z_rows * 128u, b3_atom = (uint32_t)a.n3p * 128u;
    const uint32_t img_atom = a.img_ya_rows * 128u, img_ya_bytes = img_atom * (uint32_t)((a.ks2 + 3) / 4);
    const int na3f = a.ks3 / 4;
    const int na2 = (a.ks2 + 3) / 4;

    if (warp == 8) {
        // ------------------------- stage-2 producer: A_t2 and Z -------------------------
        int issued = 0, s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k) {
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const bool tail = is_tail(iy);
            // a tail item takes one stage per plane and term: that plane's window of A_t2 and its Z
            const int x0 = tail ? slab * a.tailp : slab * BX;
            const int nsub = tail ? min(a.tailp, a.n1 - x0) : 1;
            for (int t = 0; t < NT && ok; ++t)
                for (int sp = 0; sp < nsub; ++sp) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&empty_bar[s], ph ^ 1, a.err, 41));
                    if (!ok) break;
                    ++issued;
                    mbar_arrive_expect_tx_w(&full_bar[s], a.stage_tx);
                    const int zdep = pl * NT + t;
                    const int xz = x0 + sp;
                    const uint8_t* asrc = a.img + (size_t)t * a.img_stride +
                                          (tail ? a.win_off + (uint32_t)sp * img_ya_bytes : 0u);
                    if (a.tailp) {
                        // packed items read rows 0..127 of each K atom only
                        for (int kk = 0; kk < na2; ++kk)
                            bulk_load_w(YAs(s) + kk * ya_atom, asrc + kk * img_atom, 128u * 128u, &full_bar[s]);
                    } else {
                        bulk_load_w(YAs(s), asrc, a.ya_bytes, &full_bar[s]);
                    }
                    if (a.zone) {
                        tma_load_3d_w(Zs(s), &mZ, &full_bar[s], 0, xz * a.r3, zdep);
                        for (int kk = 1; kk < na2; ++kk)
                            tma_load_3d_w(Zs(s) + kk * z_atom, &mZ, &full_bar[s], kk * AK2, xz * a.r3, zdep);
                    } else {
                        for (int kk = 0; kk < na2; ++kk)
                            for (int p = 0; p < BX; ++p)
                                tma_load_3d_w(Zs(s) + kk * z_atom + (uint32_t)(p * a.gs) * 128u, &mZ, &full_bar[s],
                                              kk * AK2, (xz + p) * a.r3, zdep);
                    }
                    if (++s == NL) { s = 0; ph ^= 1; }
                }
        }
        if (!ok)
            for (int g = (issued > NL ? issued - NL : 0); g < issued; ++g) mbar_drain(&full_bar[g % NL], (g / NL) & 1, a.err);
    } else if (warp == 10) {
        // ---------------- stage-3 producer: mu_t A_t3, and the Z L2 prefetches ----------------
        const size_t zterm = (size_t)a.n1 * a.z_plane;
        // global term g = k * nt + t; the prefetch runs nl + 2 terms ahead, across items
        auto prefetch = [&](int g) {
            const int k = g / NT, t = g - k * NT;
            if (k >= nmine) return;
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const bool tail = is_tail(iy);
            const int x0 = tail ? slab * a.tailp : slab * BX;
            const int np_ = min(tail ? a.tailp : BX, a.n1 - x0);
            bulk_prefetch_l2_w(a.zsrc + ((size_t)pl * NT * a.n1 + x0) * a.z_plane + (size_t)t * zterm,
                               (uint32_t)np_ * a.z_plane);
        };
        // (the dual-issuer form leaves the Z tiles to the copies themselves: a prefetch holds the
        // issuing warp for hundreds of cycles, which this warp cannot spare at its term rate)
        if (!DUAL)
            for (int g = 1; g <= NL + 2; ++g) prefetch(g);
        int issued = 0, s = 0, g = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k)
            for (int t = 0; t < NT; ++t, ++g) {
                ok = __all_sync(0xffffffffu, mbar_wait(&empty3[s], ph ^ 1, a.err, 46));
                if (!ok) break;
                ++issued;
                mbar_arrive_expect_tx_w(&full3[s], a.b3_bytes);
                bulk_load_w(B3s(s), a.img + (size_t)t * a.img_stride + img_ya_bytes, a.b3_bytes, &full3[s]);
                if (!DUAL && g > 0) prefetch(g + NL + 2);
                if (++s == NL3) { s = 0; ph ^= 1; }
            }
        if (!ok)
            for (int q = (issued > NL3 ? issued - NL3 : 0); q < issued; ++q) mbar_drain(&full3[q % NL3], (q / NL3) & 1, a.err);
    } else if (warp == 9 || (DUAL && warp == 12)) {
        // ------------------------------ stage-2 MMA issuer ------------------------------
        // (dual-issuer form: warp 9 takes the even terms g of this CTA's sequence, warp 12 the
        // odd ones; each walks the whole sequence to keep the ring stages and Y buffers in step.
        // Terms of different parity write different Y buffers, so their MMAs need no order, but
        // the waits do: a warp waits for the stages of term g only after the other has seen
        // those of term g - 1 arrive (a token), so that every wait finds its barrier at most one
        // phase behind, as with a single consumer)
        const int mine = DUAL ? (warp == 12 ? 1 : 0) : -1;
        const uint64_t d0 = sdesc_sw128(0);
        const int n0 = pad16c(min(a.npc, BX) * a.gs);
        const uint32_t id0 = S2TF32 ? idesc_tf32(128, n0) : idesc_bf16(128, n0);
        const bool more2 = a.nY > 1 || a.npc < BX;
        int s = 0, yb = 0, g = 0;
        uint32_t ph = 0, yph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k) {
            int pl_, slab_, iy;
            item_of(k, pl_, slab_, iy);
            const bool tail = is_tail(iy);
            const int nsub = tail ? min(a.tailp, a.n1 - slab_ * a.tailp) : 1;
            for (int t = 0; t < NT && ok; ++t, ++g) {
                if (DUAL && (g & 1) != mine) {
                    for (int sp = 0; sp < nsub; ++sp)
                        if (++s == NL) { s = 0; ph ^= 1; }
                    if (++yb == NYB) { yb = 0; yph ^= 1; }
                    continue;
                }
                const uint32_t tY = tmem + (uint32_t)yb * a.y_cols;
                // a tail item accumulates the windows of its planes into one Y buffer: each window
                // is zero outside its plane's rows, so every plane lands in its own TMEM lanes
                for (int sp = 0; sp < nsub; ++sp) {
                    bool w = true;
                    if (DUAL && sp == 0 && g > 0) w = mbar_wait(&tok2[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), a.err, 53);
                    if (w) w = mbar_wait(&full_bar[s], ph, a.err, 42);
                    // Y buffer yb was last read by stage 3 of term g - nyb
                    if (w && sp == 0 && g >= NYB) w = mbar_wait(&ybar[yb], yph ^ 1, a.err, 43);
                    ok = __all_sync(0xffffffffu, w);
                    if (!ok) break;
                    if (DUAL && sp == nsub - 1 && lane == 0) mbar_arrive(&tok2[g & 1]);
                    tc_fence_after();
                    // the item's first y tile: rows iy * 128 of the A_t2 tile (1024 descriptor units)
                    const uint64_t ya = d0 + (smem_u32(YAs(s)) >> 4) + (tail ? 0u : (uint32_t)iy * 1024u),
                                   zb = d0 + (smem_u32(Zs(s)) >> 4);
                    s2_mmas<S2TF32, KS2>(a.ks2, tY, ya, zb, ya_atom >> 4, z_atom >> 4, id0, sp > 0 ? 1u : 0u);
                    if (more2)
                        for (int i = 0; i < a.nY; ++i)
                            for (int p0 = (i == 0 ? a.npc : 0); p0 < BX; p0 += a.npc) {
                                const int N = pad16c(min(a.npc, BX - p0) * a.gs);
                                const uint32_t id2 = S2TF32 ? idesc_tf32(128, N) : idesc_bf16(128, N);
                                s2_mmas<S2TF32, KS2>(a.ks2, tY + (uint32_t)(i * a.ycol_tile + p0 * a.gs),
                                                     ya + (uint32_t)i * 1024u, zb + (uint32_t)(p0 * a.gs) * 8u,
                                                     ya_atom >> 4, z_atom >> 4, id2);
                            }
                    if (sp == nsub - 1) mma_commit_w(&s2bar[yb]);
                    mma_commit_w(&empty_bar[s]);
                    if (++s == NL) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                if (++yb == NYB) { yb = 0; yph ^= 1; }
            }
        }
        // the CTA must not release TMEM while these MMAs run
        uint64_t* fb = (DUAL && warp == 12) ? &fin2[0] : &s3fin[0];
        mma_commit_w(fb);
        mbar_drain(fb, 0, a.err);
    } else if (warp == 11 || (DUAL && warp == 13)) {
        // ---------------- stage-3 MMA issuer: every plane and y tile ----------------
        // (dual-issuer form: warp 11 takes the even terms, warp 13 the odd ones.  All terms of an
        // item accumulate into one phi, so the two hand a token back and forth: a warp issues the
        // MMAs of term g only after the other has issued those of term g - 1, with tcgen05 fences
        // around the hand-over, which keeps every MMA into phi in term order)
        const int mine = DUAL ? (warp == 13 ? 1 : 0) : -1;
        const uint64_t d0 = sdesc_sw128(0);
        const uint32_t id3 = BF3 ? idesc_bf16(128, a.n3p) : idesc_tf32(128, a.n3p);
        int s3 = 0, yb = 0, g = 0;
        uint32_t ph3 = 0, yph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k)
            for (int t = 0; t < NT; ++t, ++g) {
                if (DUAL && (g & 1) != mine) {
                    if (++s3 == NL3) { s3 = 0; ph3 ^= 1; }
                    if (++yb == NYB) { yb = 0; yph ^= 1; }
                    continue;
                }
                // BF3: Y is read once the converters have rounded it to bf16 in place
                bool w = mbar_wait(BF3 ? &cvtbar[yb] : &s2bar[yb], yph, a.err, 44);
                if (w) w = mbar_wait(&full3[s3], ph3, a.err, 48);
                // the accumulator is free once the epilogue of the previous item holds phi (BF3,
                // DUAL: once the epilogue of item k - 2 has read this item's phi buffer)
                if constexpr (PHI2) {
                    if (w && t == 0 && k > 1) w = mbar_wait(&phif[k & 1], (uint32_t)(((k - 2) >> 1) & 1), a.err, 50);
                } else {
                    if (w && t == 0 && k > 0) w = mbar_wait(&phifree, (uint32_t)((k - 1) & 1), a.err, 50);
                }
                // DUAL: term g - 1 (the other warp's) has been issued: its (g - 1) / 2-th token
                if (DUAL && w && g > 0) w = mbar_wait(&tok[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), a.err, 52);
                ok = __all_sync(0xffffffffu, w);
                if (!ok) break;
                tc_fence_after();
                const uint64_t b3 = d0 + (smem_u32(B3s(s3)) >> 4);
                const uint64_t b3t = sdesc_sw32(0) + (smem_u32(B3s(s3) + na3f * b3_atom) >> 4);
                const uint32_t tY = tmem + (uint32_t)yb * a.y_cols;
                const uint32_t acc0 = t > 0 ? 1u : 0u;
                for (int p = 0; p < BX; ++p)
                    for (int i = 0; i < a.nY; ++i) {
                        const uint32_t dT = tPhi + (PHI2 ? (uint32_t)(k & 1) * phi_cols : 0u) +
                                            (uint32_t)((p * a.nY + i) * a.n3p);
                        const uint32_t aT = tY + (uint32_t)(i * a.ycol_tile + p * a.gs);
                        if constexpr (BF3)
                            s3b_mmas<KS3>(a.ks3, dT, aT, b3, b3_atom >> 4, id3, acc0);
                        else
                            s3_mmas<KS3>(a.ks3, dT, aT, b3, b3t, b3_atom >> 4, (uint32_t)a.n3p * 2u, id3, acc0);
                    }
                if (DUAL) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tok[g & 1]);
                }
                mma_commit_w(&ybar[yb]);
                mma_commit_w(&empty3[s3]);
                // DUAL: each warp commits phi after its own last term of the item (count 2)
                if (DUAL ? t + 2 >= NT : t == NT - 1) mma_commit_w(PHI2 ? &phid[k & 1] : &phidone);
                if (++s3 == NL3) { s3 = 0; ph3 ^= 1; }
                if (++yb == NYB) { yb = 0; yph ^= 1; }
            }
        // the CTA must not release TMEM while these MMAs run
        uint64_t* fb = (DUAL && warp == 13) ? &fin2[1] : &s3fin[1];
        mma_commit_w(fb);
        mbar_drain(fb, 0, a.err);
    } else if (BF3 && warp >= 4) {
        // ---------------- BF3 converters: Y -> bf16 in place ----------------
        // Two groups of four warps (4-7 and 12-15), one warp per TMEM lane quadrant, take
        // alternate Gaussian terms.  A plane's float32 Y is read into registers 64 columns at a
        // time, rounded to bf16 pairs and written back into the first 32 of those columns (chunk
        // c into columns 32c .. 32c + 31, which chunks 0 .. c have already been read from), so
        // stage 3 finds a K-major bf16 A operand in the first gs / 2 columns of the plane.
        const int grp = warp >= 12 ? 1 : 0;
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        int yb = 0, g = 0;
        uint32_t yph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k)
            for (int t = 0; t < NT; ++t, ++g) {
                if ((g & 1) == grp) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&s2bar[yb], yph, a.err, 51));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t tY = tmem + lanes + (uint32_t)yb * a.y_cols;
                    for (int i = 0; i < a.nY; ++i)
                        for (int p = 0; p < BX; ++p) {
                            const uint32_t base = tY + (uint32_t)(i * a.ycol_tile + p * a.gs);
                            for (int c = 0; c < a.gs / 64; ++c) {
                                uint32_t v[4][16], o[2][16];
                                tmem_ld16(base + 64u * c, v[0]);
                                tmem_ld16(base + 64u * c + 16u, v[1]);
                                tmem_ld16(base + 64u * c + 32u, v[2]);
                                tmem_ld16(base + 64u * c + 48u, v[3]);
                                tmem_ld_wait();
#pragma unroll
                                for (int h = 0; h < 2; ++h)
#pragma unroll
                                    for (int j = 0; j < 8; ++j) {
                                        o[h][j] = pack_bf16x2(v[2 * h][2 * j], v[2 * h][2 * j + 1]);
                                        o[h][8 + j] = pack_bf16x2(v[2 * h + 1][2 * j], v[2 * h + 1][2 * j + 1]);
                                    }
                                tmem_st16(base + 32u * c, o[0]);
                                tmem_st16(base + 32u * c + 16u, o[1]);
                            }
                            if (a.gs % 64) {           // a last 32-column chunk
                                const int c = a.gs / 64;
                                uint32_t v0[16], v1[16], o[16];
                                tmem_ld16(base + 64u * c, v0);
                                tmem_ld16(base + 64u * c + 16u, v1);
                                tmem_ld_wait();
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    o[j] = pack_bf16x2(v0[2 * j], v0[2 * j + 1]);
                                    o[8 + j] = pack_bf16x2(v1[2 * j], v1[2 * j + 1]);
                                }
                                tmem_st16(base + 32u * c, o);
                            }
                        }
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&cvtbar[yb]);
                }
                if (++yb == NYB) { yb = 0; yph ^= 1; }
            }
    } else if (PHI2) {
        // ------- BF3 epilogue, warps 0-3 (one lane quadrant each); DUAL: warps 0-7 -------
        // phi is double-buffered in TMEM, so the epilogue reads it chunk by chunk (16 columns)
        // while the next item accumulates into the other buffer, and releases the buffer when
        // the item is done.  Each lane walks its own grid row as in the other epilogue; in the
        // dual-issuer form the two warps of a lane quadrant take alternate 16-column chunks.
        constexpr int NE = BF3 ? 4 : 8, NH = NE / 4;
        const int q = warp & 3, h = warp >> 2;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        for (int k = 0; k < nmine; ++k) {
            const bool live = mbar_wait_idle(&phid[k & 1], (uint32_t)((k >> 1) & 1), a.err, 45);
            tc_fence_after();
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const bool tail = is_tail(iy);
            const int x0 = tail ? slab * a.tailp : slab * BX;
            const PairRec rec = a.recs[a.p0 + pl];
            const bool en = (a.flags & EPI_ENERGY) != 0;
            const bool o0 = (a.flags & EPI_OUT) && a.OUT0 && rec.o0 >= 0;
            const bool o1 = (a.flags & EPI_OUT) && a.OUT1 && rec.o1 >= 0;
            const bool need0 = o0 || (en && a.emul), need1 = o1 || (en && a.emul);
            const long N3 = (long)a.n1 * a.n2 * a.n3;
            double e = 0.0;
            for (int jt = 0; live && jt < a.nT3; ++jt) {
                int x, y;
                bool rowin;
                if (tail) {
                    const int l = q * 32 + lane, pp = l / a.tail_r8, yy = l - pp * a.tail_r8;
                    x = x0 + pp;
                    y = (a.nyi - 1) * 128 + yy;
                    rowin = pp < a.tailp && yy < a.tail_rows && x < a.n1;
                } else {
                    const int p = jt / a.nY;
                    x = x0 + p;
                    y = (iy + jt - p * a.nY) * 128 + q * 32 + lane;
                    rowin = x < a.n1 && y < a.n2;
                }
                if (!(need0 || need1) || !__any_sync(0xffffffffu, rowin)) continue;
                const float wxy = rowin ? a.w1[x] * a.w2[y] : 0.f;
                const long rowoff = rowin ? ((long)x * a.n2 + y) * a.n3 : 0;
                const float* mul0 = need0 ? a.MUL0 + (long)rec.m0 * N3 + rowoff : nullptr;
                const float* mul1 = need1 ? a.MUL1 + (long)rec.m1 * N3 + rowoff : nullptr;
                float* out0 = o0 ? a.OUT0 + (long)rec.o0 * N3 + rowoff : nullptr;
                float* out1 = o1 ? a.OUT1 + (long)rec.o1 * N3 + rowoff : nullptr;
                const uint32_t tb = tPhi + lanes + (uint32_t)(k & 1) * phi_cols + (uint32_t)(jt * a.n3p);
                for (int zc = 16 * h; zc < a.n3; zc += 16 * NH) {
                    uint32_t ph[16];
                    tmem_ld16(tb + (uint32_t)zc, ph);
                    tmem_ld_wait();
                    if (!rowin) continue;
                    float4 m0v[4], m1v[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        m0v[c] = (need0 && z < a.n3) ? __ldg((const float4*)(mul0 + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        m1v[c] = (need1 && z < a.n3) ? __ldg((const float4*)(mul1 + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    float eb = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        if (z >= a.n3) break;                    // n3 % 4 == 0
                        const float4 phi = make_float4(__uint_as_float(ph[4 * c]), __uint_as_float(ph[4 * c + 1]),
                                                       __uint_as_float(ph[4 * c + 2]), __uint_as_float(ph[4 * c + 3]));
                        const float4 w3 = *(const float4*)(a.w3 + z);
                        const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
                        float4 f = phi;
                        if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
                        const float4 m0 = m0v[c], m1 = m1v[c];
                        if (o0) atomicAdd((float4*)(out0 + z), make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w));
                        if (o1) atomicAdd((float4*)(out1 + z), make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w));
                        if (en && a.emul)
                            eb += wv.x * m1.x * m0.x * phi.x + wv.y * m1.y * m0.y * phi.y + wv.z * m1.z * m0.z * phi.z +
                                  wv.w * m1.w * m0.w * phi.w;
                    }
                    e += (double)eb;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&phif[k & 1]);
            if (a.flags & EPI_ENERGY) {
                for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
                if (lane == 0) red[k & 1][warp] = e * rec.ew;
            }
            // the epilogue warps meet once per item (named barrier 1): energy partial
            asm volatile("bar.sync 1, %0;" ::"n"(NE * 32) : "memory");
            if ((a.flags & EPI_ENERGY) && warp == 0 && lane == 0) {
                double sum = 0.0;
                for (int w = 0; w < NE; ++w) sum += red[k & 1][w];
                a.epart[(long)blockIdx.x + (long)k * gridDim.x] = sum;
            }
        }
    } else {
        // ---------------- epilogue warps 0-7 ----------------
        // With two tiles per item, warp (q, h) takes tile h; with one tile, the two warps of a
        // lane quadrant split its 32-column chunks (h, h + 2, ...).  Either way a lane holds at
        // most kTpMaxZ columns of its row.
        const int q = warp & 3, h = warp >> 2;
        const bool csplit = a.nT3 == 1;
        const int jt = csplit ? 0 : h;
        const int cbase = csplit ? h : 0, cstep = csplit ? 2 : 1;
        auto chunk_of = [&](int j) { return cbase + cstep * j; };   // global 32-column chunk
        for (int k = 0; k < nmine; ++k) {
            // on an error every later wait returns at once; the warps still meet at the named
            // barrier below once per item, so none of them is left waiting there
            const bool live = mbar_wait_idle(&phidone, (uint32_t)(k & 1), a.err, 45);
            tc_fence_after();
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const bool tail = is_tail(iy);
            const int x0 = tail ? slab * a.tailp : slab * BX;
            const PairRec rec = a.recs[a.p0 + pl];
            // phi of this lane's row of tile jt (its chunks), into registers; then release the
            // accumulator
            uint32_t phr[kTpMaxZ];
            const bool has = live && jt < a.nT3;
            if (has) {
#pragma unroll
                for (int c = 0; c < kTpMaxZ / 16; ++c) {
                    const int col = 32 * chunk_of(c >> 1) + 16 * (c & 1);
                    if (col < a.n3p)
                        tmem_ld16(tPhi + ((uint32_t)(q * 32) << 16) + (uint32_t)(jt * a.n3p + col),
                                  *(uint32_t(*)[16]) & phr[16 * c]);
                }
                tmem_ld_wait();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&phifree);
            double e = 0.0;
            // this lane's grid row (x, y): in a tail item lane row l of the tile is row l % tail_r8
            // of the last y tile of plane x0 + l / tail_r8
            int x, y;
            bool rowin;
            if (tail) {
                const int l = q * 32 + lane, pp = l / a.tail_r8, yy = l - pp * a.tail_r8;
                x = x0 + pp;
                y = (a.nyi - 1) * 128 + yy;
                rowin = pp < a.tailp && yy < a.tail_rows && x < a.n1;
            } else {
                const int p = jt / a.nY;
                x = x0 + p;
                y = (iy + jt - p * a.nY) * 128 + q * 32 + lane;
                rowin = x < a.n1 && y < a.n2;
            }
            const bool en = (a.flags & EPI_ENERGY) != 0;
            const bool o0 = (a.flags & EPI_OUT) && a.OUT0 && rec.o0 >= 0;
            const bool o1 = (a.flags & EPI_OUT) && a.OUT1 && rec.o1 >= 0;
            const bool need0 = o0 || (en && a.emul), need1 = o1 || (en && a.emul);
            if (has && (need0 || need1) && __any_sync(0xffffffffu, rowin)) {
                // each lane walks its own grid row: the orbital values come with direct 16-byte
                // loads (a 64-byte row segment per chunk and orbital, all issued before use) and W
                // is updated with 16-byte vector atomics, so no chunk waits on a shared-memory
                // round trip and the pipeline keeps the shared memory for deeper operand rings
                const long N3 = (long)a.n1 * a.n2 * a.n3;
                const float wxy = rowin ? a.w1[x] * a.w2[y] : 0.f;
                const long rowoff = rowin ? ((long)x * a.n2 + y) * a.n3 : 0;
                const float* mul0 = need0 ? a.MUL0 + (long)rec.m0 * N3 + rowoff : nullptr;
                const float* mul1 = need1 ? a.MUL1 + (long)rec.m1 * N3 + rowoff : nullptr;
                float* out0 = o0 ? a.OUT0 + (long)rec.o0 * N3 + rowoff : nullptr;
                float* out1 = o1 ? a.OUT1 + (long)rec.o1 * N3 + rowoff : nullptr;
#pragma unroll
                for (int h16 = 0; h16 < kTpMaxZ / 16; ++h16) {
                    const int zc = 32 * chunk_of(h16 >> 1) + 16 * (h16 & 1);
                    if (zc >= a.n3) break;
                    if (!rowin) continue;
                    float4 m0v[4], m1v[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        m0v[c] = (need0 && z < a.n3) ? __ldg((const float4*)(mul0 + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        m1v[c] = (need1 && z < a.n3) ? __ldg((const float4*)(mul1 + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    float eb = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        if (z >= a.n3) break;                    // n3 % 4 == 0
                        const int r0 = 16 * h16 + 4 * c;
                        const float4 phi = make_float4(__uint_as_float(phr[r0]), __uint_as_float(phr[r0 + 1]),
                                                       __uint_as_float(phr[r0 + 2]), __uint_as_float(phr[r0 + 3]));
                        const float4 w3 = *(const float4*)(a.w3 + z);
                        const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
                        float4 f = phi;
                        if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
                        const float4 m0 = m0v[c], m1 = m1v[c];
                        if (o0) atomicAdd((float4*)(out0 + z), make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w));
                        if (o1) atomicAdd((float4*)(out1 + z), make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w));
                        if (en && a.emul)
                            eb += wv.x * m1.x * m0.x * phi.x + wv.y * m1.y * m0.y * phi.y + wv.z * m1.z * m0.z * phi.z +
                                  wv.w * m1.w * m0.w * phi.w;
                    }
                    e += (double)eb;
                }
            }
            if (a.flags & EPI_ENERGY) {
                for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
                if (lane == 0) red[k & 1][warp] = e * rec.ew;
            }
            // the eight epilogue warps meet once per item (named barrier 1): energy partial
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if ((a.flags & EPI_ENERGY) && warp == 0 && lane == 0) {
                double sum = 0.0;
                for (int w = 0; w < 8; ++w) sum += red[k & 1][w];
                a.epart[(long)blockIdx.x + (long)k * gridDim.x] = sum;    // the item's index
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) tmem_dealloc(tmem, a.tmem_cols);
}

// Image of the per-term operator tiles of the single-pass kernel, built once per context:
// [A_t2 tile][mu_t A_t3 tile] for every term t, byte for byte as the tensor-map loads of a load
// stage lay them out (128-byte swizzle, the 32-byte-swizzled K tail of mu_t A_t3, zero fill).
// The expansion kernel then brings each term's operators in with two plain bulk copies, which
// the copy engine streams at its byte rate, instead of walking one box row at a time.
struct ImageArgs {
    int ks2, ks3, n3p;
    uint32_t ya_rows, ya_bytes, b3_bytes;
    uint32_t stride;           // bytes per term of the image (the tiles, then any tail windows)
    uint8_t* img;
    int* err;
};

// Tail windows of the operator image (persistent kernel with packed y tiles): for term t and
// plane slot p, a copy of the A_t2 tile whose rows p * r8 .. p * r8 + rows - 1 hold A_t2's rows
// ybase .. ybase + rows - 1 and every other row is zero.  ybase and r8 are multiples of 8, so a
// row keeps its 128-byte swizzle phase and is copied verbatim.
__global__ void __launch_bounds__(256) k_tail_windows(uint8_t* img, uint32_t stride, uint32_t win_off, uint32_t ya_bytes,
                                                      uint32_t ya_rows, int na2, int ybase, int rows, int r8) {
    const int t = blockIdx.x, p = blockIdx.y;
    const uint8_t* src = img + (size_t)t * stride;
    uint8_t* dst = img + (size_t)t * stride + win_off + (size_t)p * ya_bytes;
    const int total = na2 * (int)ya_rows * 8;   // 16-byte chunks of the window
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int row = q / 8, c = q % 8, k = row / (int)ya_rows, i = row - k * (int)ya_rows;
        const int j = i - p * r8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (j >= 0 && j < rows) v = *(const uint4*)(src + ((size_t)k * ya_rows + ybase + j) * 128 + c * 16);
        *(uint4*)(dst + ((size_t)k * ya_rows + i) * 128 + c * 16) = v;
    }
}

template <bool S2TF32>
__global__ void __launch_bounds__(32, 1)
    k_operand_image(const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mA3f,
                    const __grid_constant__ CUtensorMap mA3t, ImageArgs g) {
    constexpr int AK2 = S2TF32 ? 32 : 64;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int t = blockIdx.x;
    const int na2 = (g.ks2 + 3) / 4, na3f = g.ks3 / 4, kt = g.ks3 % 4;
    const uint32_t ya_atom = g.ya_rows * 128u, b3_atom = (uint32_t)g.n3p * 128u;
    uint8_t* b3 = smem + g.ya_bytes;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
        mbar_arrive_expect_tx(&bar, g.ya_bytes + g.b3_bytes);
        for (int k = 0; k < na2; ++k) tma_load_3d(smem + k * ya_atom, &mA2, &bar, k * AK2, 0, t);
        for (int k = 0; k < na3f; ++k) tma_load_3d(b3 + k * b3_atom, &mA3f, &bar, k * 32, 0, t);
        for (int j = 0; j < kt; ++j)
            tma_load_3d(b3 + na3f * b3_atom + (uint32_t)j * g.n3p * 32u, &mA3t, &bar, na3f * 32 + 8 * j, 0, t);
    }
    __syncwarp();
    const bool ok = mbar_wait(&bar, 0, g.err, 47);
    if (!__all_sync(0xffffffffu, ok)) {
        mbar_drain(&bar, 0, g.err);
        return;
    }
    const uint4* src = (const uint4*)smem;
    uint4* dst = (uint4*)(g.img + (size_t)t * g.stride);
    for (uint32_t i = threadIdx.x; i < (g.ya_bytes + g.b3_bytes) / 16; i += 32) dst[i] = src[i];
}


// bf16 form of the persistent kernel: stage 3 also runs as kind::f16.  Stage 2 leaves Y_t in
// TMEM in float32 (y on the lanes); four converter warps (one per TMEM lane quadrant) round it to
// bf16 and write it as the K-major stage-3 A operand in shared memory (128-byte swizzle, one
// 128-row tile per plane and y tile), so stage 3 multiplies bf16 by bf16 at the full tensor rate
// instead of running as TF32 from TMEM.  phi is double-buffered in TMEM: the epilogue of item k
// reads it directly from TMEM while item k + 1 accumulates into the other buffer.
// Warp roles: 0-7 converters (two groups of four, one TMEM lane quadrant per warp, taking
// alternate terms so that one group's TMEM load round trip overlaps the other's stores), 8
// stage-2 producer, 9 stage-2 MMAs, 10 stage-3 producer and Z prefetches, 11 stage-3 MMAs, 12-15
// epilogue.
constexpr int kThreadsTb = 512;
constexpr int kMaxYs = 3;
constexpr uint32_t kTbEpiBytes = 0;                  // the epilogue reads the orbitals directly
constexpr uint32_t kYsAtom = 128u * 128u;            // one 128-row x 128-byte operand atom

template <int KS2, int KS3>
__global__ void __launch_bounds__(kThreadsTb, 1)
    k_consume_tb(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ EpiMaps em, ConsumeArgs a) {
    constexpr int AK2 = 64;                  // stage-2 elements per 128-byte atom
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kMaxLoad], empty_bar[kMaxLoad], full3[kMaxLoad], empty3[kMaxLoad];
    __shared__ uint64_t s2bar[kMaxYBuf], ybar[kMaxYBuf], ysfull[kMaxYs], ysfree[kMaxYs];
    __shared__ uint64_t phidone[2], phifree[2], s3fin[2], ebar[4];
    __shared__ uint32_t tmem_base;
    __shared__ double red[2][4];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NL = a.nload, NL3 = a.nload3, NYB = a.nyb, NYS = a.nys, BX = a.bx, NT = a.nt;
    const int nmine = (int)blockIdx.x < a.nitems ? (a.nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto item_of = [&](int k, int& pl, int& slab, int& iy) {
        const int it = (int)blockIdx.x + k * (int)gridDim.x;
        const int ps = it / a.nyi;
        iy = it - ps * a.nyi;
        pl = ps / a.nslab;
        slab = ps - pl * a.nslab;
    };
    auto YAs = [&](int s) { return smem + s * a.load_bytes; };
    auto Zs = [&](int s) { return YAs(s) + a.ya_bytes; };
    auto B3s = [&](int s) { return smem + a.a3_off + s * a.load3_bytes; };
    auto YSs = [&](int b) { return smem + a.ys_off + b * a.ys_bytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxLoad; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&full3[s], 1);
            mbar_init(&empty3[s], 1);
        }
        for (int b = 0; b < kMaxYBuf; ++b) {
            mbar_init(&s2bar[b], 1);
            mbar_init(&ybar[b], 4);
        }
        for (int b = 0; b < kMaxYs; ++b) {
            mbar_init(&ysfull[b], 4);
            mbar_init(&ysfree[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&phidone[b], 1);
            mbar_init(&phifree[b], 4);
            mbar_init(&s3fin[b], 1);
        }
        for (int w = 0; w < 4; ++w) mbar_init(&ebar[w], 1);
        fence_barrier_init();
    }
    // Z tile rows that no copy writes feed Y columns that are never converted: keep them finite
    for (int s = 0; s < NL; ++s) {
        uint4* z = (uint4*)Zs(s);
        for (int i = threadIdx.x; i < (int)(a.z_bytes / 16); i += kThreadsTb) z[i] = make_uint4(0, 0, 0, 0);
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
    const uint32_t phi_cols = (uint32_t)(a.nT3 * a.n3p);
    const uint32_t tPhi0 = tmem + (uint32_t)NYB * a.y_cols;
    const uint32_t ya_atom = a.ya_rows * 128u, z_atom = a.z_rows * 128u, b3_atom = (uint32_t)a.n3p * 128u;
    const int na2 = (a.ks2 + 3) / 4;

    if (warp == 8) {
        // ------------------------- stage-2 producer: A_t2 and Z -------------------------
        int issued = 0, s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k) {
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const int x0 = slab * BX;
            for (int t = 0; t < NT; ++t) {
                ok = __all_sync(0xffffffffu, mbar_wait(&empty_bar[s], ph ^ 1, a.err, 61));
                if (!ok) break;
                ++issued;
                mbar_arrive_expect_tx_w(&full_bar[s], a.stage_tx);
                const int zdep = pl * NT + t;
                bulk_load_w(YAs(s), a.img + (size_t)t * a.img_stride, a.ya_bytes, &full_bar[s]);
                if (a.zone) {
                    tma_load_3d_w(Zs(s), &mZ, &full_bar[s], 0, x0 * a.r3, zdep);
                    for (int kk = 1; kk < na2; ++kk)
                        tma_load_3d_w(Zs(s) + kk * z_atom, &mZ, &full_bar[s], kk * AK2, x0 * a.r3, zdep);
                } else {
                    for (int kk = 0; kk < na2; ++kk)
                        for (int p = 0; p < BX; ++p)
                            tma_load_3d_w(Zs(s) + kk * z_atom + (uint32_t)(p * a.gs) * 128u, &mZ, &full_bar[s],
                                          kk * AK2, (x0 + p) * a.r3, zdep);
                }
                if (++s == NL) { s = 0; ph ^= 1; }
            }
        }
        if (!ok)
            for (int g = (issued > NL ? issued - NL : 0); g < issued; ++g)
                mbar_drain(&full_bar[g % NL], (g / NL) & 1, a.err);
    } else if (warp == 10) {
        // ---------------- stage-3 producer: mu_t A_t3 (bf16), and the Z L2 prefetches ----------------
        const size_t zterm = (size_t)a.n1 * a.z_plane;
        auto prefetch = [&](int g) {
            const int k = g / NT, t = g - k * NT;
            if (k >= nmine) return;
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const int x0 = slab * BX;
            const int np_ = min(BX, a.n1 - x0);
            bulk_prefetch_l2_w(a.zsrc + ((size_t)pl * NT * a.n1 + x0) * a.z_plane + (size_t)t * zterm,
                               (uint32_t)np_ * a.z_plane);
        };
        for (int g = 1; g <= NL + 2; ++g) prefetch(g);
        int issued = 0, s = 0, g = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k)
            for (int t = 0; t < NT; ++t, ++g) {
                ok = __all_sync(0xffffffffu, mbar_wait(&empty3[s], ph ^ 1, a.err, 62));
                if (!ok) break;
                ++issued;
                mbar_arrive_expect_tx_w(&full3[s], a.b3_bytes);
                bulk_load_w(B3s(s), a.img + (size_t)t * a.img_stride + a.ya_bytes, a.b3_bytes, &full3[s]);
                if (g > 0) prefetch(g + NL + 2);
                if (++s == NL3) { s = 0; ph ^= 1; }
            }
        if (!ok)
            for (int q = (issued > NL3 ? issued - NL3 : 0); q < issued; ++q)
                mbar_drain(&full3[q % NL3], (q / NL3) & 1, a.err);
    } else if (warp == 9) {
        // ------------------------------ stage-2 MMA issuer ------------------------------
        const uint64_t d0 = sdesc_sw128(0);
        const int n0 = pad16c(min(a.npc, BX) * a.gs);
        const uint32_t id0 = idesc_bf16(128, n0);
        const bool more2 = a.nY > 1 || a.npc < BX;
        int s = 0, yb = 0, g = 0;
        uint32_t ph = 0, yph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k) {
            int pl_, slab_, iy;
            item_of(k, pl_, slab_, iy);
            for (int t = 0; t < NT; ++t, ++g) {
                bool w = mbar_wait(&full_bar[s], ph, a.err, 63);
                // Y buffer yb was last converted for term g - nyb
                if (w && g >= NYB) w = mbar_wait(&ybar[yb], yph ^ 1, a.err, 64);
                ok = __all_sync(0xffffffffu, w);
                if (!ok) break;
                tc_fence_after();
                const uint64_t ya = d0 + (smem_u32(YAs(s)) >> 4) + (uint32_t)iy * 1024u, zb = d0 + (smem_u32(Zs(s)) >> 4);
                const uint32_t tY = tmem + (uint32_t)yb * a.y_cols;
                s2_mmas<false, KS2>(a.ks2, tY, ya, zb, ya_atom >> 4, z_atom >> 4, id0);
                if (more2)
                    for (int i = 0; i < a.nY; ++i)
                        for (int p0 = (i == 0 ? a.npc : 0); p0 < BX; p0 += a.npc) {
                            const int N = pad16c(min(a.npc, BX - p0) * a.gs);
                            s2_mmas<false, KS2>(a.ks2, tY + (uint32_t)(i * a.ycol_tile + p0 * a.gs), ya + (uint32_t)i * 1024u,
                                                zb + (uint32_t)(p0 * a.gs) * 8u, ya_atom >> 4, z_atom >> 4,
                                                idesc_bf16(128, N));
                        }
                mma_commit_w(&s2bar[yb]);
                mma_commit_w(&empty_bar[s]);
                if (++s == NL) { s = 0; ph ^= 1; }
                if (++yb == NYB) { yb = 0; yph ^= 1; }
            }
        }
        mma_commit_w(&s3fin[0]);
        mbar_drain(&s3fin[0], 0, a.err);
    } else if (warp == 11) {
        // ------------- stage-3 MMA issuer: bf16 Y tiles (shared memory) x mu_t A_t3 -------------
        const uint64_t d0 = sdesc_sw128(0);
        const uint32_t id3 = idesc_bf16(128, a.n3p);
        int s3 = 0, ys = 0;
        uint32_t ph3 = 0, yph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k) {
            const int fb = k & 1;
            const uint32_t tPhi = tPhi0 + (uint32_t)fb * phi_cols;
            for (int t = 0; t < NT; ++t) {
                bool w = mbar_wait(&ysfull[ys], yph, a.err, 65);
                if (w) w = mbar_wait(&full3[s3], ph3, a.err, 66);
                // phi buffer fb was last read by the epilogue of item k - 2
                if (w && t == 0 && k >= 2) w = mbar_wait(&phifree[fb], (uint32_t)(((k - 2) >> 1) & 1), a.err, 67);
                ok = __all_sync(0xffffffffu, w);
                if (!ok) break;
                tc_fence_after();
                const uint64_t b3 = d0 + (smem_u32(B3s(s3)) >> 4);
                const uint64_t ya = d0 + (smem_u32(YSs(ys)) >> 4);
                for (int jt = 0; jt < a.nT3; ++jt) {
                    const uint32_t d = tPhi + (uint32_t)(jt * a.n3p);
                    const uint64_t at = ya + (uint32_t)jt * (a.ys_tile >> 4);
#pragma unroll
                    for (int kk = 0; kk < (KS3 > 0 ? KS3 : 16); ++kk) {
                        if (KS3 == 0 && kk >= a.ks3) break;
                        mma_ss_w<false>(d, at + (uint32_t)(kk >> 2) * (kYsAtom >> 4) + (uint32_t)(kk & 3) * 2u,
                                        b3 + (uint32_t)(kk >> 2) * (b3_atom >> 4) + (uint32_t)(kk & 3) * 2u, id3,
                                        (t > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                mma_commit_w(&ysfree[ys]);
                mma_commit_w(&empty3[s3]);
                if (t == NT - 1) mma_commit_w(&phidone[fb]);
                if (++s3 == NL3) { s3 = 0; ph3 ^= 1; }
                if (++ys == NYS) { ys = 0; yph ^= 1; }
            }
        }
        mma_commit_w(&s3fin[1]);
        mbar_drain(&s3fin[1], 0, a.err);
    } else if (warp < 8) {
        // ---------------- converters: Y (float32, TMEM) -> bf16 stage-3 A operand ----------------
        const int q = warp & 3, grp = warp >> 2;
        const int kpad = 16 * a.ks3;             // K of the operand tile (zero past gs)
        int yb = 0, ys = 0, g = 0;
        uint32_t yph = 0, sph = 0;
        bool ok = true;
        for (int k = 0; k < nmine && ok; ++k)
            for (int t = 0; t < NT; ++t, ++g) {
                if ((g & 1) != grp) {            // the other group's term: advance the rings only
                    if (++yb == NYB) { yb = 0; yph ^= 1; }
                    if (++ys == NYS) { ys = 0; sph ^= 1; }
                    continue;
                }
                bool w = mbar_wait(&s2bar[yb], yph, a.err, 68);
                if (w && g >= NYS) w = mbar_wait(&ysfree[ys], sph ^ 1, a.err, 69);
                ok = __all_sync(0xffffffffu, w);
                if (!ok) break;
                tc_fence_after();
                const uint32_t tY = tmem + (uint32_t)yb * a.y_cols + ((uint32_t)(q * 32) << 16);
                uint8_t* tileb = YSs(ys);
                const uint32_t row = (uint32_t)(q * 32 + lane);
                for (int jt = 0; jt < a.nT3; ++jt) {
                    const int p = jt / a.nY, i = jt - p * a.nY;
                    const uint32_t col = tY + (uint32_t)(i * a.ycol_tile + p * a.gs);
                    uint8_t* tile = tileb + jt * a.ys_tile;
                    // the columns of one 64-wide atom are loaded together and waited for once:
                    // a TMEM load round trip costs far more than the conversion itself
                    for (int a0 = 0; a0 < kpad; a0 += 64) {
                        uint32_t r[4][16];
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (a0 + 16 * c < kpad && a0 + 16 * c < a.gs) tmem_ld16(col + a0 + 16 * c, r[c]);
                        tmem_ld_wait();
                        uint8_t* at = tile + (a0 >> 6) * kYsAtom;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int g0 = a0 + 16 * c;
                            if (g0 >= kpad) break;
                            uint32_t w8[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int c0 = g0 + 2 * e;
                                const float lo = c0 < a.gs ? __uint_as_float(r[c][2 * e]) : 0.f;
                                const float hi = c0 + 1 < a.gs ? __uint_as_float(r[c][2 * e + 1]) : 0.f;
                                w8[e] = pack_bf16(lo, hi);
                            }
                            // bytes (g0 % 64) * 2 .. + 32 of this row of the atom
                            const uint32_t b0 = (uint32_t)((g0 & 63) * 2);
                            *(uint4*)(at + sw128_offset(row, b0)) = make_uint4(w8[0], w8[1], w8[2], w8[3]);
                            *(uint4*)(at + sw128_offset(row, b0 + 16)) = make_uint4(w8[4], w8[5], w8[6], w8[7]);
                        }
                    }
                }
                tc_fence_before();
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&ybar[yb]);
                    mbar_arrive(&ysfull[ys]);
                }
                if (++yb == NYB) { yb = 0; yph ^= 1; }
                if (++ys == NYS) { ys = 0; sph ^= 1; }
            }
    } else {
        // ---------------- epilogue warps 12-15: phi straight from TMEM ----------------
        // Each lane owns one grid row (x, y) of a tile and walks its z in chunks of 16: the
        // orbital values come with direct 16-byte loads (one 64-byte row segment per lane and
        // orbital, all issued before any is used) and W is updated with 16-byte vector atomics,
        // so no chunk waits on a shared-memory round trip.
        const int q = warp - 12;
        const long N3 = (long)a.n1 * a.n2 * a.n3;
        for (int k = 0; k < nmine; ++k) {
            const int fb = k & 1;
            // on an error every later wait returns at once; the four warps still meet at the
            // named barrier below once per item
            const bool live = mbar_wait_idle(&phidone[fb], (uint32_t)((k >> 1) & 1), a.err, 70);
            tc_fence_after();
            int pl, slab, iy;
            item_of(k, pl, slab, iy);
            const int x0 = slab * BX;
            const PairRec rec = a.recs[a.p0 + pl];
            const uint32_t tPhi = tPhi0 + (uint32_t)fb * phi_cols + ((uint32_t)(q * 32) << 16);
            double e = 0.0;
            const bool en = (a.flags & EPI_ENERGY) != 0;
            const bool o0 = (a.flags & EPI_OUT) && a.OUT0 && rec.o0 >= 0;
            const bool o1 = (a.flags & EPI_OUT) && a.OUT1 && rec.o1 >= 0;
            const bool need0 = o0 || (en && a.emul), need1 = o1 || (en && a.emul);
            const float* mul0 = need0 ? a.MUL0 + (long)rec.m0 * N3 : nullptr;
            const float* mul1 = need1 ? a.MUL1 + (long)rec.m1 * N3 : nullptr;
            float* out0 = o0 ? a.OUT0 + (long)rec.o0 * N3 : nullptr;
            float* out1 = o1 ? a.OUT1 + (long)rec.o1 * N3 : nullptr;
            for (int jt = 0; jt < a.nT3 && live; ++jt) {
                const int p = jt / a.nY, x = x0 + p, y = (iy + jt - p * a.nY) * 128 + q * 32 + lane;
                // the whole warp takes part in the TMEM loads; rows past the grid skip the rest
                const bool rowin = x < a.n1 && y < a.n2 && (need0 || need1);
                const float wxy = rowin ? a.w1[x] * a.w2[y] : 0.f;
                const long rowoff = rowin ? ((long)x * a.n2 + y) * a.n3 : 0;
                for (int zc = 0; zc < a.n3; zc += 16) {
                    uint32_t phr[16];
                    tmem_ld16(tPhi + (uint32_t)(jt * a.n3p + zc), phr);
                    float4 m0v[4], m1v[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        const bool zin = rowin && z < a.n3;
                        m0v[c] = (need0 && zin) ? __ldg((const float4*)(mul0 + rowoff + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        m1v[c] = (need1 && zin) ? __ldg((const float4*)(mul1 + rowoff + z)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    tmem_ld_wait();
                    if (!rowin) continue;
                    float eb = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int z = zc + 4 * c;
                        if (z >= a.n3) break;                    // n3 % 4 == 0
                        const float4 phi = make_float4(__uint_as_float(phr[4 * c]), __uint_as_float(phr[4 * c + 1]),
                                                       __uint_as_float(phr[4 * c + 2]), __uint_as_float(phr[4 * c + 3]));
                        const float4 w3 = *(const float4*)(a.w3 + z);
                        const float4 wv = make_float4(wxy * w3.x, wxy * w3.y, wxy * w3.z, wxy * w3.w);
                        float4 f = phi;
                        if (a.flags & EPI_MULW) f = make_float4(f.x * wv.x, f.y * wv.y, f.z * wv.z, f.w * wv.w);
                        const float4 m0 = m0v[c], m1 = m1v[c];
                        if (o0) atomicAdd((float4*)(out0 + rowoff + z), make_float4(-m0.x * f.x, -m0.y * f.y, -m0.z * f.z, -m0.w * f.w));
                        if (o1) atomicAdd((float4*)(out1 + rowoff + z), make_float4(-m1.x * f.x, -m1.y * f.y, -m1.z * f.z, -m1.w * f.w));
                        if (en && a.emul)
                            eb += wv.x * m1.x * m0.x * phi.x + wv.y * m1.y * m0.y * phi.y + wv.z * m1.z * m0.z * phi.z +
                                  wv.w * m1.w * m0.w * phi.w;
                    }
                    e += (double)eb;
                }
            }
            // this item's phi has been read: the stage-3 warp may reuse the buffer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&phifree[fb]);
            if (a.flags & EPI_ENERGY) {
                for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
                if (lane == 0) red[k & 1][q] = e * rec.ew;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if ((a.flags & EPI_ENERGY) && q == 0 && lane == 0) {
                double sum = 0.0;
                for (int w = 0; w < 4; ++w) sum += red[k & 1][w];
                a.epart[((long)pl * a.nslab + slab) * a.nyi + iy] = sum;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) tmem_dealloc(tmem, a.tmem_cols);
}

// Image of the bf16 persistent kernel's per-term operator tiles: [A_t2 tile][mu_t A_t3 (bf16)],
// both 128-byte swizzled K-major atoms laid out as the tile loads would write them.
template <int DUMMY>
__global__ void __launch_bounds__(32, 1)
    k_operand_image_b16(const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mA3, ImageArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int t = blockIdx.x;
    const int na2 = (g.ks2 + 3) / 4, na3 = (g.ks3 + 3) / 4;
    const uint32_t ya_atom = g.ya_rows * 128u, b3_atom = (uint32_t)g.n3p * 128u;
    uint8_t* b3 = smem + g.ya_bytes;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
        mbar_arrive_expect_tx(&bar, g.ya_bytes + g.b3_bytes);
        for (int k = 0; k < na2; ++k) tma_load_3d(smem + k * ya_atom, &mA2, &bar, k * 64, 0, t);
        for (int k = 0; k < na3; ++k) tma_load_3d(b3 + k * b3_atom, &mA3, &bar, k * 64, 0, t);
    }
    __syncwarp();
    const bool ok = mbar_wait(&bar, 0, g.err, 72);
    if (!__all_sync(0xffffffffu, ok)) {
        mbar_drain(&bar, 0, g.err);
        return;
    }
    const uint4* src = (const uint4*)smem;
    uint4* dst = (uint4*)(g.img + (size_t)t * g.stride);
    for (uint32_t i = threadIdx.x; i < (g.ya_bytes + g.b3_bytes) / 16; i += 32) dst[i] = src[i];
}

}  // namespace tcc

// ======================================================================================
// host side: tile plan and launch
// ======================================================================================

struct ConsumePlan {
    bool tb;                 // bf16 persistent kernel (stage 3 in bf16 from shared memory)
    int nys;                 // ... its Y operand tiles in shared memory
    uint32_t ys_tile, ys_bytes;
    bool ts;                 // single-pass kernel (stage 3 from TMEM) instead of the converter kernel
    bool ysplit;             // single-pass, persistent only: one work item per 128-row y tile
    int nyi;                 // work items per slab (nY with ysplit, else 1)
    int bx, nY, Nz, npc, nT3, n2p, n3p, ks2, ks3, nq, nload, na3, nyb, gs, ycol_tile;
    uint32_t ya_rows, z_rows, ya, zb, b3, a3, load, a3_off, tmem_cols, y_cols;
    int nload3;              // single-pass: stages of the stage-3 (mu_t A_t3) ring
    uint32_t load3;          // single-pass: stride of the stage-3 ring
    size_t smem;
    // y-tile items with packed tails: the last y tile of each plane has tail_rows rows; tailp
    // planes (tail_r8 = tail_rows rounded up to 8 rows each) share one item (0: not packed)
    int tailp, tail_r8, tail_rows;
    uint32_t sya_rows, sya;  // rows per K atom and bytes of the A_t2 tile in a shared-memory stage
    bool bf3;                // persistent form with Y rounded to bf16 in TMEM: stage 3 in bf16 (form 4)
    bool dual;               // persistent form with two stage-2 and two stage-3 MMA warps (form 5)
    // split kernel, y/z items (one plane, one 128-row y tile of nyi and one z part of nzi per CTA)
    bool yz;
    int nzi;
    uint32_t loadB;          // converter kernel: stride and stages of the stage-3 operand ring
    int nloadB;
    uint32_t img_stride() const { return ya + b3 + (uint32_t)tailp * ya; }
    int items_per_slab_pair(int n1) const {   // work items per pair
        if (yz) return ((n1 + bx - 1) / bx) * nyi * nzi;
        return tailp ? (n1 / bx) * (nyi - 1) + (n1 + tailp - 1) / tailp : ((n1 + bx - 1) / bx) * (ts ? nyi : 1);
    }
};

// Single-pass plan: bx planes, nload load stages and as many stage-2 output buffers in TMEM.
// With ysplit every work item covers one 128-row y tile of its planes (persistent kernel only),
// so that phi and the stage-2 buffers of planes with more than 128 rows fit TMEM.
static bool plan_ts(const tx_ctx* c, bool tf32, int bx, int nload, ConsumePlan* p, bool ysplit = false) {
    const int MK2 = tf32 ? 8 : 16;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2];
    if (bx < 1 || bx > n1 || bx > tcc::kMaxPlanes || nload < 2 || nload > tcc::kMaxLoad) return false;
    *p = ConsumePlan{};
    p->ts = true;
    p->bx = bx;
    p->n2p = pad16(n2);
    p->n3p = pad16(n3);
    p->gs = pad8(r3);                          // TMEM columns (and Z tile rows) per plane
    if (p->n2p > 256 || p->n3p > 256 || p->gs > 256) return false;
    p->nY = (n2 + 127) / 128;
    p->nyi = 1;
    if (ysplit) {
        if (p->nY < 2 || bx > 2) return false;
        p->ysplit = true;
        p->nyi = p->nY;
        p->nY = 1;
        // pack the short last y tiles of several planes into one item (one plane per slab)
        const int rows = n2 - 128 * (p->nyi - 1), r8 = pad8(rows);
        if (bx == 1 && c->consume_form != 3 && 128 / r8 >= 2) {
            p->tailp = 128 / r8;
            p->tail_r8 = r8;
            p->tail_rows = rows;
        }
    }
    p->npc = std::min(bx, 256 / p->gs);
    p->ks2 = (r2 + MK2 - 1) / MK2;
    // form 4 (bf16): stage 3 takes Y rounded to bf16 in TMEM, 32 columns at a time
    // (the persistent kernel only: at most two planes per item)
    p->bf3 = !tf32 && c->consume_form == 4 && p->gs % 32 == 0 && bx <= 2 && bx * p->nY <= 2;
    // form 5 (bf16): two warps issue the stage-2 MMAs and two the stage-3 MMAs, alternate terms
    // each (the persistent kernel only, at least two terms)
    p->dual = !tf32 && c->consume_form == 5 && bx <= 2 && bx * p->nY <= 2 && c->T >= 2;
    p->ks3 = p->bf3 ? (r3 + 15) / 16 : (r3 + 7) / 8;
    // columns of one y tile of Y: each plane chunk writes pad16(planes * gs) columns from p0 * gs
    p->ycol_tile = 0;
    for (int p0 = 0; p0 < bx; p0 += p->npc)
        p->ycol_tile = std::max(p->ycol_tile, p0 * p->gs + pad16(std::min(p->npc, bx - p0) * p->gs));
    p->y_cols = (uint32_t)(p->nY * p->ycol_tile);
    p->nT3 = bx * p->nY;
    // (forms 4 and 5 keep two phi buffers, so that the epilogue reads one while the next item
    // fills the other)
    const uint32_t phi = (uint32_t)(p->nT3 * p->n3p) * ((p->bf3 || p->dual) ? 2u : 1u);
    // one Y buffer per load stage when TMEM allows (the kernel then needs no Y-buffer barrier)
    p->nyb = std::min(nload, tcc::kMaxYBuf);
    while (p->nyb > 2 && p->nyb * p->y_cols + phi > 512) --p->nyb;
    const uint32_t cols = p->nyb * p->y_cols + phi;
    if (cols > 512) return false;
    p->tmem_cols = 32;
    while (p->tmem_cols < cols) p->tmem_cols <<= 1;
    const int na2 = (p->ks2 + 3) / 4;          // 128-byte atoms along K
    // The A_t2 tile holds the n2p loaded rows; a 128-row MMA tile reads past them into the Z tile
    // that follows (garbage rows only reach TMEM lanes that are never read), and the smem
    // allocation keeps 16 KB spare after the last stage for the same reason.
    p->ya_rows = (uint32_t)p->n2p;
    p->z_rows = (uint32_t)p->ycol_tile;         // rows every stage-2 MMA may read
    p->ya = (uint32_t)na2 * p->ya_rows * 128u;
    p->zb = (uint32_t)na2 * p->z_rows * 128u;
    p->b3 = p->bf3 ? (uint32_t)((p->ks3 + 3) / 4) * p->n3p * 128u
                   : (uint32_t)(p->ks3 / 4) * p->n3p * 128u + (uint32_t)(p->ks3 % 4) * p->n3p * 32u;
    // two rings: nload stages of [A_t2][Z] (stage 2), then as many stages of [mu_t A_t3]
    // (stage 3, up to kMaxLoad) as shared memory holds: its loads start only when stage 3 of
    // an earlier term has finished, so this ring needs the deeper lead
    // packed items read 128 rows per K atom of the A_t2 tile (or of a window): a stage keeps those
    p->sya_rows = p->tailp ? 128u : p->ya_rows;
    p->sya = (uint32_t)na2 * p->sya_rows * 128u;
    p->load = (p->sya + p->zb + 1023) & ~1023u;
    p->load3 = (p->b3 + 1023) & ~1023u;
    p->nload = nload;
    p->a3_off = p->load * (uint32_t)nload;
    // y-tile items run in the persistent kernel only: its smallest split (two stages of each
    // ring and the epilogue boxes) must fit, and an epilogue lane must hold its share of a phi
    // row (the whole row with two tiles per item, every other 32-column chunk with one)
    if (ysplit) {
        if (2 * (size_t)p->load + 2 * (size_t)p->load3 + tcc::kTpEpiBytes + 1024 > 226 * 1024) return false;
        const int lane_cols = p->nT3 == 1 ? 32 * (((p->n3p + 31) / 32 + 1) / 2) : p->n3p;
        if (p->nT3 > 2 || lane_cols > tcc::kTpMaxZ || p->nyb < 2) return false;
    }
    for (p->nload3 = tcc::kMaxLoad; p->nload3 >= 2; --p->nload3) {
        p->smem = std::max((size_t)p->a3_off + (size_t)p->load3 * p->nload3 + 16384, (size_t)tcc::kEpiBytes) + 1024;
        if (p->smem <= 226 * 1024) return true;
    }
    return false;
}

// tensor-pipe cycles per plane and term of a single-pass plan (one MMA costs max(50, N / 2))
static double ts_cost(const ConsumePlan& p) {
    double s2 = 0;
    for (int p0 = 0; p0 < p.bx; p0 += p.npc) s2 += std::max(50.0, pad16(std::min(p.npc, p.bx - p0) * p.gs) / 2.0);
    const double s3 = p.bx * std::max(50.0, p.n3p / 2.0);
    return (p.nY * p.ks2 * s2 + p.nY * p.ks3 * s3) / p.bx;
}

static bool plan_cv(const tx_ctx* c, bool tf32, bool split, int bx, int nload, int na3, ConsumePlan* p,
                    int nzi = 0);

// bf16 persistent plan (k_consume_tb): bx planes, nload stage-2 stages.  phi (double-buffered),
// at least two float32 Y buffers in TMEM; the stage-3 ring, the bf16 Y tiles and the epilogue
// boxes in shared memory.  Planes of more than 128 rows take one work item per y tile.
static bool plan_tb(const tx_ctx* c, int bx, int nload, ConsumePlan* p) {
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2];
    if (c->consume_form != 2 || bx < 1 || bx > n1 || bx > 4 || nload < 2 || nload > 4) return false;
    *p = ConsumePlan{};
    p->ts = true;
    p->tb = true;
    p->bx = bx;
    p->n2p = pad16(n2);
    p->n3p = pad16(n3);
    p->gs = pad8(r3);
    if (p->n2p > 256 || p->n3p > 256 || p->gs > 256) return false;
    const int nyf = (n2 + 127) / 128;
    p->ysplit = nyf > 1;
    p->nyi = p->ysplit ? nyf : 1;
    p->nY = p->ysplit ? 1 : nyf;
    if (p->ysplit && bx > 2) return false;
    p->npc = std::min(bx, 256 / p->gs);
    p->ks2 = (r2 + 15) / 16;
    p->ks3 = (r3 + 15) / 16;
    p->ycol_tile = 0;
    for (int p0 = 0; p0 < bx; p0 += p->npc)
        p->ycol_tile = std::max(p->ycol_tile, p0 * p->gs + pad16(std::min(p->npc, bx - p0) * p->gs));
    p->y_cols = (uint32_t)(p->nY * p->ycol_tile);
    p->nT3 = bx * p->nY;
    const uint32_t phi = 2u * (uint32_t)(p->nT3 * p->n3p);
    p->nyb = std::min(3, tcc::kMaxYBuf);
    while (p->nyb >= 2 && p->nyb * p->y_cols + phi > 512) --p->nyb;
    if (p->nyb < 2) return false;
    const uint32_t cols = p->nyb * p->y_cols + phi;
    p->tmem_cols = 32;
    while (p->tmem_cols < cols) p->tmem_cols <<= 1;
    const int na2 = (p->ks2 + 3) / 4, na3 = (p->ks3 + 3) / 4;
    p->ya_rows = (uint32_t)p->n2p;
    p->z_rows = (uint32_t)p->ycol_tile;
    p->ya = (uint32_t)na2 * p->ya_rows * 128u;
    p->zb = (uint32_t)na2 * p->z_rows * 128u;
    p->b3 = (uint32_t)na3 * p->n3p * 128u;
    p->load = (p->ya + p->zb + 1023) & ~1023u;
    p->load3 = (p->b3 + 1023) & ~1023u;
    p->ys_tile = (uint32_t)na3 * tcc::kYsAtom;
    p->ys_bytes = (uint32_t)p->nT3 * p->ys_tile;
    p->nload = nload;
    p->a3_off = p->load * (uint32_t)nload;
    auto total = [&](int nl3, int nys) {
        return (size_t)p->a3_off + (size_t)nl3 * p->load3 + (size_t)nys * p->ys_bytes + tcc::kTbEpiBytes + 1024;
    };
    // the deepest stage-3 ring with two Y tiles, then a third Y tile if it still fits
    p->nys = 2;
    for (p->nload3 = 4; p->nload3 >= 2; --p->nload3)
        if (total(p->nload3, 2) <= 226 * 1024) break;
    if (p->nload3 < 2) return false;
    if (total(p->nload3, 3) <= 226 * 1024) p->nys = 3;
    p->smem = total(p->nload3, p->nys);
    return true;
}

// tensor-pipe cycles per plane and term of a bf16 persistent plan (one MMA costs max(50, N / 2))
static double tb_cost(const ConsumePlan& p) {
    double s2 = 0;
    for (int p0 = 0; p0 < p.bx; p0 += p.npc) s2 += std::max(50.0, pad16(std::min(p.npc, p.bx - p0) * p.gs) / 2.0);
    const double s3 = p.bx * std::max(50.0, p.n3p / 2.0);
    return (p.nY * p.ks2 * s2 + p.nY * p.ks3 * s3) / p.bx;
}

static bool tb_possible(const tx_ctx* c, bool tf32, bool split) {
    if (tf32 || split || c->consume_form != 2) return false;
    ConsumePlan p;
    for (int bx = 1; bx <= 4; ++bx)
        if (plan_tb(c, bx, 2, &p)) return true;
    return false;
}

// single-pass shapes whose planes fit no TMEM plan (large n with large r) take one work item per
// y tile in the persistent kernel (unless the one-CTA-per-item form is forced); failing that,
// the converter kernel
static bool ts_fits(const tx_ctx* c, bool tf32, bool ysplit) {
    ConsumePlan p;
    for (int nl = 2; nl <= tcc::kMaxLoad; ++nl)
        if (plan_ts(c, tf32, 1, nl, &p, ysplit)) return true;
    return false;
}
static bool ts_ysplit(const tx_ctx* c, bool tf32) {
    return !ts_fits(c, tf32, false) && c->consume_form != 1 && ts_fits(c, tf32, true);
}
static bool ts_possible(const tx_ctx* c, bool tf32) { return ts_fits(c, tf32, false) || ts_ysplit(c, tf32); }

static bool plan_for(const tx_ctx* c, bool tf32, bool split, int bx, int nload, int na3, ConsumePlan* p) {
    if (tb_possible(c, tf32, split)) return plan_tb(c, bx, nload, p);
    if (!split && ts_possible(c, tf32)) return plan_ts(c, tf32, bx, nload, p, ts_ysplit(c, tf32));
    return plan_cv(c, tf32, split, bx, nload, na3, p);
}

// Converter plan (split precisions).  nzi > 0: y/z items, one plane per CTA, one 128-row y tile
// of the plane and one of nzi parts of its z columns: for planes whose phi and operand tiles do
// not fit TMEM, the register accumulator or shared memory whole.
static bool plan_cv(const tx_ctx* c, bool tf32, bool split, int bx, int nload, int na3, ConsumePlan* p, int nzi) {
    const int MK = tf32 ? 8 : 16;
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2];
    if (bx < 1 || bx > n1 || bx > tcc::kMaxPlanes || nload < 1 || nload > tcc::kMaxLoad || na3 < 1 || na3 > 2)
        return false;
    if (nzi > 0 && (bx != 1 || nzi > 16)) return false;
    *p = ConsumePlan{};
    p->bx = bx;
    p->n2p = pad16(n2);
    p->n3p = nzi > 0 ? pad16((n3 + nzi - 1) / nzi) : pad16(n3);
    p->Nz = pad16(r3);
    if (p->n2p > 256 || p->n3p > 256 || p->Nz > 256) return false;
    if (nzi > 0 && (nzi - 1) * p->n3p >= n3) return false;      // no empty z part
    p->yz = nzi > 0;
    p->nzi = nzi;
    p->nyi = nzi > 0 ? (n2 + 127) / 128 : 1;
    p->nY = nzi > 0 ? 1 : (n2 + 127) / 128;
    p->nq = std::min(4, (std::min(n2, nzi > 0 ? 128 : n2) + 31) / 32);
    p->npc = std::min(bx, 256 / p->Nz);                  // planes per stage-2 MMA (N <= 256)
    p->nT3 = nzi > 0 ? 1 : (bx * n2 + 127) / 128;
    p->ks2 = (r2 + MK - 1) / MK;
    p->ks3 = (r3 + MK - 1) / MK;
    p->y_cols = (uint32_t)(bx * p->nY * p->Nz);
    // split precisions keep the cross products in accumulators of their own (twice the columns)
    const uint32_t cols = (split ? 2u : 1u) * (p->y_cols + (uint32_t)(p->nT3 * p->n3p));
    if (cols > 512) return false;
    // ... and fold phi into registers: kMasterGroups x 16 columns per converter thread
    if (split && p->nT3 * p->n3p > 2 * 16 * tcc::kMasterGroups) return false;
    p->tmem_cols = 32;
    while (p->tmem_cols < cols) p->tmem_cols <<= 1;
    const int m = split ? 2 : 1;
    p->ya_rows = (uint32_t)(p->nY * 128);
    p->z_rows = (uint32_t)(bx * p->Nz);                   // plane p at rows p * Nz
    p->ya = (uint32_t)p->ks2 * p->ya_rows * 32u;
    p->zb = (uint32_t)p->ks2 * p->z_rows * 32u;
    p->b3 = (uint32_t)(p->ks3 * p->n3p * 32);
    p->a3 = (uint32_t)(p->ks3 * p->nT3 * 128 * 32);
    // two rings: nload stages of [A_t2][Z] (released by stage 2), then up to two stages of
    // [mu_t A_t3] (released by stage 3), then the na3 converted stage-3 A operands
    p->load = ((uint32_t)(m * (p->ya + p->zb)) + 1023) & ~1023u;
    p->loadB = ((uint32_t)(m * p->b3) + 1023) & ~1023u;
    p->nload = nload;
    p->na3 = na3;
    for (p->nloadB = std::min(tcc::kMaxLoadB, nload + 1); p->nloadB >= 1; --p->nloadB) {
        p->a3_off = p->load * nload + p->loadB * p->nloadB;
        const size_t total = (size_t)p->a3_off + (size_t)na3 * m * p->a3;
        p->smem = std::max(total, (size_t)tcc::kEpiBytes) + 1024;   // the epilogue reuses the front
        if (p->smem <= 226 * 1024) return true;
    }
    return false;
}

static bool choose_plan(const tx_ctx* c, bool tf32, bool split, ConsumePlan* best) {
    if (c->tile_bx > 0) {
        const int nl = c->tile_nstage;
        if (plan_for(c, tf32, split, c->tile_bx, nl, nl > 1 ? 2 : 1, best)) return true;
    }
    double best_score = -1;
    if (tb_possible(c, tf32, split)) {
        // least tensor-pipe time per plane and term, then the deepest stage-2 ring
        for (int nl = 4; nl >= 2; --nl)
            for (int bx = 1; bx <= 4; ++bx) {
                ConsumePlan p;
                if (!plan_tb(c, bx, nl, &p)) continue;
                const double score = 1.0 / tb_cost(p) * (0.9 + 0.03 * nl);
                if (score > best_score * 1.0001) {
                    best_score = score;
                    *best = p;
                }
            }
        return best_score > 0;
    }
    if (!split && ts_possible(c, tf32)) {
        const bool ysplit = ts_ysplit(c, tf32);
        // least tensor-pipe time per plane and term, then the deepest load pipeline
        for (int nl = tcc::kMaxLoad; nl >= 2; --nl)
            for (int bx = 1; bx <= tcc::kMaxPlanes; ++bx) {
                ConsumePlan p;
                if (!plan_ts(c, tf32, bx, nl, &p, ysplit)) continue;
                const double score = 1.0 / ts_cost(p) * (0.8 + 0.05 * nl);
                if (score > best_score * 1.0001) {
                    best_score = score;
                    *best = p;
                }
            }
        return best_score > 0;
    }
    // deepest load pipeline first, then the slab with the least padding per useful row.  With
    // more than one load stage a single converted stage-3 operand buffer still lets the loads
    // and stage 2 of the next term run under the conversion and stage 3 of this one (measured
    // on the Pt-shaped block in TF32x3, one load stage runs load, stage 2, conversion and
    // stage 3 of every term back to back), so two load stages with one operand buffer rank
    // above one load stage.
    for (int nl = tcc::kMaxLoad; nl >= 1; --nl)
        for (int bx = 1; bx <= tcc::kMaxPlanes; ++bx)
            for (int na3 = nl > 1 ? 2 : 1; na3 >= 1; --na3) {
                ConsumePlan p;
                if (!plan_for(c, tf32, split, bx, nl, na3, &p)) continue;
                const double use3 = (double)(bx * c->n[1]) / (p.nT3 * 128.0);
                const double depth = nl >= 4 ? 1.0 : (nl == 3 ? 0.95 : (nl == 2 ? 0.8 : 0.5));
                const double score = depth * use3 * (1.0 + 0.03 * std::min(bx, 8)) * (na3 == 2 ? 1.0 : 0.97) *
                                     (p.nloadB >= 2 ? 1.0 : 0.9);
                if (score > best_score) {
                    best_score = score;
                    *best = p;
                }
            }
    if (best_score > 0 || !split) return best_score > 0;
    // split precisions on planes no whole-slab plan holds: y/z items, the fewest z parts (each
    // part repeats stage 2), then the deepest pipeline
    for (int nzi = 1; nzi <= 16; ++nzi) {
        for (int nl = tcc::kMaxLoad; nl >= 1; --nl)
            for (int na3 = 2; na3 >= 1; --na3)
                if (plan_cv(c, tf32, split, 1, nl, na3, best, nzi)) return true;
    }
    return false;
}

// every (bx, stages) that fits, for the autotuner; returns the count written (<= cap)
int tc_feasible_plans(const tx_ctx* c, int* bx, int* ns, int cap) {
    const TcOperands* op = c->tc;
    if (!op) return 0;
    int k = 0;
    for (int s = tcc::kMaxLoad; s >= 1; --s)
        for (int b = 1; b <= tcc::kMaxPlanes && k < cap; ++b) {
            ConsumePlan p;
            if (plan_for(c, op->tf32, op->split, b, s, s > 1 ? 2 : 1, &p)) {
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
    *ns = p.nload;
    return true;
}

bool tc_plan_fits(const tx_ctx* c, int bx, int ns) {
    const TcOperands* op = c->tc;
    ConsumePlan p;
    return op && plan_for(c, op->tf32, op->split, bx, ns, ns > 1 ? 2 : 1, &p);
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
    return p.items_per_slab_pair(c->n[0]);
}

// Persistent form of the single-pass kernel (the epilogue of one item overlaps the main loop of
// the next): it applies where each epilogue warp holds one tile of phi in registers and the
// energy factors are the multipliers, and it splits shared memory its own way (a stage-2 ring
// of at most four stages, a stage-3 ring as deep as fits, the epilogue boxes).
struct TpSplit {
    bool on;
    int nl1, nl3;
    uint32_t a3_off, epi_off;
    size_t smem;
};

static TpSplit tp_split(const tx_ctx* c, const ConsumePlan& p, bool energy, bool emul) {
    TpSplit t{};
    // columns of one phi row an epilogue lane holds: the whole row with two tiles per item, every
    // other 32-column chunk with one
    const int lane_cols = p.nT3 == 1 ? 32 * (((p.n3p + 31) / 32 + 1) / 2) : p.n3p;
    t.on = p.ts && (c->consume_form != 1 || p.ysplit) && p.nT3 <= 2 && p.bx <= 2 && lane_cols <= tcc::kTpMaxZ &&
           p.nyb >= 2 && (!energy || emul);
    if (!t.on) return t;
    // the two rings as deep as shared memory allows, the shallower of the two first (a ring
    // turns over only when the MMAs queued ahead of its stage have run and the next tile has
    // arrived, so a shallow ring bounds the term rate); at most four stage-2 stages
    auto fits = [&](int n1, int n3) {
        return (size_t)p.load * n1 + (size_t)n3 * p.load3 + tcc::kTpEpiBytes + 1024 <= 226 * 1024;
    };
    int b1 = 0, b3 = 0;
    for (int n1 = 2; n1 <= std::min(p.nload, 4); ++n1)
        for (int n3 = 2; n3 <= tcc::kMaxLoad; ++n3)
            if (fits(n1, n3) && (std::min(n1, n3) > std::min(b1, b3) ||
                                 (std::min(n1, n3) == std::min(b1, b3) && n1 + n3 > b1 + b3))) {
                b1 = n1;
                b3 = n3;
            }
    if (b1 < 2 || b3 < 2) {
        t.on = false;
        return t;
    }
    t.nl1 = b1;
    t.a3_off = p.load * (uint32_t)t.nl1;
    t.nl3 = b3;
    t.epi_off = t.a3_off + (uint32_t)t.nl3 * p.load3;
    t.smem = (size_t)t.epi_off + tcc::kTpEpiBytes + 1024;
    return t;
}

// host-only description of the expansion plan (see tx_describe_expansion_plan)
int tc_describe_plan(const tx_ctx* c, int* out, int nout) {
    const bool tf32 = c->prec == TX_PREC_TF32 || c->prec == TX_PREC_TF32X3;
    const bool split = c->prec == TX_PREC_TF32X3 || c->prec == TX_PREC_BF16X3;
    ConsumePlan p;
    if (!choose_plan(c, tf32, split, &p)) return fail(TX_ERR_UNSUPPORTED_SHAPE, "no expansion tile plan");
    const TpSplit t = (p.ts && !p.tb) ? tp_split(c, p, false, false) : TpSplit{};
    const int v[14] = {p.tb ? 4 : (t.on ? (p.bf3 ? 5 : (p.dual ? 6 : 3)) : (p.ts ? 2 : 1)),
                       p.bx,
                       t.on ? t.nl1 : p.nload,
                       p.ts ? (t.on ? t.nl3 : p.nload3) : (p.tb ? 0 : p.nloadB),
                       p.ts ? p.nyb : 0,
                       (int)p.tmem_cols,
                       (int)(t.on ? t.smem : p.smem),
                       p.tb ? tcc::kThreadsTb
                            : (t.on ? (p.bf3 ? tcc::kThreadsTpB : (p.dual ? tcc::kThreadsTpD : tcc::kThreadsTp))
                                    : (p.ts ? tcc::kThreadsTs : tcc::kThreads)),
                       p.ks2,
                       p.ks3,
                       p.n3p,
                       p.items_per_slab_pair(c->n[0]),
                       p.tailp,
                       p.yz ? p.nzi : 0};
    for (int i = 0; i < nout && i < 14; ++i) out[i] = v[i];
    return TX_OK;
}

// operator image of the bf16 persistent kernel: [A_t2 tile][mu_t A_t3 tile], bf16, per term
static int build_image_tb(tx_ctx* c, cudaStream_t s) {
    TcOperands* op = c->tc;
    ConsumePlan p;
    bool found = false;
    for (int bx = 1; bx <= 4 && !found; ++bx) found = plan_tb(c, bx, 2, &p);
    if (!found) return fail(TX_ERR_UNSUPPORTED_SHAPE, "no bf16 expansion plan");
    const int n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2], T = c->T;
    op->img_stride = p.ya + p.b3;
    if (cudaMalloc(&op->img, (size_t)T * op->img_stride) != cudaSuccess) {
        cudaGetLastError();
        op->img = nullptr;
        return fail(TX_ERR_OOM, "expansion operator image");
    }
    CUtensorMap mA2, mA3;
    const int l2 = ldk(r2, 2), l3 = ldk(r3, 2);
    TX_TRY(make_map(&mA2, op->st.A2, 2, l2, n2, T, l2, (uint64_t)n2 * l2, 64, (uint32_t)p.n2p));
    TX_TRY(make_map(&mA3, op->st.A3, 2, l3, n3, T, l3, (uint64_t)n3 * l3, 64, (uint32_t)p.n3p));
    tcc::ImageArgs g{};
    g.ks2 = p.ks2;
    g.ks3 = p.ks3;
    g.n3p = p.n3p;
    g.ya_rows = p.ya_rows;
    g.ya_bytes = p.ya;
    g.b3_bytes = p.b3;
    g.stride = op->img_stride;
    g.img = (uint8_t*)op->img;
    g.err = c->d_err;
    const int smem = (int)op->img_stride + 1024;
    cudaFuncSetAttribute(tcc::k_operand_image_b16<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    tcc::k_operand_image_b16<0><<<(unsigned)T, 32, smem, s>>>(mA2, mA3, g);
    TX_LAUNCHED();
    return TX_OK;
}

int tc_build_operand_image(tx_ctx* c, cudaStream_t s) {
    TcOperands* op = c->tc;
    if (op->img) {
        bump_gen(c);
        cudaFree(op->img);
        op->img = nullptr;
    }
    ConsumePlan p;
    if (tb_possible(c, op->tf32, op->split)) return build_image_tb(c, s);
    if (op->split || !ts_possible(c, op->tf32)) return TX_OK;
    const bool ysplit = ts_ysplit(c, op->tf32);
    for (int nl = 2; nl <= tcc::kMaxLoad; ++nl)
        if (plan_ts(c, op->tf32, 1, nl, &p, ysplit)) break;
    // the tile shapes below depend on (n, r, precision) only, not on the slab or the stages
    const int n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2], T = c->T, eb = op->esize;
    op->img_stride = p.img_stride();
    if (p.bf3) {
        // [A_t2 tile][mu_t A_t3 tile in bf16] per term (then the packed-tile windows)
        if (cudaMalloc(&op->img, (size_t)T * op->img_stride) != cudaSuccess) {
            cudaGetLastError();
            op->img = nullptr;
            return fail(TX_ERR_OOM, "expansion operator image");
        }
        CUtensorMap mA2b, mA3b;
        const int l2 = ldk(r2, 2), l3 = ldk(r3, 2);
        TX_TRY(make_map(&mA2b, op->st.A2, 2, l2, n2, T, l2, (uint64_t)n2 * l2, 64, (uint32_t)p.n2p));
        TX_TRY(make_map(&mA3b, op->st.A3, 2, l3, n3, T, l3, (uint64_t)n3 * l3, 64, (uint32_t)p.n3p));
        tcc::ImageArgs g{};
        g.ks2 = p.ks2;
        g.ks3 = p.ks3;
        g.n3p = p.n3p;
        g.ya_rows = p.ya_rows;
        g.ya_bytes = p.ya;
        g.b3_bytes = p.b3;
        g.stride = op->img_stride;
        g.img = (uint8_t*)op->img;
        g.err = c->d_err;
        const int smem = (int)(p.ya + p.b3) + 1024;
        cudaFuncSetAttribute(tcc::k_operand_image_b16<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tcc::k_operand_image_b16<0><<<(unsigned)T, 32, smem, s>>>(mA2b, mA3b, g);
        TX_LAUNCHED();
        if (p.tailp) {
            tcc::k_tail_windows<<<dim3((unsigned)T, (unsigned)p.tailp), 256, 0, s>>>(
                (uint8_t*)op->img, op->img_stride, p.ya + p.b3, p.ya, p.ya_rows, (p.ks2 + 3) / 4, 128 * (p.nyi - 1),
                p.tail_rows, p.tail_r8);
            TX_LAUNCHED();
        }
        return TX_OK;
    }
    if (cudaMalloc(&op->img, (size_t)T * op->img_stride) != cudaSuccess) {
        cudaGetLastError();
        op->img = nullptr;
        return fail(TX_ERR_OOM, "expansion operator image");
    }
    CUtensorMap mA2, mA3f, mA3t;
    const uint32_t AK2 = op->tf32 ? 32 : 64;   // elements per 128-byte box row
    // K extents are the zero-padded row lengths (whole 32-byte sectors)
    const int l2 = ldk(r2, eb);
    TX_TRY(make_map(&mA2, op->st.A2, eb, l2, n2, T, l2, (uint64_t)n2 * l2, AK2, (uint32_t)p.n2p));
    TX_TRY(make_map(&mA3f, op->st.A3f, 4, pad8(r3), n3, T, pad8(r3), (uint64_t)n3 * pad8(r3), 32, (uint32_t)p.n3p));
    TX_TRY(make_map_sw(&mA3t, op->st.A3f, 4, pad8(r3), n3, T, pad8(r3), (uint64_t)n3 * pad8(r3), 8, (uint32_t)p.n3p,
                       CU_TENSOR_MAP_SWIZZLE_32B));
    tcc::ImageArgs g{};
    g.ks2 = p.ks2;
    g.ks3 = p.ks3;
    g.n3p = p.n3p;
    g.ya_rows = p.ya_rows;
    g.ya_bytes = p.ya;
    g.b3_bytes = p.b3;
    g.stride = op->img_stride;
    g.img = (uint8_t*)op->img;
    g.err = c->d_err;
    const int smem = (int)(p.ya + p.b3) + 1024;
    if (op->tf32) {
        cudaFuncSetAttribute(tcc::k_operand_image<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tcc::k_operand_image<true><<<(unsigned)T, 32, smem, s>>>(mA2, mA3f, mA3t, g);
    } else {
        cudaFuncSetAttribute(tcc::k_operand_image<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tcc::k_operand_image<false><<<(unsigned)T, 32, smem, s>>>(mA2, mA3f, mA3t, g);
    }
    TX_LAUNCHED();
    if (p.tailp) {
        tcc::k_tail_windows<<<dim3((unsigned)T, (unsigned)p.tailp), 256, 0, s>>>(
            (uint8_t*)op->img, op->img_stride, p.ya + p.b3, p.ya, p.ya_rows, (p.ks2 + 3) / 4, 128 * (p.nyi - 1),
            p.tail_rows, p.tail_r8);
        TX_LAUNCHED();
    }
    return TX_OK;
}

int tc_consume(const tx_ctx* c, const PairRec* recs, int p0, int np, const void* Z, const float* SA, const float* SB,
               const float* MUL0, const float* MUL1, float* OUT0, float* OUT1, const OrbCounts& cnt, int flags,
               double* epart, cudaStream_t s, bool emul) {
    const TcOperands* op = c->tc;
    ConsumePlan p;
    if (!choose_plan(c, op->tf32, op->split, &p)) return fail(TX_ERR_UNSUPPORTED_SHAPE, "no expansion tile plan");
    const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2], r2 = c->r[1], r3 = c->r[2], T = c->T;
    const TcScratch sc = tc_scratch(c);
    const int m = op->split ? 2 : 1;
    tcc::ConsumeArgs a{};
    a.n1 = n1; a.n2 = n2; a.n3 = n3; a.r2 = r2; a.r3 = r3; a.nt = T;
    a.bx = p.bx; a.R = p.bx * n2; a.nY = p.nY; a.Nz = p.Nz; a.npc = p.npc; a.nT3 = p.nT3;
    a.n2p = p.n2p; a.n3p = p.n3p; a.ks2 = p.ks2; a.ks3 = p.ks3; a.nq = p.nq;
    a.nload = p.nload; a.na3 = p.na3; a.nyb = p.nyb;
    a.ya_rows = p.ya_rows; a.z_rows = p.z_rows; a.img_ya_rows = p.ya_rows;
    a.ya_bytes = p.ya; a.z_bytes = p.zb; a.b3_bytes = p.b3; a.a3_bytes = p.a3;
    a.load_bytes = p.load; a.a3_off = p.a3_off;
    // bytes the TMA delivers per stage (out-of-range rows and columns count: they are zero-filled):
    // converter kernel, [A_t2][Z] stages and the stage-3 operand ring after them
    a.stage_tx = (uint32_t)(m * 32 * (p.ks2 * p.n2p + p.ks2 * p.bx * r3));
    a.loadB_bytes = p.loadB; a.nloadB = p.nloadB; a.b_off = p.load * (uint32_t)p.nload;
    a.stageB_tx = (uint32_t)(m * 32 * p.ks3 * p.n3p);
    a.tmem_cols = p.tmem_cols; a.y_cols = p.y_cols;
    a.p0 = p0; a.recs = recs;
    a.SA = SA; a.SB = SB; a.MUL0 = MUL0; a.MUL1 = MUL1; a.OUT0 = OUT0; a.OUT1 = OUT1;
    a.w1 = c->f_w[0]; a.w2 = c->f_w[1]; a.w3 = c->f_w[2];
    a.flags = flags; a.epart = epart; a.err = c->d_err;
    a.chunk = c->acc_chunk;     // split precisions: terms per tensor-core accumulation chunk (0: 1)
    a.emul = (SA == MUL1 && SB == MUL0 && emul) ? 1 : 0;
    const int eb = op->esize;
    const uint32_t MK = op->tf32 ? 8 : 16;
    dim3 grid((unsigned)((n1 + p.bx - 1) / p.bx), (unsigned)np);
    if (p.yz) {
        // split kernel, y/z items: one CTA per (plane, y tile, z part); A_t2 boxes of 128 rows
        a.yz = 1;
        a.nyi = p.nyi;
        a.nzi = p.nzi;
        grid.x *= (unsigned)(p.nyi * p.nzi);
        a.stage_tx = (uint32_t)(m * 32 * (p.ks2 * 128 + p.ks2 * p.bx * r3));
    }
    if (p.ts) {
        a.gs = p.gs; a.ycol_tile = p.ycol_tile; a.ns3 = std::min(p.bx, 8);
        a.nload3 = p.nload3; a.load3_bytes = p.load3;
        // bytes per stage-2 stage (128-byte rows; zero-filled parts count): A_t2, Z planes
        const int na2 = (p.ks2 + 3) / 4;
        a.stage_tx = (uint32_t)(128 * (na2 * p.n2p + na2 * p.bx * r3));
        if (!op->img || op->img_stride != (p.tb ? p.ya + p.b3 : p.img_stride()))
            return fail(TX_ERR_CUDA, "operator image missing or built for another tile shape");
        a.img = (const uint8_t*)op->img;
        a.img_stride = op->img_stride;
        a.zsrc = (const uint8_t*)Z;
        a.z_plane = (uint32_t)((size_t)r3 * sc.ld_b * eb);
        CUtensorMap mZ;
        const uint32_t AK2 = op->tf32 ? 32 : 64;   // elements per 128-byte box row
        a.zone = (p.gs == r3 && p.bx * r3 <= 256) ? 1 : 0;
        TX_TRY(make_map(&mZ, Z, eb, sc.ld_b, (uint64_t)n1 * r3, (uint64_t)np * T, sc.ld_b, (uint64_t)n1 * r3 * sc.ld_b,
                        AK2, (uint32_t)(a.zone ? p.bx * r3 : r3)));
        // epilogue tensors [orbital * n1 + x][y][z]: absent arrays take a valid stand-in map
        tcc::EpiMaps em;
        auto orb_map = [&](CUtensorMap* m, const float* base, int norb) -> int {
            if (!base || norb < 1) {
                *m = mZ;
                return TX_OK;
            }
            return make_map(m, base, 4, (uint64_t)n3, (uint64_t)n2, (uint64_t)norb * n1, (uint64_t)n3, (uint64_t)n2 * n3,
                            32, 32);
        };
        TX_TRY(orb_map(&em.m0, MUL0, cnt.mul0));
        TX_TRY(orb_map(&em.m1, MUL1, cnt.mul1));
        TX_TRY(orb_map(&em.sa, SA, cnt.sa));
        TX_TRY(orb_map(&em.sb, SB, cnt.sb));
        TX_TRY(orb_map(&em.o0, OUT0, cnt.out0));
        TX_TRY(orb_map(&em.o1, OUT1, cnt.out1));
        if (p.tb) {
            if ((flags & EPI_ENERGY) && !a.emul)
                return fail(TX_ERR_UNSUPPORTED_SHAPE, "bf16 expansion: energy sums need the symmetric pair table");
            a.nload3 = p.nload3;
            a.load3_bytes = p.load3;
            a.nys = p.nys;
            a.ys_tile = p.ys_tile;
            a.ys_bytes = p.ys_bytes;
            a.ys_off = p.a3_off + (uint32_t)p.nload3 * p.load3;
            a.epi_off = a.ys_off + (uint32_t)p.nys * p.ys_bytes;
            a.ks3 = p.ks3;
            a.nslab = (int)grid.x;
            a.nyi = p.nyi;
            a.nitems = (int)grid.x * np * p.nyi;
            int dev = 0, nsm = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            using KernTb = void (*)(const CUtensorMap, const tcc::EpiMaps, tcc::ConsumeArgs);
            KernTb kern = tcc::k_consume_tb<0, 0>;
            if (p.ks2 == 2 && p.ks3 == 2) kern = tcc::k_consume_tb<2, 2>;
            if (p.ks2 == 3 && p.ks3 == 3) kern = tcc::k_consume_tb<3, 3>;
            if (p.ks2 == 4 && p.ks3 == 4) kern = tcc::k_consume_tb<4, 4>;
            const int ps = prof_begin("tc_consume", s);
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
            kern<<<dim3((unsigned)std::min(a.nitems, nsm)), tcc::kThreadsTb, p.smem, s>>>(mZ, em, a);
            prof_end(ps, s);
            TX_LAUNCHED();
            return TX_OK;
        }
        if (8 * tcc::kEpiWarpBytes + 1024 > p.smem) return fail(TX_ERR_UNSUPPORTED_SHAPE, "expansion epilogue buffers");
        const TpSplit tps = tp_split(c, p, (flags & EPI_ENERGY) != 0, a.emul != 0);
        const bool tp = tps.on;
        if (p.ysplit && !tp)
            return fail(TX_ERR_UNSUPPORTED_SHAPE, "expansion: this grid needs the persistent kernel's y-tile items, "
                                                  "which do not apply to this call");
        size_t smem = p.smem;
        if (tp) {
            a.nload = tps.nl1;
            a.a3_off = tps.a3_off;
            a.nload3 = tps.nl3;
            a.epi_off = tps.epi_off;
            smem = tps.smem;
        }
        // instantiations with compile-time K step counts for ranks 32, 40, 48 and 64; any other
        // rank runs the dispatching form (see s2_mmas / s3_mmas)
        using Kern = void (*)(const CUtensorMap, const tcc::EpiMaps, tcc::ConsumeArgs);
        Kern kern;
        if (tp && p.bf3) {
            kern = (Kern)tcc::k_consume_tp<false, 0, 0, true>;
            if (p.ks2 == 4 && p.ks3 == 4) kern = tcc::k_consume_tp<false, 4, 4, true>;
            if (p.ks2 == 3 && p.ks3 == 3) kern = tcc::k_consume_tp<false, 3, 3, true>;
        } else if (tp && p.dual) {
            kern = (Kern)tcc::k_consume_tp<false, 0, 0, false, true>;
            if (p.ks2 == 4 && p.ks3 == 8) kern = tcc::k_consume_tp<false, 4, 8, false, true>;
            if (p.ks2 == 3 && p.ks3 == 6) kern = tcc::k_consume_tp<false, 3, 6, false, true>;
        } else if (tp) {
            kern = op->tf32 ? (Kern)tcc::k_consume_tp<true, 0, 0> : (Kern)tcc::k_consume_tp<false, 0, 0>;
#define TX_TP_CASE(TF, K2, K3) \
    if (op->tf32 == TF && p.ks2 == K2 && p.ks3 == K3) kern = tcc::k_consume_tp<TF, K2, K3>;
            TX_TP_CASE(false, 2, 4) TX_TP_CASE(false, 3, 5) TX_TP_CASE(false, 3, 6) TX_TP_CASE(false, 4, 8)
            TX_TP_CASE(true, 4, 4) TX_TP_CASE(true, 5, 5) TX_TP_CASE(true, 6, 6) TX_TP_CASE(true, 8, 8)
#undef TX_TP_CASE
        } else {
            kern = op->tf32 ? (Kern)tcc::k_consume_ts<true, 0, 0> : (Kern)tcc::k_consume_ts<false, 0, 0>;
#define TX_TS_CASE(TF, K2, K3) \
    if (op->tf32 == TF && p.ks2 == K2 && p.ks3 == K3) kern = tcc::k_consume_ts<TF, K2, K3>;
            TX_TS_CASE(false, 2, 4) TX_TS_CASE(false, 3, 5) TX_TS_CASE(false, 3, 6) TX_TS_CASE(false, 4, 8)
            TX_TS_CASE(true, 4, 4) TX_TS_CASE(true, 5, 5) TX_TS_CASE(true, 6, 6) TX_TS_CASE(true, 8, 8)
#undef TX_TS_CASE
        }
        a.nslab = (int)grid.x;
        a.nyi = p.nyi;
        a.per_pair = p.items_per_slab_pair(n1);
        a.nitems = a.per_pair * np;
        if (p.tailp) {
            if (!tp) return fail(TX_ERR_UNSUPPORTED_SHAPE, "packed y tiles need the persistent kernel");
            // every item reads 128 rows of A_t2 (or of a window) per K atom
            a.stage_tx = (uint32_t)(128 * (na2 * 128 + na2 * p.bx * r3));
            a.ya_rows = p.sya_rows;
            a.ya_bytes = p.sya;
            a.tailp = p.tailp;
            a.tail_r8 = p.tail_r8;
            a.tail_rows = p.tail_rows;
            a.win_off = p.ya + p.b3;
        }
        if (tp) {
            int dev = 0, nsm = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            grid = dim3((unsigned)std::min(a.nitems, nsm));
        }
        const int ps = prof_begin("tc_consume", s);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (p.bf3 && !tp) return fail(TX_ERR_UNSUPPORTED_SHAPE, "bf16 stage 3 in TMEM needs the persistent kernel");
        if (p.dual && !tp) return fail(TX_ERR_UNSUPPORTED_SHAPE, "the dual-issuer form needs the persistent kernel");
        kern<<<grid, tp ? (p.bf3 ? tcc::kThreadsTpB : (p.dual ? tcc::kThreadsTpD : tcc::kThreadsTp)) : tcc::kThreadsTs,
               smem, s>>>(mZ, em, a);
        prof_end(ps, s);
        TX_LAUNCHED();
        return TX_OK;
    }
    // Z of this batch: [pair][t][(x, g) rows][ld_b]; lo part after the batch's hi part
    const size_t zlo = (size_t)np * sc.z * eb;
    CUtensorMap mZ, mZlo, mA2, mA2lo, mA3, mA3lo;
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_32B;
    const int l2 = ldk(r2, eb), l3 = ldk(r3, eb);
    TX_TRY(make_map_sw(&mZ, Z, eb, sc.ld_b, (uint64_t)n1 * r3, (uint64_t)np * T, sc.ld_b, (uint64_t)n1 * r3 * sc.ld_b, MK,
                       (uint32_t)r3, sw));
    const uint32_t a2_box = p.yz ? 128u : (uint32_t)p.n2p;     // rows of one A_t2 box
    TX_TRY(make_map_sw(&mA2, op->st.A2, eb, l2, n2, T, l2, (uint64_t)n2 * l2, MK, a2_box, sw));
    TX_TRY(make_map_sw(&mA3, op->st.A3, eb, l3, n3, T, l3, (uint64_t)n3 * l3, MK, (uint32_t)p.n3p, sw));
    if (op->split) {
        TX_TRY(make_map_sw(&mZlo, (const char*)Z + zlo, eb, sc.ld_b, (uint64_t)n1 * r3, (uint64_t)np * T, sc.ld_b,
                           (uint64_t)n1 * r3 * sc.ld_b, MK, (uint32_t)r3, sw));
        TX_TRY(make_map_sw(&mA2lo, (const char*)op->st.A2 + op->st.off_lo, eb, l2, n2, T, l2, (uint64_t)n2 * l2, MK,
                           a2_box, sw));
        TX_TRY(make_map_sw(&mA3lo, (const char*)op->st.A3 + op->st.off_lo, eb, l3, n3, T, l3, (uint64_t)n3 * l3, MK,
                           (uint32_t)p.n3p, sw));
    } else {
        mZlo = mZ;
        mA2lo = mA2;
        mA3lo = mA3;
    }
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
