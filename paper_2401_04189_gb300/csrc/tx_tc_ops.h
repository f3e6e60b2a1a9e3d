// Tensor-core path: operand copies owned by the context and the per-pair scratch layout.
#pragma once

#include "tx_tc.h"

namespace tx {

inline int pad8(int v) { return (v + 7) & ~7; }
inline int pad16(int v) { return (v + 15) & ~15; }
// row length (elements) of a tensor-core operand in memory: K padded with zeros to a multiple of
// 32 bytes.  A TMA box row that ends inside a 32-byte sector of its tensor takes a slow path
// (measured: about a quarter of the full-row rate), so every map's K extent is a whole number
// of sectors and the padding is read as zeros.
inline int ldk(int k, int elem_bytes) { return elem_bytes == 2 ? pad16(k) : pad8(k); }

// Static operands, K-major with 16-byte row strides, in the operand type of the precision
// (bf16, or float32 holding TF32 values).  For the 3-pass precisions `lo` holds x - hi.
struct TcStatic {
    void* U3T;   // [r3][ld(n3)]     rows gamma, K = z        (projection, mode 3)
    void* U2T;   // [r2][ld(n2)]     rows beta,  K = y        (projection, mode 2)
    void* U1T;   // [r1][ld(n1)]     rows alpha, K = x        (projection, mode 1)
    void* A1s;   // [T*n1][ld(r1)]   rows (t,x), K = alpha    (expansion, mode 1, every term)
    void* A2;    // [T][n2][ld(r2)]  rows y, K = beta         (expansion, mode 2)
    void* A3;    // [T][n3][ld(r3)]  rows z, K = gamma, mu_t folded in (expansion, mode 3)
    void* A3f;   // the same in float32 rounded to TF32 (single-pass precisions; == A3 for tf32)
    void* A3T;   // [T][r3][ld(n3)]  rows gamma, K = z, mu_t folded in (adjoint, mode 3)
    void* A2T;   // [T][r2][ld(n2)]  rows beta,  K = y        (adjoint, mode 2)
    size_t off_lo;   // byte offset from each hi array to its lo copy (3-pass precisions)
};

struct TcOperands {
    int prec;
    bool tf32, split;
    int esize;            // bytes per operand element
    char* buf;            // one allocation for every static operand (hi, then lo)
    TcStatic st;
    int bx;               // x planes per expansion CTA
    // single-pass expansion: per Gaussian term, the shared-memory image of its operator tiles
    // ([A_t2 tile][mu_t A_t3 tile], swizzled and zero-filled as the tile loads lay them out)
    void* img;
    uint32_t img_stride;  // bytes per term
};

// per-pair scratch (elements of the operand type; doubled for split precisions)
struct TcScratch {
    size_t s1, s2, g, z;  // element counts per pair
    int ld_y, ld_x, ld_a, ld_b;
};
TcScratch tc_scratch(const tx_ctx* c);

// S1 = (SA * SB (* w)) x3 B^T with B the operand U3^T (forward projection, Bhi NULL) or a term's
// mu_t A_t3^T (the adjoint's first mode)
int tc_project_mode3(const tx_ctx* c, const PairRec* recs, int p0, int np, const float* SA, int nA, const float* SB,
                     int nB, int flags, void* S1, cudaStream_t s, const void* Bhi = nullptr);
int tc_build_operand_image(tx_ctx* c, cudaStream_t s);
// orbital counts of the arrays the expansion epilogue reads and writes (bounds of its tensors)
struct OrbCounts {
    int sa, sb, mul0, mul1, out0, out1;
};
int tc_consume(const tx_ctx* c, const PairRec* recs, int p0, int np, const void* Z, const float* SA, const float* SB,
               const float* MUL0, const float* MUL1, float* OUT0, float* OUT1, const OrbCounts& cnt, int flags, double* epart,
               cudaStream_t s, bool emul = false);
long tc_consume_blocks(const tx_ctx* c);

}  // namespace tx
