// Tensor-core (tcgen05) building blocks shared by the tensor-core translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tx_internal.h"

namespace tx {

enum TcOutType { TC_OUT_F32 = 0, TC_OUT_BF16 = 1, TC_OUT_F32_SPLIT = 2, TC_OUT_BF16_SPLIT = 3 };

// A K-major operand in global memory: element (z, row, k) at base + z*depth_stride + row*row_stride + k
// (strides in elements, 16-byte multiples); `lo` is the low part for the 3-pass precisions.
struct TcOperand {
    const void* hi;
    const void* lo;
    uint64_t k_extent, rows, depth, row_stride, depth_stride;
};

// One batched GEMM launch.  Batch b = (b1, b2) with b1 = b % nb1; operand rows are offset by
// b1*x_row1 + b2*x_row2 and the depth coordinate is b1*x_z1 + b2*x_z2.  Output element (m, n)
// of batch b goes to C + b1*c_b1 + b2*c_b2 + m*c_m + n*c_n (+ c_lo for the low part).
struct TcGemmArgs {
    int M, N, K, BN, nb1, nb2;
    int a_row1, a_row2, a_z1, a_z2;
    int b_row1, b_row2, b_z1, b_z2;
    void* C;
    long c_m, c_n, c_b1, c_b2, c_lo;
    int rdiv, cdiv;          // row / column index splits (0 = none)
    long c_mh, c_nh;         // strides of m / rdiv and n / cdiv
    int c_type;
    float alpha;
    uint32_t tmem_cols;
    int nacc;                // TMEM accumulators, one per K atom in turn (summed in float32)
    int vec;                 // set by the launcher: rows are contiguous and 16-byte aligned
    int stages;
    int* err;
};

// [depth][rows][k_extent] operand (strides in elements), box {box_k, box_rows, 1}; 128-byte swizzle
int make_map(CUtensorMap* m, const void* base, int elem_bytes, uint64_t k_extent, uint64_t rows, uint64_t depth,
             uint64_t row_stride_elems, uint64_t depth_stride_elems, uint32_t box_k, uint32_t box_rows);
// the same with the swizzle chosen by the caller (box_k x elem_bytes must not exceed its span)
int make_map_sw(CUtensorMap* m, const void* base, int elem_bytes, uint64_t k_extent, uint64_t rows, uint64_t depth,
                uint64_t row_stride_elems, uint64_t depth_stride_elems, uint32_t box_k, uint32_t box_rows,
                CUtensorMapSwizzle swizzle);
// float32 [depth][rows][k_extent] (row stride k_extent), no swizzle, box {box_k, box_rows, 1}
int make_map_f32_plain(CUtensorMap* m, const void* base, uint64_t k_extent, uint64_t rows, uint64_t depth,
                       uint32_t box_k, uint32_t box_rows);
int tc_gemm_launch(const TcOperand& A, const TcOperand& B, TcGemmArgs g, bool tf32, bool split, const char* prof,
                   cudaStream_t s);
// The same product by the row-streaming kernel where it applies (single-pass precision, K of
// at most two 128-byte atoms, contiguous 16-byte aligned output rows, N >= 128); otherwise
// tc_gemm_launch.
int tc_rows_launch(const TcOperand& A, const TcOperand& B, TcGemmArgs g, bool tf32, bool split, const char* prof,
                   cudaStream_t s);

}  // namespace tx
