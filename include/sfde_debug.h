/*
 * sfde_debug.h -- verification hooks of the GB300 SFDE library (not needed to solve problems).
 * No counterpart in the paper.
 */
#ifndef SFDE_DEBUG_H
#define SFDE_DEBUG_H
#include "sfde.h"
#ifdef __cplusplus
extern "C" {
#endif

/*
 * One tensor-core slice GEMM on device buffers, the unit every mixed-precision step is built from:
 *   Out[b] = (X[s0 + b*ds] * Mat)^T,  b = 0..batch-1,
 * X: nslices slices of R x C row-major (R = 32, 64 or a multiple of 128); MatT: Cout x C row-major
 * (Mat transposed, Cout a multiple of 32); Out: batch slices of Cout x R.  kind 0: BF16 operands and
 * output (tcgen05 kind::f16), kind 1: FP32 storage with TF32 products (kind::tf32); FP32
 * accumulation.  All pointers are device pointers, 16-byte aligned.  Synchronous.  *err_out (may be
 * NULL) receives the kernel's error word (non-zero if a bounded wait ran out -> SFDE_ETIMEOUT).
 * If reps > 0 and ms_out != NULL, the product is then repeated `reps` times back to back on the
 * legacy default stream and the average device time per launch (CUDA events) is stored in *ms_out.
 */
sfde_status sfde_debug_tc_gemm(int kind, const void* X, long long nslices, int s0, int ds, int batch,
                               int R, int C, const void* MatT, int Cout, void* Out, int* err_out,
                               int reps, float* ms_out);

#ifdef __cplusplus
}
#endif
#endif
