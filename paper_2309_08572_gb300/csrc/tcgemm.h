// Tensor-core (tcgen05 + TMA) GEMM of tcgemm.cu: internal interface.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace mpdo {

// Operand modes of the tensor-core path: the MMA element type and the number of K-segments
// of a packed complex operand (1 = plain, 3 = split hi/lo precision compensation).
enum { TC_TF32 = 0, TC_TF32X3 = 1, TC_BF16 = 2, TC_BF16X3 = 3 };
inline int tc_mode_elt(int mode) { return (mode == TC_TF32 || mode == TC_TF32X3) ? 4 : 2; }
inline int tc_mode_parts(int mode) { return (mode == TC_TF32X3 || mode == TC_BF16X3) ? 3 : 1; }
// Row stride (elements) of a packed operand with k complex columns: the real K extent
// (parts x 2k) rounded up to 16 bytes, as TMA requires.
inline long tc_pack_ld(int mode, long k) {
  const long kr = (long)tc_mode_parts(mode) * 2 * k;
  const long q = 16 / tc_mode_elt(mode);
  return (kr + q - 1) / q * q;
}

struct TcEpilogue {
  float* d = nullptr;      // FP32 output (real view), or
  double* d64 = nullptr;   // FP64 accumulation target (d64 += scale * acc)
  long ldd = 0, sd = 0;    // row and batch strides of the output, in elements
  float ar = 1.f, ai = 0.f, br = 0.f, bi = 0.f;   // complex alpha, beta (column pairs)
  int use_beta = 0;
  double scale = 1.0;
};

// Real product D[b] = A[b] B[b]^T with A (M x K), B (N x K), both K-major, elements FP32
// (read as TF32, elt = 4) or BF16 (elt = 2); leading dimensions and batch strides in
// elements (multiples of 16 bytes; 16-byte aligned bases).  bn: output tile width (64, 128
// or 256; <= 0 picks by size).  err: device int set non-zero when a pipeline wait gave up.
cudaError_t tc_gemm_real(cudaStream_t st, int elt, int M, int N, int K, const void* A, long lda,
                         long sa, const void* B, long ldb, long sb, int batch, const TcEpilogue& e,
                         int* err, int bn);
int tc_pick_bn(long M, long N, int batch);

// Pack a complex operand for tc_gemm_real (side 0: A rows; side 1: B rows in the 2 x 2 real
// embedding); see tcgemm.cu.
template <typename TIN>
cudaError_t tc_pack(cudaStream_t st, int mode, int side, int rows, int kc, const cx<TIN>* src,
                    long s_r, long s_c, long sb, int conj, int batch, void* out);

// Complex64 C[b] = alpha op(A[b]) op(B[b]) + beta C[b] on the tensor cores (ops as in cgemm:
// 0 N, 1 T, 2 C, 3 R), operands packed into ws (tc_cgemm_ws_bytes of it).
template <typename TIN>
cudaError_t tc_cgemm(cudaStream_t st, int mode, int opa, int opb, int m, int n, int k,
                     const cx<TIN>* A, long lda, long sa, const cx<TIN>* B, long ldb, long sb,
                     float2* C, long ldc, long sc, int batch, float2 alpha, float2 beta,
                     void* ws, size_t ws_bytes, int* err);
size_t tc_cgemm_ws_bytes(int mode, long m, long n, long k, int batch);

// Complex FP64 C[b] = op(A[b]) op(B[b]) of complex FP32 or FP64 operands (TA, TB: float2 or
// double2), carried to ~2^-48 of each operand row's largest entry and summed in FP64
// (error-free BF16 slices on the tensor cores; tcgemm.cu).  Long K is processed in pieces
// that fit ws, added in FP64.
template <typename TA, typename TB>
cudaError_t tc_cgemm_exact(cudaStream_t st, int opa, int opb, int m, int n, int k, const TA* A,
                           long lda, long sa, const TB* B, long ldb, long sb, double2* C, long ldc,
                           long sc, int batch, void* ws, size_t ws_bytes, int* err);
size_t tc_exact_ws_bytes(long m, long n, long k, int batch);
// One-time kernel attribute setup of tc_cgemm_exact; call it before capturing a stream that
// will run the first exact product of the process.
cudaError_t tc_exact_init();

// out[r][c] = bf16(src[r*s_r + c*s_c]) for r < rows, c < kc (row stride ldo elements): the
// K-major BF16 operands of tc_gemm_real from a real FP32 matrix in either orientation.
cudaError_t tc_pack_real_bf16(cudaStream_t st, int rows, int kc, const float* src, long s_r,
                              long s_c, void* out, long ldo);

}  // namespace mpdo
