// Complex batched GEMM on CUDA cores (FP64 and FP32 arithmetic), generic strides.
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b]; op in {N, T, C (conj-transpose),
// R (conj, no transpose)}.  Used by every contraction of the update for the FP64 and
// C64 modes and for the unit tests of the other GEMM paths.
#include "common.cuh"
#include "internal.h"

namespace mpdo {

namespace {
constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

// Inputs of precision RI, products and sums in R (RI = float, R = double: the FP32
// products are exact in FP64 and the sums carry FP64 rounding only).
template <typename RI, typename R>
__global__ void __launch_bounds__(NT) cgemm_kernel(
    int M, int N, int K, const cx<RI>* __restrict__ A, long sam, long sak, long sab, int conja,
    const cx<RI>* __restrict__ B, long sbk, long sbn, long sbb, int conjb, cx<R>* C, long scm,
    long scn, long scb, cx<R> alpha, cx<R> beta, int use_beta) {
  using T = cx<R>;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long bz = blockIdx.z;
  A += bz * sab;
  B += bz * sbb;
  C += bz * scb;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mkc<R>(0, 0);
  const bool a_kfast = (sak == 1);
  const bool b_nfast = (sbn == 1);
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      int e = tid + q * NT;
      int mi, ki;
      if (a_kfast) { mi = e / BK; ki = e % BK; } else { ki = e / BM; mi = e % BM; }
      int gm = m0 + mi, gk = k0 + ki;
      T v = mkc<R>(0, 0);
      if (gm < M && gk < K) {
        cx<RI> t = A[gm * sam + gk * sak];
        v = mkc<R>((R)t.x, conja ? -(R)t.y : (R)t.y);
      }
      As[ki][mi] = v;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      int e = tid + q * NT;
      int ni, ki;
      if (b_nfast) { ki = e / BN; ni = e % BN; } else { ni = e / BK; ki = e % BK; }
      int gn = n0 + ni, gk = k0 + ki;
      T v = mkc<R>(0, 0);
      if (gn < N && gk < K) {
        cx<RI> t = B[gk * sbk + gn * sbn];
        v = mkc<R>((R)t.x, conjb ? -(R)t.y : (R)t.y);
      }
      Bs[ki][ni] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      T v = cmul(alpha, acc[i][j]);
      T* p = C + gm * scm + gn * scn;
      if (use_beta) v = cadd(v, cmul(beta, *p));
      *p = v;
    }
  }
}
}  // namespace

template <typename RI, typename R>
cudaError_t cgemm_impl(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<RI>* A,
                       long lda, long sa, const cx<RI>* B, long ldb, long sb, cx<R>* C, long ldc,
                       long sc, int batch, cx<R> alpha, cx<R> beta) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  long sam, sak, sbk, sbn;
  int conja = (opa == OP_C || opa == OP_R), conjb = (opb == OP_C || opb == OP_R);
  if (opa == OP_N || opa == OP_R) { sam = lda; sak = 1; } else { sam = 1; sak = lda; }
  if (opb == OP_N || opb == OP_R) { sbk = ldb; sbn = 1; } else { sbk = 1; sbn = ldb; }
  int use_beta = (beta.x != 0 || beta.y != 0);
  if (k <= 0) {  // C = beta C: run with K = 0 (acc = 0)
    k = 0;
  }
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    int nb = batch - b0 < 65535 ? batch - b0 : 65535;
    dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, nb);
    count_launch();
    cgemm_kernel<RI, R><<<grid, NT, 0, st>>>(m, n, k, A + (long)b0 * sa, sam, sak, sa, conja,
                                              B + (long)b0 * sb, sbk, sbn, sb, conjb,
                                              C + (long)b0 * sc, ldc, 1, sc, alpha, beta,
                                              use_beta);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t cgemm(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<R>* A,
                  long lda, long sa, const cx<R>* B, long ldb, long sb, cx<R>* C, long ldc,
                  long sc, int batch, cx<R> alpha, cx<R> beta) {
  return cgemm_impl<R, R>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch,
                          alpha, beta);
}

cudaError_t cgemm_wide(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<float>* A,
                       long lda, long sa, const cx<float>* B, long ldb, long sb, cx<double>* C,
                       long ldc, long sc, int batch) {
  return cgemm_impl<float, double>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc,
                                   batch, mkc<double>(1, 0), mkc<double>(0, 0));
}

template cudaError_t cgemm<double>(cudaStream_t, int, int, int, int, int, const double2*, long,
                                   long, const double2*, long, long, double2*, long, long, int,
                                   double2, double2);
template cudaError_t cgemm<float>(cudaStream_t, int, int, int, int, int, const float2*, long,
                                  long, const float2*, long, long, float2*, long, long, int,
                                  float2, float2);

}  // namespace mpdo
