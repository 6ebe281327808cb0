// Internal declarations shared by the library's translation units (not the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpdo {

enum { OP_N = 0, OP_T = 1, OP_C = 2, OP_R = 3 };

template <typename R>
cudaError_t cgemm(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<R>* A,
                  long lda, long sa, const cx<R>* B, long ldb, long sb, cx<R>* C, long ldc,
                  long sc, int batch, cx<R> alpha, cx<R> beta);

// C = op(A) op(B) with an FP32 A, B of precision RB (float or double), FP64 products and
// sums (alpha 1, beta 0).
template <typename RB>
cudaError_t cgemm_wide(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<float>* A,
                       long lda, long sa, const cx<RB>* B, long ldb, long sb, cx<double>* C,
                       long ldc, long sc, int batch);

// C = op(A) op(B) with an FP64 A and an FP32 B, FP64 products and sums (alpha 1, beta 0).
cudaError_t cgemm_dx(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<double>* A,
                     long lda, long sa, const cx<float>* B, long ldb, long sb, cx<double>* C,
                     long ldc, long sc, int batch);

// Workspace of the Hermitian eigensolver (capacity n_cap).
template <typename R>
struct EigWork {
  int n_cap = 0;
  cx<R>* ap = nullptr;   // padded working matrix
  cx<R>* vp = nullptr;   // padded eigenvector accumulator
  int* counters = nullptr;  // [0..1] rotation counters, [2] sweeps used
};

template <typename R>
size_t eig_work_bytes(int n_cap);
// padded size used by the eigensolver; each active pair-round of the block Jacobi does
// 3 * 16 * 16 * padded_n complex multiply-adds (rows, columns and eigenvectors)
int eig_padded_n(int n);
double eig_flops_per_count(int n, bool fp64);
template <typename R>
void eig_work_bind(EigWork<R>& w, void* base, int n_cap);

// Eigendecomposition of the Hermitian n x n row-major matrix a (not modified).
// w: device double[n] descending; v: device n x n row-major, eigenvectors in columns.
template <typename R>
cudaError_t heig(cudaStream_t st, int n, const cx<R>* a, long lda, cx<R>* v, long ldv,
                 double* w, EigWork<R>& work, int max_sweeps);

// One-CTA FP32 Jacobi solve (n <= kSmemJacobiMaxF32) of a Hermitian matrix of precision RI
// (rounded to FP32 on load), eigenvectors written in precision RO; w, counters as for heig.
constexpr int kSmemJacobiMaxF32 = 118;
template <typename RI, typename RO>
cudaError_t heig_smem_f32(cudaStream_t st, int n, const cx<RI>* a, long lda, cx<RO>* v, long ldv,
                          double* w, int* counters, int max_sweeps);

// One-sided Jacobi on the n x r factor L (row-major, ld lr; r <= 128) of W = L L^+, computed
// in precision R in one CTA's shared memory (n * r * sizeof(cx<R>) <= kOsjMaxSmem, plus the
// FP64 copy with finish64): U (n x r, ld ldu) = eigenvectors of W, w (r) = eigenvalues,
// descending.  finish64 (R = float): FP64 sweeps after the FP32 ones.  counters[2..3] =
// sweeps, rotations.
constexpr size_t kOsjMaxSmem = 200 * 1024;
template <typename RI, typename R, typename RO>
cudaError_t osj(cudaStream_t st, int n, int r, const cx<RI>* L, int lr, cx<RO>* U, int ldu,
                double* w, int* counters, int finish64);

// Workspace of the mixed-precision eigensolver (capacity n_cap).
struct MixGraphs;   // captured level sequences (eigmix.cu)
struct MixWork {
  int n_cap = 0;
  double2 *x = nullptr, *tz = nullptr, *tz2 = nullptr, *s = nullptr, *ie = nullptr;
  float2 *a32 = nullptr, *y32 = nullptr;
  double *lam = nullptr, *w32 = nullptr, *scan = nullptr;
  unsigned int* ticket = nullptr;   // CTA ticket of the fused refinement (0 between launches)
  int* cid = nullptr;               // cluster of each column in the final refinement pass
  unsigned char* sepf = nullptr;    // neighbour separation flags of levels wider than 4096
  EigWork<float> ew;
  MixGraphs* graphs = nullptr;   // created on first use; freed by mix_work_release
  bool use_graphs = true;
  cudaEvent_t block_ev = nullptr; // when set, level read-backs wait on it (blocking sync)
  double* hpin = nullptr;         // mapped pinned host area of the level scalars (lazy)
  double* hpin_dev = nullptr;     // its device address
  // Tensor-core workspace lent by the caller: when set, products of at least tc_min_macs
  // complex multiply-adds run as error-free BF16 slice products (tc_cgemm_exact) instead of
  // CUDA-core FP64; tcerr is the device flag of their pipeline waits.
  void* tcws = nullptr;
  size_t tcws_bytes = 0;
  int* tcerr = nullptr;
  double tc_min_macs = 0;
};
size_t mix_work_bytes(int n_cap);
void mix_work_bind(MixWork& w, void* base, int n_cap);
// Destroys the captured graphs (the device workspace itself belongs to the caller).
void mix_work_release(MixWork& w);
// Eigenpairs of the FP64 Hermitian matrix a (n x n, row-major, lda), descending, resolved
// down to floor * lambda_max: FP32 Jacobi levels with FP64 refinement.  Synchronises the
// stream once per level.
// *flops_out (may be NULL): executed flops (FP32 rotations plus FP64 products).
// max_vals > 0: stop after the level at which at least max_vals leading pairs are resolved;
// the remaining eigenvalues and eigenvector columns are written as zeros.
cudaError_t heig_mixed(cudaStream_t st, int n, const double2* a, long lda, double2* v, long ldv,
                       double* w, double floor, MixWork& wk, int* levels_out,
                       double* flops_out = nullptr, int max_vals = 0);

}  // namespace mpdo
