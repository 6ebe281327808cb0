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

// C = op(A) op(B) with FP32 inputs and FP64 products and sums (alpha 1, beta 0).
cudaError_t cgemm_wide(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<float>* A,
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
template <typename R>
void eig_work_bind(EigWork<R>& w, void* base, int n_cap);

// Eigendecomposition of the Hermitian n x n row-major matrix a (not modified).
// w: device double[n] descending; v: device n x n row-major, eigenvectors in columns.
template <typename R>
cudaError_t heig(cudaStream_t st, int n, const cx<R>* a, long lda, cx<R>* v, long ldv,
                 double* w, EigWork<R>& work, int max_sweeps);

}  // namespace mpdo
