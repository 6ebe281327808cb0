// Mixed-precision Hermitian eigensolver for the FP64 Gram matrices of the mixed mode:
// FP32 Jacobi sweeps plus FP64 residual products.
//
// FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU and a one-CTA Jacobi solve is
// bound by the ALUs of one SM, so FP64 sweeps would dominate the update.  Here the sweeps
// run in FP32 and FP64 appears only in dense products, which spread over many SMs:
//
//   level l, orthonormal FP64 basis X (n x m, X = I at level 0):
//     B = X^+ A X (FP64) -> FP32 Jacobi of B -> Y;  Z = X Y (FP64)
//     refinement (Ogita and Aishima, "Iterative refinement for symmetric eigenvalue
//     decomposition", 2018), `passes` times:
//       S = Z^+ A Z, G = Z^+ Z, lam_i = S_ii / G_ii,
//       E_ij = (S_ij - lam_j G_ij) / (lam_j - lam_i) for separated pairs with a
//              resolved member, -G_ij / 2 otherwise;  E_ii = (1 - G_ii) / 2;  Z <- Z (I + E)
//     pairs with lam > tau * lam_max(l) (a leading run) are final; the other columns of Z
//     span the next level's basis, because FP32 sweeps resolve eigenvectors only down to
//     ~n eps_32 lam_max(l)
//   until the largest remaining lam falls below floor * lam_max(0) or nothing remains.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace mpdo {

namespace {

// FP32 sweeps give eigenvectors to ~m eps_32 lam_max / gap.  A refinement pass squares that
// error only while it is small, so pairs are corrected only when their gap exceeds
// 100 m eps_32 lam_max (error <= 1e-2, 1e-4 after one pass, 1e-8 after two); closer pairs
// stay a cluster (orthonormalised only: any basis of a cluster is an eigenbasis to within
// the cluster's width).  Resolved eigenvalues lie above kTau lam_max, two decades per level,
// so that neighbours in a geometric spectrum stay separated.
constexpr double kTau = 1e-2;
constexpr double kGapPerDim = 100 * 6e-8;
constexpr int kPasses = 2;
constexpr int kMaxLevels = 8;

// lam_i = S_ii / G_ii; out[0] = lam_max; out[1] = length of the leading run with
// lam > tau lam_max; out[2] = max lam over the rest
__global__ void mix_scan_kernel(int m, const double2* __restrict__ S,
                                const double2* __restrict__ G, double* lam, double* out) {
  __shared__ double red[1024];
  const int tid = threadIdx.x;
  double mx = -1e300;
  for (int i = tid; i < m; i += blockDim.x) {
    double g = G[(long)i * m + i].x;
    double l = g > 0 ? S[(long)i * m + i].x / g : 0.0;
    lam[i] = l;
    mx = fmax(mx, l);
  }
  red[tid] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
    __syncthreads();
  }
  const double lmax = red[0];
  __syncthreads();
  if (tid == 0) {
    int nl = 0;
    while (nl < m && lam[nl] > kTau * lmax) ++nl;
    double rest = 0.0;
    for (int i = nl; i < m; ++i) rest = fmax(rest, lam[i]);
    out[0] = lmax;
    out[1] = (double)nl;
    out[2] = rest;
  }
}

// IE = I + E (see the file comment)
__global__ void mix_correction_kernel(int m, int n, const double2* __restrict__ S,
                                      const double2* __restrict__ G,
                                      const double* __restrict__ lam,
                                      const double* __restrict__ scan, double lam0,
                                      double2* IE) {
  const double lmax = scan[0];
  // separated: above the FP32 resolution of this level and above the FP64 rounding of the
  // products with A (~n eps_64 lam_0), below which eigenvectors are not defined
  const double sep = fmax(kGapPerDim * (m > 10 ? m : 10) * lmax, 100.0 * n * 1.1e-16 * lam0);
  const int nl = (int)scan[1];
  long total = (long)m * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    double2 g = G[e];
    double2 r;
    if (i == j) {
      r = make_double2(1.0 + 0.5 * (1.0 - g.x), 0.0);
    } else {
      double d = lam[j] - lam[i];
      bool resolved = (i < nl) || (j < nl);
      if (resolved && fabs(d) > sep) {
        double2 s = S[e];
        r = make_double2((s.x - lam[j] * g.x) / d, (s.y - lam[j] * g.y) / d);
      } else {
        r = make_double2(-0.5 * g.x, -0.5 * g.y);
      }
    }
    IE[e] = r;
  }
}

cudaError_t gemm64(cudaStream_t st, int opa, int opb, int m, int n, int k, const double2* A,
                   long lda, const double2* B, long ldb, double2* C, long ldc) {
  return cgemm<double>(st, opa, opb, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1,
                       make_double2(1, 0), make_double2(0, 0));
}

}  // namespace

size_t mix_work_bytes(int n_cap) {
  size_t sq = (size_t)n_cap * n_cap;
  return 7 * sq * sizeof(double2) + 2 * sq * sizeof(float2) + 4 * (size_t)n_cap * 8 +
         eig_work_bytes<float>(n_cap) + 8 * 256;
}

void mix_work_bind(MixWork& w, void* base, int n_cap) {
  size_t sq = (size_t)n_cap * n_cap;
  char* p = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  w.n_cap = n_cap;
  w.x = reinterpret_cast<double2*>(take(sq * 16));
  w.z = reinterpret_cast<double2*>(take(sq * 16));
  w.z2 = reinterpret_cast<double2*>(take(sq * 16));
  w.t = reinterpret_cast<double2*>(take(sq * 16));
  w.s = reinterpret_cast<double2*>(take(sq * 16));
  w.g = reinterpret_cast<double2*>(take(sq * 16));
  w.ie = reinterpret_cast<double2*>(take(sq * 16));
  w.a32 = reinterpret_cast<float2*>(take(sq * 8));
  w.y32 = reinterpret_cast<float2*>(take(sq * 8));
  w.lam = reinterpret_cast<double*>(take((size_t)n_cap * 8));
  w.w32 = reinterpret_cast<double*>(take((size_t)n_cap * 8));
  w.scan = reinterpret_cast<double*>(take(64));
  eig_work_bind<float>(w.ew, take(eig_work_bytes<float>(n_cap)), n_cap);
}

cudaError_t heig_mixed(cudaStream_t st, int n, const double2* a, long lda, double2* v, long ldv,
                       double* w, double floor, MixWork& wk, int* levels_out,
                       double* flops_out) {
  double flops = 0.0;
  auto gf = [&](int mm, int nn, int kk) { flops += 8.0 * mm * nn * (double)kk; };
  int hcnt[4];
  if (n <= 0) return cudaSuccess;
  if (n > wk.n_cap) return cudaErrorInvalidValue;
  int m = n, off = 0, level = 0;
  double lam0 = 0.0;
  double hscan[3];
  for (;; ++level) {
    // B = X^+ A X (level 0: B = A), rounded to FP32 for the sweeps
    const double2* B = a;
    long ldbm = lda;
    if (level > 0) {
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.x, m, wk.t, m));
      MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.x, m, wk.t, m, wk.s, m));
      gf(n, m, n);
      gf(m, m, n);
      B = wk.s;
      ldbm = m;
    }
    MPDO_CUDA_TRY((convert<double, float>(st, m, m, B, ldbm, wk.a32, m)));
    MPDO_CUDA_TRY(heig<float>(st, m, wk.a32, m, wk.y32, m, wk.w32, wk.ew, 20));
    // Z = X Y
    if (level == 0) {
      MPDO_CUDA_TRY((convert<float, double>(st, n, m, wk.y32, m, wk.z, m)));
    } else {
      MPDO_CUDA_TRY((convert<float, double>(st, m, m, wk.y32, m, wk.ie, m)));
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, wk.x, m, wk.ie, m, wk.z, m));
      gf(n, m, m);
    }
    for (int pass = 0; pass < kPasses; ++pass) {
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.z, m, wk.t, m));
      MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.z, m, wk.t, m, wk.s, m));
      MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.z, m, wk.z, m, wk.g, m));
      count_launch(2);
      mix_scan_kernel<<<1, 1024, 0, st>>>(m, wk.s, wk.g, wk.lam, wk.scan);
      MPDO_CUDA_TRY(cudaGetLastError());
      long tot = (long)m * m;
      int blocks = (int)std::min<long>((tot + 255) / 256, 4096);
      if (level == 0 && pass == 0) {
        // lam_0 (largest eigenvalue) for the absolute separation floor
        MPDO_CUDA_TRY(cudaMemcpyAsync(hscan, wk.scan, sizeof(hscan), cudaMemcpyDeviceToHost, st));
        MPDO_CUDA_TRY(cudaStreamSynchronize(st));
        lam0 = hscan[0];
      }
      mix_correction_kernel<<<blocks, 256, 0, st>>>(m, n, wk.s, wk.g, wk.lam, wk.scan, lam0,
                                                    wk.ie);
      MPDO_CUDA_TRY(cudaGetLastError());
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, wk.z, m, wk.ie, m, wk.z2, m));
      gf(n, m, n);
      gf(m, m, n);
      gf(m, m, n);
      gf(n, m, m);
      std::swap(wk.z, wk.z2);
    }
    // Rayleigh quotients of the refined vectors and the split of this level
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.z, m, wk.t, m));
    MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.z, m, wk.t, m, wk.s, m));
    MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.z, m, wk.z, m, wk.g, m));
    count_launch();
    mix_scan_kernel<<<1, 1024, 0, st>>>(m, wk.s, wk.g, wk.lam, wk.scan);
    MPDO_CUDA_TRY(cudaGetLastError());
    gf(n, m, n);
    gf(m, m, n);
    gf(m, m, n);
    MPDO_CUDA_TRY(cudaMemcpyAsync(hscan, wk.scan, sizeof(hscan), cudaMemcpyDeviceToHost, st));
    MPDO_CUDA_TRY(cudaMemcpyAsync(hcnt, wk.ew.counters, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    MPDO_CUDA_TRY(cudaStreamSynchronize(st));
    flops += hcnt[3] * eig_flops_per_count(m, false);
    int nl = (int)hscan[1];
    const bool last = (nl >= m) || level + 1 >= kMaxLevels || !(hscan[2] > floor * lam0) ||
                      nl == 0;
    const int take = last ? m : nl;
    // final columns and values of this level
    MPDO_CUDA_TRY(cudaMemcpy2DAsync(v + off, ldv * sizeof(double2), wk.z, m * sizeof(double2),
                                    take * sizeof(double2), n, cudaMemcpyDeviceToDevice, st));
    MPDO_CUDA_TRY(cudaMemcpyAsync(w + off, wk.lam, take * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
    off += take;
    if (last) break;
    // the unresolved columns become the next basis
    const int mr = m - nl;
    MPDO_CUDA_TRY(cudaMemcpy2DAsync(wk.x, mr * sizeof(double2), wk.z + nl, m * sizeof(double2),
                                    mr * sizeof(double2), n, cudaMemcpyDeviceToDevice, st));
    m = mr;
  }
  if (levels_out) *levels_out = level + 1;
  if (flops_out) *flops_out = flops;
  return cudaSuccess;
}

}  // namespace mpdo
