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
// 100 m eps_32 lam_max (error <= 1e-2 at worst, ~1e-6 in practice, squared by the pass); closer pairs
// stay a cluster (orthonormalised only: any basis of a cluster is an eigenbasis to within
// the cluster's width).  Resolved eigenvalues lie above kTau lam_max, two decades per level,
// so that neighbours in a geometric spectrum stay separated.
constexpr double kTau = 1e-2;
constexpr double kGapPerDim = 100 * 6e-8;
constexpr int kPasses = 1;
constexpr int kMaxLevels = 8;

// One refinement step's scalars and correction, one CTA.  S = SG[:, 0:m], G = SG[:, m:2m]
// (row stride 2m).  lam_i = S_ii / G_ii; scan[0] = lam_max, scan[1] = length of the leading
// run with lam > kTau lam_max, scan[2] = max lam over the rest; IE = I + E (file comment).
// lam0 <= 0: this is level 0 and lam_max is lam_0.
__global__ void __launch_bounds__(1024) mix_refine_kernel(int m, int n,
                                                          const double2* __restrict__ SG,
                                                          double lam0, double* lam, double* scan,
                                                          double2* IE) {
  __shared__ double red[32];
  __shared__ double s_lmax;
  __shared__ int s_nl;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const long ld = 2L * m;
  double mx = -1e300;
  for (int i = tid; i < m; i += blockDim.x) {
    double g = SG[(long)i * ld + m + i].x;
    double l = g > 0 ? SG[(long)i * ld + i].x / g : 0.0;
    lam[i] = l;
    mx = fmax(mx, l);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    double v = -1e300;
    for (int k = 0; k < nw; ++k) v = fmax(v, red[k]);
    int nl = 0;
    while (nl < m && lam[nl] > kTau * v) ++nl;
    double rest = 0.0;
    for (int i = nl; i < m; ++i) rest = fmax(rest, lam[i]);
    scan[0] = v;
    scan[1] = (double)nl;
    scan[2] = rest;
    s_lmax = v;
    s_nl = nl;
  }
  __syncthreads();
  const double lmax = s_lmax;
  const int nl = s_nl;
  const double l0 = lam0 > 0 ? lam0 : lmax;
  // separated: above the FP32 resolution of this level and above the FP64 rounding of the
  // products with A (~n eps_64 lam_0), below which eigenvectors are not defined
  const double sep = fmax(kGapPerDim * (m > 10 ? m : 10) * lmax, 100.0 * n * 1.1e-16 * l0);
  for (long e = tid; e < (long)m * m; e += blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    double2 g = SG[(long)i * ld + m + j];
    double2 r;
    if (i == j) {
      r = make_double2(1.0 + 0.5 * (1.0 - g.x), 0.0);
    } else {
      double d = lam[j] - lam[i];
      bool resolved = (i < nl) || (j < nl);
      if (resolved && fabs(d) > sep) {
        double2 sv = SG[(long)i * ld + j];
        r = make_double2((sv.x - lam[j] * g.x) / d, (sv.y - lam[j] * g.y) / d);
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
  return 8 * sq * sizeof(double2) + 2 * sq * sizeof(float2) + 4 * (size_t)n_cap * 8 +
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
  w.tz = reinterpret_cast<double2*>(take(2 * sq * 16));
  w.tz2 = reinterpret_cast<double2*>(take(2 * sq * 16));
  w.s = reinterpret_cast<double2*>(take(2 * sq * 16));
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
  // Z lives in the right half of tz ([T | Z], row stride 2m) so that S and G come from one
  // product Z^+ [T | Z]
  for (;; ++level) {
    const long l2 = 2L * m;
    double2* T = wk.tz;
    double2* Z = wk.tz + m;
    // B = X^+ A X (level 0: B = A), rounded to FP32 for the sweeps
    const double2* B = a;
    long ldbm = lda;
    if (level > 0) {
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.x, m, T, l2));
      MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.x, m, T, l2, wk.s, m));
      gf(n, m, n);
      gf(m, m, n);
      B = wk.s;
      ldbm = m;
    }
    MPDO_CUDA_TRY((convert<double, float>(st, m, m, B, ldbm, wk.a32, m)));
    MPDO_CUDA_TRY(heig<float>(st, m, wk.a32, m, wk.y32, m, wk.w32, wk.ew, 20));
    // Z = X Y
    if (level == 0) {
      MPDO_CUDA_TRY((convert<float, double>(st, n, m, wk.y32, m, Z, l2)));
    } else {
      MPDO_CUDA_TRY((convert<float, double>(st, m, m, wk.y32, m, wk.ie, m)));
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, wk.x, m, wk.ie, m, Z, l2));
      gf(n, m, m);
    }
    for (int pass = 0; pass < kPasses; ++pass) {
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, Z, l2, T, l2));     // T = A Z
      MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, 2 * m, n, Z, l2, T, l2, wk.s, l2));  // [S | G]
      count_launch();
      mix_refine_kernel<<<1, 1024, 0, st>>>(m, n, wk.s, level == 0 ? 0.0 : lam0, wk.lam,
                                            wk.scan, wk.ie);
      MPDO_CUDA_TRY(cudaGetLastError());
      double2* Z2 = wk.tz2 + m;
      MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, Z, l2, wk.ie, m, Z2, l2));
      gf(n, m, n);
      gf(m, 2 * m, n);
      gf(n, m, m);
      std::swap(wk.tz, wk.tz2);
      T = wk.tz;
      Z = wk.tz + m;
    }
    // the last pass's Rayleigh quotients (second-order accurate for the refined vectors)
    // and the split of this level
    MPDO_CUDA_TRY(cudaMemcpyAsync(hscan, wk.scan, sizeof(hscan), cudaMemcpyDeviceToHost, st));
    MPDO_CUDA_TRY(cudaMemcpyAsync(hcnt, wk.ew.counters, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    MPDO_CUDA_TRY(cudaStreamSynchronize(st));
    flops += hcnt[3] * eig_flops_per_count(m, false);
    if (level == 0) lam0 = hscan[0];
    int nl = (int)hscan[1];
    const bool last = (nl >= m) || level + 1 >= kMaxLevels || !(hscan[2] > floor * lam0) ||
                      nl == 0;
    const int take = last ? m : nl;
    // final columns and values of this level
    MPDO_CUDA_TRY(cudaMemcpy2DAsync(v + off, ldv * sizeof(double2), Z, l2 * sizeof(double2),
                                    take * sizeof(double2), n, cudaMemcpyDeviceToDevice, st));
    MPDO_CUDA_TRY(cudaMemcpyAsync(w + off, wk.lam, take * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
    off += take;
    if (last) break;
    // the unresolved columns become the next basis
    const int mr = m - nl;
    MPDO_CUDA_TRY(cudaMemcpy2DAsync(wk.x, mr * sizeof(double2), Z + nl, l2 * sizeof(double2),
                                    mr * sizeof(double2), n, cudaMemcpyDeviceToDevice, st));
    m = mr;
  }
  if (levels_out) *levels_out = level + 1;
  if (flops_out) *flops_out = flops;
  return cudaSuccess;
}

}  // namespace mpdo
