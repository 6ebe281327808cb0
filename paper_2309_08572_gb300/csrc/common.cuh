// Shared device helpers for the MPDO kernels: complex arithmetic on float2/double2,
// launch checks.  Internal header (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

template <typename R> struct CxOf;
template <> struct CxOf<double> { using T = double2; };
template <> struct CxOf<float> { using T = float2; };
template <typename R> using cx = typename CxOf<R>::T;

template <typename R> __host__ __device__ __forceinline__ cx<R> mkc(R re, R im) {
  cx<R> z; z.x = re; z.y = im; return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x; a.y += b.y; return a;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x; a.y -= b.y; return a;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C z; z.x = a.x * b.x + a.y * b.y; z.y = a.y * b.x - a.x * b.y; return z;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cconjmul(C a, C b) {
  C z; z.x = a.x * b.x + a.y * b.y; z.y = a.x * b.y - a.y * b.x; return z;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
  a.x *= s; a.y *= s; return a;
}
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __host__ __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) {
  return a.x * a.x + a.y * a.y;
}

// Round-robin pairing (circle method) of `players` (even) indices: pair k of round `round`,
// rounds 0 .. players - 2 meet every pair once; player players - 1 stays fixed.
__device__ __forceinline__ void tourney(int round, int k, int players, int& a, int& b) {
  const int m = players - 1;
  if (k == 0) {
    a = m;
    b = round % m;
  } else {
    a = (round + k) % m;
    b = (round - k + m) % m;
  }
}

// Scalars produced by one update step on the device and read by the host driver.
struct StepScalars {
  int keep;        // bond values kept
  int kkeep;       // inner values kept
  int rank_g;      // rank of the left Gram
  int flags;       // bit 0: numeric problem (NaN / zero state)
  double tot;      // sum of all bond eigenvalues (= tr rho before the cut)
  double kept;     // sum of the kept ones
  double renorm;   // sqrt(tot / kept)
  double ktot;     // inner: sum of all w
  double theta;    // PPT angle
  int infeasible;
  int clamped;
  double trpre;    // ||theta||^2 of the two-site block before the channel (FP64)
};

// Device-side accumulation of the per-call truncation statistics.
struct DevStats {
  double disc_bond_w;
  double disc_kraus_w;
  double ppt_theta_min;
  int ppt_infeasible;
  int ppt_clamped;
  int chi_used_max;
  int k_used_max;
  int n_updates;
  int numeric_error;
};

// Count of kernels launched by this library (all handles), for throughput reports.
#include <atomic>
namespace mpdo {
extern std::atomic<long long> g_launches;
inline void count_launch(long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace mpdo

#define MPDO_CUDA_TRY(expr)                                 \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return _e;                       \
  } while (0)
