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
#include <unordered_map>
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
constexpr int kMaxLevels = 8;

// One refinement step's scalars and correction, one CTA.  S = SG[:, 0:m], G = SG[:, m:2m]
// (row stride 2m).  lam_i = S_ii / G_ii; scan[0] = lam_max, scan[1] = length of the leading
// run with lam > kTau lam_max, scan[2] = max lam over the rest; IE = I + E (file comment).
// lam0 <= 0: this is level 0 and lam_max is lam_0.
__global__ void __launch_bounds__(1024) mix_refine_kernel(int m, int n,
                                                          const double2* __restrict__ SG,
                                                          int level0, double* lam, double* scan,
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
    if (level0) scan[4] = v;   // lam_0, kept for the later levels
    s_lmax = v;
    s_nl = nl;
  }
  __syncthreads();
  const double lmax = s_lmax;
  const int nl = s_nl;
  const double l0 = level0 ? lmax : scan[4];
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

// One captured graph per (input matrix, n, m, level 0 or not): the launches of a level up
// to its host read-back run as one graph launch instead of ~12 kernel launches.
struct MixKey {
  const void* a;
  long lda;
  int n, m, lev0;
  bool operator==(const MixKey& o) const {
    return a == o.a && lda == o.lda && n == o.n && m == o.m && lev0 == o.lev0;
  }
};
struct MixKeyHash {
  size_t operator()(const MixKey& k) const {
    size_t h = std::hash<const void*>()(k.a);
    h ^= std::hash<long>()(k.lda) + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    h ^= std::hash<long>()(((long)k.n << 32) ^ ((long)k.m << 1) ^ k.lev0) + (h << 6) + (h >> 2);
    return h;
  }
};
struct MixGraphs {
  std::unordered_map<MixKey, std::pair<cudaGraphExec_t, int>, MixKeyHash> map;
};

void mix_work_release(MixWork& w) {
  if (w.hpin) cudaFreeHost(w.hpin);
  w.hpin = nullptr;
  if (!w.graphs) return;
  for (auto& kv : w.graphs->map) cudaGraphExecDestroy(kv.second.first);
  delete w.graphs;
  w.graphs = nullptr;
}

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

namespace {
constexpr int kPasses = 2;
inline double2* mix_result(MixWork& wk, int m) { return ((kPasses & 1) ? wk.tz2 : wk.tz) + m; }

// The launches of one level up to the read-back (no host synchronisation inside).
// Level 0 reads B = A; later levels project on the basis in wk.x.  Refined vectors end in
// the right half of tz2 ([T | Z] layout, row stride 2m).
cudaError_t enqueue_level(cudaStream_t st, int n, int m, bool lev0, const double2* a, long lda,
                          MixWork& wk, double& flops) {
  auto gf = [&](int mm, int nn, int kk) { flops += 8.0 * mm * nn * (double)kk; };
  const long l2 = 2L * m;
  double2* T = wk.tz;
  double2* Z = wk.tz + m;
  const double2* B = a;
  long ldbm = lda;
  if (!lev0) {
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.x, m, T, l2));
    MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.x, m, T, l2, wk.s, m));
    gf(n, m, n);
    gf(m, m, n);
    B = wk.s;
    ldbm = m;
  }
  MPDO_CUDA_TRY((convert<double, float>(st, m, m, B, ldbm, wk.a32, m)));
  MPDO_CUDA_TRY(heig<float>(st, m, wk.a32, m, wk.y32, m, wk.w32, wk.ew, 20));
  if (lev0) {
    MPDO_CUDA_TRY((convert<float, double>(st, n, m, wk.y32, m, Z, l2)));
  } else {
    MPDO_CUDA_TRY((convert<float, double>(st, m, m, wk.y32, m, wk.ie, m)));
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, wk.x, m, wk.ie, m, Z, l2));
    gf(n, m, m);
  }
  // refinement passes: T = A Z, [S | G] = Z^+ [T | Z], I + E, Z' = Z (I + E); the buffers
  // alternate between tz and tz2, so the result lies in mix_result(wk, m)
  double2* cur = wk.tz;
  double2* nxt = wk.tz2;
  for (int pass = 0; pass < kPasses; ++pass) {
    double2* Tc = cur;
    double2* Zc = cur + m;
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, Zc, l2, Tc, l2));
    MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, 2 * m, n, Zc, l2, Tc, l2, wk.s, l2));
    count_launch();
    mix_refine_kernel<<<1, 1024, 0, st>>>(m, n, wk.s, (lev0 && pass == 0) ? 1 : 0, wk.lam,
                                          wk.scan, wk.ie);
    MPDO_CUDA_TRY(cudaGetLastError());
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, m, Zc, l2, wk.ie, m, nxt + m, l2));
    gf(n, m, n);
    gf(m, 2 * m, n);
    gf(n, m, m);
    std::swap(cur, nxt);
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t heig_mixed(cudaStream_t st, int n, const double2* a, long lda, double2* v, long ldv,
                       double* w, double floor, MixWork& wk, int* levels_out,
                       double* flops_out) {
  double flops = 0.0;
  if (n <= 0) return cudaSuccess;
  if (n > wk.n_cap) return cudaErrorInvalidValue;
  if (!wk.hpin) MPDO_CUDA_TRY(cudaMallocHost((void**)&wk.hpin, 8 * sizeof(double)));
  double* hscan = wk.hpin;                          // [0..2]
  int* hcnt = reinterpret_cast<int*>(wk.hpin + 4);  // [0..3]
  int m = n, off = 0, level = 0;
  double lam0 = 0.0;
  for (;; ++level) {
    const long l2 = 2L * m;
    const bool lev0 = (level == 0);
    // graphs only for one-CTA sweeps (m <= 118) on a capturable stream
    bool launched = false;
    double lflops = 0.0;
    if (wk.use_graphs && m <= 118 && st != 0 && st != cudaStreamLegacy &&
        st != cudaStreamPerThread) {
      if (!wk.graphs) wk.graphs = new MixGraphs();
      MixKey key{a, lda, n, m, lev0 ? 1 : 0};
      auto it = wk.graphs->map.find(key);
      if (it == wk.graphs->map.end()) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t e2 = enqueue_level(st, n, m, lev0, a, lda, wk, lflops);
          e = cudaStreamEndCapture(st, &g);
          if (e2 != cudaSuccess) e = e2;
          size_t nodes = 0;
          if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nodes);
          // the capture counted its kernels without launching them
          count_launch(-(long long)nodes);
          cudaGraphExec_t ex = nullptr;
          if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
          if (g) cudaGraphDestroy(g);
          if (e == cudaSuccess) it = wk.graphs->map.emplace(key, std::make_pair(ex, (int)nodes)).first;
        }
        if (e != cudaSuccess) {
          cudaGetLastError();
          wk.use_graphs = false;   // not capturable here: launch directly from now on
        }
      }
      if (wk.use_graphs && it != wk.graphs->map.end()) {
        MPDO_CUDA_TRY(cudaGraphLaunch(it->second.first, st));
        count_launch(it->second.second);
        launched = true;
      }
    }
    if (!launched) MPDO_CUDA_TRY(enqueue_level(st, n, m, lev0, a, lda, wk, lflops));
    // flops of the level's products (same count whether captured or not)
    {
      auto gfl = [&](int mm, int nn, int kk) { flops += 8.0 * mm * nn * (double)kk; };
      if (!lev0) { gfl(n, m, n); gfl(m, m, n); gfl(n, m, m); }
      for (int pass = 0; pass < kPasses; ++pass) {
        gfl(n, m, n);
        gfl(m, 2 * m, n);
        gfl(n, m, m);
      }
    }
    double2* Z = mix_result(wk, m);   // refined vectors
    MPDO_CUDA_TRY(cudaMemcpyAsync(hscan, wk.scan, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPDO_CUDA_TRY(cudaMemcpyAsync(hcnt, wk.ew.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (wk.block_ev) {
      MPDO_CUDA_TRY(cudaEventRecord(wk.block_ev, st));
      MPDO_CUDA_TRY(cudaEventSynchronize(wk.block_ev));
    } else {
      MPDO_CUDA_TRY(cudaStreamSynchronize(st));
    }
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
