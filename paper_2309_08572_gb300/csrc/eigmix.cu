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

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace cg = cooperative_groups;

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

// Level scalars in wk.scan: [0] lam_max of the pass, [1] nl = length of the leading run
// with lam > kTau lam_max, [2] largest lam after that run, [3] lam_max of level 0's last
// pass, [4] lam_max of level 0's first pass (lam_0 of the separation floor), [5] Jacobi
// rotations of the level, [6] 1 when this level is the last, [7] columns it emits.
constexpr int kScan = 8;

// One refinement step's scalars and correction, run by one CTA.  S = SG[:, 0:m],
// G = SG[:, m:2m] (row stride 2m), written by other CTAs of the same launch (read through
// L2).  lam_i = S_ii / G_ii; IE = I + E (file comment).  The final pass also decides
// whether the level is the last one.
__device__ void refine_step(int m, int n, const double2* SG, int level0, int final_pass,
                            int level, double floor, const int* rot, double* lam, double* scan,
                            double2* IE) {
  __shared__ double red[32];
  __shared__ double s_lmax;
  __shared__ int s_nl;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const long ld = 2L * m;
  double mx = -1e300;
  for (int i = tid; i < m; i += blockDim.x) {
    double g = __ldcg(&SG[(long)i * ld + m + i].x);
    double l = g > 0 ? __ldcg(&SG[(long)i * ld + i].x) / g : 0.0;
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
    if (final_pass) {
      if (level == 0) scan[3] = v;
      const double top = scan[3];
      const bool last = (nl >= m) || (level + 1 >= kMaxLevels) || !(rest > floor * top) ||
                        nl == 0;
      scan[5] = rot ? (double)rot[3] : 0.0;
      scan[6] = last ? 1.0 : 0.0;
      scan[7] = last ? (double)m : (double)nl;
    }
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
    double2 g = __ldcg(&SG[(long)i * ld + m + j]);
    double2 r;
    if (i == j) {
      r = make_double2(1.0 + 0.5 * (1.0 - g.x), 0.0);
    } else {
      double d = lam[j] - lam[i];
      bool resolved = (i < nl) || (j < nl);
      if (resolved && fabs(d) > sep) {
        double2 sv = __ldcg(&SG[(long)i * ld + j]);
        r = make_double2((sv.x - lam[j] * g.x) / d, (sv.y - lam[j] * g.y) / d);
      } else {
        r = make_double2(-0.5 * g.x, -0.5 * g.y);
      }
    }
    IE[e] = r;
  }
}

constexpr int RT = 16;   // output tile of the fused products (one element per thread)

// [S | G] = Z^+ [T | Z] (m x 2m, row stride 2m) from TZ = [T | Z] (n x 2m, row stride 2m),
// then the refinement step, run by the CTA that finishes last (a ticket counter in global
// memory; no CTA waits on another).  The ticket returns to 0 for the next launch.  FP64
// runs at 2 FMA per clock per SM, so each output tile's K loop (over n) is split over the
// CTAs of a thread-block cluster (dims (splits, 1, 1)); the partial sums meet in rank 0
// through distributed shared memory, added in rank order.
__global__ void __launch_bounds__(RT * RT) sg_refine_kernel(
    int m, int n, const double2* __restrict__ TZ, double2* SG, int level0, int final_pass,
    int level, double floor, const int* rot, double* lam, double* scan, double2* IE,
    unsigned int* ticket, int splits) {
  __shared__ double2 As[RT][RT + 1];   // [k][i]
  __shared__ double2 Bs[RT][RT + 1];   // [k][j]
  __shared__ double2 part[RT * RT];
  __shared__ int s_last;
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank();
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
  const int i0 = blockIdx.y * RT, j0 = (blockIdx.x / splits) * RT;
  const long ld = 2L * m;
  const int kc = ((n + splits * RT - 1) / (splits * RT)) * RT;
  const int kb = s * kc, ke = min(n, kb + kc);
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = kb; k0 < ke; k0 += RT) {
    const int k = k0 + ty;
    double2 za = make_double2(0.0, 0.0), tb = make_double2(0.0, 0.0);
    if (k < ke && i0 + tx < m) za = cconj(TZ[(long)k * ld + m + i0 + tx]);
    if (k < ke && j0 + tx < 2 * m) tb = TZ[(long)k * ld + j0 + tx];
    As[ty][tx] = za;
    Bs[ty][tx] = tb;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RT; ++kk) cfma(acc, As[kk][ty], Bs[kk][tx]);
    __syncthreads();
  }
  part[threadIdx.x] = acc;
  cluster.sync();
  if (s == 0) {
    double2 sum = part[threadIdx.x];
    for (int q = 1; q < splits; ++q) sum = cadd(sum, cluster.map_shared_rank(part, q)[threadIdx.x]);
    if (i0 + ty < m && j0 + tx < 2 * m) SG[(long)(i0 + ty) * ld + j0 + tx] = sum;
  }
  cluster.sync();   // rank 0 has read every partial before the cluster leaves
  if (s != 0) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int total = (gridDim.x / splits) * gridDim.y;
    s_last = (atomicAdd(ticket, 1u) == total - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  refine_step(m, n, SG, level0, final_pass, level, floor, rot, lam, scan, IE);
  if (threadIdx.x == 0) *ticket = 0u;
}

// K slices of a small FP64 product: enough to bring the CTAs towards one per SM, each
// slice at least 16 long (one tile step), at most 8 (portable cluster size).
inline int split_count(long tiles, int K) {
  int s = 1;
  while (s < 8 && tiles * (2 * s) <= 152 && K >= 16 * (2 * s)) s *= 2;
  return s;
}

// The level's last product Z' = Z (I + E) (Z: n x m, row stride ldz), routed by the level's
// scalars: columns j < take go to v[:, off + j] (with w[off + j] = lam_j); when the level is
// not the last, columns j >= nl go to the next basis x[:, j - nl] (row stride m - nl).
__global__ void __launch_bounds__(RT * RT) level_out_kernel(
    int n, int m, const double2* __restrict__ Z, long ldz, const double2* __restrict__ IE,
    const double* scan, const double* lam, double2* v, long ldv, double* w, int off,
    double2* x, double* hscan) {
  __shared__ double2 As[RT][RT + 1];   // [k][row]
  __shared__ double2 Bs[RT][RT + 1];   // [k][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
  const int r0 = blockIdx.y * RT, j0 = blockIdx.x * RT;
  const bool last = scan[6] != 0.0;
  const int nl = (int)scan[1];
  const int take = last ? m : nl;
  const int mr = m - nl;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < m; k0 += RT) {
    double2 za = make_double2(0.0, 0.0), eb = make_double2(0.0, 0.0);
    if (r0 + ty < n && k0 + tx < m) za = Z[(long)(r0 + ty) * ldz + k0 + tx];
    if (k0 + ty < m && j0 + tx < m) eb = IE[(long)(k0 + ty) * m + j0 + tx];
    As[tx][ty] = za;
    Bs[ty][tx] = eb;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RT; ++kk) cfma(acc, As[kk][ty], Bs[kk][tx]);
    __syncthreads();
  }
  const int r = r0 + ty, j = j0 + tx;
  if (r < n && j < m) {
    if (j < take)
      v[(long)r * ldv + off + j] = acc;
    else if (!last && j >= nl)
      x[(long)r * mr + (j - nl)] = acc;
  }
  if (blockIdx.y == 0 && ty == 0 && j < take) w[off + j] = lam[j];
  // the level's scalars, straight into the mapped host area (no copy launch)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kScan) {
    hscan[threadIdx.x] = scan[threadIdx.x];
    __threadfence_system();
  }
}

cudaError_t gemm64(cudaStream_t st, int opa, int opb, int m, int n, int k, const double2* A,
                   long lda, const double2* B, long ldb, double2* C, long ldc) {
  return cgemm<double>(st, opa, opb, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1,
                       make_double2(1, 0), make_double2(0, 0));
}

}  // namespace

// One captured graph per level shape: (input matrix, n, m, level, outputs, floor).  The
// launches of a level run as one graph launch instead of ~8; its scalars reach the host
// through mapped pinned memory, written by the level's last kernel.
struct MixKey {
  const void* a;
  long lda;
  int n, m, level;
  const void* v;
  long ldv;
  const void* w;
  double floor;
  bool operator==(const MixKey& o) const {
    return a == o.a && lda == o.lda && n == o.n && m == o.m && level == o.level && v == o.v &&
           ldv == o.ldv && w == o.w && floor == o.floor;
  }
};
struct MixKeyHash {
  size_t operator()(const MixKey& k) const {
    auto mix = [](size_t h, size_t x) {
      return h ^ (x + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2));
    };
    size_t h = std::hash<const void*>()(k.a);
    h = mix(h, std::hash<long>()(k.lda));
    h = mix(h, std::hash<long>()(((long)k.n << 32) ^ ((long)k.m << 8) ^ k.level));
    h = mix(h, std::hash<const void*>()(k.v));
    h = mix(h, std::hash<long>()(k.ldv));
    h = mix(h, std::hash<const void*>()(k.w));
    h = mix(h, std::hash<double>()(k.floor));
    return h;
  }
};
struct MixGraphs {
  std::unordered_map<MixKey, std::pair<cudaGraphExec_t, int>, MixKeyHash> map;
};

void mix_work_release(MixWork& w) {
  if (w.hpin) cudaFreeHost(w.hpin);
  w.hpin = nullptr;
  w.hpin_dev = nullptr;
  if (!w.graphs) return;
  for (auto& kv : w.graphs->map) cudaGraphExecDestroy(kv.second.first);
  delete w.graphs;
  w.graphs = nullptr;
}

size_t mix_work_bytes(int n_cap) {
  size_t sq = (size_t)n_cap * n_cap;
  return 8 * sq * sizeof(double2) + 2 * sq * sizeof(float2) + 4 * (size_t)n_cap * 8 +
         eig_work_bytes<float>(n_cap) + 10 * 256;
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
  w.scan = reinterpret_cast<double*>(take(kScan * sizeof(double)));
  w.ticket = reinterpret_cast<unsigned int*>(take(64));
  eig_work_bind<float>(w.ew, take(eig_work_bytes<float>(n_cap)), n_cap);
}

namespace {
constexpr int kPasses = 2;

// Floating-point work of one level's products (8 real flops per complex multiply-add).
double level_flops(int n, int m, bool lev0) {
  auto g = [](int a, int b, int c) { return 8.0 * a * b * (double)c; };
  double f = 0.0;
  if (!lev0) f += g(n, m, n) + g(m, m, n) + g(n, m, m);   // X^+ A X and Z = X Y
  f += g(n, m, n);                                          // T = A Z
  for (int pass = 0; pass < kPasses; ++pass) {
    f += g(m, 2 * m, n);                                    // [S | G]
    f += (pass + 1 < kPasses) ? 2 * g(n, m, m) : g(n, m, m); // [T | Z] (I + E) or Z (I + E)
  }
  return f;
}

// The launches of one level; its last kernel also writes the level's scalars to the mapped
// host area (no host synchronisation inside, so a level can be captured as one graph).  Level 0 reads
// B = A; later levels project on the basis in wk.x, which the level's last product replaces
// with the unresolved columns.  The refinement carries T along: after a pass,
// [T | Z] <- [T | Z] (I + E) = [A Z' | Z'], so A enters only the first product.
cudaError_t enqueue_level(cudaStream_t st, int n, int m, int level, const double2* a, long lda,
                          double2* v, long ldv, double* w, double floor, MixWork& wk) {
  const bool lev0 = (level == 0);
  const long l2 = 2L * m;
  double2* T = wk.tz;
  double2* Z = wk.tz + m;
  const double2* B = a;
  long ldbm = lda;
  if (!lev0) {
    MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, wk.x, m, T, l2));
    MPDO_CUDA_TRY(gemm64(st, OP_C, OP_N, m, m, n, wk.x, m, T, l2, wk.s, m));
    B = wk.s;
    ldbm = m;
  }
  if (m <= kSmemJacobiMaxF32) {
    // the FP32 sweeps read the FP64 matrix and write the vectors in the precision needed
    if (lev0) {
      MPDO_CUDA_TRY((heig_smem_f32<double, double>(st, m, B, ldbm, Z, l2, wk.w32,
                                                   wk.ew.counters, 20)));
    } else {
      MPDO_CUDA_TRY((heig_smem_f32<double, float>(st, m, B, ldbm, wk.y32, m, wk.w32,
                                                  wk.ew.counters, 20)));
      MPDO_CUDA_TRY(cgemm_dx(st, OP_N, OP_N, n, m, m, wk.x, m, 0, wk.y32, m, 0, Z, l2, 0, 1));
    }
  } else {
    MPDO_CUDA_TRY((convert<double, float>(st, m, m, B, ldbm, wk.a32, m)));
    MPDO_CUDA_TRY(heig<float>(st, m, wk.a32, m, wk.y32, m, wk.w32, wk.ew, 20));
    if (lev0)
      MPDO_CUDA_TRY((convert<float, double>(st, n, m, wk.y32, m, Z, l2)));
    else
      MPDO_CUDA_TRY(cgemm_dx(st, OP_N, OP_N, n, m, m, wk.x, m, 0, wk.y32, m, 0, Z, l2, 0, 1));
  }
  MPDO_CUDA_TRY(gemm64(st, OP_N, OP_N, n, m, n, a, lda, Z, l2, T, l2));
  double2* cur = wk.tz;
  double2* nxt = wk.tz2;
  const dim3 gsg((2 * m + RT - 1) / RT, (m + RT - 1) / RT);
  const int splits = split_count((long)gsg.x * gsg.y, n);
  for (int pass = 0; pass < kPasses; ++pass) {
    const int final_pass = (pass + 1 == kPasses);
    count_launch();
    {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(gsg.x * splits, gsg.y);
      cfg.blockDim = dim3(RT * RT);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = splits;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      MPDO_CUDA_TRY(cudaLaunchKernelEx(&cfg, sg_refine_kernel, m, n, (const double2*)cur, wk.s,
                                       (lev0 && pass == 0) ? 1 : 0, final_pass, level, floor,
                                       (const int*)wk.ew.counters, wk.lam, wk.scan, wk.ie,
                                       wk.ticket, splits));
    }
    if (!final_pass) {
      // [T | Z] (I + E): two products sharing the right factor (batch of 2, offset m)
      MPDO_CUDA_TRY(cgemm<double>(st, OP_N, OP_N, n, m, m, cur, l2, m, wk.ie, m, 0, nxt, l2, m,
                                  2, make_double2(1, 0), make_double2(0, 0)));
      std::swap(cur, nxt);
    } else {
      count_launch();
      const dim3 gout((m + RT - 1) / RT, (n + RT - 1) / RT);
      level_out_kernel<<<gout, RT * RT, 0, st>>>(n, m, cur + m, l2, wk.ie, wk.scan, wk.lam, v,
                                                 ldv, w, n - m, wk.x, wk.hpin_dev);
      MPDO_CUDA_TRY(cudaGetLastError());
    }
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t heig_mixed(cudaStream_t st, int n, const double2* a, long lda, double2* v, long ldv,
                       double* w, double floor, MixWork& wk, int* levels_out,
                       double* flops_out, int max_vals) {
  double flops = 0.0;
  if (n <= 0) return cudaSuccess;
  if (n > wk.n_cap) return cudaErrorInvalidValue;
  if (!wk.hpin) {
    MPDO_CUDA_TRY(cudaHostAlloc((void**)&wk.hpin, kScan * sizeof(double), cudaHostAllocMapped));
    MPDO_CUDA_TRY(cudaHostGetDevicePointer((void**)&wk.hpin_dev, wk.hpin, 0));
  }
  const double* hscan = wk.hpin;
  int m = n, level = 0;
  for (;; ++level) {
    // graphs only for one-CTA sweeps (m <= 118) on a capturable stream
    bool launched = false;
    if (wk.use_graphs && m <= kSmemJacobiMaxF32 && st != 0 && st != cudaStreamLegacy &&
        st != cudaStreamPerThread) {
      if (!wk.graphs) wk.graphs = new MixGraphs();
      MixKey key{a, lda, n, m, level, v, ldv, w, floor};
      auto it = wk.graphs->map.find(key);
      if (it == wk.graphs->map.end()) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t e2 = enqueue_level(st, n, m, level, a, lda, v, ldv, w, floor, wk);
          e = cudaStreamEndCapture(st, &g);
          if (e2 != cudaSuccess) e = e2;
          // kernel nodes of the graph (the capture counted them without launching them)
          size_t nodes = 0;
          if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nodes);
          std::vector<cudaGraphNode_t> list(nodes);
          if (e == cudaSuccess && nodes) e = cudaGraphGetNodes(g, list.data(), &nodes);
          int kernels = 0;
          for (size_t q = 0; e == cudaSuccess && q < nodes; ++q) {
            cudaGraphNodeType ty;
            e = cudaGraphNodeGetType(list[q], &ty);
            if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
          }
          count_launch(-(long long)kernels);
          cudaGraphExec_t ex = nullptr;
          if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
          if (g) cudaGraphDestroy(g);
          if (e == cudaSuccess) it = wk.graphs->map.emplace(key, std::make_pair(ex, kernels)).first;
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
    if (!launched) MPDO_CUDA_TRY(enqueue_level(st, n, m, level, a, lda, v, ldv, w, floor, wk));
    if (wk.block_ev) {
      MPDO_CUDA_TRY(cudaEventRecord(wk.block_ev, st));
      MPDO_CUDA_TRY(cudaEventSynchronize(wk.block_ev));
    } else {
      MPDO_CUDA_TRY(cudaStreamSynchronize(st));
    }
    flops += level_flops(n, m, level == 0) + hscan[5] * eig_flops_per_count(m, false);
    const int nl = (int)hscan[1];
    // the device decided (scan[6]); the bounds below only guard the host loop
    if (hscan[6] != 0.0 || nl <= 0 || nl >= m || level + 1 >= kMaxLevels) break;
    // enough leading pairs resolved for the caller: the rest is reported as zero
    const int resolved = n - m + nl;
    if (max_vals > 0 && resolved >= max_vals) {
      MPDO_CUDA_TRY(cudaMemset2DAsync(v + resolved, ldv * sizeof(double2), 0,
                                      (size_t)(n - resolved) * sizeof(double2), n, st));
      MPDO_CUDA_TRY(cudaMemsetAsync(w + resolved, 0, (size_t)(n - resolved) * sizeof(double), st));
      break;
    }
    m -= nl;
  }
  if (levels_out) *levels_out = level + 1;
  if (flops_out) *flops_out = flops;
  return cudaSuccess;
}

}  // namespace mpdo
