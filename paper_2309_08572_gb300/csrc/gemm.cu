// Complex batched GEMM on CUDA cores (FP64 and FP32 arithmetic), generic strides.
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b]; op in {N, T, C (conj-transpose),
// R (conj, no transpose)}.  Used by every contraction of the update for the FP64 and
// C64 modes and for the unit tests of the other GEMM paths.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/mpdo.h"
#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace mpdo {

namespace {
constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

// Inputs of precisions RA and RB, products and sums in R (float inputs, R = double: the
// FP32 products are exact in FP64 and the sums carry FP64 rounding only).
template <typename RA, typename RB, typename R>
__global__ void __launch_bounds__(NT) cgemm_kernel(
    int M, int N, int K, const cx<RA>* __restrict__ A, long sam, long sak, long sab, int conja,
    const cx<RB>* __restrict__ B, long sbk, long sbn, long sbb, int conjb, cx<R>* C, long scm,
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
        cx<RA> t = A[gm * sam + gk * sak];
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
        cx<RB> t = B[gk * sbk + gn * sbn];
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
// 16 x 16 output tiles, one element per thread: for small products, where 64 x 64 tiles
// would occupy only a few SMs (FP64 runs at 2 FMA per clock per SM, so spreading matters).
constexpr int ST = 16;
template <typename RA, typename RB, typename R>
__global__ void __launch_bounds__(ST * ST) cgemm_small_kernel(
    int M, int N, int K, const cx<RA>* __restrict__ A, long sam, long sak, long sab, int conja,
    const cx<RB>* __restrict__ B, long sbk, long sbn, long sbb, int conjb, cx<R>* C, long scm,
    long scn, long scb, cx<R> alpha, cx<R> beta, int use_beta) {
  using T = cx<R>;
  __shared__ T As[ST][ST + 1];   // [k][m]
  __shared__ T Bs[ST][ST + 1];   // [k][n]
  const int tx = threadIdx.x % ST, ty = threadIdx.x / ST;
  const int m0 = blockIdx.y * ST, n0 = blockIdx.x * ST;
  const long bz = blockIdx.z;
  A += bz * sab;
  B += bz * sbb;
  C += bz * scb;
  T acc = mkc<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += ST) {
    {
      // A tile: thread (ty, tx) loads m = m0 + ty, k = k0 + tx
      int gm = m0 + ty, gk = k0 + tx;
      T v = mkc<R>(0, 0);
      if (gm < M && gk < K) {
        cx<RA> t = A[gm * sam + gk * sak];
        v = mkc<R>((R)t.x, conja ? -(R)t.y : (R)t.y);
      }
      As[tx][ty] = v;
      // B tile: k = k0 + ty, n = n0 + tx
      int gk2 = k0 + ty, gn = n0 + tx;
      T u = mkc<R>(0, 0);
      if (gn < N && gk2 < K) {
        cx<RB> t = B[gk2 * sbk + gn * sbn];
        u = mkc<R>((R)t.x, conjb ? -(R)t.y : (R)t.y);
      }
      Bs[ty][tx] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ST; ++kk) cfma(acc, As[kk][ty], Bs[kk][tx]);
    __syncthreads();
  }
  const int gm = m0 + ty, gn = n0 + tx;
  if (gm < M && gn < N) {
    T v = cmul(alpha, acc);
    T* p = C + gm * scm + gn * scn;
    if (use_beta) v = cadd(v, cmul(beta, *p));
    *p = v;
  }
}

// Split-K form of the 16 x 16 tile kernel for FP64 products with few output tiles and a
// long K: FP64 runs at 2 FMA per clock per SM, so one tile's K loop is spread over the
// CTAs of a thread-block cluster (cluster dims (splits, 1, 1): CTA rank s takes the s-th
// K slice).  The partial sums meet in rank 0's registers through distributed shared
// memory, added in rank order, so the result does not depend on scheduling.
template <typename RA, typename RB, typename R>
__global__ void __launch_bounds__(ST * ST) cgemm_small_split_kernel(
    int M, int N, int K, const cx<RA>* __restrict__ A, long sam, long sak, long sab, int conja,
    const cx<RB>* __restrict__ B, long sbk, long sbn, long sbb, int conjb, cx<R>* C, long scm,
    long scn, long scb, cx<R> alpha, cx<R> beta, int use_beta, int splits) {
  using T = cx<R>;
  __shared__ T As[ST][ST + 1];
  __shared__ T Bs[ST][ST + 1];
  __shared__ T part[ST * ST];
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank();
  const int tx = threadIdx.x % ST, ty = threadIdx.x / ST;
  const int m0 = blockIdx.y * ST, n0 = (blockIdx.x / splits) * ST;
  const long bz = blockIdx.z;
  A += bz * sab;
  B += bz * sbb;
  C += bz * scb;
  // K slices: whole multiples of ST, rank order
  const int kc = ((K + splits * ST - 1) / (splits * ST)) * ST;
  const int kb = s * kc, ke = min(K, kb + kc);
  T acc = mkc<R>(0, 0);
  for (int k0 = kb; k0 < ke; k0 += ST) {
    {
      int gm = m0 + ty, gk = k0 + tx;
      T v = mkc<R>(0, 0);
      if (gm < M && gk < ke) {
        cx<RA> t = A[gm * sam + gk * sak];
        v = mkc<R>((R)t.x, conja ? -(R)t.y : (R)t.y);
      }
      As[tx][ty] = v;
      int gk2 = k0 + ty, gn = n0 + tx;
      T u = mkc<R>(0, 0);
      if (gn < N && gk2 < ke) {
        cx<RB> t = B[gk2 * sbk + gn * sbn];
        u = mkc<R>((R)t.x, conjb ? -(R)t.y : (R)t.y);
      }
      Bs[ty][tx] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ST; ++kk) cfma(acc, As[kk][ty], Bs[kk][tx]);
    __syncthreads();
  }
  part[threadIdx.x] = acc;
  cluster.sync();
  if (s == 0) {
    T sum = part[threadIdx.x];
    for (int q = 1; q < splits; ++q) sum = cadd(sum, cluster.map_shared_rank(part, q)[threadIdx.x]);
    const int gm = m0 + ty, gn = n0 + tx;
    if (gm < M && gn < N) {
      T v = cmul(alpha, sum);
      T* p = C + gm * scm + gn * scn;
      if (use_beta) v = cadd(v, cmul(beta, *p));
      *p = v;
    }
  }
  cluster.sync();   // rank 0 has read every partial before the cluster leaves
}

// Number of K slices for a small-tile FP64 product: enough to bring the tiles of the grid
// towards one per SM, each slice at least 16 long (one tile step), at most 8 (portable
// cluster size).
inline int split_count(long tiles, int K) {
  int s = 1;
  while (s < 8 && tiles * (2 * s) <= 152 && K >= 16 * (2 * s)) s *= 2;
  return s;
}

// Tile-shape table of the autotuner (mpdo_autotune_gemm): per precision (0: FP64 products,
// 1: FP32), per bucket of the 16 x 16 output-tile count (log2, 0..10) and of K (log2(K/16),
// 0..8), the kernel choice: 0 = size rules above (untuned), 1 = 64 x 64 tiles, 2 = 16 x 16
// tiles, 3/4/5 = 16 x 16 tiles with K split over a cluster of 2/4/8.
constexpr int kTileBuckets = 11, kKBuckets = 9, kChoices = 5;
std::atomic<signed char> g_choice[2][kTileBuckets][kKBuckets];

inline int log2_ceil(long x) {
  int b = 0;
  while ((1L << b) < x) ++b;
  return b;
}
inline int tile_bucket(long tiles16) { return std::min(kTileBuckets - 1, log2_ceil(std::max(1L, tiles16))); }
inline int k_bucket(int K) { return std::min(kKBuckets - 1, std::max(0, log2_ceil(std::max(1, K)) - 4)); }
}  // namespace

template <typename RA, typename RB, typename R>
cudaError_t cgemm_impl(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<RA>* A,
                       long lda, long sa, const cx<RB>* B, long ldb, long sb, cx<R>* C, long ldc,
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
  const long big_tiles = (long)((n + BN - 1) / BN) * ((m + BM - 1) / BM) * batch;
  const long tiles16 = (long)((n + ST - 1) / ST) * ((m + ST - 1) / ST) * batch;
  const int choice =
      g_choice[sizeof(R) == 8 ? 0 : 1][tile_bucket(tiles16)][k_bucket(k)].load(std::memory_order_relaxed);
  const bool small = choice == 0 ? big_tiles < 152 : choice >= 2;
  for (int b0 = 0; b0 < batch; b0 += 65535) {
    int nb = batch - b0 < 65535 ? batch - b0 : 65535;
    count_launch();
    if (small && (sizeof(R) == 8 || choice >= 3)) {
      const long tiles = (long)((n + ST - 1) / ST) * ((m + ST - 1) / ST) * nb;
      int splits = choice == 0 ? split_count(tiles, k) : (choice >= 3 ? 1 << (choice - 2) : 1);
      while (splits > 1 && k < 16 * splits) splits >>= 1;   // every slice at least one step
      if (splits > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(((n + ST - 1) / ST) * splits, (m + ST - 1) / ST, nb);
        cfg.blockDim = dim3(ST * ST);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = splits;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(
            &cfg, cgemm_small_split_kernel<RA, RB, R>, m, n, k, A + (long)b0 * sa, sam, sak, sa,
            conja, B + (long)b0 * sb, sbk, sbn, sb, conjb, C + (long)b0 * sc, (long)ldc, 1L, sc,
            alpha, beta, use_beta, splits);
        if (e != cudaSuccess) return e;
        continue;
      }
    }
    if (small) {
      dim3 g2((n + ST - 1) / ST, (m + ST - 1) / ST, nb);
      cgemm_small_kernel<RA, RB, R><<<g2, ST * ST, 0, st>>>(
          m, n, k, A + (long)b0 * sa, sam, sak, sa, conja, B + (long)b0 * sb, sbk, sbn, sb, conjb,
          C + (long)b0 * sc, ldc, 1, sc, alpha, beta, use_beta);
      continue;
    }
    dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, nb);
    cgemm_kernel<RA, RB, R><<<grid, NT, 0, st>>>(m, n, k, A + (long)b0 * sa, sam, sak, sa, conja,
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
  return cgemm_impl<R, R, R>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch,
                          alpha, beta);
}

template <typename RB>
cudaError_t cgemm_wide(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<float>* A,
                       long lda, long sa, const cx<RB>* B, long ldb, long sb, cx<double>* C,
                       long ldc, long sc, int batch) {
  return cgemm_impl<float, RB, double>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc,
                                       batch, mkc<double>(1, 0), mkc<double>(0, 0));
}
template cudaError_t cgemm_wide<float>(cudaStream_t, int, int, int, int, int, const float2*,
                                       long, long, const float2*, long, long, double2*, long,
                                       long, int);
template cudaError_t cgemm_wide<double>(cudaStream_t, int, int, int, int, int, const float2*,
                                        long, long, const double2*, long, long, double2*, long,
                                        long, int);

cudaError_t cgemm_dx(cudaStream_t st, int opa, int opb, int m, int n, int k, const cx<double>* A,
                     long lda, long sa, const cx<float>* B, long ldb, long sb, cx<double>* C,
                     long ldc, long sc, int batch) {
  return cgemm_impl<double, float, double>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc,
                                           sc, batch, mkc<double>(1, 0), mkc<double>(0, 0));
}

template cudaError_t cgemm<double>(cudaStream_t, int, int, int, int, int, const double2*, long,
                                   long, const double2*, long, long, double2*, long, long, int,
                                   double2, double2);
template cudaError_t cgemm<float>(cudaStream_t, int, int, int, int, int, const float2*, long,
                                  long, const float2*, long, long, float2*, long, long, int,
                                  float2, float2);

}  // namespace mpdo

// ------------------------------------------------------------------ autotuner
namespace mpdo {
void set_global_error(const char* msg);
}

extern "C" int mpdo_autotune_gemm(int prec, void* stream, int reps, int* n_tuned) {
  using namespace mpdo;
  if (prec != 0 && prec != 1) {
    set_global_error("mpdo_autotune_gemm: prec must be 0 (FP64) or 1 (FP32)");
    return MPDO_ERR_ARG;
  }
  if (n_tuned) *n_tuned = 0;
  auto& table = g_choice[prec];
  if (reps <= 0) {   // back to the size rules
    for (auto& row : table)
      for (auto& c : row) c.store(0, std::memory_order_relaxed);
    return MPDO_OK;
  }
  reps = std::min(reps, 50);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t elt = prec == 0 ? sizeof(double2) : sizeof(float2);
  // largest representative shape: 2^10 tiles of 16 x 16 (512 x 512), K = 4096
  const long mmax = 512, kmax = 16L << (kKBuckets - 1);
  void *a = nullptr, *b = nullptr, *c = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (c) cudaFree(c);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&a, mmax * kmax * elt) != cudaSuccess || cudaMalloc(&b, kmax * mmax * elt) != cudaSuccess ||
      cudaMalloc(&c, mmax * mmax * elt) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    release();
    set_global_error("mpdo_autotune_gemm: allocation failed");
    return MPDO_ERR_OOM;
  }
  cudaError_t err = cudaMemsetAsync(a, 0, mmax * kmax * elt, st);
  if (err == cudaSuccess) err = cudaMemsetAsync(b, 0, kmax * mmax * elt, st);
  int tuned = 0;
  for (int tb = 0; tb < kTileBuckets && err == cudaSuccess; ++tb)
    for (int kb = 0; kb < kKBuckets && err == cudaSuccess; ++kb) {
      // representative shape of the bucket: 2^tb tiles, K = 16 * 2^kb
      const int m = 16 << ((tb + 1) / 2), n = 16 << (tb / 2), k = 16 << kb;
      float best = 1e30f;
      int best_c = 0;
      for (int ch = 1; ch <= kChoices && err == cudaSuccess; ++ch) {
        if (ch >= 3 && k < 16 * (1 << (ch - 2))) continue;   // slices shorter than one step
        table[tb][kb].store((signed char)ch, std::memory_order_relaxed);
        auto run = [&]() {
          return prec == 0
                     ? cgemm<double>(st, OP_N, OP_N, m, n, k, (const double2*)a, k, 0,
                                     (const double2*)b, n, 0, (double2*)c, n, 0, 1,
                                     make_double2(1, 0), make_double2(0, 0))
                     : cgemm<float>(st, OP_N, OP_N, m, n, k, (const float2*)a, k, 0,
                                    (const float2*)b, n, 0, (float2*)c, n, 0, 1,
                                    make_float2(1, 0), make_float2(0, 0));
        };
        err = run();   // warm-up
        float t_min = 1e30f;
        for (int r = 0; r < reps && err == cudaSuccess; ++r) {
          err = cudaEventRecord(e0, st);
          if (err == cudaSuccess) err = run();
          if (err == cudaSuccess) err = cudaEventRecord(e1, st);
          if (err == cudaSuccess) err = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
          t_min = std::min(t_min, ms);
        }
        if (err == cudaSuccess && t_min < best) {
          best = t_min;
          best_c = ch;
        }
      }
      table[tb][kb].store((signed char)best_c, std::memory_order_relaxed);
      if (best_c) ++tuned;
    }
  release();
  if (err != cudaSuccess) {
    for (auto& row : table)
      for (auto& cc : row) cc.store(0, std::memory_order_relaxed);
    cudaGetLastError();
    set_global_error(cudaGetErrorString(err));
    return MPDO_ERR_CUDA;
  }
  if (n_tuned) *n_tuned = tuned;
  return MPDO_OK;
}
