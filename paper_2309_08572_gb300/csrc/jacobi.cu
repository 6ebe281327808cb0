// Parallel two-sided block Jacobi eigensolver for Hermitian matrices (FP64 / FP32).
//
// The columns are split into blocks of JW = 8; every round pairs the blocks by a
// round-robin tournament and one CTA per pair diagonalises its 16 x 16 principal
// sub-matrix with scalar cyclic Jacobi rotations in shared memory (GVL sym.schur2 with
// the complex phase factored out), then applies the accumulated 16 x 16 unitary to its
// rows (phase A) and, after a grid-wide barrier, to its columns and to the eigenvector
// accumulator (phase B).  Pairs in one round touch disjoint rows/columns, so phases A
// and B need only the two barriers of a cooperative launch.  A sweep in which no pair
// rotated ends the iteration.  Cost per sweep ~6 n^3 complex MACs; the matrix stays in
// L2 (it is at most a few MB).
#include <cooperative_groups.h>
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "../../include/mpdo.h"

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace mpdo {
namespace {

constexpr int JW = 8;          // block width
constexpr int JS = 2 * JW;     // sub-problem size
constexpr int JT = 256;        // threads per CTA
constexpr int CH = 64;         // staged chunk (columns in phase A, rows in phase B)
// Sweeps of the 16x16 sub-problem per block-pair visit.  One sweep per visit is the
// classic one-sided-update choice: the outer rounds keep rotating the pair, so a fully
// converged sub-problem buys little and costs 15 warp rounds per extra sweep.
constexpr int kInnerSweeps = 1;


template <typename R> struct Tol;
template <> struct Tol<double> { static constexpr double rel = 1e-15, abs = 2.2e-16; };
// FP32: absolute threshold only.  Eigenvalues below ~eps |A| are not resolved in FP32
// whatever the rotations do (every FP32 cut sits above 10 eps, and the mixed solver
// resolves the small ones in its next level), so pairs whose coupling is below eps |A|
// are left alone; this saves the sweeps a relative threshold spends on them.
template <> struct Tol<float> { static constexpr float rel = 0.f, abs = 6e-8f; };

template <typename R>
__global__ void pad_copy_kernel(int n, int np, const cx<R>* __restrict__ a, long lda,
                                cx<R>* __restrict__ ap, cx<R>* __restrict__ vp, int* counters) {
  long total = (long)np * np;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int i = (int)(e / np), j = (int)(e % np);
    cx<R> v = mkc<R>(0, 0);
    if (i < n && j < n) v = a[(long)i * lda + j];
    ap[e] = v;
    vp[e] = mkc<R>(i == j ? 1 : 0, 0);
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) counters[threadIdx.x] = 0;
}

template <typename R>
__global__ void __launch_bounds__(JT) jacobi_coop_kernel(int np, int nblk, cx<R>* ap,
                                                         cx<R>* vp, int* counters,
                                                         int max_sweeps) {
  using T = cx<R>;
  cg::grid_group grid = cg::this_grid();
  __shared__ T S[JS][JS + 1];
  __shared__ T U[JS][JS + 1];
  __shared__ T X[JS][CH + 1];
  __shared__ int idx[JS];
  __shared__ R rc[JS / 2], rs[JS / 2];
  __shared__ T re[JS / 2];
  __shared__ int ra[JS / 2], rb[JS / 2], rflag[JS / 2];
  __shared__ int any_rot;
  __shared__ R s_anorm;
  const int tid = threadIdx.x;

  // |A| scale for the absolute rotation floor: sum of |diag|, reduced in a fixed order so
  // that every CTA (and every run) uses the same threshold
  {
    __shared__ R wpart[JT / 32];
    R part = 0;
    for (int i = tid; i < np; i += JT) part += fabs(ap[(long)i * np + i].x);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) wpart[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      R t = 0;
      for (int k = 0; k < JT / 32; ++k) t += wpart[k];
      s_anorm = t;
    }
  }
  __syncthreads();
  const R atol = Tol<R>::abs * s_anorm;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nblk - 1; ++round) {
      int bi, bj;
      tourney(round, blockIdx.x, nblk, bi, bj);
      if (tid < JS) idx[tid] = (tid < JW) ? bi * JW + tid : bj * JW + (tid - JW);
      __syncthreads();
      // ---- load the 16x16 principal sub-matrix, U = I
      for (int e = tid; e < JS * JS; e += JT) {
        int a = e / JS, b = e % JS;
        S[a][b] = ap[(long)idx[a] * np + idx[b]];
        U[a][b] = mkc<R>(a == b ? 1 : 0, 0);
      }
      __syncthreads();
      // ---- scalar cyclic Jacobi on S, by warp 0 alone (warp-level barriers only)
      if (tid < 32) {
        const int lane = tid;
        int rot_seen = 0;
        for (int inner = 0; inner < kInnerSweeps; ++inner) {
          int any_inner_w = 0;
          for (int r = 0; r < JS - 1; ++r) {
            int f = 0;
            if (lane < JS / 2) {
              int a, b;
              tourney(r, lane, JS, a, b);
              if (a > b) { int t = a; a = b; b = t; }
              T g = S[a][b];
              R ag = sqrt(cabs2(g));
              R al = S[a][a].x, be = S[b][b].x;
              f = (ag > Tol<R>::rel * sqrt(fabs(al * be))) && (ag > atol);
              ra[lane] = a; rb[lane] = b; rflag[lane] = f;
              if (f) {
                R tau = (be - al) / (2 * ag);
                R t = (tau >= 0 ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
                R c = R(1) / sqrt(R(1) + t * t);
                rc[lane] = c; rs[lane] = t * c;
                re[lane] = mkc<R>(g.x / ag, g.y / ag);
              }
            }
            const unsigned any_f = __ballot_sync(0xffffffffu, f);
            __syncwarp();
            if (!any_f) continue;
            any_inner_w = 1;
            // rows: S <- U^+ S on rows (a, b)
            for (int e = lane; e < (JS / 2) * JS; e += 32) {
              int p = e / JS, col = e % JS;
              if (!rflag[p]) continue;
              int a = ra[p], b = rb[p];
              R c = rc[p], s = rs[p];
              T ee = re[p];
              T x = S[a][col], y = S[b][col];
              S[a][col] = csub(cscale(x, c), cscale(cmul(ee, y), s));
              S[b][col] = cadd(cscale(cmulc(x, ee), s), cscale(y, c));
            }
            __syncwarp();
            // cols: S <- S U and U_acc <- U_acc U on cols (a, b)
            for (int e = lane; e < (JS / 2) * JS * 2; e += 32) {
              int which = e / ((JS / 2) * JS);
              int e2 = e % ((JS / 2) * JS);
              int p = e2 / JS, row = e2 % JS;
              if (!rflag[p]) continue;
              int a = ra[p], b = rb[p];
              R c = rc[p], s = rs[p];
              T ee = re[p];
              if (which) {
                T x = U[row][a], y = U[row][b];
                U[row][a] = csub(cscale(x, c), cscale(cmulc(y, ee), s));
                U[row][b] = cadd(cscale(cmul(x, ee), s), cscale(y, c));
              } else {
                T x = S[row][a], y = S[row][b];
                S[row][a] = csub(cscale(x, c), cscale(cmulc(y, ee), s));
                S[row][b] = cadd(cscale(cmul(x, ee), s), cscale(y, c));
              }
            }
            __syncwarp();
          }
          rot_seen |= any_inner_w;
          if (!any_inner_w) break;
        }
        if (lane == 0) any_rot = rot_seen;
      }
      __syncthreads();
      const int active = any_rot;
      // One Newton-Schulz polar step U <- U (3I - U^+U)/2 removes the drift of the
      // accumulated rotations from unitarity (quadratic in the drift), so repeated
      // applications do not scale the spectrum.
      if (active) {
        for (int e = tid; e < JS * JS; e += JT) {
          int a = e / JS, b = e % JS;
          T acc = mkc<R>(0, 0);
          for (int r = 0; r < JS; ++r) cfma(acc, cconj(U[r][a]), U[r][b]);
          X[a][b] = acc;                      // G = U^+ U (X used as scratch)
        }
        __syncthreads();
        T nu[JS * JS / JT > 0 ? JS * JS / JT : 1];
        int q = 0;
        for (int e = tid; e < JS * JS; e += JT, ++q) {
          int a = e / JS, b = e % JS;
          T acc = cscale(U[a][b], R(1.5));
          for (int r = 0; r < JS; ++r) cfma(acc, cscale(U[a][r], R(-0.5)), X[r][b]);
          nu[q] = acc;
        }
        __syncthreads();
        q = 0;
        for (int e = tid; e < JS * JS; e += JT, ++q) U[e / JS][e % JS] = nu[q];
        __syncthreads();
      }
      // ---- phase A: rows idx of A <- U^+ A[idx, :], in column chunks staged in smem
      if (active) {
        for (int c0 = 0; c0 < np; c0 += CH) {
          int cw = min(CH, np - c0);
          for (int e = tid; e < JS * CH; e += JT) {
            int a = e / CH, c = e % CH;
            X[a][c] = (c < cw) ? ap[(long)idx[a] * np + c0 + c] : mkc<R>(0, 0);
          }
          __syncthreads();
          for (int e = tid; e < JS * CH; e += JT) {
            int a = e / CH, c = e % CH;
            if (c >= cw) continue;
            T acc = mkc<R>(0, 0);
            for (int b = 0; b < JS; ++b) cfma(acc, cconj(U[b][a]), X[b][c]);
            ap[(long)idx[a] * np + c0 + c] = acc;
          }
          __syncthreads();
        }
      }
      grid.sync();
      // ---- phase B: columns idx of A and V <- (.) U, in row chunks staged in smem
      if (active) {
        for (int r0 = 0; r0 < 2 * np; r0 += CH) {
          int rw = min(CH, 2 * np - r0);
          for (int e = tid; e < CH * JS; e += JT) {
            int r = e / JS, b = e % JS;
            int gr = r0 + r;
            if (r < rw) {
              const T* rowp = (gr < np) ? ap + (long)gr * np : vp + (long)(gr - np) * np;
              X[b][r] = rowp[idx[b]];
            }
          }
          __syncthreads();
          for (int e = tid; e < CH * JS; e += JT) {
            int r = e / JS, a = e % JS;
            int gr = r0 + r;
            if (r >= rw) continue;
            T acc = mkc<R>(0, 0);
            for (int b = 0; b < JS; ++b) cfma(acc, X[b][r], U[b][a]);
            T* rowp = (gr < np) ? ap + (long)gr * np : vp + (long)(gr - np) * np;
            rowp[idx[a]] = acc;
          }
          __syncthreads();
        }
        if (tid == 0) {
          atomicAdd(&counters[sweep & 1], 1);
          atomicAdd(&counters[3], 1);  // active pair-rounds, for the flop count
        }
      }
      grid.sync();
      if (round == 0 && blockIdx.x == 0 && tid == 0) counters[(sweep + 1) & 1] = 0;
    }
    int done = (atomicAdd(&counters[sweep & 1], 0) == 0);
    if (done) { ++sweep; break; }
  }
  if (blockIdx.x == 0 && tid == 0) counters[2] = sweep;
}

// Sort the eigenvalues (diagonal of the converged matrix, positions < n) descending
// and gather the matching columns of V.  One CTA, bitonic sort on a power of two.
template <typename R>
__global__ void eig_finalize_kernel(int n, int np, const cx<R>* __restrict__ ap,
                                    const cx<R>* __restrict__ vp, cx<R>* v, long ldv,
                                    double* w) {
  extern __shared__ unsigned char smem_raw[];
  int P = 1;
  while (P < n) P <<= 1;
  double* key = reinterpret_cast<double*>(smem_raw);
  int* val = reinterpret_cast<int*>(key + P);
  __shared__ int s_nan;
  if (threadIdx.x == 0) s_nan = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    double kv = -INFINITY;
    if (i < n) {
      kv = (double)ap[(long)i * np + i].x;
      if (!isfinite(kv)) { s_nan = 1; kv = -INFINITY; }
    }
    key[i] = kv;
    val[i] = i;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool desc = ((i & k) == 0);
          double ki = key[i], kl = key[l];
          bool sw = desc ? (ki < kl) : (ki > kl);
          if (sw) {
            key[i] = kl; key[l] = ki;
            int t = val[i]; val[i] = val[l]; val[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = (s_nan && i == 0) ? NAN : key[i];
  long total = (long)n * n;
  for (long e = threadIdx.x; e < total; e += blockDim.x) {
    int i = (int)(e / n), k = (int)(e % n);
    int col = val[k];
    col = (col >= 0 && col < n) ? col : k;
    v[(long)i * ldv + k] = vp[(long)i * np + col];
  }
}

// ---------------------------------------------------------------------------------------
// Single-CTA cyclic Jacobi with the whole problem resident in shared memory: the Hermitian
// matrix A and the accumulator V live in shared memory; each round of the round-robin
// ordering rotates np/2 disjoint index pairs at once (GVL sym.schur2 with the complex
// phase factored out): rotation parameters, then one pass over the 2x2 blocks of A (row
// and column rotation together) and the columns of V, with a block barrier after each.  Rotations act on A itself (two-sided),
// so eigenvectors are accurate to eps |A| / gap.  Used for n <= smem_jacobi_max<R>().
// The input (precision RI) is rounded to R on load and the eigenvectors are written in
// precision RO, so a solve of an FP64 matrix in FP32 sweeps needs no conversion launches.
constexpr int SJ_THREADS = 1024;

template <typename R, typename RI, typename RO>
__global__ void __launch_bounds__(SJ_THREADS) jacobi_smem_kernel(int n, int np,
                                                                 const cx<RI>* __restrict__ a,
                                                                 long lda, cx<RO>* v, long ldv,
                                                                 double* w, int* counters,
                                                                 int max_sweeps) {
  using T = cx<R>;
  extern __shared__ unsigned char sj_raw[];
  T* A = reinterpret_cast<T*>(sj_raw);       // row-major np x np
  T* V = A + (size_t)np * np;
  __shared__ R s_anorm;
  __shared__ int s_rot;
  __shared__ double s_key[128];
  __shared__ int s_val[128];
  __shared__ R pc[64], ps[64];
  __shared__ T pe[64];
  __shared__ int pp[64], pq[64], pf[64];
  const int tid = threadIdx.x, lane = tid & 31;
  const int nthr = blockDim.x;
  const int half = np / 2;
  for (int e = tid; e < np * np; e += nthr) {
    int i = e / np, j = e % np;
    T z = mkc<R>(0, 0);
    if (i < n && j < n) {
      const cx<RI> t = a[(long)i * lda + j];
      z = mkc<R>((R)t.x, (R)t.y);
    }
    A[e] = z;
    V[e] = mkc<R>(i == j ? 1 : 0, 0);
  }
  if (tid == 0) s_anorm = 0;
  __syncthreads();
  if (tid < 32) {
    R part = 0;
    for (int i = lane; i < n; i += 32) part += fabs(A[(size_t)i * np + i].x);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_anorm = part;
  }
  __syncthreads();
  const R atol = Tol<R>::abs * s_anorm;
  int sweep = 0;
  int total_rot = 0;   // thread 0: rotations applied (pair-rounds with an active pair)
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int k = tid; k < half; k += nthr) {
        int p, q;
        tourney(r, k, np, p, q);
        if (p > q) { int t = p; p = q; q = t; }
        T g = A[(size_t)p * np + q];
        R ag = sqrt(cabs2(g));
        R al = A[(size_t)p * np + p].x, be = A[(size_t)q * np + q].x;
        int f = (ag > Tol<R>::rel * sqrt(fabs(al * be))) && (ag > atol);
        pp[k] = p; pq[k] = q; pf[k] = f;
        if (f) {
          R tau = (be - al) / (2 * ag);
          R t = (tau >= 0 ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
          R c = R(1) / sqrt(R(1) + t * t);
          pc[k] = c; ps[k] = t * c;
          pe[k] = mkc<R>(g.x / ag, g.y / ag);
          atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
      // The disjoint pairs partition the indices, so A' = J^+ A J splits into independent
      // 2x2 blocks: block (a, b) holds rows {p_a, q_a} x columns {p_b, q_b} and needs only
      // the rotations of pairs a and b.  One pass updates every block (and the columns of
      // V), with no barrier between the row and the column rotation.
      for (int e = tid; e < half * half; e += nthr) {
        const int ka = e / half, kb = e - ka * half;
        const int fa = pf[ka], fb = pf[kb];
        if (!fa && !fb) continue;
        const int pa = pp[ka], qa = pq[ka], pb = pp[kb], qb = pq[kb];
        const R ca = fa ? pc[ka] : R(1), sa = fa ? ps[ka] : R(0);
        const R cb = fb ? pc[kb] : R(1), sb = fb ? ps[kb] : R(0);
        const T ea = fa ? pe[ka] : mkc<R>(1, 0), eb = fb ? pe[kb] : mkc<R>(1, 0);
        T* rp = A + (size_t)pa * np;
        T* rq = A + (size_t)qa * np;
        const T x0 = rp[pb], x1 = rp[qb], y0 = rq[pb], y1 = rq[qb];
        // rows (pair a): p' = c x - s e y, q' = s x conj(e) + c y
        const T u0 = csub(cscale(x0, ca), cscale(cmul(ea, y0), sa));
        const T u1 = csub(cscale(x1, ca), cscale(cmul(ea, y1), sa));
        const T w0 = cadd(cscale(cmulc(x0, ea), sa), cscale(y0, ca));
        const T w1 = cadd(cscale(cmulc(x1, ea), sa), cscale(y1, ca));
        // columns (pair b): p' = c x - s y conj(e), q' = s x e + c y
        rp[pb] = csub(cscale(u0, cb), cscale(cmulc(u1, eb), sb));
        rp[qb] = cadd(cscale(cmul(u0, eb), sb), cscale(u1, cb));
        rq[pb] = csub(cscale(w0, cb), cscale(cmulc(w1, eb), sb));
        rq[qb] = cadd(cscale(cmul(w0, eb), sb), cscale(w1, cb));
      }
      for (int e = tid; e < np * half; e += nthr) {
        const int row = e / half, kb = e - row * half;
        if (!pf[kb]) continue;
        const int p = pp[kb], q = pq[kb];
        const R c = pc[kb], sn = ps[kb];
        const T ee = pe[kb];
        T* vr = V + (size_t)row * np;
        const T x = vr[p], y = vr[q];
        vr[p] = csub(cscale(x, c), cscale(cmulc(y, ee), sn));
        vr[q] = cadd(cscale(cmul(x, ee), sn), cscale(y, c));
      }
      __syncthreads();
    }
    if (tid == 0) total_rot += s_rot;
    // every thread reads the count before thread 0 resets it for the next sweep (a thread
    // that read the reset value would leave the loop alone and break the block barriers)
    const int rotated = s_rot;
    __syncthreads();
    if (rotated == 0) { ++sweep; break; }
  }
  // eigenvalues = diagonal; sort descending (n <= 128)
  __shared__ int s_nan;
  if (tid == 0) s_nan = 0;
  __syncthreads();
  int P = 2;
  while (P < n) P <<= 1;                       // n <= 118 -> P <= 128
  for (int c = tid; c < P; c += nthr) {
    double key = -INFINITY;
    if (c < n) {
      key = (double)A[(size_t)c * np + c].x;
      if (!isfinite(key)) { s_nan = 1; key = -INFINITY; }
    }
    s_key[c] = key;
    s_val[c] = c;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int c = tid; c < P; c += nthr) {
        int l = c ^ j;
        if (l > c) {
          bool desc = ((c & k) == 0);
          double ki = s_key[c], kl = s_key[l];
          if (desc ? (ki < kl) : (ki > kl)) {
            s_key[c] = kl; s_key[l] = ki;
            int t = s_val[c]; s_val[c] = s_val[l]; s_val[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  // a non-finite input is reported as a NaN leading eigenvalue (callers flag it); the
  // gather index is clamped so a broken permutation can never leave the arrays
  for (int i = tid; i < n; i += nthr) w[i] = (s_nan && i == 0) ? NAN : s_key[i];
  for (int e = tid; e < n * n; e += nthr) {
    int i = e / n, k = e % n;
    int col = s_val[k];
    col = (col >= 0 && col < n) ? col : k;
    const T t = V[(size_t)i * np + col];
    v[(long)i * ldv + k] = mkc<RO>((RO)t.x, (RO)t.y);
  }
  if (tid == 0 && counters) {
    counters[2] = sweep;
    counters[3] = total_rot;   // each rotates 2 rows and 2 columns of A and 2 columns of V
  }
}

template <typename R>
constexpr int smem_jacobi_max() { return sizeof(R) == 8 ? 84 : 118; }

inline int padded_n(int n) {
  int nblk = (n + JW - 1) / JW;
  if (nblk < 2) nblk = 2;
  if (nblk & 1) ++nblk;
  return nblk * JW;
}

template <typename R, typename RI, typename RO>
cudaError_t smem_jacobi_launch(cudaStream_t st, int n, const cx<RI>* a, long lda, cx<RO>* v,
                               long ldv, double* w, int* counters, int max_sweeps) {
  const int np2 = n + (n & 1);
  const size_t sm = 2ull * np2 * np2 * sizeof(cx<R>);
  const int smax = smem_jacobi_max<R>() + (smem_jacobi_max<R>() & 1);
  // once per instantiation (a thread-safe static initialiser)
  static const cudaError_t attr = cudaFuncSetAttribute(
      jacobi_smem_kernel<R, RI, RO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(2ull * smax * smax * sizeof(cx<R>)));
  MPDO_CUDA_TRY(attr);
  count_launch();
  const int thr = std::min(SJ_THREADS, std::max(64, ((np2 / 2) * np2 + 31) / 32 * 32));
  jacobi_smem_kernel<R, RI, RO><<<1, thr, sm, st>>>(n, np2, a, lda, v, ldv, w, counters,
                                                    max_sweeps);
  return cudaGetLastError();
}

}  // namespace

template <typename RI, typename RO>
cudaError_t heig_smem_f32(cudaStream_t st, int n, const cx<RI>* a, long lda, cx<RO>* v, long ldv,
                          double* w, int* counters, int max_sweeps) {
  if (n <= 0) return cudaSuccess;
  if (n > kSmemJacobiMaxF32) return cudaErrorInvalidValue;
  return smem_jacobi_launch<float, RI, RO>(st, n, a, lda, v, ldv, w, counters, max_sweeps);
}
template cudaError_t heig_smem_f32<double, double>(cudaStream_t, int, const double2*, long,
                                                   double2*, long, double*, int*, int);
template cudaError_t heig_smem_f32<double, float>(cudaStream_t, int, const double2*, long,
                                                  float2*, long, double*, int*, int);

int eig_padded_n(int n) { return padded_n(n); }

// Executed rotation flops per unit of counters[3] (8 real flops per complex element update):
// the one-CTA kernel counts applied rotations (each updates 2 rows and 2 columns of A and 2
// columns of V, n elements each: 6 n updates); the block kernel counts active pair-rounds
// (3 x 16 x 16 x n_pad complex multiply-adds).
double eig_flops_per_count(int n, bool fp64) {
  const int smax = fp64 ? 84 : 118;
  if (n <= smax) return 8.0 * 6.0 * (double)(n + (n & 1));
  return 8.0 * 3 * 256 * (double)padded_n(n);
}

template <typename R>
size_t eig_work_bytes(int n_cap) {
  size_t np = padded_n(n_cap);
  return 2 * np * np * sizeof(cx<R>) + 256;
}

template <typename R>
void eig_work_bind(EigWork<R>& w, void* base, int n_cap) {
  size_t np = padded_n(n_cap);
  w.n_cap = n_cap;
  w.ap = reinterpret_cast<cx<R>*>(base);
  w.vp = w.ap + np * np;
  w.counters = reinterpret_cast<int*>(w.vp + np * np);
}

template <typename R>
cudaError_t heig(cudaStream_t st, int n, const cx<R>* a, long lda, cx<R>* v, long ldv,
                 double* w, EigWork<R>& work, int max_sweeps) {
  if (n <= 0) return cudaSuccess;
  if (n > work.n_cap) return cudaErrorInvalidValue;
  if (n <= smem_jacobi_max<R>())
    return smem_jacobi_launch<R, R, R>(st, n, a, lda, v, ldv, w, work.counters, max_sweeps);
  int np = padded_n(n);
  int nblk = np / JW;
  long total = (long)np * np;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch(3);
  pad_copy_kernel<R><<<blocks, 256, 0, st>>>(n, np, a, lda, work.ap, work.vp, work.counters);
  MPDO_CUDA_TRY(cudaGetLastError());
  int grid = nblk / 2;
  void* args[] = {&np, &nblk, &work.ap, &work.vp, &work.counters, &max_sweeps};
  MPDO_CUDA_TRY(cudaLaunchCooperativeKernel((void*)jacobi_coop_kernel<R>, dim3(grid),
                                            dim3(JT), args, 0, st));
  int P = 1;
  while (P < n) P <<= 1;
  size_t sm = (size_t)P * (sizeof(double) + sizeof(int));
  // sort keys beyond n = 2048 exceed the default 48 KB of shared memory (with the kernel's
  // static flag): opt in up to n = 16384, 192 KB (once per instantiation)
  static const cudaError_t fattr = cudaFuncSetAttribute(
      eig_finalize_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(16384 * (sizeof(double) + sizeof(int))));
  MPDO_CUDA_TRY(fattr);
  if (P > 16384) return cudaErrorInvalidValue;
  eig_finalize_kernel<R><<<1, 1024, sm, st>>>(n, np, work.ap, work.vp, v, ldv, w);
  return cudaGetLastError();
}

template size_t eig_work_bytes<double>(int);
template size_t eig_work_bytes<float>(int);
template void eig_work_bind<double>(EigWork<double>&, void*, int);
template void eig_work_bind<float>(EigWork<float>&, void*, int);
template cudaError_t heig<double>(cudaStream_t, int, const double2*, long, double2*, long,
                                  double*, EigWork<double>&, int);
template cudaError_t heig<float>(cudaStream_t, int, const float2*, long, float2*, long,
                                 double*, EigWork<float>&, int);

}  // namespace mpdo

// ---------------------------------------------------------------------------------------
// Allocation-free eigensolver entry point (mpdo_heig_noalloc, declared in mpdo.h).
// Its scratch -- the padded working matrix, the eigenvector accumulator and the sweep
// counters -- is one file-scope device array sized for n <= MPDO_HEIG_NOALLOC_NMAX, so a
// call performs no device allocation.  Host code cannot use the array's name as a device
// address; the address is looked up with cudaGetSymbolAddress once per device (first call
// with that device current) and passed to the kernels.
namespace {
constexpr int kNoAllocNMax = MPDO_HEIG_NOALLOC_NMAX;
constexpr size_t kNoAllocBytes = 2ull * kNoAllocNMax * kNoAllocNMax * sizeof(double2) + 256;
static_assert(kNoAllocNMax % (2 * mpdo::JW) == 0, "maximum must be a whole number of block pairs");
static __device__ __align__(256) unsigned char g_heig_scratch[kNoAllocBytes];
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
// per device: the CUDA context the address was looked up in, and the address.  A device
// reset (or a primary context destroyed and created again) loads the module anew, possibly
// elsewhere, so the address is looked up again whenever the current context changes.
void* g_scratch_ctx[kMaxDevices] = {};
void* g_scratch_addr[kMaxDevices] = {};
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
void* current_context() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<CtxGetCurrentFn>(nullptr);
    }
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  CUcontext c = nullptr;
  if (fn) fn(&c);
  return c;
}
}  // namespace

namespace mpdo {
void set_global_error(const char* msg);
}

extern "C" int mpdo_heig_noalloc(int prec, int n, void* a, void* v, double* w, int* sweeps,
                                 void* stream) {
  using namespace mpdo;
  if (prec != 0 && prec != 1) {
    set_global_error("mpdo_heig_noalloc: prec must be 0 (complex128) or 1 (complex64)");
    return MPDO_ERR_ARG;
  }
  if (n < 1 || n > kNoAllocNMax) {
    set_global_error("mpdo_heig_noalloc: n must be in 1..MPDO_HEIG_NOALLOC_NMAX (192)");
    return MPDO_ERR_ARG;
  }
  if (!a || !v || !w) {
    set_global_error("mpdo_heig_noalloc: null matrix, vector or eigenvalue pointer");
    return MPDO_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error("mpdo_heig_noalloc: no usable current CUDA device");
    return MPDO_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    void* ctx = current_context();
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_heig_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error("mpdo_heig_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return MPDO_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = current_context();
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* counters;
  if (prec == 0) {
    EigWork<double> wk;
    eig_work_bind<double>(wk, base, kNoAllocNMax);
    counters = wk.counters;
    e = heig<double>(st, n, static_cast<const double2*>(a), n, static_cast<double2*>(v), n, w,
                     wk, 30);
  } else {
    EigWork<float> wk;
    eig_work_bind<float>(wk, base, kNoAllocNMax);
    counters = wk.counters;
    e = heig<float>(st, n, static_cast<const float2*>(a), n, static_cast<float2*>(v), n, w, wk,
                    20);
  }
  if (e == cudaSuccess && sweeps) {
    e = cudaMemcpyAsync(sweeps, counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return MPDO_ERR_CUDA;
  }
  return MPDO_OK;
}

// =======================================================================================
// Eigenpairs of a Hermitian PSD matrix from its pivoted Cholesky factor W ~ L L^+:
// one-sided (Hestenes) Jacobi on the columns of L.  Pairs of columns are rotated until
// mutually orthogonal (|a_p^+ a_q| <= tol |a_p| |a_q|); then sigma_k = |a_k| and the unit
// columns are the eigenvectors of L L^+ with eigenvalues sigma_k^2.  The rotations never
// form a Gram matrix, so small eigenvalues keep their relative accuracy (Demmel and
// Veselic): the factor's graded columns need no square of the precision.  One CTA; L lives
// column-major in shared memory; warp w handles pair slots w, w + nw, ... of each round.
namespace mpdo {
namespace {

template <typename R>
struct OsjTol;
template <> struct OsjTol<double> { static constexpr double v = 1e-14; };
template <> struct OsjTol<float> { static constexpr double v = 2e-6; };

// Sweeps over the column pairs of A (column-major, n x rp, precision of T) until no pair
// is rotated; returns the rotations applied (thread 0).
template <typename T>
__device__ int osj_sweeps(T* A, int n, int rp, int max_sweeps, double tol, int* s_rot,
                          int* sweeps_out) {
  using R = decltype(T{}.x);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int sweep = 0, total = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *s_rot = 0;
    __syncthreads();
    for (int round = 0; round < rp - 1; ++round) {
      for (int slot = warp; slot < rp / 2; slot += nw) {
        int p, q;
        tourney(round, slot, rp, p, q);
        T* ap = A + (size_t)p * n;
        T* aq = A + (size_t)q * n;
        R al = 0, be = 0, gr = 0, gi = 0;
        for (int i = lane; i < n; i += 32) {
          T x = ap[i], y = aq[i];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;     // conj(x) y
          gi += x.x * y.y - x.y * y.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        const R ag = sqrt(gr * gr + gi * gi);
        if (!(ag > (R)tol * sqrt(al * be)) || !(ag > 0)) continue;
        // with b_q = conj(e) a_q (e = g/|g|) the pair's Gram is real: [[al, |g|], [|g|, be]]
        const R zeta = (be - al) / (2 * ag);
        const R t = (zeta >= 0 ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
        const R c = R(1) / sqrt(R(1) + t * t), s = c * t;
        const R er = gr / ag, ei = gi / ag;   // e
        for (int i = lane; i < n; i += 32) {
          T x = ap[i], y = aq[i];
          T b;   // conj(e) y
          b.x = er * y.x + ei * y.y;
          b.y = er * y.y - ei * y.x;
          T xn, yn;
          xn.x = c * x.x - s * b.x; xn.y = c * x.y - s * b.y;
          yn.x = s * x.x + c * b.x; yn.y = s * x.y + c * b.y;
          ap[i] = xn;
          aq[i] = yn;
        }
        if (lane == 0) atomicAdd(s_rot, 1);
      }
      __syncthreads();
    }
    if (tid == 0) total += *s_rot;
    const int any = *s_rot;
    __syncthreads();
    if (any == 0) { ++sweep; break; }
  }
  *sweeps_out = sweep;
  return total;
}

// Column norms, descending sort and output of the unit columns (A column-major n x rp).
template <typename T, typename RO>
__device__ void osj_output(const T* A, int n, int r, int rp, cx<RO>* U, int ldu, double* w,
                           double* s_key, int* s_val) {
  using R = decltype(T{}.x);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int P = 2;
  while (P < rp) P <<= 1;
  for (int c = warp; c < P; c += nw) {
    double nn = 0.0;
    if (c < r) {
      const T* ac = A + (size_t)c * n;
      for (int i = lane; i < n; i += 32) nn += (double)ac[i].x * ac[i].x + (double)ac[i].y * ac[i].y;
      for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if (lane == 0) {
      s_key[c] = (c < r && isfinite(nn)) ? nn : -1.0;
      s_val[c] = c;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int c = tid; c < P; c += blockDim.x) {
        int l = c ^ j;
        if (l > c) {
          bool desc = ((c & k) == 0);
          double kc = s_key[c], kl = s_key[l];
          if (desc ? (kc < kl) : (kc > kl)) {
            s_key[c] = kl; s_key[l] = kc;
            int t2 = s_val[c]; s_val[c] = s_val[l]; s_val[l] = t2;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int k = tid; k < r; k += blockDim.x) w[k] = s_key[k] > 0 ? s_key[k] : 0.0;
  for (long e = tid; e < (long)n * r; e += blockDim.x) {
    int i = (int)(e / r), k = (int)(e % r);
    int col = s_val[k];
    col = (col >= 0 && col < r) ? col : k;
    double nk = s_key[k];
    T x = A[(size_t)col * n + i];
    R inv = nk > 0 ? (R)(1.0 / sqrt(nk)) : R(0);
    U[(long)i * ldu + k] = mkc<RO>((RO)(x.x * inv), (RO)(x.y * inv));
  }
}

// R: precision of the sweeps.  finish64 (R = float only): after the FP32 sweeps the
// rotated columns are widened and the sweeps continue in FP64 (a few, from near
// orthogonality), so the columns end orthogonal to FP64 precision; the FP32 phase's
// rounding perturbs each direction by ~1e-7 relative, which mixed precision accepts.
template <typename RI, typename R, typename RO>
__global__ void __launch_bounds__(1024) osj_kernel(int n, int r, const cx<RI>* __restrict__ L,
                                                   int lr, cx<RO>* U, int ldu, double* w,
                                                   int max_sweeps, int finish64, int* counters) {
  using T = cx<R>;
  extern __shared__ __align__(16) unsigned char osj_raw[];
  const int rp = r + (r & 1);
  T* A = reinterpret_cast<T*>(osj_raw);          // column c at A + c * n
  __shared__ int s_rot;
  __shared__ double s_key[128];
  __shared__ int s_val[128];
  const int tid = threadIdx.x;
  for (int e = tid; e < n * rp; e += blockDim.x) {
    int c = e / n, i = e - c * n;
    cx<RI> x = (c < r) ? L[(long)i * lr + c] : mkc<RI>(0, 0);
    A[e] = mkc<R>((R)x.x, (R)x.y);
  }
  __syncthreads();
  int sweeps = 0, sweeps2 = 0;
  int total = osj_sweeps<T>(A, n, rp, max_sweeps, OsjTol<R>::v, &s_rot, &sweeps);
  if (finish64 && sizeof(R) == 4) {
    // widen into the region after the FP32 columns (16-byte aligned)
    double2* A2 = reinterpret_cast<double2*>(osj_raw + (((size_t)n * rp * sizeof(T) + 15) & ~(size_t)15));
    for (int e = tid; e < n * rp; e += blockDim.x) A2[e] = make_double2((double)A[e].x, (double)A[e].y);
    __syncthreads();
    total += osj_sweeps<double2>(A2, n, rp, max_sweeps, OsjTol<double>::v, &s_rot, &sweeps2);
    osj_output<double2, RO>(A2, n, r, rp, U, ldu, w, s_key, s_val);
  } else {
    osj_output<T, RO>(A, n, r, rp, U, ldu, w, s_key, s_val);
  }
  if (tid == 0 && counters) {
    counters[2] = sweeps + sweeps2;
    counters[3] = total;
  }
}

}  // namespace

template <typename RI, typename R, typename RO>
cudaError_t osj(cudaStream_t st, int n, int r, const cx<RI>* L, int lr, cx<RO>* U, int ldu,
                double* w, int* counters, int finish64) {
  if (n < 1 || r < 1 || r > 128) return cudaErrorInvalidValue;
  const int rp = r + (r & 1);
  size_t sm = (size_t)n * rp * sizeof(cx<R>);
  if (finish64 && sizeof(R) == 4) sm = ((sm + 15) & ~(size_t)15) + (size_t)n * rp * sizeof(double2);
  if (sm > kOsjMaxSmem) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    MPDO_CUDA_TRY(cudaFuncSetAttribute(osj_kernel<RI, R, RO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kOsjMaxSmem));
    attr = true;
  }
  int thr = std::min(1024, std::max(64, (rp / 2) * 32));
  count_launch();
  osj_kernel<RI, R, RO><<<1, thr, sm, st>>>(n, r, L, lr, U, ldu, w, 30, finish64, counters);
  return cudaGetLastError();
}
template cudaError_t osj<double, double, double>(cudaStream_t, int, int, const double2*, int,
                                                 double2*, int, double*, int*, int);
template cudaError_t osj<double, float, double>(cudaStream_t, int, int, const double2*, int,
                                                double2*, int, double*, int*, int);
template cudaError_t osj<float, float, float>(cudaStream_t, int, int, const float2*, int,
                                              float2*, int, double*, int*, int);

}  // namespace mpdo
