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
//     pairs with lam > tau * lam_max(l) (a leading run ending where a column is separated
//     from the next) are final; the other columns of Z span the next level's basis,
//     because FP32 sweeps resolve eigenvectors only down to ~n eps_32 lam_max(l)
//   until the largest remaining lam falls below floor * lam_max(0) or nothing remains.
#include <cuda_runtime.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgemm.h"

namespace cg = cooperative_groups;

namespace mpdo {

namespace {

// A refinement pass squares the eigenvector error of a pair only while it is small: the
// first-order correction E_ij = (S_ij - lam_j G_ij) / (lam_j - lam_i) is the pair's mixing
// angle, so a pair is corrected when |E_ij| is below a bound (and its gap exceeds the FP64
// rounding of the products, ~n eps_64 lam_0).  The step leaves errors of order |E|^2 in the
// columns' norms and mutual angles, so the bound is kNewtonMax in the first pass and
// kNewtonFinal in the last (whose errors no later pass removes): a pair at angle 1e-2 after
// the sweeps is at 1e-4 after the first pass and at 1e-8 after the last, with norms and
// angles off by at most ~1e-8.  Levels wider than kThreePassMin (whose FP32 vectors from
// the block Jacobi carry angles up to ~m eps_32 lam_max / gap) take a third pass, the first
// one accepting angles up to kNewtonWide.  Other pairs -- those the FP32 sweeps could not
// separate -- are orthonormalised only, and in the final pass short runs of them are
// settled by Rayleigh-Ritz (ritz_cluster).  Resolved eigenvalues lie above kTau lam_max,
// two decades per level, the range FP32 sweeps resolve relative to the level's largest.
constexpr double kTau = 1e-2;
constexpr double kNewtonMax = 1e-2;
constexpr double kNewtonFinal = 1e-4;
constexpr double kNewtonWide = 1e-1;
constexpr int kThreePassMin = 1024;
constexpr int kMaxLevels = 24;

// Whether the pair (i, j) takes the first-order correction, |E_ij| < emax (see
// kNewtonMax); symmetric in i and j (evaluated on the entry above the diagonal).
__device__ __forceinline__ bool pair_separated(const double2* SG, long ld, int m,
                                               const double* lam, int i0, int j0, double fsep,
                                               double emax) {
  const int i = i0 < j0 ? i0 : j0, j = i0 < j0 ? j0 : i0;
  const double d = lam[j] - lam[i];
  if (!(fabs(d) > fsep)) return false;
  const double2 sv = __ldcg(&SG[(long)i * ld + j]);
  const double2 g = __ldcg(&SG[(long)i * ld + m + j]);
  const double ex = sv.x - lam[j] * g.x, ey = sv.y - lam[j] * g.y;
  return sqrt(ex * ex + ey * ey) < emax * fabs(d);
}

// Level scalars in wk.scan: [0] lam_max of the pass, [1] nl = length of the leading run
// with lam > kTau lam_max, [2] largest lam after that run, [3] lam_max of level 0's last
// pass, [4] lam_max of level 0's first pass (lam_0 of the separation floor), [5] Jacobi
// rotations of the level, [6] 1 when this level is the last, [7] columns it emits.
constexpr int kScan = 8;

// Largest cluster solved by Rayleigh-Ritz in the final refinement pass, the most clusters
// one pass settles, and the most columns whose separation flags live in shared memory
// (larger levels keep them in the workspace).
constexpr int kRitzMax = 16;
constexpr int kMaxClusters = 1024;
constexpr int kSepMax = 4096;

// Block-wide reductions of the refinement CTA (blockDim.x a multiple of 32, <= 1024); every
// thread gets the result.
__device__ double block_max(double x, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  double v = red[0];
  for (int k = 1; k < nw; ++k) v = fmax(v, red[k]);
  return v;
}
__device__ int block_min_int(int x, int* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  int v = red[0];
  for (int k = 1; k < nw; ++k) v = min(v, red[k]);
  return v;
}
__device__ int block_max_int(int x, int* red) { return -block_min_int(-x, red); }

// Rayleigh-Ritz on one cluster C = [c0, c0 + c) of the final pass (all threads of the CTA):
// its block of [S | G] gives the pencil (S_CC, G_CC); with P = I - (G_CC - I) / 2
// (G_CC^-1/2 to first order) the Hermitian H = P^+ S_CC P is diagonalised by FP64 Jacobi
// rotations, H = Q D Q^+.  IE, filled with I + E outside the cluster blocks, becomes
// (I + E) B on the cluster's columns with B = P Q (its rows outside C carry their
// corrections along the rotation), and lam[C] the eigenvalues, both in descending order.
__device__ void ritz_cluster(int m, const double2* SG, int c0, int c, double* lam, double2* IE) {
  __shared__ double2 Hs[kRitzMax][kRitzMax + 1];
  __shared__ double2 Ps[kRitzMax][kRitzMax + 1];
  __shared__ double2 Qs[kRitzMax][kRitzMax + 1];
  __shared__ double rc[kRitzMax / 2], rs[kRitzMax / 2];
  __shared__ double2 rz[kRitzMax / 2];
  __shared__ int rp[kRitzMax / 2], rq[kRitzMax / 2], rf[kRitzMax / 2];
  __shared__ int s_rot, s_perm[kRitzMax];
  __shared__ double s_atol;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long ld = 2L * m;
  const int cp = c + (c & 1), half = cp / 2;
  for (int e = tid; e < kRitzMax * kRitzMax; e += nt) {
    const int a = e / kRitzMax, b = e % kRitzMax;
    double2 sv = make_double2(0.0, 0.0), pv = make_double2(a == b ? 1.0 : 0.0, 0.0);
    if (a < c && b < c) {
      sv = __ldcg(&SG[(long)(c0 + a) * ld + c0 + b]);
      const double2 g = __ldcg(&SG[(long)(c0 + a) * ld + m + c0 + b]);
      pv = make_double2((a == b ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y);
    }
    Hs[a][b] = sv;
    Ps[a][b] = pv;
  }
  __syncthreads();
  for (int e = tid; e < c * c; e += nt) {   // Qs = S_CC P
    const int a = e / c, b = e % c;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < c; ++k) cfma(acc, Hs[a][k], Ps[k][b]);
    Qs[a][b] = acc;
  }
  __syncthreads();
  for (int e = tid; e < c * c; e += nt) {   // Hs = P^+ (S_CC P)
    const int a = e / c, b = e % c;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < c; ++k) cfma(acc, cconj(Ps[k][a]), Qs[k][b]);
    Hs[a][b] = acc;
  }
  __syncthreads();
  for (int e = tid; e < c * c; e += nt) {   // Hermitian part
    const int a = e / c, b = e % c;
    if (a < b) {
      const double2 x = Hs[a][b], y = Hs[b][a];
      const double2 hh = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      Hs[a][b] = hh;
      Hs[b][a] = cconj(hh);
    }
  }
  __syncthreads();
  for (int e = tid; e < kRitzMax * kRitzMax; e += nt) {
    const int a = e / kRitzMax, b = e % kRitzMax;
    Qs[a][b] = make_double2(a == b ? 1.0 : 0.0, 0.0);
    if (a == b) Hs[a][a].y = 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int a = 0; a < c; ++a) t += fabs(Hs[a][a].x);
    s_atol = 1e-18 * t;
  }
  for (int sweep = 0; sweep < 12; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < cp - 1; ++r) {
      if (tid < half) {
        int p, q;
        tourney(r, tid, cp, p, q);
        if (p > q) { const int t = p; p = q; q = t; }
        const double2 g = Hs[p][q];
        const double ag = sqrt(cabs2(g));
        const double al = Hs[p][p].x, be = Hs[q][q].x;
        const int f = (ag > s_atol) && (ag > 1e-15 * sqrt(fabs(al * be)));
        rp[tid] = p;
        rq[tid] = q;
        rf[tid] = f;
        if (f) {
          const double tau = (be - al) / (2.0 * ag);
          const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cc = 1.0 / sqrt(1.0 + t * t);
          rc[tid] = cc;
          rs[tid] = t * cc;
          rz[tid] = make_double2(g.x / ag, g.y / ag);
          atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
      // the disjoint pairs split H' = J^+ H J into 2 x 2 blocks (rows of pair a, columns
      // of pair b); Q's columns rotate with pair b
      for (int e = tid; e < half * half; e += nt) {
        const int ka = e / half, kb = e - ka * half;
        const int fa = rf[ka], fb = rf[kb];
        if (!fa && !fb) continue;
        const int pa = rp[ka], qa = rq[ka], pb = rp[kb], qb = rq[kb];
        const double ca = fa ? rc[ka] : 1.0, sa = fa ? rs[ka] : 0.0;
        const double cb = fb ? rc[kb] : 1.0, sb = fb ? rs[kb] : 0.0;
        const double2 ea = fa ? rz[ka] : make_double2(1.0, 0.0);
        const double2 eb = fb ? rz[kb] : make_double2(1.0, 0.0);
        const double2 x0 = Hs[pa][pb], x1 = Hs[pa][qb], y0 = Hs[qa][pb], y1 = Hs[qa][qb];
        const double2 u0 = csub(cscale(x0, ca), cscale(cmul(ea, y0), sa));
        const double2 u1 = csub(cscale(x1, ca), cscale(cmul(ea, y1), sa));
        const double2 w0 = cadd(cscale(cmulc(x0, ea), sa), cscale(y0, ca));
        const double2 w1 = cadd(cscale(cmulc(x1, ea), sa), cscale(y1, ca));
        Hs[pa][pb] = csub(cscale(u0, cb), cscale(cmulc(u1, eb), sb));
        Hs[pa][qb] = cadd(cscale(cmul(u0, eb), sb), cscale(u1, cb));
        Hs[qa][pb] = csub(cscale(w0, cb), cscale(cmulc(w1, eb), sb));
        Hs[qa][qb] = cadd(cscale(cmul(w0, eb), sb), cscale(w1, cb));
      }
      for (int e = tid; e < cp * half; e += nt) {
        const int row = e / half, kb = e - row * half;
        if (!rf[kb]) continue;
        const int p = rp[kb], q = rq[kb];
        const double cc = rc[kb], sn = rs[kb];
        const double2 ee = rz[kb];
        const double2 x = Qs[row][p], y = Qs[row][q];
        Qs[row][p] = csub(cscale(x, cc), cscale(cmulc(y, ee), sn));
        Qs[row][q] = cadd(cscale(cmul(x, ee), sn), cscale(y, cc));
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  if (tid == 0) {
    for (int a = 0; a < c; ++a) s_perm[a] = a;
    for (int a = 0; a < c; ++a)
      for (int b = a + 1; b < c; ++b)
        if (Hs[s_perm[b]][s_perm[b]].x > Hs[s_perm[a]][s_perm[a]].x) {
          const int t = s_perm[a];
          s_perm[a] = s_perm[b];
          s_perm[b] = t;
        }
  }
  __syncthreads();
  // B = P Q with its columns sorted, into Ps (P is read before the barrier below)
  double2 bv[(kRitzMax * kRitzMax + 255) / 256];
  int nb = 0;
  for (int e = tid; e < c * c; e += nt, ++nb) {
    const int a = e / c, b = e % c;
    const int col = s_perm[b];
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < c; ++k) cfma(acc, Ps[a][k], Qs[k][col]);
    bv[nb] = acc;
  }
  __syncthreads();
  nb = 0;
  for (int e = tid; e < c * c; e += nt, ++nb) Ps[e / c][e % c] = bv[nb];
  for (int b = tid; b < c; b += nt) lam[c0 + b] = Hs[s_perm[b]][s_perm[b]].x;
  __syncthreads();
  // IE[:, C] <- IE[:, C] B: the cluster's own block is the identity there, i.e. B itself
  for (int i = tid; i < m; i += nt) {
    double2* row = IE + (long)i * m + c0;
    if (i >= c0 && i < c0 + c) {
      for (int b = 0; b < c; ++b) row[b] = Ps[i - c0][b];
      continue;
    }
    double2 x[kRitzMax];
    for (int k = 0; k < c; ++k) x[k] = row[k];
    for (int b = 0; b < c; ++b) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < c; ++k) cfma(acc, x[k], Ps[k][b]);
      row[b] = acc;
    }
  }
  __syncthreads();
}

// I + E of a pass (file comment) for the resolved run [0, nl): pairs that are separated
// (bound emax) take the first-order correction, the others are orthonormalised; with cid,
// pairs inside one Ritz cluster get the identity (the Ritz step sets their block).
__device__ void fill_ie(int m, const double2* SG, const double* lam, double2* IE, int nl,
                        double fsep, double emax, const int* cid) {
  const long ld = 2L * m;
  // one thread per pair i <= j: the pair's separation is decided once, from the entry above
  // the diagonal, and both entries are written
  for (long e = threadIdx.x; e < (long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    if (j < i) continue;
    if (cid && cid[i] >= 0 && cid[i] == cid[j]) {
      IE[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      if (j != i) IE[(long)j * m + i] = make_double2(0.0, 0.0);
      continue;
    }
    const double2 gij = __ldcg(&SG[(long)i * ld + m + j]);
    if (i == j) {
      IE[e] = make_double2(1.0 + 0.5 * (1.0 - gij.x), 0.0);
      continue;
    }
    const double2 gji = __ldcg(&SG[(long)j * ld + m + i]);
    const double li = lam[i], lj = lam[j], d = lj - li;
    bool newton = false;
    double2 sij, sji;
    if ((i < nl || j < nl) && fabs(d) > fsep) {
      sij = __ldcg(&SG[(long)i * ld + j]);
      const double ex = sij.x - lj * gij.x, ey = sij.y - lj * gij.y;
      newton = sqrt(ex * ex + ey * ey) < emax * fabs(d);
      if (newton) sji = __ldcg(&SG[(long)j * ld + i]);
    }
    if (newton) {
      IE[e] = make_double2((sij.x - lj * gij.x) / d, (sij.y - lj * gij.y) / d);
      IE[(long)j * m + i] = make_double2((sji.x - li * gji.x) / -d, (sji.y - li * gji.y) / -d);
    } else {
      IE[e] = make_double2(-0.5 * gij.x, -0.5 * gij.y);
      IE[(long)j * m + i] = make_double2(-0.5 * gji.x, -0.5 * gji.y);
    }
  }
}

// One refinement step's scalars and correction, run by one CTA of 256 threads.
// S = SG[:, 0:m], G = SG[:, m:2m] (row stride 2m), possibly written by other CTAs of the
// same launch (read through L2).  lam_i = S_ii / G_ii; IE = I + E.  The final pass
// (FINAL) also settles the short clusters by Rayleigh-Ritz, takes the resolved run on a
// clean boundary and decides whether the level is the last one; its scratch (flags and
// cluster list) exists only in that instantiation.  sepg: workspace for the neighbour
// separation flags of levels wider than kSepMax.
template <bool FINAL>
__device__ void refine_step(int m, int n, const double2* SG, int level0, int level,
                            double floor, const int* rot, double* lam, double* scan, double2* IE,
                            int* cid, double emax, unsigned char* sepg) {
  __shared__ double red[32];
  __shared__ int ired[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long ld = 2L * m;
  double mx = -1e300;
  for (int i = tid; i < m; i += nt) {
    double g = __ldcg(&SG[(long)i * ld + m + i].x);
    double l = g > 0 ? __ldcg(&SG[(long)i * ld + i].x) / g : 0.0;
    lam[i] = l;
    mx = fmax(mx, l);
  }
  const double v = block_max(mx, red);
  if (tid == 0 && level0) scan[4] = v;   // lam_0, kept for the later levels
  __syncthreads();
  const double l0 = level0 ? v : scan[4];
  // gaps below the FP64 rounding of the products with A (~n eps_64 lam_0) define no
  // eigenvectors
  const double fsep = 100.0 * n * 1.1e-16 * l0;
  int nl;
  double vf = v;
  if constexpr (!FINAL) {
    // the leading run above kTau lam_max (it only selects the pairs that take corrections)
    int f = m;
    for (int i = tid; i < m; i += nt)
      if (!(lam[i] > kTau * v)) f = min(f, i);
    nl = block_min_int(f, ired);
    fill_ie(m, SG, lam, IE, nl, fsep, emax, nullptr);
  } else {
    __shared__ unsigned char s_sep[kSepMax];
    __shared__ int s_cl0[kMaxClusters], s_cln[kMaxClusters];
    __shared__ int s_ncl;
    unsigned char* sep = m <= kSepMax ? s_sep : sepg;
    // columns at or below kTau lam_max go to the next level whatever happens here
    int f0 = m;
    for (int i = tid; i < m; i += nt)
      if (!(lam[i] > kTau * v)) f0 = min(f0, i);
    f0 = block_min_int(f0, ired);
    // neighbour separation, then the runs of unseparated neighbours that start above f0:
    // short ones become Ritz clusters (cid = first index), longer ones (or beyond
    // kMaxClusters) cid = -2
    for (int i = tid; i < m; i += nt) {
      sep[i] = (i + 1 < m) ? (pair_separated(SG, ld, m, lam, i, i + 1, fsep, kNewtonFinal) ? 1 : 0) : 1;
      cid[i] = -1;
    }
    __syncthreads();
    if (tid == 0) {
      int ncl = 0;
      for (int i = 0; i < f0;) {
        int j = i;
        while (j + 1 < m && !sep[j]) ++j;   // run [i, j]
        const int len = j - i + 1;
        if (len >= 2) {
          const bool ritz = len <= kRitzMax && ncl < kMaxClusters;
          if (ritz) {
            s_cl0[ncl] = i;
            s_cln[ncl] = len;
            ++ncl;
          }
          for (int t = i; t <= j; ++t) cid[t] = ritz ? i : -2;
        }
        i = j + 1;
      }
      s_ncl = ncl;
    }
    __syncthreads();
    // resolved run: every column above kTau lam_max and outside long runs, ending on a
    // clean boundary -- its last column separated from the first one left to the next
    // level (so the columns passed on carry no mixing with resolved ones)
    int f = m;
    for (int i = tid; i < m; i += nt)
      if (!(lam[i] > kTau * v) || cid[i] == -2) f = min(f, i);
    f = block_min_int(f, ired);
    int best = 0;
    for (int k = 1 + tid; k <= f; k += nt) {
      const bool clean = (k == m) || (sep[k - 1] && !(cid[k - 1] >= 0 && cid[k - 1] == cid[k]));
      if (clean) best = max(best, k);
    }
    nl = block_max_int(best, ired);
    fill_ie(m, SG, lam, IE, nl, fsep, emax, cid);
    __syncthreads();
    const int ncl = s_ncl;
    for (int q = 0; q < ncl; ++q) ritz_cluster(m, SG, s_cl0[q], s_cln[q], lam, IE);
    double mx2 = -1e300;
    for (int i = tid; i < m; i += nt) mx2 = fmax(mx2, lam[i]);
    vf = block_max(mx2, red);
  }
  double rst = 0.0;
  for (int i = nl + tid; i < m; i += nt) rst = fmax(rst, lam[i]);
  const double rest = block_max(rst, red);
  if (tid == 0) {
    scan[0] = vf;
    scan[1] = (double)nl;
    scan[2] = rest;
    if constexpr (FINAL) {
      if (level == 0) scan[3] = vf;
      const double top = scan[3];
      const bool last = (nl >= m) || (level + 1 >= kMaxLevels) || !(rest > floor * top) ||
                        nl == 0;
      scan[5] = rot ? (double)rot[3] : 0.0;
      scan[6] = last ? 1.0 : 0.0;
      scan[7] = last ? (double)m : (double)nl;
    }
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
    unsigned int* ticket, int splits, int* cid, double emax, unsigned char* sepg) {
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
  refine_step<false>(m, n, SG, level0, level, floor, rot, lam, scan, IE, cid, emax, sepg);
  if (threadIdx.x == 0) *ticket = 0u;
}

// The refinement step alone, on [S | G] formed by a separate product (one CTA).
__global__ void __launch_bounds__(RT * RT) refine_kernel(int m, int n, const double2* SG,
                                                         int level0, int final_pass, int level,
                                                         double floor, const int* rot, double* lam,
                                                         double* scan, double2* IE, int* cid,
                                                         double emax, unsigned char* sepg) {
  if (final_pass)
    refine_step<true>(m, n, SG, level0, level, floor, rot, lam, scan, IE, cid, emax, sepg);
  else
    refine_step<false>(m, n, SG, level0, level, floor, rot, lam, scan, IE, cid, emax, sepg);
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
// With P != NULL the product was formed already (P: n x m, row stride ldp) and is only routed.
__global__ void __launch_bounds__(RT * RT) level_out_kernel(
    int n, int m, const double2* __restrict__ Z, long ldz, const double2* __restrict__ IE,
    const double* scan, const double* lam, double2* v, long ldv, double* w, int off,
    double2* x, double* hscan, const double2* __restrict__ P, long ldp) {
  __shared__ double2 As[RT][RT + 1];   // [k][row]
  __shared__ double2 Bs[RT][RT + 1];   // [k][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
  const int r0 = blockIdx.y * RT, j0 = blockIdx.x * RT;
  const bool last = scan[6] != 0.0;
  const int nl = (int)scan[1];
  const int take = last ? m : nl;
  const int mr = m - nl;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; P == nullptr && k0 < m; k0 += RT) {
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
  if (P != nullptr && r < n && j < m) acc = P[(long)r * ldp + j];
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

// Products with FP64 results of the solver: error-free BF16 slice products on the tensor
// cores (carried to ~2^-48 of each operand row's largest entry, summed in FP64) when the
// caller lent their workspace and the product is large enough; CUDA-core FP64 otherwise.
bool tc_route(const MixWork& wk, long m, long n, long k, int batch) {
  return wk.tcws != nullptr && (double)m * n * k * batch >= wk.tc_min_macs && m >= 16 && n >= 16;
}

// Unit norm for the columns a level emits (v[:, off + j], j < the level's take): the last
// pass leaves norm errors of order its corrections squared.  One CTA per column.
__global__ void __launch_bounds__(128) normalize_out_kernel(int n, int m, const double* scan,
                                                            double2* v, long ldv, int off) {
  __shared__ double red[4];
  const bool last = scan[6] != 0.0;
  const int take = last ? m : (int)scan[1];
  const int j = blockIdx.x;
  if (j >= take) return;
  double2* col = v + off + j;
  double ss = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) ss += cabs2(col[(long)r * ldv]);
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  const double t = red[0] + red[1] + red[2] + red[3];
  if (!(t > 0.0)) return;
  const double sc = 1.0 / sqrt(t);
  for (int r = threadIdx.x; r < n; r += blockDim.x) col[(long)r * ldv] = cscale(col[(long)r * ldv], sc);
}

cudaError_t gemm64(cudaStream_t st, const MixWork& wk, int opa, int opb, int m, int n, int k,
                   const double2* A, long lda, long sa, const double2* B, long ldb, long sb,
                   double2* C, long ldc, long sc, int batch) {
  if (tc_route(wk, m, n, k, batch))
    return tc_cgemm_exact<double2, double2>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc,
                                            sc, batch, wk.tcws, wk.tcws_bytes, wk.tcerr);
  return cgemm<double>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch,
                       make_double2(1, 0), make_double2(0, 0));
}

// FP64 basis times FP32 rotations.
cudaError_t gemm64x(cudaStream_t st, const MixWork& wk, int m, int n, int k, const double2* A,
                    long lda, const float2* B, long ldb, double2* C, long ldc) {
  if (tc_route(wk, m, n, k, 1))
    return tc_cgemm_exact<double2, float2>(st, OP_N, OP_N, m, n, k, A, lda, 0, B, ldb, 0, C, ldc,
                                           0, 1, wk.tcws, wk.tcws_bytes, wk.tcerr);
  return cgemm_dx(st, OP_N, OP_N, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1);
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
  return 8 * sq * sizeof(double2) + 2 * sq * sizeof(float2) + 6 * (size_t)n_cap * 8 +
         eig_work_bytes<float>(n_cap) + 12 * 256;
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
  w.cid = reinterpret_cast<int*>(take((size_t)n_cap * sizeof(int)));
  w.sepf = reinterpret_cast<unsigned char*>(take((size_t)n_cap));
  eig_work_bind<float>(w.ew, take(eig_work_bytes<float>(n_cap)), n_cap);
}

namespace {
// refinement passes of a level and the angle bound of pass p (kNewtonFinal in the last)
inline int level_passes(int m) { return m > kThreePassMin ? 3 : 2; }
inline double pass_bound(int passes, int p) {
  if (p + 1 == passes) return kNewtonFinal;
  return (passes == 3 && p == 0) ? kNewtonWide : kNewtonMax;
}

// Floating-point work of one level's products (8 real flops per complex multiply-add).
double level_flops(int n, int m, bool lev0) {
  auto g = [](int a, int b, int c) { return 8.0 * a * b * (double)c; };
  double f = 0.0;
  if (!lev0) f += g(n, m, n) + g(m, m, n) + g(n, m, m);   // X^+ A X and Z = X Y
  f += g(n, m, n);                                          // T = A Z
  const int passes = level_passes(m);
  for (int pass = 0; pass < passes; ++pass) {
    f += g(m, 2 * m, n);                                    // [S | G]
    f += (pass + 1 < passes) ? 2 * g(n, m, m) : g(n, m, m); // [T | Z] (I + E) or Z (I + E)
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
    MPDO_CUDA_TRY(gemm64(st, wk, OP_N, OP_N, n, m, n, a, lda, 0, wk.x, m, 0, T, l2, 0, 1));
    MPDO_CUDA_TRY(gemm64(st, wk, OP_C, OP_N, m, m, n, wk.x, m, 0, T, l2, 0, wk.s, m, 0, 1));
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
      MPDO_CUDA_TRY(gemm64x(st, wk, n, m, m, wk.x, m, wk.y32, m, Z, l2));
    }
  } else {
    MPDO_CUDA_TRY((convert<double, float>(st, m, m, B, ldbm, wk.a32, m)));
    // block Jacobi: large m needs more than 20 sweeps to converge (it stops once no pair rotates)
    MPDO_CUDA_TRY(heig<float>(st, m, wk.a32, m, wk.y32, m, wk.w32, wk.ew, 40));
    if (lev0)
      MPDO_CUDA_TRY((convert<float, double>(st, n, m, wk.y32, m, Z, l2)));
    else
      MPDO_CUDA_TRY(gemm64x(st, wk, n, m, m, wk.x, m, wk.y32, m, Z, l2));
  }
  MPDO_CUDA_TRY(gemm64(st, wk, OP_N, OP_N, n, m, n, a, lda, 0, Z, l2, 0, T, l2, 0, 1));
  double2* cur = wk.tz;
  double2* nxt = wk.tz2;
  const dim3 gsg((2 * m + RT - 1) / RT, (m + RT - 1) / RT);
  const int splits = split_count((long)gsg.x * gsg.y, n);
  // [S | G] = Z^+ [T | Z] and the refinement step: one fused CUDA-core launch (passes before
  // the last), or the product followed by a one-CTA step
  const bool tc_sg = tc_route(wk, m, 2L * m, n, 1);
  const int passes = level_passes(m);
  for (int pass = 0; pass < passes; ++pass) {
    const int final_pass = (pass + 1 == passes);
    const double emax = pass_bound(passes, pass);
    if (tc_sg || final_pass) {
      // the final pass's step (Ritz clusters, level decisions) runs as its own one-CTA
      // launch, so the fused product keeps the light step's small footprint
      MPDO_CUDA_TRY(gemm64(st, wk, OP_C, OP_N, m, 2 * m, n, cur + m, l2, 0, cur, l2, 0, wk.s, l2,
                           0, 1));
      count_launch();
      refine_kernel<<<1, RT * RT, 0, st>>>(m, n, wk.s, (lev0 && pass == 0) ? 1 : 0, final_pass,
                                           level, floor, (const int*)wk.ew.counters, wk.lam,
                                           wk.scan, wk.ie, wk.cid, emax, wk.sepf);
      MPDO_CUDA_TRY(cudaGetLastError());
    } else {
      count_launch();
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
                                       wk.ticket, splits, wk.cid, emax, wk.sepf));
    }
    if (!final_pass) {
      // [T | Z] (I + E): two products sharing the right factor (batch of 2, offset m)
      MPDO_CUDA_TRY(gemm64(st, wk, OP_N, OP_N, n, m, m, cur, l2, m, wk.ie, m, 0, nxt, l2, m, 2));
      std::swap(cur, nxt);
    } else {
      // Z (I + E), fused with the routing on the CUDA cores, or formed on the tensor cores
      // (into the free half of the other buffer) and then routed
      const double2* P = nullptr;
      if (tc_route(wk, n, m, m, 1)) {
        MPDO_CUDA_TRY(gemm64(st, wk, OP_N, OP_N, n, m, m, cur + m, l2, 0, wk.ie, m, 0, nxt, l2, 0,
                             1));
        P = nxt;
      }
      count_launch();
      const dim3 gout((m + RT - 1) / RT, (n + RT - 1) / RT);
      level_out_kernel<<<gout, RT * RT, 0, st>>>(n, m, cur + m, l2, wk.ie, wk.scan, wk.lam, v,
                                                 ldv, w, n - m, wk.x, wk.hpin_dev, P, l2);
      MPDO_CUDA_TRY(cudaGetLastError());
      count_launch();
      normalize_out_kernel<<<m, 128, 0, st>>>(n, m, wk.scan, v, ldv, n - m);
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
  if (wk.tcws) MPDO_CUDA_TRY(tc_exact_init());   // outside any capture below
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
