// Elementwise and small kernels of the MPDO update, observables and sampling.
// Every kernel here is memory- or latency-bound; the contractions are in gemm.cu.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace mpdo {
namespace {

inline int nblocks(long total, int threads = 256, int cap = 16384) {
  long b = (total + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// out[i0][i2][i1][i3] = in[i0][i1][i2][i3]
template <typename T>
__global__ void swap12_kernel(long n0, long n1, long n2, long n3, const T* __restrict__ in,
                              T* __restrict__ out) {
  long total = n0 * n1 * n2 * n3;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long i3 = e % n3;
    long r = e / n3;
    long i1 = r % n1;
    r /= n1;
    long i2 = r % n2;
    long i0 = r / n2;
    // e enumerates the OUTPUT [i0][i2][i1][i3]
    out[e] = in[((i0 * n1 + i1) * n2 + i2) * n3 + i3];
  }
}

// site [l][s][k][r] -> [r][s][k][l]
template <typename T>
__global__ void reverse_site_kernel(int dl, int d, int k, int dr, const T* __restrict__ in,
                                    T* __restrict__ out) {
  long total = (long)dl * d * k * dr;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    // output index [r][s][k][l]
    long l = e % dl;
    long t = e / dl;
    long kk = t % k;
    t /= k;
    long s = t % d;
    long r = t / d;
    out[e] = in[((l * d + s) * k + kk) * dr + r];
  }
}

// A[l][s][k][r] <- sum_s' U[s][s'] A[l][s'][k][r]
template <typename R>
__global__ void one_site_kernel(int dl, int k, int dr, const cx<R>* __restrict__ u,
                                cx<R>* a) {
  long plane = (long)k * dr;
  long total = (long)dl * plane;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long l = e / plane, q = e % plane;
    cx<R>* base = a + l * 3 * plane + q;
    cx<R> x0 = base[0], x1 = base[plane], x2 = base[2 * plane];
    for (int s = 0; s < 3; ++s) {
      cx<R> acc = mkc<R>(0, 0);
      cfma(acc, u[s * 3 + 0], x0);
      cfma(acc, u[s * 3 + 1], x1);
      cfma(acc, u[s * 3 + 2], x2);
      base[s * plane] = acc;
    }
  }
}

template <typename R>
__global__ void product_state_kernel(cx<R> v0, cx<R> v1, cx<R> v2, cx<R>* base, long stride,
                                     int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    base[i * stride + 0] = v0;
    base[i * stride + 1] = v1;
    base[i * stride + 2] = v2;
  }
}

// rs/irs from the left-Gram spectrum sigma (descending): numerical rank cut.
template <typename R>
__global__ void gram_mask_kernel(int n, const double* __restrict__ sig, double gtol,
                                 R* rs, R* irs, StepScalars* sc) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  double s0 = sig[0];
  bool bad = !(s0 > 0.0) || !isfinite(s0);
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double s = sig[c];
    if (!bad && s > gtol * s0) {
      rs[c] = (R)sqrt(s);
      irs[c] = (R)(1.0 / sqrt(s));
      atomicAdd(&cnt, 1);
    } else {
      rs[c] = 0;
      irs[c] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sc->rank_g = cnt;
    // first flag write of an update: starts the update's flags afresh
    sc->flags = bad ? 1 : 0;
  }
}

// R[c][x] = rs[c] conj(V[x][c]); Vs[x][c] = V[x][c] irs[c]; Vr[x][c] = V[x][c] rs[c]
template <typename R>
__global__ void gram_factor_kernel(int n, const cx<R>* __restrict__ v, const R* __restrict__ rs,
                                   const R* __restrict__ irs, cx<R>* rmat, cx<R>* vs, cx<R>* vr) {
  long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int x = (int)(e / n), c = (int)(e % n);
    cx<R> val = v[e];
    vs[e] = cscale(val, irs[c]);
    vr[e] = cscale(val, rs[c]);
    rmat[(long)c * n + x] = cscale(cconj(val), rs[c]);
  }
}

// Phi[(S,s,b),(S2,s2,b2)] = sum_{t,t2} C[(S,s,t),(S2,s2,t2)] Gj[(b,t),(b2,t2)]
template <typename R>
__global__ void build_phi_kernel(int dm, const cx<R>* __restrict__ ct,
                                 const cx<R>* __restrict__ gj, cx<R>* phi) {
  long n = 9L * dm;
  long total = n * n;
  long ldg = 3L * dm;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long row = e / n, col = e % n;
    int ss = (int)(row / dm), b = (int)(row % dm);     // ss = S*3 + s
    int ss2 = (int)(col / dm), b2 = (int)(col % dm);
    cx<R> acc = mkc<R>(0, 0);
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int t2 = 0; t2 < 3; ++t2)
        cfma(acc, ct[(ss * 3 + t) * 27 + ss2 * 3 + t2], gj[(b * 3 + t) * ldg + b2 * 3 + t2]);
    phi[e] = acc;
  }
}

// Bond cut on the spectrum lam (descending, n): keep <= chi values above htol*lam0.
// The total weight is the trace of the matrix itself (noise-free in expectation), not
// the sum of the positive computed eigenvalues, which is biased upward by the noise floor.
template <typename R>
__global__ void bond_select_kernel(int n, const double* __restrict__ lam, const cx<R>* __restrict__ hm,
                                   long ldh, double htol, int chi, StepScalars* sc, DevStats* st) {
  __shared__ double red_tot[256], red_kept[256];
  __shared__ int s_keep;
  double l0 = lam[0];
  bool bad = !(l0 > 0.0) || !isfinite(l0);
  if (threadIdx.x == 0) {
    int k = 0;
    if (!bad) {
      while (k < n && k < chi && lam[k] > htol * l0) ++k;
    }
    if (k < 1) k = 1;
    s_keep = k;
  }
  __syncthreads();
  int keep = s_keep;
  double t = 0, kp = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    t += (double)hm[(long)i * ldh + i].x;
    if (i < keep) kp += lam[i] > 0 ? lam[i] : 0.0;
  }
  red_tot[threadIdx.x] = t;
  red_kept[threadIdx.x] = kp;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red_tot[threadIdx.x] += red_tot[threadIdx.x + s];
      red_kept[threadIdx.x] += red_kept[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tot = red_tot[0], kept = red_kept[0];
    sc->keep = keep;
    sc->tot = tot;
    sc->kept = kept;
    sc->renorm = (kept > 0) ? sqrt(tot / kept) : 0.0;
    if (bad || !(kept > 0) || !isfinite(tot)) sc->flags |= 1;
    st->disc_bond_w += (tot > 0) ? (tot - kept) / tot : 0.0;
    if (keep > st->chi_used_max) st->chi_used_max = keep;
    st->n_updates += 1;
  }
}

// Q[(b',T,m),(b,t)] = renorm * sum_{S,s} conj(W[(S,s,b)][b']) E[m][(S,T),(s,t)]
template <typename R>
__global__ void make_q_kernel(int dm, int keep, int m_ops, const cx<R>* __restrict__ w,
                              const cx<R>* __restrict__ e, const StepScalars* sc, cx<R>* q) {
  long cols = 3L * dm;
  long rows = (long)keep * 3 * m_ops;
  long total = rows * cols;
  R ren = (R)sc->renorm;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    long row = idx / cols, col = idx % cols;
    int m = (int)(row % m_ops);
    long r2 = row / m_ops;
    int T = (int)(r2 % 3);
    int bp = (int)(r2 / 3);
    int b = (int)(col / 3), t = (int)(col % 3);
    const cx<R>* em = e + (long)m * 81;
    cx<R> acc = mkc<R>(0, 0);
#pragma unroll
    for (int S = 0; S < 3; ++S)
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        cx<R> wv = w[((long)(S * 3 + s) * dm + b) * keep + bp];
        cfma(acc, cconj(wv), em[(S * 3 + T) * 9 + s * 3 + t]);
      }
    q[idx] = cscale(acc, ren);
  }
}

// Inner-index cut + purity-preserving truncation (Sec. III.D Eqs. xiformula / ppt with
// T = 1, P = identity; theta = 0 when infeasible; clamp negatives; keep the trace).
// Writes f[k] = sqrt(Lambda~_k / w_k) for k < kk.
// Partial sums of tr W (diagonal real parts) and ||W||_F^2 over the n x n matrix wm, one pair
// per CTA of a fixed grid (kNormBlocks), so the final sum is deterministic.
constexpr int kNormBlocks = 64;
template <typename R>
__global__ void __launch_bounds__(256) gram_norms_kernel(int n, const cx<R>* __restrict__ wm,
                                                         double* parts) {
  __shared__ double rt[256], rf[256];
  double t = 0, f2 = 0;
  const long total = (long)n * n;
  for (long e = blockIdx.x * 256L + threadIdx.x; e < total; e += 256L * kNormBlocks) {
    const cx<R> v = wm[e];
    f2 += (double)v.x * v.x + (double)v.y * v.y;
    if (e / n == e % n) t += (double)v.x;
  }
  rt[threadIdx.x] = t;
  rf[threadIdx.x] = f2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rt[threadIdx.x] += rt[threadIdx.x + s];
      rf[threadIdx.x] += rf[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    parts[2 * blockIdx.x] = rt[0];
    parts[2 * blockIdx.x + 1] = rf[0];
  }
}

template <typename R>
__global__ void kraus_select_kernel(int n, const double* __restrict__ w, const double* parts,
                                    double kcut, int kmax, int use_ppt, double* f,
                                    StepScalars* sc, DevStats* st, double* trace) {
  // total weight tr W and sum of squared weights ||W||_F^2 (= sum w^2 for the Hermitian W,
  // whatever part of its spectrum was resolved), from the matrix in FP64: the per-CTA partial
  // sums of gram_norms_kernel, added here in a fixed order
  __shared__ double red_t[kNormBlocks], red_f[kNormBlocks];
  if (threadIdx.x < kNormBlocks) {
    red_t[threadIdx.x] = parts[2 * threadIdx.x];
    red_f[threadIdx.x] = parts[2 * threadIdx.x + 1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 1; b < kNormBlocks; ++b) {
      red_t[0] += red_t[b];
      red_f[0] += red_f[b];
    }
  }
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double w0 = w[0] > 0 ? w[0] : 0.0;
  bool bad = !(w0 > 0.0) || !isfinite(w0);
  int kk = 0;
  if (!bad) {
    double thr = kcut * kcut * w0;
    while (kk < n && kk < kmax && w[kk] > thr) ++kk;
  }
  if (kk < 1) kk = 1;
  double sum = red_t[0], sq = red_f[0], sumk = 0, sqk = 0;
  for (int i = 0; i < kk; ++i) {
    double v = w[i] > 0 ? w[i] : 0.0;
    sumk += v;
    sqk += v * v;
  }
  // The trace the truncation keeps (reading A2) is carried in FP64 across updates: the
  // channel multiplies it by tr(theta')/tr(theta) of this block (bond total sc->tot over
  // sc->trpre, both FP64 sums of the same stored tensors), so rounding of the stored
  // tensors and of the products that form the new centre does not accumulate in the norm.
  double target = sum;
  if (trace && sc->trpre > 0 && sc->tot > 0 && isfinite(*trace)) {
    target = *trace * (sc->tot / sc->trpre);
    *trace = target;
  }

  double theta = 0.0;
  int infeas = 0, clamped = 0;
  double lt[1024];
  if (use_ppt && !bad) {
    double nl = sqrt(sq), nlp = sqrt(sqk);
    double nt = sqrt((double)n), ntp = sqrt((double)kk);
    double cos_phi = sum / (nl * nt);
    double cos_sig = sumk / (nlp * ntp);
    if (cos_sig > 1.0) cos_sig = 1.0;
    double ratio = nt * cos_phi / ntp;
    if (ratio > 1.0) { infeas = 1; theta = 0.0; } else { theta = acos(ratio); }
    double sigma = acos(cos_sig);
    double x = (sigma == 0.0) ? 0.0 : tan(theta) / tan(sigma) - 1.0;
    double lsum = 0;
    for (int i = 0; i < kk; ++i) {
      double lp = w[i] > 0 ? w[i] : 0.0;
      double v = (sigma == 0.0) ? lp : lp + x * (lp - nlp * cos_sig / ntp);
      if (v < 0) { v = 0; ++clamped; }
      lt[i] = v;
      lsum += v;
    }
    double sc_tr = (lsum > 0) ? target / lsum : 0.0;
    for (int i = 0; i < kk; ++i) lt[i] *= sc_tr;
  } else {
    double sc_tr = (sumk > 0) ? target / sumk : 0.0;
    for (int i = 0; i < kk; ++i) lt[i] = (w[i] > 0 ? w[i] : 0.0) * sc_tr;
  }
  for (int i = 0; i < kk; ++i) {
    double wi = w[i];
    f[i] = (wi > 0) ? sqrt(lt[i] / wi) : 0.0;
  }
  sc->kkeep = kk;
  sc->ktot = sum;
  sc->theta = theta;
  sc->infeasible = infeas;
  sc->clamped = clamped;
  if (bad) sc->flags |= 1;
  st->disc_kraus_w += (sum > 0) ? (sum - sumk) / sum : 0.0;
  if (use_ppt && theta < st->ppt_theta_min) st->ppt_theta_min = theta;
  st->ppt_infeasible += infeas;
  st->ppt_clamped += clamped;
  if (kk > st->k_used_max) st->k_used_max = kk;
}

// ||theta||^2 of the two-site block before the channel, from the two Gram matrices:
// sum_{s,b,b'} G_i[(s,b'),(s,b)] sum_t G_j[(b,t),(b',t)]  (G_i, G_j: 3D x 3D, index s*D+b
// resp. b*3+t), accumulated in FP64 into sc->trpre.  One CTA.
template <typename R>
__global__ void trace_pre_kernel(int dm, const cx<R>* __restrict__ gi, const cx<R>* __restrict__ gj,
                                 StepScalars* sc) {
  __shared__ double red[256];
  const long n3 = 3L * dm;
  double t = 0;
  for (long e = threadIdx.x; e < (long)dm * dm; e += blockDim.x) {
    const int b = (int)(e / dm), bp = (int)(e % dm);
    double gtr = 0, gti = 0;
    for (int q = 0; q < 3; ++q) {
      const cx<R> v = gj[(long)(b * 3 + q) * n3 + bp * 3 + q];
      gtr += (double)v.x;
      gti += (double)v.y;
    }
    for (int s = 0; s < 3; ++s) {
      const cx<R> v = gi[(long)(s * dm + bp) * n3 + s * dm + b];
      t += (double)v.x * gtr - (double)v.y * gti;
    }
  }
  red[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) sc->trpre = red[0];
}

// out = sum |a_e|^2 over n complex entries, in FP64 (one CTA; the norm of the centre site).
template <typename R>
__global__ void sumsq_kernel(long n, const cx<R>* __restrict__ a, double* out) {
  __shared__ double red[256];
  double t = 0;
  for (long e = threadIdx.x; e < n; e += blockDim.x) {
    const cx<R> v = a[e];
    t += (double)v.x * v.x + (double)v.y * v.y;
  }
  red[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// out = in with its 6 axes reordered: out axis i is in axis perm[i] (dims of in: d[0..5]).
template <typename T>
__global__ void permute6_kernel(const T* __restrict__ in, T* __restrict__ out, int d0, int d1,
                                int d2, int d3, int d4, int d5, int p0, int p1, int p2, int p3,
                                int p4, int p5) {
  const int d[6] = {d0, d1, d2, d3, d4, d5};
  const int p[6] = {p0, p1, p2, p3, p4, p5};
  long st[6];
  st[5] = 1;
  for (int i = 4; i >= 0; --i) st[i] = st[i + 1] * d[i + 1];
  const long total = st[0] * d[0];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long rem = e, off = 0;
    for (int i = 5; i >= 0; --i) {
      const int od = d[p[i]];
      const long idx = rem % od;
      rem /= od;
      off += idx * st[p[i]];
    }
    out[e] = in[off];
  }
}

// R[(a,b)][s][s'][(r,r')] (a, b < dl; s, s' < 3; r, r' < dr): mode 0 keeps it, mode 1 zeroes
// the blocks s != s' (the diagonal transfer of the collision probability), mode 2 writes the
// trace over s into tr[(a,b)][(r,r')] instead.
template <typename T>
__global__ void rho_site_kernel(long dl2, long dr2, T* r, T* tr, int mode) {
  const long total = dl2 * 9 * dr2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long q = e % dr2, ss = (e / dr2) % 9, ab = e / (9 * dr2);
    const int s = (int)(ss / 3), s2 = (int)(ss % 3);
    if (mode == 1) {
      if (s != s2) { r[e].x = 0; r[e].y = 0; }
    } else if (mode == 2 && s == 0 && s2 == 0) {
      T v = r[e];
      const T v1 = r[e + 4 * dr2], v2 = r[e + 8 * dr2];
      v.x += v1.x + v2.x;
      v.y += v1.y + v2.y;
      tr[ab * dr2 + q] = v;
    }
  }
}

// Deterministic FP64 contractions of environments into parts[blockIdx]: mode 0:
// sum_e Re(x[e] y[e]); mode 1: sum_{(ab),(cd)} Re(c[(ab),(cd)] u[ab] u[cd]) with n2 = dim of
// (ab).  A second pass (one CTA) adds the parts in order.
template <typename T>
__global__ void __launch_bounds__(256) env_dot_kernel(long n2, const T* __restrict__ x,
                                                      const T* __restrict__ y, int mode,
                                                      double* parts) {
  __shared__ double red[256];
  double t = 0;
  const long total = mode == 0 ? n2 : n2 * n2;
  for (long e = blockIdx.x * 256L + threadIdx.x; e < total; e += 256L * gridDim.x) {
    if (mode == 0) {
      t += (double)x[e].x * y[e].x - (double)x[e].y * y[e].y;
    } else {
      const long i = e / n2, j = e % n2;
      // c[(ab),(cd)] u[ab] u[cd]
      const double ur = (double)y[i].x * y[j].x - (double)y[i].y * y[j].y;
      const double ui = (double)y[i].x * y[j].y + (double)y[i].y * y[j].x;
      t += (double)x[e].x * ur - (double)x[e].y * ui;
    }
  }
  red[threadIdx.x] = t;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = red[0];
}
__global__ void sum_parts_kernel(int n, const double* parts, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += parts[i];
    *out = s;
  }
}

// Vks[kappa][k] = V[kappa][k] * f[k], k < kk (V has leading dimension ldv)
template <typename R, typename RO>
__global__ void scale_vk_kernel(int n, int kk, const cx<R>* __restrict__ v, long ldv,
                                const double* __restrict__ f, cx<RO>* out) {
  long total = (long)n * kk;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int r = (int)(e / kk), c = (int)(e % kk);
    cx<R> t = cscale(v[(long)r * ldv + c], (R)f[c]);
    out[e] = mkc<RO>((RO)t.x, (RO)t.y);
  }
}

// Energy automaton, one-site step: from F0, FZ, F1 (= env^T A for the three states)
// form G0 = P F0, GZ = Z F0, G1 = P F1 + (-h X - bJ Z) F0 - J Z FZ on the s index.
// Layout of F*: [l'][s][k][r] with plane = k*dr; proj = 1 uses P = |0><0|+|1><1|,
// proj = 0 uses the identity.  Six automata are stacked: [0..2] projected, [3..5] raw.
template <typename R>
__global__ void energy_mix_kernel(int dl, int plane, const cx<R>* __restrict__ f, long fstride,
                                  cx<R>* g, long gstride, double J, double hx, double bz) {
  long total = (long)dl * plane;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long l = e / plane, q = e % plane;
    long off = l * 3 * plane + q;
    for (int proj = 1; proj >= 0; --proj) {
      int base = proj ? 0 : 3;
      const cx<R>* f0 = f + (base + 0) * fstride + off;
      const cx<R>* fz = f + (base + 1) * fstride + off;
      const cx<R>* f1 = f + (base + 2) * fstride + off;
      cx<R>* g0 = g + (base + 0) * gstride + off;
      cx<R>* gz = g + (base + 1) * gstride + off;
      cx<R>* g1 = g + (base + 2) * gstride + off;
      cx<R> a0 = f0[0], a1 = f0[plane], a2 = f0[2 * plane];
      cx<R> z0 = fz[0], z1 = fz[plane];
      cx<R> b0 = f1[0], b1 = f1[plane], b2 = f1[2 * plane];
      // G0
      g0[0] = a0;
      g0[plane] = a1;
      g0[2 * plane] = proj ? mkc<R>(0, 0) : a2;
      // GZ: Z = diag(1, -1, 0)
      gz[0] = a0;
      gz[plane] = cscale(a1, R(-1));
      gz[2 * plane] = mkc<R>(0, 0);
      // G1 = P F1 + (-h X - bJ Z) F0 - J Z FZ  (X swaps s' <- s on the qubit levels)
      R h = (R)hx, bj = (R)(bz * J), jj = (R)J;
      cx<R> o0 = cadd(b0, cadd(cscale(a1, -h), cscale(a0, -bj)));
      o0 = cadd(o0, cscale(z0, -jj));
      cx<R> o1 = cadd(b1, cadd(cscale(a0, -h), cscale(a1, bj)));
      o1 = cadd(o1, cscale(z1, jj));
      g1[0] = o0;
      g1[plane] = o1;
      g1[2 * plane] = proj ? mkc<R>(0, 0) : b2;
    }
  }
}

// ----------------------------------------------------------------- sampling
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                             uint32_t& c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
  uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

// Philox4x32-10 (Salmon et al., SC'11) on counter (site, sample, 0, 0), key = seed.
__device__ double philox_uniform(uint64_t seed, uint32_t sample, uint32_t site) {
  uint32_t c0 = site, c1 = sample, c2 = 0, c3 = 0;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
  uint64_t v = ((uint64_t)c0 << 21) | (uint64_t)(c1 >> 11);
  return (double)v * 0x1.0p-53;
}

// q[smp][v] = sum_{r,r'} Ev[smp][v][r][r'] Rt[r][r'] ; pick v; copy chosen env.
template <typename R>
__global__ void sample_pick_kernel(int dr, const cx<R>* __restrict__ ev, const cx<R>* __restrict__ rt,
                                   uint64_t seed, int site, int site_user, int n_sites,
                                   cx<R>* env_out, uint8_t* bits, double* probs, int last) {
  int smp = blockIdx.x;
  long plane = (long)dr * dr;
  const cx<R>* base = ev + (long)smp * 3 * plane;
  __shared__ double red[3][256];
  double q[3] = {0, 0, 0};
  for (long e = threadIdx.x; e < plane; e += blockDim.x) {
    cx<R> rv = rt[e];
    for (int v = 0; v < 3; ++v) {
      cx<R> x = base[v * plane + e];
      q[v] += (double)x.x * rv.x - (double)x.y * rv.y;
    }
  }
  for (int v = 0; v < 3; ++v) red[v][threadIdx.x] = q[v];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 3; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  __shared__ int pick;
  if (threadIdx.x == 0) {
    double q0 = red[0][0] > 0 ? red[0][0] : 0, q1 = red[1][0] > 0 ? red[1][0] : 0,
           q2 = red[2][0] > 0 ? red[2][0] : 0;
    double tot = q0 + q1 + q2;
    double u = philox_uniform(seed, (uint32_t)smp, (uint32_t)site_user);
    int v = 2;
    if (u < q0 / tot) v = 0;
    else if (u < (q0 + q1) / tot) v = 1;
    pick = v;
    bits[(long)smp * n_sites + site_user] = (uint8_t)v;
    if (last) {
      double pv = (v == 0) ? red[0][0] : (v == 1 ? red[1][0] : red[2][0]);
      probs[smp] = pv;
    }
  }
  __syncthreads();
  const cx<R>* src = base + pick * plane;
  for (long e = threadIdx.x; e < plane; e += blockDim.x) env_out[(long)smp * plane + e] = src[e];
}

// Newton-Schulz polar step for a near-isometry A with Gram G = A^+A (n x n):
// P = (3I - G)/2 (applied to A) and Q = (I + G)/2 (applied to the other factor), so that
// A P has unit Gram to second order and (A P)(Q B) = A B - A E^2 B / 4 with E = G - I.
template <typename R>
__global__ void polar_factors_kernel(int n, const cx<R>* __restrict__ g, cx<R>* pm, cx<R>* qm) {
  long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    cx<R> v = g[e];
    R d = (i == j) ? R(1) : R(0);
    pm[e] = mkc<R>((R)1.5 * d - (R)0.5 * v.x, (R)(-0.5) * v.y);
    qm[e] = mkc<R>((R)0.5 * d + (R)0.5 * v.x, (R)0.5 * v.y);
  }
}

// Inner-index truncation through the dual Gram W' = B^+B (used when B has fewer columns
// than rows): with W' y_k = w_k y_k, the kept rows of the new centre are
// f_k x_k^+ B = f_k sqrt(w_k) y_k^+  (x_k = B y_k / sqrt(w_k)), so no product with B is needed.
template <typename R, typename RO>
__global__ void dual_rows_kernel(int kk, int cols, const cx<R>* __restrict__ y, long ldy,
                                 const double* __restrict__ f, const double* __restrict__ w,
                                 cx<RO>* out) {
  long total = (long)kk * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int k = (int)(e / cols), c = (int)(e % cols);
    double wk = w[k] > 0 ? w[k] : 0.0;
    R sc = (R)(f[k] * sqrt(wk));
    cx<R> t = cscale(cconj(y[(long)c * ldy + k]), sc);
    out[e] = mkc<RO>((RO)t.x, (RO)t.y);
  }
}

// Pivoted Cholesky of the Hermitian PSD n x n matrix w (precision R, n <= 1024): W ~ L L^+
// with L n x r (row-major, row stride lr), greedy diagonal pivoting, stopping once the
// largest remaining diagonal is <= tol * tr W or after rmax (<= 128) columns.
// *rout = r; *resid = largest remaining diagonal / tr W.
// The rows are shared out over the CTAs of a thread-block cluster (row i belongs to rank
// i mod S; FP64 runs at 2 FMA per clock per SM, so the column updates want several SMs).
// Per column, one cluster barrier: each CTA posts its best remaining diagonal in shared
// memory (two slots, alternating by column, so a slot is rewritten only after every CTA
// has passed the next barrier), then every CTA reads all posts through distributed shared
// memory and takes the same pivot.  Sums and the pivot choice follow rank order, so the
// factor does not depend on scheduling.
template <typename R>
__global__ void __launch_bounds__(1024) pchol_kernel(int n, const cx<R>* __restrict__ w,
                                                     int rmax, double tol, cx<R>* L, int lr,
                                                     int* rout, double* resid) {
  using T = cx<R>;
  cg::cluster_group cluster = cg::this_cluster();
  const int S = (int)cluster.num_blocks(), c = (int)cluster.block_rank();
  __shared__ double d[1024];        // remaining diagonal of this CTA's rows (local index)
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ T lp[128];
  __shared__ double post_v[2];      // this CTA's best remaining diagonal, by column parity
  __shared__ int post_i[2];
  __shared__ double post_tr;        // this CTA's share of the trace
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int nloc = (n - c + S - 1) / S;   // rows c, c + S, ...
  double tp = 0.0;
  for (int li = tid; li < nloc; li += blockDim.x) {
    const int i = c + li * S;
    double v = (double)w[(long)i * n + i].x;
    d[li] = v > 0 ? v : 0.0;
    tp += d[li];
  }
  for (int o = 16; o > 0; o >>= 1) tp += __shfl_xor_sync(0xffffffffu, tp, o);
  if (lane == 0) rv[wid] = tp;
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int k = 0; k < nw; ++k) t += rv[k];
    post_tr = t;
  }
  cluster.sync();
  double tr = 0.0;
  for (int q = 0; q < S; ++q) tr += *cluster.map_shared_rank(&post_tr, q);
  int r = 0;
  double last = 0.0;
  for (int j = 0; j < rmax; ++j) {
    const int par = j & 1;
    double bv = -1.0;
    int bi = -1;
    for (int li = tid; li < nloc; li += blockDim.x)
      if (d[li] > bv) { bv = d[li]; bi = c + li * S; }
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi >= 0 && (bi < 0 || oi < bi))) { bv = ov; bi = oi; }
    }
    if (lane == 0) { rv[wid] = bv; ri[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = -1;
      for (int k = 0; k < nw; ++k)
        if (rv[k] > b || (rv[k] == b && ri[k] >= 0 && (p < 0 || ri[k] < p))) { b = rv[k]; p = ri[k]; }
      post_v[par] = b;
      post_i[par] = p;
    }
    cluster.sync();   // posts of column j complete; columns < j of L visible
    double dp = -1.0;
    int p = -1;
    for (int q = 0; q < S; ++q) {
      const double v = cluster.map_shared_rank(post_v, q)[par];
      const int i = cluster.map_shared_rank(post_i, q)[par];
      if (v > dp || (v == dp && i >= 0 && (p < 0 || i < p))) { dp = v; p = i; }
    }
    last = dp;
    if (!(dp > tol * tr) || p < 0) break;
    for (int k = tid; k < j; k += blockDim.x) lp[k] = __ldcg(&L[(long)p * lr + k]);
    __syncthreads();
    const R inv = (R)(1.0 / sqrt(dp));
    for (int li = tid; li < nloc; li += blockDim.x) {
      const int i = c + li * S;
      T acc = w[(long)i * n + p];
      const T* lrow = L + (long)i * lr;
      for (int k = 0; k < j; ++k) {
        T a = lrow[k], b = lp[k];
        // acc -= a * conj(b)
        acc.x -= a.x * b.x + a.y * b.y;
        acc.y -= a.y * b.x - a.x * b.y;
      }
      T lij = mkc<R>(acc.x * inv, acc.y * inv);
      if (i == p) lij = mkc<R>((R)sqrt(dp), R(0));
      L[(long)i * lr + j] = lij;
      double nd = (i == p) ? 0.0 : d[li] - ((double)lij.x * lij.x + (double)lij.y * lij.y);
      d[li] = nd > 0 ? nd : 0.0;
    }
    __syncthreads();
    r = j + 1;
    last = 0.0;
  }
  if (r == rmax) {
    // largest remaining diagonal over the cluster (posted in the free slot)
    double b = 0.0;
    for (int li = tid; li < nloc; li += blockDim.x) b = fmax(b, d[li]);
    for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    if (lane == 0) rv[wid] = b;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int k = 0; k < nw; ++k) t = fmax(t, rv[k]);
      post_v[rmax & 1] = t;
    }
    cluster.sync();
    last = 0.0;
    for (int q = 0; q < S; ++q) last = fmax(last, cluster.map_shared_rank(post_v, q)[rmax & 1]);
  }
  if (c == 0 && tid == 0) {
    *rout = r;
    *resid = tr > 0 ? last / tr : 0.0;
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// zs[i][c] = z[i][c] / sqrt(s_c) (0 where s_c <= 0): eigenvectors of L L^+ from those of L^+ L
template <typename R>
__global__ void lift_kernel(int r, const cx<R>* __restrict__ z, const double* __restrict__ s,
                            cx<R>* zs) {
  long total = (long)r * r;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int c = (int)(e % r);
    double sc = s[c] > 0 ? 1.0 / sqrt(s[c]) : 0.0;
    zs[e] = cscale(z[e], (R)sc);
  }
}

}  // namespace

// ------------------------------------------------------------- launchers
// Rows x cols complex matrix copied between precisions (strided rows on both sides).
template <typename Ri, typename Ro>
__global__ void convert_kernel(int rows, int cols, const cx<Ri>* __restrict__ in, long ldi,
                               cx<Ro>* __restrict__ out, long ldo) {
  long total = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long r = e / cols, c = e % cols;
    cx<Ri> v = in[r * ldi + c];
    out[r * ldo + c] = mkc<Ro>((Ro)v.x, (Ro)v.y);
  }
}

template <typename Ri, typename Ro>
cudaError_t convert(cudaStream_t st, int rows, int cols, const cx<Ri>* in, long ldi, cx<Ro>* out,
                    long ldo) {
  long total = (long)rows * cols;
  if (total <= 0) return cudaSuccess;
  count_launch();
  convert_kernel<Ri, Ro><<<nblocks(total), 256, 0, st>>>(rows, cols, in, ldi, out, ldo);
  return cudaGetLastError();
}
template cudaError_t convert<float, double>(cudaStream_t, int, int, const cx<float>*, long,
                                            cx<double>*, long);
template cudaError_t convert<double, float>(cudaStream_t, int, int, const cx<double>*, long,
                                            cx<float>*, long);

template <typename T>
cudaError_t swap12(cudaStream_t st, long n0, long n1, long n2, long n3, const T* in, T* out) {
  long total = n0 * n1 * n2 * n3;
  if (total <= 0) return cudaSuccess;
  count_launch();
  swap12_kernel<T><<<nblocks(total), 256, 0, st>>>(n0, n1, n2, n3, in, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t reverse_site(cudaStream_t st, int dl, int d, int k, int dr, const T* in, T* out) {
  long total = (long)dl * d * k * dr;
  count_launch();
  reverse_site_kernel<T><<<nblocks(total), 256, 0, st>>>(dl, d, k, dr, in, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t one_site(cudaStream_t st, int dl, int k, int dr, const cx<R>* u, cx<R>* a) {
  long total = (long)dl * k * dr;
  count_launch();
  one_site_kernel<R><<<nblocks(total), 256, 0, st>>>(dl, k, dr, u, a);
  return cudaGetLastError();
}
template <typename R>
cudaError_t product_state(cudaStream_t st, const double* v, cx<R>* base, long stride, int n) {
  count_launch();
  product_state_kernel<R><<<(n + 127) / 128, 128, 0, st>>>(
      mkc<R>((R)v[0], (R)v[1]), mkc<R>((R)v[2], (R)v[3]), mkc<R>((R)v[4], (R)v[5]), base, stride,
      n);
  return cudaGetLastError();
}
template <typename R>
cudaError_t gram_mask(cudaStream_t st, int n, const double* sig, double gtol, R* rs, R* irs,
                      StepScalars* sc) {
  count_launch();
  gram_mask_kernel<R><<<1, 256, 0, st>>>(n, sig, gtol, rs, irs, sc);
  return cudaGetLastError();
}
template <typename R>
cudaError_t gram_factor(cudaStream_t st, int n, const cx<R>* v, const R* rs, const R* irs,
                        cx<R>* rmat, cx<R>* vs, cx<R>* vr) {
  count_launch();
  gram_factor_kernel<R><<<nblocks((long)n * n), 256, 0, st>>>(n, v, rs, irs, rmat, vs, vr);
  return cudaGetLastError();
}
template <typename R>
cudaError_t build_phi(cudaStream_t st, int dm, const cx<R>* ct, const cx<R>* gj, cx<R>* phi) {
  long n = 9L * dm;
  count_launch();
  build_phi_kernel<R><<<nblocks(n * n), 256, 0, st>>>(dm, ct, gj, phi);
  return cudaGetLastError();
}
template <typename R>
cudaError_t bond_select(cudaStream_t st, int n, const double* lam, const cx<R>* hm, long ldh,
                        double htol, int chi, StepScalars* sc, DevStats* ds) {
  count_launch();
  bond_select_kernel<R><<<1, 256, 0, st>>>(n, lam, hm, ldh, htol, chi, sc, ds);
  return cudaGetLastError();
}
template <typename R>
cudaError_t make_q(cudaStream_t st, int dm, int keep, int m_ops, const cx<R>* w, const cx<R>* e,
                   const StepScalars* sc, cx<R>* q) {
  long total = (long)keep * 3 * m_ops * 3 * dm;
  count_launch();
  make_q_kernel<R><<<nblocks(total), 256, 0, st>>>(dm, keep, m_ops, w, e, sc, q);
  return cudaGetLastError();
}
template <typename R>
cudaError_t kraus_select(cudaStream_t st, int n, const double* w, const cx<R>* wm, int ntr,
                         double kcut, int kmax, int use_ppt, double* f, StepScalars* sc,
                         DevStats* ds, double* trace) {
  // the partial sums live after the kept scale factors f (at most 1024 of them)
  double* parts = f + 1024;
  count_launch(2);
  gram_norms_kernel<R><<<kNormBlocks, 256, 0, st>>>(ntr, wm, parts);
  kraus_select_kernel<R><<<1, 256, 0, st>>>(n, w, parts, kcut, kmax, use_ppt, f, sc, ds, trace);
  return cudaGetLastError();
}
template <typename R>
cudaError_t trace_pre(cudaStream_t st, int dm, const cx<R>* gi, const cx<R>* gj, StepScalars* sc) {
  count_launch();
  trace_pre_kernel<R><<<1, 256, 0, st>>>(dm, gi, gj, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t permute6(cudaStream_t st, const int* d, const int* p, const T* in, T* out) {
  long total = 1;
  for (int i = 0; i < 6; ++i) total *= d[i];
  count_launch();
  permute6_kernel<T><<<nblocks(total), 256, 0, st>>>(in, out, d[0], d[1], d[2], d[3], d[4], d[5],
                                                     p[0], p[1], p[2], p[3], p[4], p[5]);
  return cudaGetLastError();
}
template <typename R>
cudaError_t rho_site(cudaStream_t st, long dl2, long dr2, cx<R>* r, cx<R>* tr, int mode) {
  count_launch();
  rho_site_kernel<cx<R>><<<nblocks(dl2 * 9 * dr2), 256, 0, st>>>(dl2, dr2, r, tr, mode);
  return cudaGetLastError();
}
constexpr int kDotBlocks = 64;
template <typename R>
cudaError_t env_dot(cudaStream_t st, long n2, const cx<R>* x, const cx<R>* y, int mode,
                    double* parts, double* out) {
  count_launch(2);
  env_dot_kernel<cx<R>><<<kDotBlocks, 256, 0, st>>>(n2, x, y, mode, parts);
  sum_parts_kernel<<<1, 32, 0, st>>>(kDotBlocks, parts, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t sumsq(cudaStream_t st, long n, const cx<R>* a, double* out) {
  count_launch();
  sumsq_kernel<R><<<1, 256, 0, st>>>(n, a, out);
  return cudaGetLastError();
}
template <typename R, typename RO>
cudaError_t scale_vk(cudaStream_t st, int n, int kk, const cx<R>* v, long ldv, const double* f,
                     cx<RO>* out) {
  count_launch();
  scale_vk_kernel<R, RO><<<nblocks((long)n * kk), 256, 0, st>>>(n, kk, v, ldv, f, out);
  return cudaGetLastError();
}
template <typename R>
cudaError_t energy_mix(cudaStream_t st, int dl, int plane, const cx<R>* f, long fstride,
                       cx<R>* g, long gstride, double J, double hx, double bz) {
  count_launch();
  energy_mix_kernel<R><<<nblocks((long)dl * plane), 256, 0, st>>>(dl, plane, f, fstride, g,
                                                                    gstride, J, hx, bz);
  return cudaGetLastError();
}
template <typename R>
cudaError_t sample_pick(cudaStream_t st, int n_samples, int dr, const cx<R>* ev, const cx<R>* rt,
                        uint64_t seed, int site, int site_user, int n_sites, cx<R>* env_out,
                        uint8_t* bits, double* probs, int last) {
  count_launch();
  sample_pick_kernel<R><<<n_samples, 256, 0, st>>>(dr, ev, rt, seed, site, site_user, n_sites,
                                                   env_out, bits, probs, last);
  return cudaGetLastError();
}

template <typename R>
cudaError_t polar_factors(cudaStream_t st, int n, const cx<R>* g, cx<R>* pm, cx<R>* qm) {
  count_launch();
  polar_factors_kernel<R><<<nblocks((long)n * n), 256, 0, st>>>(n, g, pm, qm);
  return cudaGetLastError();
}

template <typename R, typename RO>
cudaError_t dual_rows(cudaStream_t st, int kk, int cols, const cx<R>* y, long ldy, const double* f,
                      const double* w, cx<RO>* out) {
  count_launch();
  dual_rows_kernel<R, RO><<<nblocks((long)kk * cols), 256, 0, st>>>(kk, cols, y, ldy, f, w, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t pchol(cudaStream_t st, int n, const cx<R>* w, int rmax, double tol, cx<R>* L, int lr,
                  int* rout, double* resid) {
  if (n < 1 || n > 1024 || rmax < 1 || rmax > 128) return cudaErrorInvalidValue;
  // cluster of S CTAs, at least 32 rows each, at most 8 (portable cluster size)
  const int S = std::min(8, std::max(1, n / 32));
  const int rows = (n + S - 1) / S;
  const int threads = std::min(1024, std::max(64, (rows + 31) / 32 * 32));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S);
  cfg.blockDim = dim3(threads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = S;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, pchol_kernel<R>, n, w, rmax, tol, L, lr, rout, resid);
}
template cudaError_t pchol<float>(cudaStream_t, int, const float2*, int, double, float2*, int,
                                  int*, double*);
template cudaError_t pchol<double>(cudaStream_t, int, const double2*, int, double, double2*, int,
                                   int*, double*);
template <typename R>
cudaError_t lift(cudaStream_t st, int r, const cx<R>* z, const double* s, cx<R>* zs) {
  count_launch();
  lift_kernel<R><<<nblocks((long)r * r), 256, 0, st>>>(r, z, s, zs);
  return cudaGetLastError();
}
template cudaError_t lift<double>(cudaStream_t, int, const double2*, const double*, double2*);
template cudaError_t lift<float>(cudaStream_t, int, const float2*, const double*, float2*);

#define INST(R)                                                                               \
  template cudaError_t swap12<cx<R>>(cudaStream_t, long, long, long, long, const cx<R>*,     \
                                     cx<R>*);                                               \
  template cudaError_t reverse_site<cx<R>>(cudaStream_t, int, int, int, int, const cx<R>*,   \
                                           cx<R>*);                                         \
  template cudaError_t one_site<R>(cudaStream_t, int, int, int, const cx<R>*, cx<R>*);      \
  template cudaError_t product_state<R>(cudaStream_t, const double*, cx<R>*, long, int);     \
  template cudaError_t gram_mask<R>(cudaStream_t, int, const double*, double, R*, R*,       \
                                    StepScalars*);                                          \
  template cudaError_t gram_factor<R>(cudaStream_t, int, const cx<R>*, const R*, const R*,  \
                                      cx<R>*, cx<R>*, cx<R>*);                              \
  template cudaError_t build_phi<R>(cudaStream_t, int, const cx<R>*, const cx<R>*, cx<R>*); \
  template cudaError_t make_q<R>(cudaStream_t, int, int, int, const cx<R>*, const cx<R>*,   \
                                 const StepScalars*, cx<R>*);                               \
  template cudaError_t energy_mix<R>(cudaStream_t, int, int, const cx<R>*, long, cx<R>*,    \
                                     long, double, double, double);                         \
  template cudaError_t bond_select<R>(cudaStream_t, int, const double*, const cx<R>*, long,  \
                                      double, int, StepScalars*, DevStats*);                 \
  template cudaError_t kraus_select<R>(cudaStream_t, int, const double*, const cx<R>*, int,   \
                                       double, int, int, double*, StepScalars*, DevStats*,   \
                                       double*);                                             \
  template cudaError_t trace_pre<R>(cudaStream_t, int, const cx<R>*, const cx<R>*,           \
                                    StepScalars*);                                           \
  template cudaError_t polar_factors<R>(cudaStream_t, int, const cx<R>*, cx<R>*, cx<R>*);   \
  template cudaError_t sumsq<R>(cudaStream_t, long, const cx<R>*, double*);                 \
  template cudaError_t permute6<cx<R>>(cudaStream_t, const int*, const int*, const cx<R>*,    \
                                       cx<R>*);                                              \
  template cudaError_t rho_site<R>(cudaStream_t, long, long, cx<R>*, cx<R>*, int);           \
  template cudaError_t env_dot<R>(cudaStream_t, long, const cx<R>*, const cx<R>*, int,       \
                                  double*, double*);                                          \
  template cudaError_t sample_pick<R>(cudaStream_t, int, int, const cx<R>*, const cx<R>*,   \
                                      uint64_t, int, int, int, cx<R>*, uint8_t*, double*, int);
INST(double)
INST(float)
#undef INST

#define INST2(R, RO)                                                                          \
  template cudaError_t scale_vk<R, RO>(cudaStream_t, int, int, const cx<R>*, long,           \
                                       const double*, cx<RO>*);                              \
  template cudaError_t dual_rows<R, RO>(cudaStream_t, int, int, const cx<R>*, long,          \
                                        const double*, const double*, cx<RO>*);
INST2(double, double)
INST2(float, float)
INST2(double, float)
#undef INST2

}  // namespace mpdo
