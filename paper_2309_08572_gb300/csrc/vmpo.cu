// Vectorized MPO engine with purity-preserving truncation on the bond (the paper's main
// engine: Sec. III.A "vectorized MPO", Sec. III.D Eqs. xiformula and ppt, App. B).
//
// rho is an MPS over the doubled index eta = (s, s') (d^2 = 9 per site), site tensors
// A_n[l][eta][r] in complex128, kept in mixed-canonical form for the Frobenius inner product.
// A two-site op acts on the pair (eta_i, eta_j) as its superoperator (built on the host from
// the op's Kraus set).  One update, centre at i (right-to-left updates run on the mirrored
// chain, as in the MPDO engine):
//   theta  = A_i A_j                       ((9 D_l) x (9 D_r), [l][eta_i][eta_j][r])
//   theta' = S theta on (eta_i, eta_j)     (81 x 81 superoperator, batched over l)
//   theta' = U Lambda V^+                  (eigenpairs of theta' theta'^+, FP64 Jacobi;
//                                           Lambda = sqrt of the eigenvalues above the cut,
//                                           V^+ = Lambda^-1 U^+ theta')
//   T_k    = (L (x) tau)^T U[:, k] * V^+[k, :] (tau (x) R)   (trace environment: L, R the
//            contractions of the sites left of i / right of j with tau[(s,s')] = delta_ss')
//   keep the chi largest: naive (unchanged) or PPT's values with this T (trace and
//   xi = tr rho^2 / tr rho^2 of the bond kept);  A_i <- U_keep, A_j <- diag(Lambda~) V^+_keep.
// The left trace environment of the new centre is updated from the new A_i; the right ones
// are recomputed after every change of direction.  Observables: tr(O rho) contracts each
// site with o[(s,s')] = O[s', s]; the TFIM energies run as a three-state automaton per
// projector (identity / qubit projector), one kernel per site.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/mpdo.h"
#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgemm.h"

namespace mpdo {
void set_global_error(const char* msg);
}

using namespace mpdo;

namespace {

using zc = std::complex<double>;

// Scalars of one vMPO update read by the host.
struct VScalars {
  int nz;        // Schmidt values above the cut
  int keep;      // kept
  int infeasible;
  int clamped;
  int flags;     // bit 0: numeric problem
  double theta;  // PPT angle
  double disc;   // discarded weight fraction (sum of Lambda^2)
};

// Cut and truncation of the Schmidt values (eigenvalues lam of theta' theta'^+, descending):
// nz = count above cut^2 lam_0, keep = min(nz, chi); mode 1 = PPT with the trace environment
// T_k = Re(tl_k trw_k) / Lambda_k (trw carries the factor Lambda_k of U^+ theta'; Eqs.
// xiformula, ppt; theta = 0 when infeasible, negative values clamped, rescaled so that
// T'.Lambda~ = T.Lambda); out[k] = Lambda~_k (k < keep), sv[k] = sqrt(lam_k) for k < nz.
__global__ void vmpo_cut_kernel(int n, const double* __restrict__ lam, const double2* __restrict__ tl,
                                const double2* __restrict__ tr, double cut2, int chi, int mode,
                                double* sv, double* out, VScalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double l0 = lam[0];
  VScalars s{};
  if (!(l0 > 0.0) || !isfinite(l0)) {
    s.flags = 1;
    s.nz = s.keep = 1;
    *sc = s;
    return;
  }
  int nz = 0;
  while (nz < n && lam[nz] > cut2 * l0) ++nz;
  if (nz < 1) nz = 1;
  const int keep = nz < chi ? nz : chi;
  double tot = 0, kept = 0;
  for (int k = 0; k < nz; ++k) {
    sv[k] = sqrt(fmax(lam[k], 0.0));
    tot += lam[k];
    if (k < keep) kept += lam[k];
  }
  s.nz = nz;
  s.keep = keep;
  s.disc = tot > 0 ? (tot - kept) / tot : 0.0;
  if (mode == 0) {
    for (int k = 0; k < keep; ++k) out[k] = sv[k];
  } else {
    double lt = 0, nl = 0, nt = 0, lpt = 0, nlp = 0, ntp = 0;
    for (int k = 0; k < nz; ++k) {
      // T_k = Re(tl_k tr_k) (real for a Hermitian rho up to near-degeneracies)
      const double t = (tl[k].x * tr[k].x - tl[k].y * tr[k].y) / sv[k];
      lt += sv[k] * t;
      nl += sv[k] * sv[k];
      nt += t * t;
      if (k < keep) {
        lpt += sv[k] * t;
        nlp += sv[k] * sv[k];
        ntp += t * t;
      }
    }
    nl = sqrt(nl);
    nt = sqrt(nt);
    nlp = sqrt(nlp);
    ntp = sqrt(ntp);
    const double cos_phi = lt / (nl * nt);
    double cos_sig = lpt / (nlp * ntp);
    if (cos_sig > 1.0) cos_sig = 1.0;
    const double ratio = nt * cos_phi / ntp;
    double th;
    if (ratio > 1.0 || !(ntp > 0)) {
      s.infeasible = 1;
      th = 0.0;
    } else {
      th = acos(ratio);
    }
    s.theta = th;
    const double sig = acos(cos_sig);
    const double x = (sig == 0.0) ? 0.0 : tan(th) / tan(sig) - 1.0;
    double dot = 0;
    for (int k = 0; k < keep; ++k) {
      const double t = (tl[k].x * tr[k].x - tl[k].y * tr[k].y) / sv[k];
      double v = (sig == 0.0) ? sv[k] : sv[k] + x * (sv[k] - nlp * cos_sig * t / ntp);
      if (v < 0) {
        v = 0;
        ++s.clamped;
      }
      out[k] = v;
      dot += v * t;
    }
    const double scale = (dot != 0.0) ? lt / dot : 0.0;
    for (int k = 0; k < keep; ++k) out[k] *= scale;
  }
  *sc = s;
}

// x[(l, eta)] = env[l] tau[eta] (side 0) or x[(eta, r)] = tau[eta] env[r] (side 1)
__global__ void trace_vec_kernel(int d, const double2* __restrict__ env, int side, double2* x) {
  const int total = 9 * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int eta = side == 0 ? e % 9 : e / d;
    const int b = side == 0 ? e / 9 : e % d;
    const bool diag = (eta == 0 || eta == 4 || eta == 8);
    x[e] = diag ? env[b] : make_double2(0.0, 0.0);
  }
}

// rows k < keep of vh (ld ldv) scaled by f[k] / sv[k] (f = Lambda~ or 1 for the isometry)
__global__ void scale_rows_kernel(int keep, int cols, const double2* __restrict__ in, long ldi,
                                  const double* __restrict__ num, const double* __restrict__ den,
                                  double2* out, long ldo) {
  const long total = (long)keep * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e / cols), c = (int)(e % cols);
    const double f = (num ? num[k] : 1.0) / den[k];
    const double2 v = in[(long)k * ldi + c];
    out[(long)k * ldo + c] = make_double2(v.x * f, v.y * f);
  }
}

// The energy automaton on one site: for projector p (0: identity, 1: qubit projector),
// states s = 0 (no term yet), 1 (a Z waiting for its partner), 2 (term complete):
//   E0' = E0 T[P], E1' = E0 T[PZP], E2' = E2 T[P] - J E1 T[PZP] + E0 T[P H1 P]
// with T[O](E)[r] = sum_{l,eta} E[l] o[eta] A[l,eta,r], o[(s,s')] = O[s',s];
// env in/out: [2 projectors][3 states][dl | dr].
__global__ void vmpo_energy_kernel(int dl, int dr, const double2* __restrict__ a,
                                   const double2* __restrict__ ein, double2* eout,
                                   const double2* __restrict__ ovec /* [2][3][9] */, double J) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= dr) return;
  for (int p = 0; p < 2; ++p) {
    const double2* op = ovec + p * 27;   // [0] P, [1] PZP, [2] P H1 P
    const double2* e0 = ein + (p * 3 + 0) * dl;
    const double2* e1 = ein + (p * 3 + 1) * dl;
    const double2* e2 = ein + (p * 3 + 2) * dl;
    double2 n0 = make_double2(0, 0), n1 = n0, n2 = n0;
    for (int l = 0; l < dl; ++l) {
      double2 t[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
      for (int eta = 0; eta < 9; ++eta) {
        const double2 av = a[((long)l * 9 + eta) * dr + r];
        for (int q = 0; q < 3; ++q) t[q] = cadd(t[q], cmul(op[q * 9 + eta], av));
      }
      n0 = cadd(n0, cmul(e0[l], t[0]));
      n1 = cadd(n1, cmul(e0[l], t[1]));
      n2 = cadd(n2, cadd(cmul(e2[l], t[0]), cadd(cscale(cmul(e1[l], t[1]), -J), cmul(e0[l], t[2]))));
    }
    eout[(p * 3 + 0) * dr + r] = n0;
    eout[(p * 3 + 1) * dr + r] = n1;
    eout[(p * 3 + 2) * dr + r] = n2;
  }
}

// product state: site s, eta = (t, t') -> v_t conj(v_t') (v host-side complex128 in device copy)
__global__ void vmpo_product_kernel(const double* v, double2* base, long stride, int n) {
  const int s = blockIdx.x, eta = threadIdx.x;
  if (s >= n || eta >= 9) return;
  const int si = eta / 3, sp = eta % 3;
  const double re = v[2 * si] * v[2 * sp] + v[2 * si + 1] * v[2 * sp + 1];
  const double im = v[2 * si + 1] * v[2 * sp] - v[2 * si] * v[2 * sp + 1];
  base[(long)s * stride + eta] = make_double2(re, im);
}

// mirrored site: [l][eta][r] -> [r][eta][l]
__global__ void vmpo_reverse_kernel(int dl, int dr, const double2* __restrict__ in, double2* out) {
  const long total = (long)dl * 9 * dr;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e % dr), eta = (int)((e / dr) % 9), l = (int)(e / (9L * dr));
    out[((long)r * 9 + eta) * dl + l] = in[e];
  }
}

inline int nblk(long n) { return (int)std::min<long>((n + 255) / 256, 4096); }

}  // namespace

struct VOp {
  int site = 0;
  std::vector<zc> s, sm;   // pair superoperator and its mirror (sites swapped), 81 x 81
};

struct mpdo_vmpo_s {
  int n = 0, chi = 0, mode = 1;
  double cut2 = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  bool rev = false;
  int centre = 0;                 // user coordinates
  std::vector<int> bond;          // storage coordinates, size n + 1
  size_t site_cap = 0;
  double2* sites = nullptr;
  double2 *th = nullptr, *th2 = nullptr, *H = nullptr, *U = nullptr, *Vh = nullptr;
  double2 *S = nullptr, *x = nullptr, *tl = nullptr, *tr = nullptr, *ov = nullptr;
  double2 *Lenv = nullptr, *Renv = nullptr, *etmp = nullptr, *ebuf = nullptr;
  double *lam = nullptr, *sv = nullptr, *lt = nullptr;
  EigWork<double> eig;
  void* eigmem = nullptr;
  // tensor-core form (mpdo_vmpo_set_precision 1): exact-slice products and the mixed solver
  int tc = 0;
  MixWork mixw;
  void* mixmem = nullptr;
  void* tcws = nullptr;
  size_t tcws_bytes = 0;
  int* tcerr = nullptr;
  int* htcerr = nullptr;   // pinned
  double sv_req = 0;       // requested cut (Schmidt values, relative)
  VScalars* dsc = nullptr;
  VScalars* hsc = nullptr;
  std::vector<void*> allocs;
  std::string err;
  double2* site(int s) const { return sites + (size_t)s * site_cap; }
};

namespace {

int vfail(mpdo_vmpo h, int code, const std::string& msg) {
  if (h) h->err = msg;
  set_global_error(msg.c_str());
  return code;
}
#define VK(expr)                                                                     \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess)                                                           \
      return vfail(h, MPDO_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

int valloc(mpdo_vmpo h, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return vfail(h, MPDO_ERR_OOM, "vmpo: device allocation of " + std::to_string(bytes) + " bytes");
  }
  h->allocs.push_back(*p);
  if (cudaMemsetAsync(*p, 0, bytes ? bytes : 16, h->st) != cudaSuccess) {
    cudaGetLastError();
    return vfail(h, MPDO_ERR_CUDA, "vmpo: clearing a new buffer");
  }
  return MPDO_OK;
}

cudaError_t g64(cudaStream_t st, int opa, int opb, int m, int n, int k, const double2* A, long lda,
                long sa, const double2* B, long ldb, long sb, double2* C, long ldc, long sc,
                int batch) {
  return cgemm<double>(st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch,
                       make_double2(1, 0), make_double2(0, 0));
}

// Products of the update: in the tensor-core form, those of at least 2^21 complex
// multiply-adds (both output sides >= 16) as error-free BF16 slice products summed in FP64
// (carried to ~2^-48 of each operand row's largest entry); FP64 CUDA cores otherwise.
cudaError_t u64(mpdo_vmpo h, int opa, int opb, int m, int n, int k, const double2* A, long lda,
                long sa, const double2* B, long ldb, long sb, double2* C, long ldc, long sc,
                int batch) {
  if (h->tc && m >= 16 && n >= 16 && (double)m * n * k * batch >= (double)(1 << 21))
    return tc_cgemm_exact<double2, double2>(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C,
                                            ldc, sc, batch, h->tcws, h->tcws_bytes, h->tcerr);
  return g64(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch);
}

// right trace environments Renv[n] (right of site n, storage coords) for all n
int right_envs(mpdo_vmpo h) {
  const long cap = h->chi;
  double2 one = make_double2(1, 0);
  VK(cudaMemcpyAsync(h->Renv + (long)(h->n - 1) * cap, &one, sizeof(double2), cudaMemcpyHostToDevice,
                     h->st));
  for (int s = h->n - 1; s >= 1; --s) {
    const int dl = h->bond[s], dr = h->bond[s + 1];
    // x[(eta, r)] = tau[eta] R[r];  Renv[s-1][l] = sum A[l, (eta, r)] x[(eta, r)]
    count_launch();
    trace_vec_kernel<<<nblk(9L * dr), 256, 0, h->st>>>(dr, h->Renv + (long)s * cap, 1, h->x);
    VK(cudaGetLastError());
    VK(g64(h->st, OP_N, OP_N, dl, 1, 9 * dr, h->site(s), 9L * dr, 0, h->x, 1, 0,
           h->Renv + (long)(s - 1) * cap, 1, 0, 1));
  }
  return MPDO_OK;
}

// left trace environment of site s+1 from that of site s and site s's tensor
int left_env_step(mpdo_vmpo h, int s) {
  const long cap = h->chi;
  const int dl = h->bond[s], dr = h->bond[s + 1];
  count_launch();
  trace_vec_kernel<<<nblk(9L * dl), 256, 0, h->st>>>(dl, h->Lenv + (long)s * cap, 0, h->x);
  VK(cudaGetLastError());
  VK(g64(h->st, OP_N, OP_N, 1, dr, 9 * dl, h->x, 9L * dl, 0, h->site(s), dr, 0,
         h->Lenv + (long)(s + 1) * cap, dr, 0, 1));
  return MPDO_OK;
}

int left_envs_to(mpdo_vmpo h, int upto) {
  double2 one = make_double2(1, 0);
  VK(cudaMemcpyAsync(h->Lenv, &one, sizeof(double2), cudaMemcpyHostToDevice, h->st));
  for (int s = 0; s < upto; ++s) {
    int rc = left_env_step(h, s);
    if (rc) return rc;
  }
  return MPDO_OK;
}

int reverse(mpdo_vmpo h) {
  for (int s = 0; s <= (h->n - 1) / 2; ++s) {
    const int t = h->n - 1 - s;
    const size_t ns = (size_t)h->bond[s] * 9 * h->bond[s + 1];
    const size_t nt = (size_t)h->bond[t] * 9 * h->bond[t + 1];
    count_launch();
    vmpo_reverse_kernel<<<nblk(ns), 256, 0, h->st>>>(h->bond[s], h->bond[s + 1], h->site(s), h->th);
    if (t != s) {
      count_launch();
      vmpo_reverse_kernel<<<nblk(nt), 256, 0, h->st>>>(h->bond[t], h->bond[t + 1], h->site(t),
                                                      h->th2);
    }
    VK(cudaGetLastError());
    VK(cudaMemcpyAsync(h->site(t), h->th, ns * sizeof(double2), cudaMemcpyDeviceToDevice, h->st));
    if (t != s)
      VK(cudaMemcpyAsync(h->site(s), h->th2, nt * sizeof(double2), cudaMemcpyDeviceToDevice, h->st));
  }
  std::reverse(h->bond.begin(), h->bond.end());
  h->rev = !h->rev;
  return MPDO_OK;
}

// one update on storage bond (i, i+1), centre at i; the centre moves to i+1
int update(mpdo_vmpo h, int i, const VOp& op, mpdo_trunc_stats* acc) {
  cudaStream_t st = h->st;
  const int dl = h->bond[i], dm = h->bond[i + 1], dr = h->bond[i + 2];
  const int rows = 9 * dl, cols = 9 * dr;
  const std::vector<zc>& S = h->rev ? op.sm : op.s;
  VK(cudaMemcpyAsync(h->S, S.data(), 81 * 81 * sizeof(double2), cudaMemcpyHostToDevice, st));
  // theta = A_i A_j ; theta' = S on (eta_i, eta_j), batched over l
  VK(u64(h, OP_N, OP_N, rows, cols, dm, h->site(i), dm, 0, h->site(i + 1), cols, 0, h->th, cols,
         0, 1));
  VK(u64(h, OP_N, OP_N, 81, dr, 81, h->S, 81, 0, h->th, dr, 81L * dr, h->th2, dr, 81L * dr, dl));
  // Schmidt decomposition through the Gram theta' theta'^+: FP64 Jacobi, or in the
  // tensor-core form the mixed solver (FP32 Jacobi levels, FP64 refinement) resolved below
  // a tenth of the cut -- in naive mode only the chi + 1 leading pairs (PPT needs T and
  // Lambda of every Schmidt pair)
  VK(u64(h, OP_N, OP_C, rows, rows, cols, h->th2, cols, 0, h->th2, cols, 0, h->H, rows, 0, 1));
  if (h->tc)
    VK(heig_mixed(st, rows, h->H, rows, h->U, rows, h->lam, 0.1 * h->cut2, h->mixw, nullptr,
                  nullptr, h->mode == 1 ? 0 : h->chi + 1));
  else
    VK(heig<double>(st, rows, h->H, rows, h->U, rows, h->lam, h->eig, 30));
  // trace environment: tl = (L (x) tau)^T U ; W = U^+ theta' (row k = Lambda_k V^+_k) ;
  // trw = W (tau (x) R)
  count_launch();
  trace_vec_kernel<<<nblk(rows), 256, 0, st>>>(dl, h->Lenv + (long)i * h->chi, 0, h->x);
  VK(cudaGetLastError());
  VK(g64(st, OP_N, OP_N, 1, rows, rows, h->x, rows, 0, h->U, rows, 0, h->tl, rows, 0, 1));
  VK(u64(h, OP_C, OP_N, rows, cols, rows, h->U, rows, 0, h->th2, cols, 0, h->th, cols, 0, 1));
  count_launch();
  trace_vec_kernel<<<nblk(cols), 256, 0, st>>>(dr, h->Renv + (long)(i + 1) * h->chi, 1,
                                                h->x + rows);
  VK(cudaGetLastError());
  VK(g64(st, OP_N, OP_N, rows, 1, cols, h->th, cols, 0, h->x + rows, 1, 0, h->tr, 1, 0, 1));
  count_launch();
  vmpo_cut_kernel<<<1, 32, 0, st>>>(rows, h->lam, h->tl, h->tr, h->cut2, h->chi, h->mode, h->sv,
                                    h->lt, h->dsc);
  VK(cudaGetLastError());
  VK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(VScalars), cudaMemcpyDeviceToHost, st));
  if (h->tc) VK(cudaMemcpyAsync(h->htcerr, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  VK(cudaStreamSynchronize(st));
  if (h->tc && *h->htcerr) return vfail(h, MPDO_ERR_TIMEOUT, "vmpo: a tensor-core pipeline wait gave up");
  if (h->hsc->flags & 1) return vfail(h, MPDO_ERR_NUMERIC, "vmpo: zero or non-finite state");
  const int keep = h->hsc->keep;
  // A_i <- U_keep ; A_{i+1} <- diag(Lambda~ / Lambda) W_keep
  VK(cudaMemcpy2DAsync(h->site(i), keep * sizeof(double2), h->U, rows * sizeof(double2),
                       keep * sizeof(double2), rows, cudaMemcpyDeviceToDevice, st));
  count_launch();
  scale_rows_kernel<<<nblk((long)keep * cols), 256, 0, st>>>(keep, cols, h->th, cols, h->lt, h->sv,
                                                             h->site(i + 1), cols);
  VK(cudaGetLastError());
  h->bond[i + 1] = keep;
  int rc = left_env_step(h, i);
  if (rc) return rc;
  if (acc) {
    acc->disc_bond_w += h->hsc->disc;
    acc->ppt_infeasible += h->hsc->infeasible;
    acc->ppt_clamped += h->hsc->clamped;
    if (h->mode == 1 && h->hsc->theta < acc->ppt_theta_min) acc->ppt_theta_min = h->hsc->theta;
    acc->chi_used_max = std::max(acc->chi_used_max, keep);
    acc->n_updates += 1;
  }
  return MPDO_OK;
}

// host: the pair superoperator of a Kraus set (81 x 81 complex), re-indexed from the
// two-site row-major vec ((s_i,s_j),(s'_i,s'_j)) to the MPO pair ((s_i,s'_i),(s_j,s'_j));
// mirrored: the two sites swapped
void pair_superop(const double* ops, int m, bool mirror, std::vector<zc>& out) {
  out.assign(81 * 81, zc(0, 0));
  for (int q = 0; q < m; ++q) {
    const double* e = ops + 2 * 81 * q;
    auto E = [&](int r, int c) { return zc(e[2 * (r * 9 + c)], e[2 * (r * 9 + c) + 1]); };
    // S[(a,b),(c,d)] = E[a][c] conj(E[b][d]) on two-site indices a = (si,sj) etc.
    for (int si = 0; si < 3; ++si)
      for (int sj = 0; sj < 3; ++sj)
        for (int pi = 0; pi < 3; ++pi)
          for (int pj = 0; pj < 3; ++pj)
            for (int ti = 0; ti < 3; ++ti)
              for (int tj = 0; tj < 3; ++tj)
                for (int ui = 0; ui < 3; ++ui)
                  for (int uj = 0; uj < 3; ++uj) {
                    // ket (si,sj) <- (ti,tj), bra (pi,pj) <- (ui,uj)
                    const zc v = E(si * 3 + sj, ti * 3 + tj) * std::conj(E(pi * 3 + pj, ui * 3 + uj));
                    int etai = si * 3 + pi, etaj = sj * 3 + pj;    // output MPO pair
                    int mui = ti * 3 + ui, muj = tj * 3 + uj;      // input MPO pair
                    if (mirror) {
                      std::swap(etai, etaj);
                      std::swap(mui, muj);
                    }
                    out[(etai * 9 + etaj) * 81 + mui * 9 + muj] += v;
                  }
  }
}

}  // namespace

extern "C" {

int mpdo_vmpo_create(int n_sites, int chi_max, int use_ppt, double sv_cutoff,
                     const double* init_site_vec, void* cuda_stream, mpdo_vmpo* out) {
  if (n_sites < 2 || chi_max < 1 || chi_max > 256 || !out)
    return vfail(nullptr, MPDO_ERR_ARG, "vmpo: n_sites >= 2 and chi_max in 1..256 required");
  std::unique_ptr<mpdo_vmpo_s> hp(new (std::nothrow) mpdo_vmpo_s());
  if (!hp) return vfail(nullptr, MPDO_ERR_OOM, "vmpo: host allocation");
  mpdo_vmpo h = hp.get();
  h->n = n_sites;
  h->chi = chi_max;
  h->mode = use_ppt ? 1 : 0;
  // Gram eigenvalues resolve to ~1e-16 of the largest: Schmidt values below sqrt(1e-15) of
  // the largest are numerical zeros whatever cut is asked for
  const double sv = sv_cutoff > 0 ? sv_cutoff : 1e-14;
  h->sv_req = sv;
  h->cut2 = std::max(sv * sv, 1e-15);
  if (cuda_stream) {
    h->st = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return vfail(nullptr, MPDO_ERR_CUDA, "vmpo: stream creation");
    }
    h->own_stream = true;
  }
  h->bond.assign(n_sites + 1, 1);
  const long D = chi_max, n9 = 9 * D;
  h->site_cap = (size_t)D * 9 * D;
  auto A = [&](void** p, size_t count) { return valloc(h, p, count * sizeof(double2)); };
  int rc;
  if ((rc = A((void**)&h->sites, h->site_cap * n_sites)) || (rc = A((void**)&h->th, n9 * n9)) ||
      (rc = A((void**)&h->th2, n9 * n9)) || (rc = A((void**)&h->H, n9 * n9)) ||
      (rc = A((void**)&h->U, n9 * n9)) || (rc = A((void**)&h->S, 81 * 81)) ||
      (rc = A((void**)&h->x, 2 * n9)) || (rc = A((void**)&h->tl, n9)) ||
      (rc = A((void**)&h->tr, n9)) || (rc = A((void**)&h->ov, 64)) ||
      (rc = A((void**)&h->Lenv, (size_t)(n_sites + 1) * D)) ||
      (rc = A((void**)&h->Renv, (size_t)(n_sites + 1) * D)) ||
      (rc = A((void**)&h->ebuf, 12 * D)) ||
      (rc = valloc(h, (void**)&h->lam, n9 * sizeof(double))) ||
      (rc = valloc(h, (void**)&h->sv, n9 * sizeof(double))) ||
      (rc = valloc(h, (void**)&h->lt, n9 * sizeof(double))) ||
      (rc = valloc(h, (void**)&h->dsc, sizeof(VScalars))) ||
      (rc = valloc(h, &h->eigmem, eig_work_bytes<double>((int)n9)))) {
    mpdo_vmpo_destroy(hp.release());
    return rc;
  }
  eig_work_bind<double>(h->eig, h->eigmem, (int)n9);
  if (cudaMallocHost((void**)&h->hsc, sizeof(VScalars)) != cudaSuccess) {
    cudaGetLastError();
    mpdo_vmpo_destroy(hp.release());
    return vfail(nullptr, MPDO_ERR_OOM, "vmpo: pinned host allocation");
  }
  double pl[6] = {1.0 / std::sqrt(2.0), 0, 1.0 / std::sqrt(2.0), 0, 0, 0};
  const double* v = init_site_vec ? init_site_vec : pl;
  double* dv = nullptr;
  if ((rc = valloc(h, (void**)&dv, 6 * sizeof(double)))) {
    mpdo_vmpo_destroy(hp.release());
    return rc;
  }
  cudaMemcpyAsync(dv, v, 6 * sizeof(double), cudaMemcpyHostToDevice, h->st);
  count_launch();
  vmpo_product_kernel<<<n_sites, 32, 0, h->st>>>(dv, h->sites, (long)h->site_cap, n_sites);
  if (cudaGetLastError() != cudaSuccess || (rc = right_envs(h)) || (rc = left_envs_to(h, 0)) ||
      cudaStreamSynchronize(h->st) != cudaSuccess) {
    mpdo_vmpo_destroy(hp.release());
    return rc ? rc : vfail(nullptr, MPDO_ERR_CUDA, "vmpo: initial state");
  }
  *out = hp.release();
  return MPDO_OK;
}

int mpdo_vmpo_apply_layer(mpdo_vmpo h, const mpdo_layer* layer, mpdo_trunc_stats* stats) {
  if (!h || !layer || layer->n_ops < 0 || (layer->n_ops > 0 && !layer->ops))
    return vfail(h, MPDO_ERR_ARG, "vmpo: bad layer");
  std::vector<VOp> ops(layer->n_ops);
  for (int k = 0; k < layer->n_ops; ++k) {
    const mpdo_op& op = layer->ops[k];
    if (op.kind != 2 || op.site < 0 || op.site > h->n - 2 || op.n_kraus < 1 || !op.ops)
      return vfail(h, MPDO_ERR_ARG, "vmpo: ops must be two-site channels within the chain");
    for (int a = 0; a < 2 * 81 * op.n_kraus; ++a)
      if (!std::isfinite(op.ops[a])) return vfail(h, MPDO_ERR_NUMERIC, "vmpo: non-finite op");
    ops[k].site = op.site;
    pair_superop(op.ops, op.n_kraus, false, ops[k].s);
    pair_superop(op.ops, op.n_kraus, true, ops[k].sm);
  }
  mpdo_trunc_stats acc{};
  acc.ppt_theta_min = 1e300;
  for (const VOp& op : ops) {
    const int i = op.site;
    bool ltr;
    if (h->centre == i) ltr = true;
    else if (h->centre == i + 1) ltr = false;
    else return vfail(h, MPDO_ERR_STATE, "vmpo: two-site op does not touch the centre");
    int rc;
    if (ltr == h->rev) {
      // the storage runs along the update direction: mirror, then rebuild the environments
      if ((rc = reverse(h)) || (rc = right_envs(h))) return rc;
      const int cs = h->rev ? h->n - 1 - h->centre : h->centre;
      if ((rc = left_envs_to(h, cs))) return rc;
    }
    const int is = h->rev ? h->n - 2 - i : i;
    if ((rc = update(h, is, op, &acc))) return rc;
    h->centre = ltr ? i + 1 : i;
  }
  if (stats) *stats = acc;
  return MPDO_OK;
}

int mpdo_vmpo_expect_energy(mpdo_vmpo h, double J, double hx, double b, double* e_raw,
                            double* e_success, double* success_prob, double* trace) {
  if (!h) return vfail(nullptr, MPDO_ERR_ARG, "vmpo: null handle");
  // operator vectors o[(s,s')] = O[s', s] for P in {I, Pi_q}: P, P Z P, P (-hx X - b J Z) P
  double2 ov[54];
  for (int p = 0; p < 2; ++p) {
    const double pr[3] = {1, 1, p == 0 ? 1.0 : 0.0};
    for (int s = 0; s < 3; ++s)
      for (int t = 0; t < 3; ++t) {
        // O[t][s] with t = bra index s', s = ket index
        const double P = (s == t) ? pr[s] : 0.0;
        const double z = (s == t && s < 2) ? (s == 0 ? 1.0 : -1.0) : 0.0;
        const double xq = ((s == 0 && t == 1) || (s == 1 && t == 0)) ? 1.0 : 0.0;
        const double h1 = -hx * xq - b * J * z;
        ov[p * 27 + 0 * 9 + s * 3 + t] = make_double2(P, 0);
        ov[p * 27 + 1 * 9 + s * 3 + t] = make_double2(pr[s] * pr[t] * z, 0);
        ov[p * 27 + 2 * 9 + s * 3 + t] = make_double2(pr[s] * pr[t] * h1, 0);
      }
  }
  VK(cudaMemcpyAsync(h->ov, ov, sizeof(ov), cudaMemcpyHostToDevice, h->st));
  // env [2][3][D]: start E0 = 1, E1 = E2 = 0 for both projectors
  const long D = h->chi;
  double2* ein = h->ebuf;
  double2* eout = h->ebuf + 6 * D;
  // packed [projector][state][bond] with the bond dimension 1 of the chain's left end
  std::vector<double2> init(6 * D, make_double2(0, 0));
  init[0] = make_double2(1, 0);
  init[3] = make_double2(1, 0);
  VK(cudaMemcpyAsync(ein, init.data(), sizeof(double2) * 6 * D, cudaMemcpyHostToDevice, h->st));
  for (int s = 0; s < h->n; ++s) {
    const int dl = h->bond[s], dr = h->bond[s + 1];
    count_launch();
    vmpo_energy_kernel<<<(dr + 127) / 128, 128, 0, h->st>>>(dl, dr, h->site(s), ein, eout, h->ov,
                                                          J);
    VK(cudaGetLastError());
    std::swap(ein, eout);
  }
  double2 res[6];
  for (int q = 0; q < 6; ++q)
    VK(cudaMemcpyAsync(&res[q], ein + q, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
  VK(cudaStreamSynchronize(h->st));
  // the final bond dimension is 1: state q of projector p sits at ein[(p*3+q)*1]
  const double norm = res[0].x, tot = res[2].x, ps = res[3].x, tots = res[5].x;
  if (!(norm != 0) || !std::isfinite(norm)) return vfail(h, MPDO_ERR_NUMERIC, "vmpo: zero trace");
  if (e_raw) *e_raw = tot / norm;
  if (e_success) *e_success = ps != 0 ? tots / ps : NAN;
  if (success_prob) *success_prob = ps;
  if (trace) *trace = norm;
  return MPDO_OK;
}

int mpdo_vmpo_purity(mpdo_vmpo h, double* purity) {
  if (!h || !purity) return vfail(h, MPDO_ERR_ARG, "vmpo: null argument");
  // canonical gauge: <<rho|rho>> is the centre's squared Frobenius norm
  const int c = h->rev ? h->n - 1 - h->centre : h->centre;
  const long cnt = (long)h->bond[c] * 9 * h->bond[c + 1];
  double* d = h->lam;
  VK(sumsq<double>(h->st, cnt, h->site(c), d));
  VK(cudaMemcpyAsync(purity, d, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  VK(cudaStreamSynchronize(h->st));
  return MPDO_OK;
}

int mpdo_vmpo_collision(mpdo_vmpo h, double* collision) {
  if (!h || !collision) return vfail(h, MPDO_ERR_ARG, "vmpo: null argument");
  // rho_xx = prod_n A_n[., (s_n, s_n), .]: E <- sum_s A_s^T E A_s (D x D, the pair of copies)
  // and t <- sum_s t A_s (the trace), with A_s = A_n[:, (s, s), :] (rows of stride 9 D_r);
  // the site order of the storage does not matter for a sum over all x
  const long D = h->chi;
  double2* E = h->th;              // D x D
  double2* En = E + D * D;         // D x D
  double2* T = En + D * D;         // 3 x D x D
  double2* t = T + 3 * D * D;      // D
  double2* tn = t + D;             // D
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  VK(cudaMemcpyAsync(E, &one, sizeof(double2), cudaMemcpyHostToDevice, h->st));
  VK(cudaMemcpyAsync(t, &one, sizeof(double2), cudaMemcpyHostToDevice, h->st));
  for (int s = 0; s < h->n; ++s) {
    const int dl = h->bond[s], dr = h->bond[s + 1];
    const double2* A = h->site(s);
    const long la = 9L * dr, sd = 4L * dr;   // diagonal eta = 0, 4, 8
    // T_s = E A_s, batched over the three diagonal entries
    VK(cgemm<double>(h->st, OP_N, OP_N, dl, dr, dl, E, dl, 0, A, la, sd, T, dr, (long)dl * dr, 3,
                     one, zero));
    for (int q = 0; q < 3; ++q) {
      VK(cgemm<double>(h->st, OP_T, OP_N, dr, dr, dl, A + q * sd, la, 0, T + (long)q * dl * dr, dr,
                       0, En, dr, 0, 1, one, q ? one : zero));
      VK(cgemm<double>(h->st, OP_N, OP_N, 1, dr, dl, t, dl, 0, A + q * sd, la, 0, tn, dr, 0, 1,
                       one, q ? one : zero));
    }
    std::swap(E, En);
    std::swap(t, tn);
  }
  double2 r[2];
  VK(cudaMemcpyAsync(&r[0], E, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
  VK(cudaMemcpyAsync(&r[1], t, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
  VK(cudaStreamSynchronize(h->st));
  if (!(r[1].x != 0) || !std::isfinite(r[1].x)) return vfail(h, MPDO_ERR_NUMERIC, "vmpo: zero trace");
  *collision = r[0].x / (r[1].x * r[1].x);
  return MPDO_OK;
}

int mpdo_vmpo_get_dims(mpdo_vmpo h, int* bond_dims, int* centre) {
  if (!h) return vfail(nullptr, MPDO_ERR_ARG, "vmpo: null handle");
  for (int u = 0; u < h->n - 1; ++u) {
    const int s = h->rev ? h->n - 1 - u : u;
    if (bond_dims) bond_dims[u] = h->rev ? h->bond[s] : h->bond[s + 1];
  }
  if (centre) *centre = h->centre;
  return MPDO_OK;
}

int mpdo_vmpo_set_precision(mpdo_vmpo h, int mode) {
  if (!h || (mode != 0 && mode != 1)) return vfail(h, MPDO_ERR_ARG, "vmpo: mode must be 0 or 1");
  if (mode == 1 && !h->mixmem) {
    const int n9 = 9 * h->chi;
    const size_t tw = (size_t)256 << 20;
    int rc;
    if ((rc = valloc(h, &h->mixmem, mix_work_bytes(n9))) || (rc = valloc(h, &h->tcws, tw)) ||
        (rc = valloc(h, (void**)&h->tcerr, sizeof(int)))) {
      h->mixmem = nullptr;
      return rc;
    }
    if (cudaMallocHost((void**)&h->htcerr, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h->htcerr = nullptr;
      h->mixmem = nullptr;
      return vfail(h, MPDO_ERR_OOM, "vmpo: pinned host allocation");
    }
    *h->htcerr = 0;
    mix_work_bind(h->mixw, h->mixmem, n9);
    h->mixw.tcws = h->tcws;
    h->mixw.tcws_bytes = tw;
    h->mixw.tcerr = h->tcerr;
    h->mixw.tc_min_macs = (double)(1 << 21);
    h->tcws_bytes = tw;
  }
  h->tc = mode;
  // the mixed solver resolves eigenvalues to ~1e-14 of the largest: numerical zeros below
  // 10 x that in the tensor-core form, below 1e-15 in FP64
  h->cut2 = std::max(h->sv_req * h->sv_req, mode ? 1e-13 : 1e-15);
  VK(cudaStreamSynchronize(h->st));
  return MPDO_OK;
}

int mpdo_vmpo_destroy(mpdo_vmpo h) {
  if (!h) return MPDO_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  mix_work_release(h->mixw);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->htcerr) cudaFreeHost(h->htcerr);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
  return MPDO_OK;
}

}  // extern "C"
