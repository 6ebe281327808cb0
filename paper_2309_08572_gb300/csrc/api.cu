// C ABI of libmpdo: handle management, the two-site MPDO update driver, observables and
// sampling.  The arithmetic of every step runs in the kernels of gemm.cu, jacobi.cu and
// kernels.cu; this file only sequences them and moves a few scalars to the host.
//
// Update of a bond (i, i+1) with the orthogonality centre at i (Sec. III.A, Fig. 2c):
// with M_i = A_i as [(l,k_i) x (s_i,b)] and N_j = A_{i+1} as [(b,s_j) x (k_j,r)],
//   G_i = M_i^+ M_i,  G_j = N_j N_j^+                               (Gram matrices)
//   G_i = V diag(sigma) V^+,  R = diag(sqrt sigma) V^+             (left factor)
//   Phi[(S,s,b),(S',s',b')] = sum_{t,t'} C[(S,s,t),(S',s',t')] G_j[(b,t),(b',t')]
//       with C = sum_{m,T} E_m[(S,T),(s,t)] conj(E_m[(S',T),(s',t')])
//   H = (I (x) R) Phi (I (x) R)^+ = Z Z^+ for the reduced two-site tensor Z
// The eigenpairs (lambda = s^2, u) of H give the truncated SVD of theta' = (M_i (x) I) Y:
//   new A_i  = (M_i (x) I)(I (x) V sigma^-1/2) u        (left-orthonormal)
//   new A_j  = renorm * ((I (x) V sigma^1/2) u)^+ Gamma (I (x) N_j), Gamma = the channel,
// whose inner index (m, k_j) is then truncated by the eigenpairs of its Gram matrix and
// the purity-preserving rescaling (Sec. III.D).  Right-to-left updates run on the
// mirrored chain (site order and the l/r bond indices swapped, channel sites swapped).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/mpdo.h"
#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgemm.h"

using namespace mpdo;

namespace mpdo {
std::atomic<long long> g_launches{0};
}

namespace {
thread_local std::string g_err;
}

namespace mpdo {
// handle-less error message, read back by mpdo_last_error(NULL)
void set_global_error(const char* msg) { g_err = msg ? msg : ""; }
}

namespace {

struct DevOp {
  int kind = 2;
  int site = 0;
  int m = 1;
  void* e = nullptr;      // M x 81 (precision of the handle)
  void* em = nullptr;     // mirrored (sites swapped)
  void* ct = nullptr;     // 27 x 27
  void* ctm = nullptr;    // mirrored
  void* u = nullptr;      // kind 1: 3x3
};

}  // namespace

struct mpdo_dlayer_s {
  std::vector<DevOp> ops;
  void* mem = nullptr;
};

struct mpdo_ctx {
  mpdo_config cfg{};
  cudaStream_t st = nullptr;
  std::string err;
  int n = 0, chi = 0, kmax = 0, mmax = 1;
  int n_cap = 0, chi_cap = 0, kmax_cap = 0;   // allocation capacity (mpdo_reconfigure)
  int use_ppt = 1;
  int device = 0;
  bool own_stream = false;
  bool dbl = true;     // complex128 state and arithmetic
  bool rev = false;    // chain stored mirrored
  int centre = 0;      // user coordinates
  double gtol = 0, htol = 0, kcut = 0;
  int max_sweeps = 30;
  std::vector<int> bond;  // storage coords, size n+1
  std::vector<int> kd;    // storage coords, size n
  size_t elt = 16;        // bytes per complex
  size_t site_cap = 0;    // complex elements per site
  void* sites = nullptr;   // one arena: site s at s * site_cap elements
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<void*> allocs;
  void *wPol, *wQol, *wGa;   // polar correction of the new left tensor (keep x keep)
  void *wM, *wGi, *wGj, *wVg, *wR, *wVs, *wVr, *wPhi, *wX, *wH, *wU, *wVgen, *wW, *wTmp, *wQ,
      *wWB, *wBp, *wWK, *wVk, *wVks, *wCn, *wRs, *wIrs, *eigmem;
  double *wSig, *wLam, *wWv, *wF;
  EigWork<double> eig64;
  EigWork<float> eig32;
  // FP32 site tensors with FP64 Gram matrices and small-matrix arithmetic (cfg.gram_fp64)
  bool mixed = false;
  // complex64 products on the tensor cores (MPDO_TF32X3 / MPDO_BF16X3): the operand mode
  // (TC_TF32X3 / TC_BF16X3, -1 = CUDA-core GEMMs), the packing workspace and the device flag
  // the pipeline sets when one of its bounded waits gives up
  int tcmode = -1;
  void* tcws = nullptr;
  size_t tcws_bytes = 0;
  int* tcerr = nullptr;
  int* htcerr = nullptr;   // pinned
  double tc_min_macs = 0;  // routing threshold (kTcMinMacs; MPDO_TC_MIN_MACS overrides)
  // Waits for the host read-backs of the update: spinning (cudaStreamSynchronize) for one
  // circuit; blocking on an event (the thread sleeps) while the batch executor runs many
  // circuits, whose spinning host threads would otherwise take every core.
  cudaEvent_t bev = nullptr;
  bool block_sync = false;
  // inner eigenproblem through a pivoted Cholesky (see inner_eig)
  void *wL = nullptr, *wGs = nullptr, *wZ = nullptr, *wLg = nullptr;
  struct PcOut { int r; int pad; double resid; };
  PcOut* dpc = nullptr;
  PcOut* hpc = nullptr;       // pinned
  MixWork mixw;              // mixed-precision eigensolver workspace (mixed only)
  void* mixmem = nullptr;
  size_t eltm = 16;          // bytes per complex of the Gram-derived matrices
  void* wAcM = nullptr;      // polar-corrected left factor in FP64 (mixed only)
  StepScalars* dsc = nullptr;
  StepScalars* hsc = nullptr;  // pinned
  double* dtrace = nullptr;    // trace of the state, carried in FP64 across updates
  double htrace0 = 1.0;        // its initial value (host copy, source of the upload)
  DevStats* dstats = nullptr;
  DevStats* hstats = nullptr;  // pinned
  // identity two-site channel (one op, uploaded at create) for the left-to-right order
  mpdo_dlayer_s ident;
  // staging for host layers
  mpdo_dlayer_s staged;
  size_t staged_cap = 0;
  unsigned char* hstage = nullptr;   // pinned host staging of staged layers
  size_t hstage_cap = 0;
  // lazily allocated observable buffers
  void* obs = nullptr;
  size_t obs_bytes = 0;
  // optional per-class kernel timing (0: GEMM, 1: eigensolver, 2: other kernels)
  struct ProfRec { int cls; int e0; double flops; int slot; double per_count; };
  int prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0;
  std::vector<ProfRec> prof_recs;
  double prof_ms[3] = {0, 0, 0};
  long long prof_cnt[3] = {0, 0, 0};
  double prof_flops[3] = {0, 0, 0};
  int* prof_counts = nullptr;   // pinned: active pair-rounds of profiled eigensolves
  int prof_nslots = 0, prof_slot = 0;

  void* site(int s) const { return static_cast<char*>(sites) + (size_t)s * site_cap * elt; }
};

namespace {

int fail(mpdo_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_err = msg;
  return code;
}
int cuda_fail(mpdo_ctx* h, cudaError_t e, const char* where) {
  return fail(h, MPDO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(expr)                                          \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #expr); \
  } while (0)

int prof_begin(mpdo_ctx* h, int cls) {
  if (!(h->prof_mask & (1 << cls)) || h->prof_used + 2 > (int)h->prof_ev.size()) return -1;
  int i = h->prof_used;
  h->prof_used += 2;
  cudaEventRecord(h->prof_ev[i], h->st);
  return i;
}
void prof_end(mpdo_ctx* h, int cls, int i, double flops, int slot = -1, double per_count = 0) {
  if (i < 0) return;
  cudaEventRecord(h->prof_ev[i + 1], h->st);
  h->prof_recs.push_back({cls, i, flops, slot, per_count});
}
// called after the stream has been synchronised
void prof_drain(mpdo_ctx* h) {
  for (const auto& r : h->prof_recs) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->prof_ev[r.e0], h->prof_ev[r.e0 + 1]) == cudaSuccess) {
      h->prof_ms[r.cls] += ms;
      h->prof_cnt[r.cls] += 1;
      h->prof_flops[r.cls] += r.flops;
      if (r.slot >= 0) h->prof_flops[r.cls] += r.per_count * h->prof_counts[r.slot];
    }
  }
  cudaGetLastError();
  h->prof_recs.clear();
  h->prof_used = 0;
  h->prof_slot = 0;
}
#define PO(expr)                     \
  do {                               \
    int _pi = prof_begin(h, 2);      \
    CK(expr);                        \
    prof_end(h, 2, _pi, 0.0);        \
  } while (0)

template <typename R>
cx<R> one() { return mkc<R>(1, 0); }
template <typename R>
cx<R> zero() { return mkc<R>(0, 0); }

template <typename R>
EigWork<R>& eigw(mpdo_ctx* h);
template <>
EigWork<double>& eigw<double>(mpdo_ctx* h) { return h->eig64; }
template <>
EigWork<float>& eigw<float>(mpdo_ctx* h) { return h->eig32; }

// Device memory of a handle: through the config's hooks when given, else cudaMalloc.
void* dmalloc(mpdo_ctx* h, size_t bytes) {
  if (h->cfg.alloc) return h->cfg.alloc(bytes, h->cfg.alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dfree(mpdo_ctx* h, void* p) {
  if (!p) return;
  if (h->cfg.alloc) h->cfg.free(p, h->cfg.alloc_ctx);
  else cudaFree(p);
}

int alloc_dev(mpdo_ctx* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  *p = dmalloc(h, bytes);
  if (!*p) return fail(h, MPDO_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  // no handle buffer ever starts with stale contents of earlier allocations
  cudaError_t e = cudaMemsetAsync(*p, 0, bytes, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    dfree(h, *p);
    *p = nullptr;
    return fail(h, MPDO_ERR_CUDA, "clearing a new device buffer failed");
  }
  h->allocs.push_back(*p);
  return MPDO_OK;
}

cudaError_t sync_stream(mpdo_ctx* h) {
  if (h->block_sync && h->bev) {
    cudaError_t e = cudaEventRecord(h->bev, h->st);
    return e == cudaSuccess ? cudaEventSynchronize(h->bev) : e;
  }
  return cudaStreamSynchronize(h->st);
}

int read_scalars(mpdo_ctx* h) {
  CK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(StepScalars), cudaMemcpyDeviceToHost, h->st));
  if (h->tcerr) CK(cudaMemcpyAsync(h->htcerr, h->tcerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(sync_stream(h));
  prof_drain(h);
  if (h->tcerr && *h->htcerr)
    return fail(h, MPDO_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait gave up");
  if (h->hsc->flags & 1) return fail(h, MPDO_ERR_NUMERIC, "zero or non-finite state in update");
  return MPDO_OK;
}

// Products at least this large (complex multiply-adds, both output sides >= kTcMinSide) run on
// the tensor cores in the MPDO_TF32X3 / MPDO_BF16X3 modes; smaller ones stay on the CUDA-core
// kernels, whose single launch has less latency than packing plus a pipelined tile.
constexpr double kTcMinMacs = 1 << 21;
constexpr int kTcMinSide = 16;

// Products with FP64 outputs in the tensor-core forms with FP64 Grams (mixed form): the
// error-free slice products on the BF16 tensor cores (tc_cgemm_exact) when large enough.
inline bool tc_exact_route(const mpdo_ctx* h, int m, int n, int k, int batch) {
  return h->tcmode >= 0 && h->mixed && (double)m * n * k * batch >= h->tc_min_macs &&
         m >= kTcMinSide && n >= kTcMinSide && k >= 1;
}
template <typename TA, typename TB>
cudaError_t pexact(mpdo_ctx* h, int opa, int opb, int m, int n, int k, const TA* A, long lda,
                   long sa, const TB* B, long ldb, long sb, double2* C, long ldc, long sc,
                   int batch) {
  int pi = prof_begin(h, 0);
  cudaError_t e = tc_cgemm_exact<TA, TB>(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc,
                                         sc, batch, h->tcws, h->tcws_bytes, h->tcerr);
  prof_end(h, 0, pi, 8.0 * m * n * (double)k * batch);
  return e;
}

template <typename R>
cudaError_t pgemm(mpdo_ctx* h, int opa, int opb, int m, int n, int k, const cx<R>* A, long lda,
                  long sa, const cx<R>* B, long ldb, long sb, cx<R>* C, long ldc, long sc,
                  int batch) {
  if constexpr (std::is_same<R, double>::value) {
    if (tc_exact_route(h, m, n, k, batch))
      return pexact<double2, double2>(h, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc,
                                      batch);
  }
  if constexpr (std::is_same<R, float>::value) {
    if (h->tcmode >= 0 && (double)m * n * k * batch >= h->tc_min_macs && m >= kTcMinSide &&
        n >= kTcMinSide && k >= 1) {
      int pi = prof_begin(h, 0);
      cudaError_t e = tc_cgemm<float>(h->st, h->tcmode, opa, opb, m, n, k, A, lda, sa, B, ldb,
                                      sb, C, ldc, sc, batch, make_float2(1.f, 0.f),
                                      make_float2(0.f, 0.f), h->tcws, h->tcws_bytes, h->tcerr);
      prof_end(h, 0, pi, 8.0 * m * n * (double)k * batch);
      return e;
    }
  }
  int pi = prof_begin(h, 0);
  cudaError_t e = cgemm<R>(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch,
                           one<R>(), zero<R>());
  prof_end(h, 0, pi, 8.0 * m * n * (double)k * batch);
  return e;
}
// floor: eigenpairs below floor * lambda_max need not be resolved (used by the mixed mode).
// kMixedEigMax: largest factor rank taken through the lifted route (the factor buffer holds
// 128 columns); the mixed solver itself serves any n up to the handle's capacity (one-CTA
// FP32 sweeps up to n = 118, the cooperative FP32 block Jacobi above, FP64 refinement).
// max_vals > 0: only that many leading pairs are needed (the rest come back as zeros).
constexpr int kMixedEigMax = 118;
template <typename R>
cudaError_t peig(mpdo_ctx* h, int n, const cx<R>* a, long lda, cx<R>* v, long ldv, double* w,
                 double floor, int max_vals = 0) {
  int pi = prof_begin(h, 1);
  const int sweeps = std::is_same<R, double>::value ? 30 : 20;
  cudaError_t e;
  if constexpr (std::is_same<R, double>::value) {
    if (h->mixed && n <= h->mixw.n_cap) {
      double fl = 0.0;
      e = heig_mixed(h->st, n, a, lda, v, ldv, w, floor, h->mixw, nullptr, &fl, max_vals);
      prof_end(h, 1, pi, fl);
      return e;
    }
  }
  e = heig<R>(h->st, n, a, lda, v, ldv, w, eigw<R>(h), sweeps);
  if (pi >= 0 && e == cudaSuccess && h->prof_slot < h->prof_nslots) {
    // executed flops: 8 real flops per complex MAC, 3*16*16*np MACs per active pair-round
    int slot = h->prof_slot++;
    e = cudaMemcpyAsync(&h->prof_counts[slot], eigw<R>(h).counters + 3, sizeof(int),
                        cudaMemcpyDeviceToHost, h->st);
    prof_end(h, 1, pi, 0.0, slot, eig_flops_per_count(n, std::is_same<R, double>::value));
  } else {
    prof_end(h, 1, pi, 0.0);
  }
  return e;
}

// Gram-type product with storage-precision inputs and small-matrix-precision output:
// FP32 inputs with FP64 products and sums when RS = float and RM = double.
template <typename RS, typename RM>
cudaError_t pgram(mpdo_ctx* h, int opa, int opb, int m, int n, int k, const cx<RS>* A, long lda,
                  const cx<RS>* B, long ldb, cx<RM>* C, long ldc) {
  if constexpr (std::is_same<RS, RM>::value) {
    return pgemm<RS>(h, opa, opb, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1);
  } else {
    if (tc_exact_route(h, m, n, k, 1))
      return pexact<float2, float2>(h, opa, opb, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1);
    int pi = prof_begin(h, 0);
    cudaError_t e = cgemm_wide<float>(h->st, opa, opb, m, n, k, A, lda, 0, B, ldb, 0, C, ldc, 0, 1);
    prof_end(h, 0, pi, 8.0 * m * n * (double)k);
    return e;
  }
}

// FP32 A times B of precision RB with FP64 products and sums (mixed mode).
template <typename RB>
cudaError_t pwide(mpdo_ctx* h, int opa, int opb, int m, int n, int k, const cx<float>* A,
                  long lda, long sa, const cx<RB>* B, long ldb, long sb, cx<double>* C, long ldc,
                  long sc, int batch) {
  if (tc_exact_route(h, m, n, k, batch))
    return pexact<float2, cx<RB>>(h, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch);
  int pi = prof_begin(h, 0);
  cudaError_t e =
      cgemm_wide<RB>(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch);
  prof_end(h, 0, pi, 8.0 * m * n * (double)k * batch);
  return e;
}

// a8: eigenpairs of the inner Gram W (nin x nin, in wWK).  Small problems: all of them by
// Jacobi.  Larger ones: only the leading part matters (at most k_max are kept; the total
// weight comes from tr W and the PPT's |w|^2 from the eigenvalues, where the tail below the
// factor's tolerance is negligible), so W ~ L L^+ by a pivoted Cholesky stopping at
// kInnerTol64 (FP64 mode) or kInnerTol (FP32 factor) of tr W, and the eigenpairs of W are
// lifted from those of the r x r matrix L^+ L: u_c = L z_c / sqrt(s_c).  A factor that
// reaches kInnerRmax columns above the tolerance falls back to the full solve.
// Eigenvectors go to wVk (row stride nin); returns their count.
constexpr int kInnerDirect = 32;

// Stopping tolerance of the factor for a cut at `cut` of the largest eigenvalue: 1% of the
// cut, but not below what the factor's precision resolves (FP64 ~1e-15 of the trace;
// FP32 ~1e-7, used only in C64 mode whose cuts sit at 6e-7).
inline double pc_tol(const mpdo_ctx* h, double cut) {
  const double floor = (h->dbl || h->mixed) ? 1e-16 : 2e-7;
  return std::max(0.01 * cut, floor);
}
constexpr double kInnerTol = 1e-7;
constexpr double kInnerTol64 = 1e-14;
constexpr double kInnerTolMixed = 1e-10;
constexpr int kInnerRmax = 128;

// Eigenpairs of the PSD Gram g (n x n, Gram precision RM) through its pivoted Cholesky
// factor g ~ L L^+ (stopping at tol * tr g) and one-sided Jacobi on L: eigenvectors to
// v (row stride ldv), eigenvalues to w, descending (FP64 factor and rotations for FP64
// Grams, FP32 for FP32 Grams).
// *nvals = r on success (columns r..n-1 of v and w[r..n) zeroed when zero_tail), 0 when
// the factor does not fit (rank above the shared-memory cap) and the caller must solve
// otherwise.  One host synchronisation (the rank).
template <typename RM>
int pc_eig(mpdo_ctx* h, int n, const cx<RM>* g, cx<RM>* v, long ldv, double* w, double tol,
           bool zero_tail, int* nvals) {
  cudaStream_t st = h->st;
  *nvals = 0;
  if (n < 1 || n > 1024) return MPDO_OK;
  const size_t rbytes = std::is_same<RM, double>::value ? 16 : 8;
  int rcap = (int)std::min<size_t>(128, kOsjMaxSmem / (rbytes * (size_t)n));
  rcap -= rcap & 1;
  const int rmax = std::min(n, rcap);
  if (rmax < 1) return MPDO_OK;
  int pi = prof_begin(h, 1);
  if constexpr (std::is_same<RM, double>::value) {
    CK(pchol<double>(st, n, g, rmax, tol, static_cast<double2*>(h->wLg), kInnerRmax,
                     &h->dpc->r, &h->dpc->resid));
  } else {
    CK(pchol<float>(st, n, g, rmax, tol, static_cast<float2*>(h->wLg), kInnerRmax, &h->dpc->r,
                    &h->dpc->resid));
  }
  CK(cudaMemcpyAsync(h->hpc, h->dpc, sizeof(mpdo_ctx::PcOut), cudaMemcpyDeviceToHost, st));
  CK(sync_stream(h));
  const int r = h->hpc->r;
  if (r < 1 || (r >= rmax && r < n && h->hpc->resid > tol)) {
    prof_end(h, 1, pi, 0.0);
    prof_drain(h);
    return MPDO_OK;
  }
  int* cnt = eigw<RM>(h).counters;
  if constexpr (std::is_same<RM, double>::value) {
    const double2* L = static_cast<const double2*>(h->wLg);
    CK((osj<double, double, double>(st, n, r, L, kInnerRmax, v, (int)ldv, w, cnt, 0)));
  } else {
    const float2* L = static_cast<const float2*>(h->wLg);
    CK((osj<float, float, float>(st, n, r, L, kInnerRmax, v, (int)ldv, w, cnt, 0)));
  }
  if (zero_tail && r < n) {
    CK(cudaMemset2DAsync(v + r, ldv * sizeof(cx<RM>), 0, (n - r) * sizeof(cx<RM>), n, st));
    CK(cudaMemsetAsync(w + r, 0, (n - r) * sizeof(double), st));
  }
  // executed flops: per rotation 3 dot products and 2 column updates of n complex entries
  // (8 real flops each); the rotation count is read back with the profile
  if (pi >= 0 && h->prof_slot < h->prof_nslots) {
    int slot = h->prof_slot++;
    CK(cudaMemcpyAsync(&h->prof_counts[slot], cnt + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    prof_end(h, 1, pi, 0.0, slot, 8.0 * 5 * (double)n);
  } else {
    prof_end(h, 1, pi, 0.0);
  }
  *nvals = r;
  return MPDO_OK;
}

// Eigenpairs of the PSD Gram g (n x n) through a pivoted Cholesky factor g ~ L L^+
// (stopping at tol * tr g, at most rmax columns; FP64 factor for FP64 Grams, FP32 for
// FP32 Grams) and the eigenpairs of the r x r matrix L^+ L (solved down to floor of its
// largest), lifted as u = L z / sqrt(s): eigenvectors to v (row stride ldv), eigenvalues
// to w, descending.  *nvals = r, or 0 when the factor needs more than rmax columns (the
// caller solves the full problem).  zero_tail: columns r..n-1 of v and w[r..n) zeroed.
template <typename RM>
int lift_eig(mpdo_ctx* h, int n, const cx<RM>* g, cx<RM>* v, long ldv, double* w, double tol,
             int rmax, double floor, bool zero_tail, int* nvals, int max_vals = 0) {
  using TM = cx<RM>;
  cudaStream_t st = h->st;
  *nvals = 0;
  rmax = std::min(rmax, n);
  if (n < 1 || n > 1024 || rmax < 1) return MPDO_OK;
  TM* L = static_cast<TM*>(h->wLg);
  int pi = prof_begin(h, 2);
  CK(pchol<RM>(st, n, g, rmax, tol, L, kInnerRmax, &h->dpc->r, &h->dpc->resid));
  prof_end(h, 2, pi, 0.0);
  CK(cudaMemcpyAsync(h->hpc, h->dpc, sizeof(mpdo_ctx::PcOut), cudaMemcpyDeviceToHost, st));
  CK(sync_stream(h));
  prof_drain(h);
  const int r = h->hpc->r;
  if (r < 1 || (r >= rmax && r < n && h->hpc->resid > tol)) return MPDO_OK;
  TM* Gs = static_cast<TM*>(h->wGs);
  TM* Z = static_cast<TM*>(h->wZ);
  CK(pgemm<RM>(h, OP_C, OP_N, r, r, n, L, kInnerRmax, 0, L, kInnerRmax, 0, Gs, r, 0, 1));
  CK(peig<RM>(h, r, Gs, r, Z, r, w, floor, max_vals));
  PO(lift<RM>(st, r, Z, w, Gs));
  CK(pgemm<RM>(h, OP_N, OP_N, n, r, r, L, kInnerRmax, 0, Gs, r, 0, v, ldv, 0, 1));
  if (zero_tail && r < n) {
    CK(cudaMemset2DAsync(v + r, ldv * sizeof(TM), 0, (n - r) * sizeof(TM), n, st));
    CK(cudaMemsetAsync(w + r, 0, (n - r) * sizeof(double), st));
  }
  *nvals = r;
  return MPDO_OK;
}

template <typename RM>
int inner_eig(mpdo_ctx* h, int nin, int* nvals) {
  cx<RM>* W = static_cast<cx<RM>*>(h->wWK);
  cx<RM>* V = static_cast<cx<RM>*>(h->wVk);
  int rc;
  if (h->dbl) {
    // FP64 mode: factor + one-sided Jacobi when the rank fits; the Kraus tail below the
    // tolerance is negligible for the cut and the PPT sums
    int nv = 0;
    rc = pc_eig<RM>(h, nin, W, V, nin, h->wWv, kInnerTol64, false, &nv);
    if (rc) return rc;
    if (nv > 0) {
      *nvals = nv;
      return MPDO_OK;
    }
  }
  if (nin <= kInnerDirect) {
    CK(peig<RM>(h, nin, W, nin, V, nin, h->wWv, 1e-10));
    *nvals = nin;
    return MPDO_OK;
  }
  // FP64 and mixed modes: FP64 factor (down to 1e-14 resp. 1e-10 of the trace); C64: FP32
  // factor down to its floor.  (An FP32 factor of the FP64 Gram in mixed mode resolved the
  // kept Kraus directions only to ~1e-7 of the largest weight, which moved energies by
  // up to 1e-5 where two weights at the cut were close.)  Mixed: L^+ L stays within the
  // mixed solver's size.
  const double tol = h->dbl ? kInnerTol64 : h->mixed ? kInnerTolMixed : kInnerTol;
  int nv = 0;
  // at most k_max pairs are kept (the PPT's sum of squares comes from ||W||_F), so the
  // solver may stop once k_max + 1 leading pairs are resolved
  rc = lift_eig<RM>(h, nin, W, V, nin, h->wWv, tol, h->mixed ? kMixedEigMax : kInnerRmax, 1e-10,
                    false, &nv, h->kmax + 1);
  if (rc) return rc;
  if (nv == 0) {
    // at most k_max pairs are kept; the PPT's sum of squares comes from ||W||_F
    CK(peig<RM>(h, nin, W, nin, V, nin, h->wWv, 1e-10, h->kmax + 1));
    nv = nin;
  }
  *nvals = nv;
  return MPDO_OK;
}

// ------------------------------------------------------------------ the update
// RS: precision of the site tensors and of the large contractions (a4, a7, a10);
// RM: precision of the Gram matrices and everything derived from them (a2 outputs, a3,
// a5, a6, a8, a9 and the factors that feed a7 and a10).
template <typename RS, typename RM>
int update_lr(mpdo_ctx* h, int i, const DevOp& op, bool mirrored, int chi, int kmax,
              int use_ppt) {
  using T = cx<RS>;
  using TM = cx<RM>;
  cudaStream_t st = h->st;
  const int dl = h->bond[i], ki = h->kd[i], dm = h->bond[i + 1], kj = h->kd[i + 1],
            dr = h->bond[i + 2];
  const int M = op.m;
  const int n3 = 3 * dm, n9 = 9 * dm;
  T* ai = static_cast<T*>(h->site(i));
  T* aj = static_cast<T*>(h->site(i + 1));
  const T* E = static_cast<const T*>(mirrored ? op.em : op.e);
  const TM* Ct = static_cast<const TM*>(mirrored ? op.ctm : op.ct);
  T* wM = static_cast<T*>(h->wM);
  TM* wGi = static_cast<TM*>(h->wGi);
  TM* wGj = static_cast<TM*>(h->wGj);
  TM* wVg = static_cast<TM*>(h->wVg);
  TM* wR = static_cast<TM*>(h->wR);
  TM* wVs = static_cast<TM*>(h->wVs);
  TM* wVr = static_cast<TM*>(h->wVr);
  TM* wPhi = static_cast<TM*>(h->wPhi);
  TM* wX = static_cast<TM*>(h->wX);
  TM* wH = static_cast<TM*>(h->wH);
  TM* wU = static_cast<TM*>(h->wU);
  TM* wVgen = static_cast<TM*>(h->wVgen);
  T* wW = static_cast<T*>(h->wW);
  T* wTmp = static_cast<T*>(h->wTmp);
  T* wQ = static_cast<T*>(h->wQ);
  T* wWB = static_cast<T*>(h->wWB);
  T* wBp = static_cast<T*>(h->wBp);
  TM* wWK = static_cast<TM*>(h->wWK);
  TM* wVk = static_cast<TM*>(h->wVk);
  T* wVks = static_cast<T*>(h->wVks);
  T* wCn = static_cast<T*>(h->wCn);
  RM* wRs = static_cast<RM*>(h->wRs);
  RM* wIrs = static_cast<RM*>(h->wIrs);

  int rc;
  // a2: Gram matrices of the two site tensors
  PO(swap12<T>(st, dl, 3, ki, dm, ai, wM));
  CK((pgram<RS, RM>(h, OP_C, OP_N, n3, n3, dl * ki, wM, n3, wM, n3, wGi, n3)));
  CK((pgram<RS, RM>(h, OP_N, OP_C, n3, n3, kj * dr, aj, (long)kj * dr, aj, (long)kj * dr, wGj,
                    n3)));
  PO(trace_pre<RM>(st, dm, wGi, wGj, h->dsc));
  // a3: left factor from the eigendecomposition of G_i (numerical rank by gtol)
  {
    int nv = 0;
    // FP64 mode: FP64 factor + one-sided Jacobi.  Mixed: FP64 factor and the mixed solver
    // on L^+ L (rank r instead of 3D; rotating an FP32 copy of the factor instead loses the
    // small eigenvalues: its rounding is relative to whole columns, not to eigen-
    // directions), the factor route on larger ranks.  C64: the FP32 Jacobi solver.
    if (h->mixed) {
      rc = lift_eig<RM>(h, n3, wGi, wVg, n3, h->wSig, pc_tol(h, h->gtol), kMixedEigMax,
                        0.1 * h->gtol, true, &nv);
      if (rc) return rc;
    }
    if (nv == 0 && (h->dbl || (h->mixed && n3 > h->mixw.n_cap))) {
      rc = pc_eig<RM>(h, n3, wGi, wVg, n3, h->wSig, pc_tol(h, h->gtol), true, &nv);
      if (rc) return rc;
    }
    if (nv == 0) CK(peig<RM>(h, n3, wGi, n3, wVg, n3, h->wSig, 0.1 * h->gtol));
  }
  PO(gram_mask<RM>(st, n3, h->wSig, h->gtol, wRs, wIrs, h->dsc));
  PO(gram_factor<RM>(st, n3, wVg, wRs, wIrs, wR, wVs, wVr));
  // a4/a5: Phi from the channel and G_j, then H = (I x R) Phi (I x R)^+
  PO(build_phi<RM>(st, dm, Ct, wGj, wPhi));
  CK(pgemm<RM>(h, OP_N, OP_N, n3, n9, n3, wR, n3, 0, wPhi, n9, (long)n3 * n9, wX, n9,
               (long)n3 * n9, 3));
  CK(pgemm<RM>(h, OP_N, OP_C, n9, n3, n3, wX, n9, n3, wR, n3, 0, wH, n9, n3, 3));
  // a6: bond eigenpairs and cut
  {
    int nv = 0;
    if (h->mixed) {
      rc = lift_eig<RM>(h, n9, wH, wU, n9, h->wLam, pc_tol(h, h->htol), kMixedEigMax,
                        0.1 * h->htol, true, &nv, chi + 1);
      if (rc) return rc;
    }
    if (nv == 0 && (h->dbl || (h->mixed && n9 > h->mixw.n_cap))) {
      rc = pc_eig<RM>(h, n9, wH, wU, n9, h->wLam, pc_tol(h, h->htol), true, &nv);
      if (rc) return rc;
    }
    // at most chi pairs are kept: the (chi+1)-th decides nothing more (the discarded weight
    // comes from tr H)
    if (nv == 0) CK(peig<RM>(h, n9, wH, n9, wU, n9, h->wLam, 0.1 * h->htol, chi + 1));
  }
  PO(bond_select<RM>(st, n9, h->wLam, wH, n9, h->htol, chi, h->dsc, h->dstats));
  rc = read_scalars(h);
  if (rc) return rc;
  const int keep = h->hsc->keep;
  // a7: split.  Vgen = (I x V sigma^-1/2) U_keep
  CK(pgemm<RM>(h, OP_N, OP_N, n3, keep, n3, wVs, n3, 0, wU, n9, (long)n3 * n9, wVgen, keep,
               (long)n3 * keep, 3));
  // The left factor A = (M_i x I)(I x V sigma^-1/2) U_keep is an isometry only up to the
  // error of the small-sigma eigenvectors of G_i, amplified by sigma^-1/2.  One
  // Newton-Schulz polar step (Higham) restores it: A <- A (3I - A^+A)/2.  The centre
  // factor is then the projection of the two-site block onto the kept left vectors,
  // W_s' = M_i^+ A_s' (= (I x V sigma^1/2) U_keep when the eigenpairs are exact), so that
  // theta' = A A^+ theta holds to rounding whatever the eigenvector error.
  const int rows = dl * ki * 3;
  if constexpr (!std::is_same<RS, RM>::value) {
    // Mixed precision: A, its polar step and W in FP64 from the stored FP32 M_i.  Rounding
    // M_i Vgen to FP32 before the step would be amplified by sigma^-1/2 of the smallest
    // kept sigma (down to 1e-13 of the largest here), beyond what one step can repair.
    TM* aM = static_cast<TM*>(h->wTmp);
    TM* acM = static_cast<TM*>(h->wAcM);
    TM* gaM = static_cast<TM*>(h->wGa);
    TM* polM = static_cast<TM*>(h->wPol);
    TM* qolM = static_cast<TM*>(h->wQol);
    CK(pwide<RM>(h, OP_N, OP_N, dl * ki, keep, n3, wM, n3, 0, wVgen, keep, (long)n3 * keep, aM,
                 3L * keep, keep, 3));
    CK(pgemm<RM>(h, OP_C, OP_N, keep, keep, rows, aM, keep, 0, aM, keep, 0, gaM, keep, 0, 1));
    PO(polar_factors<RM>(st, keep, gaM, polM, qolM));
    CK(pgemm<RM>(h, OP_N, OP_N, rows, keep, keep, aM, keep, 0, polM, keep, 0, acM, keep, 0, 1));
    // W in FP64 into wVgen (no longer needed), then rounded to the storage precision
    CK(pwide<RM>(h, OP_C, OP_N, n3, keep, dl * ki, wM, n3, 0, acM, 3L * keep, keep, wVgen, keep,
                 (long)n3 * keep, 3));
    CK((convert<RM, RS>(st, n9, keep, wVgen, keep, wW, keep)));
    CK((convert<RM, RS>(st, rows, keep, acM, keep, wWB, keep)));
  } else {
    T* wGa = static_cast<T*>(h->wGa);
    T* wPol = static_cast<T*>(h->wPol);
    T* wQol = static_cast<T*>(h->wQol);
    CK(pgemm<RS>(h, OP_N, OP_N, dl * ki, keep, n3, wM, n3, 0, wVgen, keep, (long)n3 * keep,
                 wTmp, 3L * keep, keep, 3));
    CK(pgemm<RS>(h, OP_C, OP_N, keep, keep, rows, wTmp, keep, 0, wTmp, keep, 0, wGa, keep, 0, 1));
    PO(polar_factors<RS>(st, keep, wGa, wPol, wQol));
    CK(pgemm<RS>(h, OP_N, OP_N, rows, keep, keep, wTmp, keep, 0, wPol, keep, 0, wWB, keep, 0, 1));
    CK(pgemm<RS>(h, OP_C, OP_N, n3, keep, dl * ki, wM, n3, 0, wWB, 3L * keep, keep, wW, keep,
                 (long)n3 * keep, 3));
  }
  PO(swap12<T>(st, dl, ki, 3, keep, wWB, ai));
  PO(make_q<RS>(st, dm, keep, M, wW, E, h->dsc, wQ));
  CK(pgemm<RS>(h, OP_N, OP_N, keep * 3 * M, kj * dr, n3, wQ, n3, 0, aj, (long)kj * dr, 0, wWB,
               (long)kj * dr, 0, 1));
  // a8: inner-index Gram of the new centre and its eigenpairs
  const int KM = M * kj;
  const long colsB = (long)keep * 3 * dr;
  PO(swap12<T>(st, 1, (long)keep * 3, KM, dr, wWB, wBp));
  int kk;
  if (colsB < KM) {
    // the inner Gram W = B B^+ has rank <= colsB: diagonalise the smaller dual B^+ B
    const int nc = (int)colsB;
    CK((pgram<RS, RM>(h, OP_C, OP_N, nc, nc, KM, wBp, colsB, wBp, colsB, wWK, nc)));
    int nv;
    rc = inner_eig<RM>(h, nc, &nv);
    if (rc) return rc;
    // a9: cut + PPT (FP64 scalars); tr(B^+B) = tr(B B^+)
    PO(kraus_select<RM>(st, nv, h->wWv, wWK, nc, h->kcut, kmax, use_ppt, h->wF, h->dsc,
                        h->dstats, h->dtrace));
    rc = read_scalars(h);
    if (rc) return rc;
    kk = h->hsc->kkeep;
    // a10: kept rows f_k sqrt(w_k) y_k^+
    PO((dual_rows<RM, RS>(st, kk, nc, wVk, nc, h->wF, h->wWv, wCn)));
  } else {
    CK((pgram<RS, RM>(h, OP_N, OP_C, KM, KM, colsB, wBp, colsB, wBp, colsB, wWK, KM)));
    int nv;
    rc = inner_eig<RM>(h, KM, &nv);
    if (rc) return rc;
    // a9: cut + PPT (FP64 scalars)
    PO(kraus_select<RM>(st, nv, h->wWv, wWK, KM, h->kcut, kmax, use_ppt, h->wF, h->dsc,
                        h->dstats, h->dtrace));
    rc = read_scalars(h);
    if (rc) return rc;
    kk = h->hsc->kkeep;
    // a10: apply the inner isometry with the PPT scales
    PO((scale_vk<RM, RS>(st, KM, kk, wVk, KM, h->wF, wVks)));
    CK(pgemm<RS>(h, OP_C, OP_N, kk, colsB, KM, wVks, kk, 0, wBp, colsB, 0, wCn, colsB, 0, 1));
  }
  PO(swap12<T>(st, 1, kk, (long)keep * 3, dr, wCn, aj));
  h->bond[i + 1] = keep;
  h->kd[i + 1] = kk;
  return MPDO_OK;
}

// Mirror the chain in place: site s <-> site N-1-s with [l][s][k][r] -> [r][s][k][l].
// Each pair goes through the two B_j work buffers (each at least one site's capacity).
template <typename R>
int reverse_chain(mpdo_ctx* h) {
  using T = cx<R>;
  T* t1 = static_cast<T*>(h->wWB);
  T* t2 = static_cast<T*>(h->wBp);
  const size_t elt = sizeof(T);
  for (int s = 0; s <= (h->n - 1) / 2; ++s) {
    int t = h->n - 1 - s;
    size_t ns = (size_t)h->bond[s] * 3 * h->kd[s] * h->bond[s + 1];
    size_t nt = (size_t)h->bond[t] * 3 * h->kd[t] * h->bond[t + 1];
    PO(reverse_site<T>(h->st, h->bond[s], 3, h->kd[s], h->bond[s + 1],
                       static_cast<const T*>(h->site(s)), t1));
    if (t != s)
      PO(reverse_site<T>(h->st, h->bond[t], 3, h->kd[t], h->bond[t + 1],
                         static_cast<const T*>(h->site(t)), t2));
    CK(cudaMemcpyAsync(h->site(t), t1, ns * elt, cudaMemcpyDeviceToDevice, h->st));
    if (t != s) CK(cudaMemcpyAsync(h->site(s), t2, nt * elt, cudaMemcpyDeviceToDevice, h->st));
  }
  std::reverse(h->bond.begin(), h->bond.end());
  std::reverse(h->kd.begin(), h->kd.end());
  h->rev = !h->rev;
  return MPDO_OK;
}

template <typename R, typename RM>
int apply_ops(mpdo_ctx* h, const std::vector<DevOp>& ops, int chi, int kmax, int use_ppt) {
  for (const DevOp& op : ops) {
    if (op.kind == 1) {
      int s = h->rev ? h->n - 1 - op.site : op.site;
      int rc = MPDO_OK;
      PO(one_site<R>(h->st, h->bond[s], h->kd[s], h->bond[s + 1],
                     static_cast<const cx<R>*>(op.u), static_cast<cx<R>*>(h->site(s))));
      (void)rc;
      continue;
    }
    int i = op.site;
    bool ltr;
    if (h->centre == i) ltr = true;
    else if (h->centre == i + 1) ltr = false;
    else
      return fail(h, MPDO_ERR_STATE, "two-site op on bond (" + std::to_string(i) + "," +
                                         std::to_string(i + 1) + ") does not touch centre " +
                                         std::to_string(h->centre));
    // storage must run left->right along the update direction
    if (ltr == h->rev) {
      int rc = reverse_chain<R>(h);
      if (rc) return rc;
    }
    int is = h->rev ? h->n - 2 - i : i;
    int rc = update_lr<R, RM>(h, is, op, h->rev, chi, kmax, use_ppt);
    if (rc) return rc;
    h->centre = ltr ? i + 1 : i;
  }
  return MPDO_OK;
}

// ----------------------------------------------------------- op preparation
using zc = std::complex<double>;

void channel_c(const zc* e, int m, zc* c) {
  // C[(S,s,t),(S2,s2,t2)] = sum_{m,T} E_m[(S,T),(s,t)] conj(E_m[(S2,T),(s2,t2)])
  for (int a = 0; a < 729; ++a) c[a] = 0;
  for (int mm = 0; mm < m; ++mm) {
    const zc* em = e + mm * 81;
    for (int S = 0; S < 3; ++S)
      for (int s = 0; s < 3; ++s)
        for (int t = 0; t < 3; ++t)
          for (int S2 = 0; S2 < 3; ++S2)
            for (int s2 = 0; s2 < 3; ++s2)
              for (int t2 = 0; t2 < 3; ++t2) {
                zc acc = 0;
                for (int T = 0; T < 3; ++T)
                  acc += em[(S * 3 + T) * 9 + s * 3 + t] *
                         std::conj(em[(S2 * 3 + T) * 9 + s2 * 3 + t2]);
                c[(S * 9 + s * 3 + t) * 27 + S2 * 9 + s2 * 3 + t2] += acc;
              }
  }
}

void mirror_ops(const zc* e, int m, zc* out) {
  for (int mm = 0; mm < m; ++mm)
    for (int S = 0; S < 3; ++S)
      for (int T = 0; T < 3; ++T)
        for (int s = 0; s < 3; ++s)
          for (int t = 0; t < 3; ++t)
            out[mm * 81 + (T * 3 + S) * 9 + t * 3 + s] = e[mm * 81 + (S * 3 + T) * 9 + s * 3 + t];
}

// Build device copies of a host layer into `dl` (memory from one cudaMalloc).
int prepare_layer(mpdo_ctx* h, const mpdo_layer* layer, mpdo_dlayer_s* dl, bool staged) {
  if (!layer || layer->n_ops < 0 || (layer->n_ops > 0 && !layer->ops))
    return fail(h, MPDO_ERR_ARG, "null layer");
  const int elt = (int)h->elt;
  size_t total = 0;
  for (int k = 0; k < layer->n_ops; ++k) {
    const mpdo_op& op = layer->ops[k];
    if (!op.ops) return fail(h, MPDO_ERR_ARG, "op " + std::to_string(k) + " has no data");
    if (op.kind == 2) {
      // uploaded layers may serve any chain length up to the capacity (checked again when
      // applied); staged layers are applied to the current chain
      if (op.site < 0 || op.site > (staged ? h->n : h->n_cap) - 2)
        return fail(h, MPDO_ERR_ARG, "two-site op site out of range");
      if (op.n_kraus < 1 || op.n_kraus > h->mmax)
        return fail(h, MPDO_ERR_ARG, "n_kraus " + std::to_string(op.n_kraus) +
                                         " outside 1..m_max=" + std::to_string(h->mmax));
      if ((size_t)op.n_kraus * h->kmax > 1024)
        return fail(h, MPDO_ERR_ARG, "n_kraus*k_max exceeds 1024");
      // same layout as the copy loop below: each part starts on a 16-byte boundary
      const size_t sizes[4] = {(size_t)op.n_kraus * 81 * elt, (size_t)op.n_kraus * 81 * elt,
                               729 * h->eltm, 729 * h->eltm};
      for (size_t sz : sizes) total = ((total + 15) & ~(size_t)15) + sz;
    } else if (op.kind == 1) {
      if (op.site < 0 || op.site > (staged ? h->n : h->n_cap) - 1)
        return fail(h, MPDO_ERR_ARG, "one-site op site");
      if (op.n_kraus != 1) return fail(h, MPDO_ERR_ARG, "one-site op needs n_kraus == 1");
      total += 9 * elt;
    } else {
      return fail(h, MPDO_ERR_ARG, "op kind must be 1 or 2");
    }
    total = (total + 255) & ~(size_t)255;
  }
  // host staging buffer of the converted data: the handle's pinned buffer for staged
  // layers (reused; the copy below completes before the next layer is prepared)
  std::vector<unsigned char> tmp;
  unsigned char* hbuf = nullptr;
  if (staged) {
    if (h->hstage_cap < total + 256) {
      if (h->hstage) cudaFreeHost(h->hstage);
      h->hstage = nullptr;
      h->hstage_cap = 0;
      if (cudaMallocHost((void**)&h->hstage, total + 256) != cudaSuccess) {
        cudaGetLastError();
        h->hstage = nullptr;
        return fail(h, MPDO_ERR_OOM, "pinned layer staging");
      }
      h->hstage_cap = total + 256;
    }
    hbuf = h->hstage;
  } else {
    tmp.resize(total + 256);
    hbuf = tmp.data();
  }
  dl->ops.clear();
  size_t off = 0;
  for (int k = 0; k < layer->n_ops; ++k) {
    const mpdo_op& op = layer->ops[k];
    DevOp d;
    d.kind = op.kind;
    d.site = op.site;
    d.m = op.n_kraus;
    const int nval = op.kind == 2 ? op.n_kraus * 81 : 9;
    std::vector<zc> e(nval);
    for (int a = 0; a < nval; ++a) {
      double re = op.ops[2 * a], im = op.ops[2 * a + 1];
      if (!std::isfinite(re) || !std::isfinite(im))
        return fail(h, MPDO_ERR_NUMERIC, "non-finite value in op " + std::to_string(k));
      e[a] = zc(re, im);
    }
    // (data, count, double precision?): Kraus operators in the storage precision, the
    // channel partial traces (inputs of Phi) in the Gram precision
    struct Part { const zc* p; int n; bool dbl; };
    std::vector<Part> parts;
    std::vector<zc> em, ct(729), ctm(729);
    if (op.kind == 2) {
      em.resize(nval);
      mirror_ops(e.data(), op.n_kraus, em.data());
      channel_c(e.data(), op.n_kraus, ct.data());
      channel_c(em.data(), op.n_kraus, ctm.data());
      const bool gd = h->eltm == 16;
      parts = {{e.data(), nval, h->dbl}, {em.data(), nval, h->dbl}, {ct.data(), 729, gd},
               {ctm.data(), 729, gd}};
    } else {
      // one-site ops must be unitary to keep the canonical gauge
      double dev = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          zc acc = 0;
          for (int c = 0; c < 3; ++c) acc += std::conj(e[c * 3 + a]) * e[c * 3 + b];
          dev = std::max(dev, std::abs(acc - (a == b ? 1.0 : 0.0)));
        }
      if (dev > 1e-10) return fail(h, MPDO_ERR_ARG, "one-site op is not unitary");
      parts = {{e.data(), nval, h->dbl}};
    }
    size_t starts[4];
    for (size_t p = 0; p < parts.size(); ++p) {
      off = (off + 15) & ~(size_t)15;
      starts[p] = off;
      for (int a = 0; a < parts[p].n; ++a) {
        zc v = parts[p].p[a];
        if (parts[p].dbl) {
          double* dst = reinterpret_cast<double*>(hbuf + off) + 2 * a;
          dst[0] = v.real(); dst[1] = v.imag();
        } else {
          float* dst = reinterpret_cast<float*>(hbuf + off) + 2 * a;
          dst[0] = (float)v.real(); dst[1] = (float)v.imag();
        }
      }
      off += (size_t)parts[p].n * (parts[p].dbl ? 16 : 8);
    }
    off = (off + 255) & ~(size_t)255;
    // pointers are filled after the device buffer exists (store offsets for now)
    if (op.kind == 2) {
      d.e = (void*)starts[0]; d.em = (void*)starts[1]; d.ct = (void*)starts[2]; d.ctm = (void*)starts[3];
    } else {
      d.u = (void*)starts[0];
    }
    dl->ops.push_back(d);
  }
  void* dev = nullptr;
  if (staged) {
    if (h->staged_cap < total) {
      if (h->staged.mem) {
        CK(cudaStreamSynchronize(h->st));
        dfree(h, h->staged.mem);
        h->staged.mem = nullptr;
        h->staged_cap = 0;
      }
      h->staged.mem = dmalloc(h, total + 256);
      if (!h->staged.mem) return fail(h, MPDO_ERR_OOM, "layer staging");
      h->staged_cap = total;
    }
    dev = h->staged.mem;
  } else {
    dev = dmalloc(h, total + 256);
    if (!dev) return fail(h, MPDO_ERR_OOM, "layer upload");
    dl->mem = dev;
  }
  CK(cudaMemcpyAsync(dev, hbuf, total, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));  // host buffer is freed on return
  char* base = static_cast<char*>(dev);
  for (DevOp& d : dl->ops) {
    if (d.kind == 2) {
      d.e = base + (size_t)d.e; d.em = base + (size_t)d.em;
      d.ct = base + (size_t)d.ct; d.ctm = base + (size_t)d.ctm;
    } else {
      d.u = base + (size_t)d.u;
    }
  }
  return MPDO_OK;
}

int reset_stats(mpdo_ctx* h) {
  DevStats z{};
  z.ppt_theta_min = 1e300;
  *h->hstats = z;
  CK(cudaMemcpyAsync(h->dstats, h->hstats, sizeof(DevStats), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemsetAsync(h->dsc, 0, sizeof(StepScalars), h->st));
  return MPDO_OK;
}

int read_stats(mpdo_ctx* h, mpdo_trunc_stats* out) {
  CK(cudaMemcpyAsync(h->hstats, h->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  prof_drain(h);
  if (out) {
    const DevStats& s = *h->hstats;
    out->disc_bond_w = s.disc_bond_w;
    out->disc_kraus_w = s.disc_kraus_w;
    out->ppt_theta_min = s.ppt_theta_min;
    out->ppt_infeasible = s.ppt_infeasible;
    out->ppt_clamped = s.ppt_clamped;
    out->chi_used_max = s.chi_used_max;
    out->k_used_max = s.k_used_max;
    out->n_updates = s.n_updates;
  }
  return MPDO_OK;
}

int run_ops(mpdo_ctx* h, const std::vector<DevOp>& ops, mpdo_trunc_stats* stats, int chi,
            int kmax, int use_ppt) {
  for (const DevOp& op : ops)
    if (op.site < 0 || op.site > h->n - (op.kind == 2 ? 2 : 1))
      return fail(h, MPDO_ERR_ARG, "op site " + std::to_string(op.site) + " outside the chain of " +
                                       std::to_string(h->n) + " sites");
  int rc = reset_stats(h);
  if (rc) return rc;
  // left-to-right order: a layer that starts on bond (0,1) with the centre elsewhere first
  // brings the centre to site 0 by identity two-site updates
  if (h->cfg.order == 0 && !ops.empty() && h->centre != 0) {
    const DevOp* first = nullptr;
    for (const DevOp& op : ops)
      if (op.kind == 2) { first = &op; break; }
    if (first && first->site == 0) {
      std::vector<DevOp> moves;
      for (int i = h->centre - 1; i >= 0; --i) {
        DevOp d = h->ident.ops[0];
        d.site = i;
        moves.push_back(d);
      }
      rc = h->dbl     ? apply_ops<double, double>(h, moves, chi, kmax, use_ppt)
           : h->mixed ? apply_ops<float, double>(h, moves, chi, kmax, use_ppt)
                      : apply_ops<float, float>(h, moves, chi, kmax, use_ppt);
      if (rc) return rc;
    }
  }
  rc = h->dbl     ? apply_ops<double, double>(h, ops, chi, kmax, use_ppt)
       : h->mixed ? apply_ops<float, double>(h, ops, chi, kmax, use_ppt)
                  : apply_ops<float, float>(h, ops, chi, kmax, use_ppt);
  if (rc) return rc;
  return read_stats(h, stats);
}

int init_state(mpdo_ctx* h, const double* v) {
  double pl[6] = {1.0 / std::sqrt(2.0), 0, 1.0 / std::sqrt(2.0), 0, 0, 0};
  if (!v) v = pl;
  for (int a = 0; a < 6; ++a)
    if (!std::isfinite(v[a])) return fail(h, MPDO_ERR_NUMERIC, "non-finite initial vector");
  std::fill(h->bond.begin(), h->bond.end(), 1);
  std::fill(h->kd.begin(), h->kd.end(), 1);
  h->rev = false;
  h->centre = 0;
  CK(cudaMemsetAsync(h->dsc, 0, sizeof(StepScalars), h->st));
  // tr rho of the product state: |v|^(2N)
  h->htrace0 = std::pow(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3] + v[4] * v[4] +
                            v[5] * v[5],
                        (double)h->n);
  CK(cudaMemcpyAsync(h->dtrace, &h->htrace0, sizeof(double), cudaMemcpyHostToDevice, h->st));
  if (h->dbl)
    CK(product_state<double>(h->st, v, static_cast<double2*>(h->sites), (long)h->site_cap, h->n));
  else
    CK(product_state<float>(h->st, v, static_cast<float2*>(h->sites), (long)h->site_cap, h->n));
  CK(cudaStreamSynchronize(h->st));
  return MPDO_OK;
}

// ---------------------------------------------------------------- observables
// FP64 product of an FP64 environment-side operand and a site tensor of precision RS.
template <typename RS>
cudaError_t penv(mpdo_ctx* h, int opa, int opb, int m, int n, int k, const cx<double>* A,
                 long lda, long sa, const cx<RS>* B, long ldb, long sb, cx<double>* C, long ldc,
                 long sc, int batch) {
  if constexpr (std::is_same<RS, double>::value) {
    return pgemm<double>(h, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch);
  } else {
    if (tc_exact_route(h, m, n, k, batch))
      return pexact<double2, float2>(h, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc,
                                     batch);
    int pi = prof_begin(h, 0);
    cudaError_t e = cgemm_dx(h->st, opa, opb, m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, batch);
    prof_end(h, 0, pi, 8.0 * m * n * (double)k * batch);
    return e;
  }
}

// a11: the environments and the energy automata are FP64 whatever the storage precision
// (FP32 site tensors are read and widened in the GEMMs): an FP32 transfer chain loses
// ~1e-5 of the trace over 100 sites.
template <typename R>
int energy(mpdo_ctx* h, double J, double hx, double bz, double out[7]) {
  using T = cx<R>;
  using TD = cx<double>;
  cudaStream_t st = h->st;
  const long chi = h->chi, K = h->kmax;
  const long env = chi * chi, fsz = chi * 3 * K * chi;
  size_t need = (2 * 6 * env + 2 * 6 * fsz) * sizeof(TD) + 1024;
  if (h->obs_bytes < need) {
    if (h->obs) {
      CK(cudaStreamSynchronize(st));
      dfree(h, h->obs);
    }
    h->obs = dmalloc(h, need);
    if (!h->obs) { h->obs_bytes = 0; return fail(h, MPDO_ERR_OOM, "energy buffers"); }
    h->obs_bytes = need;
  }
  TD* ebuf[2] = {static_cast<TD*>(h->obs), static_cast<TD*>(h->obs) + 6 * env};
  TD* F = ebuf[1] + 6 * env;
  TD* G = F + 6 * fsz;
  // initial envs (1x1): E0 = 1, EZ = 0, E1 = 0 for both automata
  TD init[6] = {one<double>(), zero<double>(), zero<double>(),
                one<double>(), zero<double>(), zero<double>()};
  for (int a = 0; a < 6; ++a)
    CK(cudaMemcpyAsync(ebuf[0] + a * env, &init[a], sizeof(TD), cudaMemcpyHostToDevice, st));
  int cur = 0;
  for (int s = 0; s < h->n; ++s) {
    const int dl = h->bond[s], k = h->kd[s], dr = h->bond[s + 1];
    const T* A = static_cast<const T*>(h->site(s));
    const long cols = 3L * k * dr;
    // F[a] = E[a]^T A   (dl x cols)
    CK(penv<R>(h, OP_T, OP_N, dl, (int)cols, dl, ebuf[cur], dl, env, A, cols, 0, F, cols, fsz,
               6));
    PO(energy_mix<double>(st, dl, (int)(k * dr), F, fsz, G, fsz, J, hx, bz));
    // E'[a] = G[a]^T conj(A2), both as (dl*3*k) x dr
    CK(penv<R>(h, OP_T, OP_R, dr, dr, dl * 3 * k, G, dr, fsz, A, dr, 0, ebuf[1 - cur], dr, env,
               6));
    cur = 1 - cur;
  }
  TD res[6];
  for (int a = 0; a < 6; ++a)
    CK(cudaMemcpyAsync(&res[a], ebuf[cur] + a * env, sizeof(TD), cudaMemcpyDeviceToHost, st));
  // the trace carried in FP64 by the updates (the norm the truncations keep)
  double cnorm = 0;
  CK(cudaMemcpyAsync(&cnorm, h->dtrace, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(sync_stream(h));
  prof_drain(h);
  for (int a = 0; a < 6; ++a) out[a] = res[a].x;
  out[6] = cnorm;
  return MPDO_OK;
}

// ------------------------------------------------------- second-order observables
// Environments of two copies of rho (Sec. III.E): one site of rho is the operator
// R[(a,b)][s][s'][(r,r')] = sum_k A[a,s,k,r] conj(A[b,s',k,r']); two copies contract site by
// site, crossed (tr rho^2: copy 1 [s][s'] with copy 2 [s'][s]), diagonal (collision) or
// traced per copy (which factorises into the plain trace environment squared).  In the
// storage precision of the sites, with FP64 final contractions.
template <typename R>
int second_order(mpdo_ctx* h, int cut, double out[5]) {
  using T = cx<R>;
  cudaStream_t st = h->st;
  const int N = h->n;
  int dmax = 1;
  for (int b : h->bond) dmax = std::max(dmax, b);
  const long d2 = (long)dmax * dmax, d4 = d2 * d2;
  const double bytes = (double)sizeof(T) * (6.0 * 9 * d4 + 8.0 * d4 + 4.0 * d2 +
                                            (double)h->site_cap) + 4096;
  if (bytes > (double)((size_t)32 << 30))
    return fail(h, MPDO_ERR_ARG, "second-order environments need " + std::to_string(bytes / 1e9) +
                                     " GB at bond dimension " + std::to_string(dmax) +
                                     " (limit 32 GB)");
  void* mem = dmalloc(h, (size_t)bytes);
  if (!mem) return fail(h, MPDO_ERR_OOM, "second-order environment buffers");
  struct Guard {
    mpdo_ctx* h;
    void* p;
    ~Guard() {
      cudaStreamSynchronize(h->st);
      dfree(h, p);
    }
  } guard{h, mem};
  T* Ap = static_cast<T*>(mem);
  T* Rf = Ap + h->site_cap;
  T* Rp = Rf + 9 * d4;
  T* Rd = Rp + 9 * d4;     // diagonal copy of Rp (collision)
  T* W = Rd + 9 * d4;
  T* W2 = W + 9 * d4;
  T* RS = W2 + 9 * d4;
  T* CL = RS + 9 * d4;     // crossed left env
  T* CD = CL + d4;         // diagonal left env
  T* CR = CD + d4;         // crossed right env
  T* tmp = CR + d4;        // 2 d4
  T* eL = tmp + 2 * d4;
  T* eR = eL + d2;
  T* etmp = eR + d2;       // 2 d2
  T* Tr = etmp + 2 * d2;   // trace over s of R: dl^2 x dr^2 <= d4
  double* parts = reinterpret_cast<double*>(Tr + d4);
  double* res = parts + 64;   // 6 results
  const T o = one<R>();
  // site n: Rp (and the diagonal copy / trace) from its tensor
  auto site_rho = [&](int n, int* dl_o, int* dr_o) -> int {
    const int dl = h->bond[n], k = h->kd[n], dr = h->bond[n + 1];
    const T* A = static_cast<const T*>(h->site(n));
    PO(swap12<T>(st, (long)dl * 3, k, dr, 1, A, Ap));
    const int rows = 3 * dl * dr;
    CK(pgemm<R>(h, OP_N, OP_C, rows, rows, k, Ap, k, 0, Ap, k, 0, Rf, rows, 0, 1));
    const int dd[6] = {dl, 3, dr, dl, 3, dr}, pp[6] = {0, 3, 1, 4, 2, 5};
    PO(permute6<T>(st, dd, pp, Rf, Rp));
    *dl_o = dl;
    *dr_o = dr;
    return MPDO_OK;
  };
  // left crossed transfer: env (dl^2 x dl^2) -> out (dr^2 x dr^2) with site operator r
  auto left_cross = [&](const T* r, int dl, int dr, const T* env, T* outp) -> int {
    const long l2 = (long)dl * dl, r2 = (long)dr * dr;
    CK(pgemm<R>(h, OP_T, OP_N, (int)(9 * r2), (int)l2, (int)l2, r, 9 * r2, 0, env, l2, 0, W, l2,
                0, 1));
    const int dw[6] = {3, 3, dr, dr, dl, dl}, pw[6] = {2, 3, 0, 1, 4, 5};
    PO(permute6<T>(st, dw, pw, W, W2));
    const int drs[6] = {dl, dl, 3, 3, dr, dr}, prs[6] = {3, 2, 0, 1, 4, 5};
    PO(permute6<T>(st, drs, prs, r, RS));
    CK(pgemm<R>(h, OP_N, OP_N, (int)r2, (int)r2, (int)(9 * l2), W2, 9 * l2, 0, RS, r2, 0, outp,
                r2, 0, 1));
    return MPDO_OK;
  };
  int rc;
  const T init = o;
  CK(cudaMemcpyAsync(CL, &init, sizeof(T), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(CD, &init, sizeof(T), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(eL, &init, sizeof(T), cudaMemcpyHostToDevice, st));
  // left sweep over all sites: crossed env saved at the cut, diagonal env and plain trace env
  T* CLcut = tmp + d4;     // crossed env at the cut
  T* eLcut = etmp + d2;
  for (int n = 0; n < N; ++n) {
    if (n == cut) {
      const long c2 = (long)h->bond[n] * h->bond[n];
      CK(cudaMemcpyAsync(CLcut, CL, sizeof(T) * c2 * c2, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(eLcut, eL, sizeof(T) * c2, cudaMemcpyDeviceToDevice, st));
    }
    int dl, dr;
    if ((rc = site_rho(n, &dl, &dr))) return rc;
    const long l2 = (long)dl * dl, r2 = (long)dr * dr;
    CK(cudaMemcpyAsync(Rd, Rp, sizeof(T) * 9 * l2 * r2, cudaMemcpyDeviceToDevice, st));
    PO(rho_site<R>(st, l2, r2, Rd, nullptr, 1));
    PO(rho_site<R>(st, l2, r2, Rp, Tr, 2));
    if ((rc = left_cross(Rp, dl, dr, CL, tmp))) return rc;
    CK(cudaMemcpyAsync(CL, tmp, sizeof(T) * r2 * r2, cudaMemcpyDeviceToDevice, st));
    if ((rc = left_cross(Rd, dl, dr, CD, tmp))) return rc;
    CK(cudaMemcpyAsync(CD, tmp, sizeof(T) * r2 * r2, cudaMemcpyDeviceToDevice, st));
    CK(pgemm<R>(h, OP_N, OP_N, 1, (int)r2, (int)l2, eL, l2, 0, Tr, r2, 0, etmp, r2, 0, 1));
    CK(cudaMemcpyAsync(eL, etmp, sizeof(T) * r2, cudaMemcpyDeviceToDevice, st));
  }
  // right sweep from the far end down to the cut: crossed and plain envs
  CK(cudaMemcpyAsync(CR, &init, sizeof(T), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(eR, &init, sizeof(T), cudaMemcpyHostToDevice, st));
  for (int n = N - 1; n >= cut; --n) {
    int dl, dr;
    if ((rc = site_rho(n, &dl, &dr))) return rc;
    const long l2 = (long)dl * dl, r2 = (long)dr * dr;
    PO(rho_site<R>(st, l2, r2, Rp, Tr, 2));
    // Z[(a,b,s,s'),(x,y)] = Rp (9 l2 x r2) CR (r2 x r2); CR' = Z RS^T with RS = Rp, s <-> s'
    CK(pgemm<R>(h, OP_N, OP_N, (int)(9 * l2), (int)r2, (int)r2, Rp, r2, 0, CR, r2, 0, W, r2, 0,
                1));
    const int dd[6] = {dl, dl, 3, 3, dr, dr}, pp[6] = {0, 1, 3, 2, 4, 5};
    PO(permute6<T>(st, dd, pp, Rp, RS));
    CK(pgemm<R>(h, OP_N, OP_T, (int)l2, (int)l2, (int)(9 * r2), W, 9 * r2, 0, RS, 9 * r2, 0, tmp,
                l2, 0, 1));
    CK(cudaMemcpyAsync(CR, tmp, sizeof(T) * l2 * l2, cudaMemcpyDeviceToDevice, st));
    CK(pgemm<R>(h, OP_N, OP_N, (int)l2, 1, (int)r2, Tr, r2, 0, eR, 1, 0, etmp, 1, 0, 1));
    CK(cudaMemcpyAsync(eR, etmp, sizeof(T) * l2, cudaMemcpyDeviceToDevice, st));
  }
  const long c2 = (long)h->bond[cut] * h->bond[cut];
  PO(env_dot<R>(st, c2 * c2, CLcut, CR, 0, parts, res + 0));      // tr rho^2
  PO(env_dot<R>(st, c2, CLcut, eR, 1, parts, res + 1));           // tr rho_L^2
  PO(env_dot<R>(st, c2, CR, eLcut, 1, parts, res + 2));           // tr rho_R^2
  PO(env_dot<R>(st, c2, eLcut, eR, 0, parts, res + 3));           // tr rho
  double hres[4];
  CK(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, st));
  // the diagonal env ends as the 1 x 1 sum_x <x|rho|x>^2
  T cd;
  CK(cudaMemcpyAsync(&cd, CD, sizeof(T), cudaMemcpyDeviceToHost, st));
  CK(sync_stream(h));
  prof_drain(h);
  for (int a = 0; a < 4; ++a) out[a] = hres[a];
  out[4] = (double)cd.x;
  return MPDO_OK;
}

template <typename R>
int sample(mpdo_ctx* h, int ns, uint64_t seed, uint8_t* bits, double* probs) {
  using T = cx<R>;
  cudaStream_t st = h->st;
  if (h->rev) {
    int rc = reverse_chain<R>(h);
    if (rc) return rc;
  }
  const int N = h->n;
  const long chi = h->chi, K = h->kmax;
  const long env = chi * chi, fsz = chi * 3 * K * chi;
  // chunk of samples processed together
  long chunk = (long)((size_t)1 << 30) / (long)(sizeof(T) * (2 * fsz + 5 * env));
  if (chunk < 1) chunk = 1;
  if (chunk > ns) chunk = ns;
  size_t renv_bytes = (size_t)(N + 1) * env * sizeof(T);
  size_t need = renv_bytes + (size_t)sizeof(T) * (fsz + chunk * (2 * fsz + 5 * env) + env) +
                (size_t)ns * (N + 8) + 4096;
  void* mem = dmalloc(h, need);
  if (!mem) return fail(h, MPDO_ERR_OOM, "sampling buffers");
  struct Guard {
    mpdo_ctx* h;
    void* p;
    ~Guard() {
      cudaStreamSynchronize(h->st);
      dfree(h, p);
    }
  } guard{h, mem};
  T* renv = static_cast<T*>(mem);                 // R_n, n = 0..N, each env
  T* Y = renv + (N + 1) * env;                    // fsz
  T* Ecur = Y + fsz;                              // chunk * env
  T* Ef = Ecur + chunk * env;                     // chunk * fsz
  T* Fp = Ef + chunk * fsz;                       // chunk * fsz
  T* Ev = Fp + chunk * fsz;                       // chunk * 3 * env
  T* Enext = Ev + chunk * 3 * env;                // chunk * env
  uint8_t* dbits = reinterpret_cast<uint8_t*>(Enext + chunk * env);
  double* dprob = reinterpret_cast<double*>(((uintptr_t)(dbits + (size_t)ns * N) + 15) & ~15);
  // right environments with the identity: R_N = 1
  T o = one<R>();
  CK(cudaMemcpyAsync(renv + (long)N * env, &o, sizeof(T), cudaMemcpyHostToDevice, st));
  for (int s = N - 1; s >= 0; --s) {
    const int dl = h->bond[s], k = h->kd[s], dr = h->bond[s + 1];
    const T* A = static_cast<const T*>(h->site(s));
    // Y = A (dl*3k x dr) R_{s+1} (dr x dr);  R_s = Y (dl x 3k*dr) A^+
    CK(pgemm<R>(h, OP_N, OP_N, dl * 3 * k, dr, dr, A, dr, 0, renv + (long)(s + 1) * env, dr, 0,
                Y, dr, 0, 1));
    CK(pgemm<R>(h, OP_N, OP_C, dl, dl, 3L * k * dr, Y, 3L * k * dr, 0, A, 3L * k * dr, 0,
                renv + (long)s * env, dl, 0, 1));
  }
  for (long c0 = 0; c0 < ns; c0 += chunk) {
    const int cn = (int)std::min<long>(chunk, ns - c0);
    // per-sample environments are packed: sample q at Ecur + q * dl * dl (dl = 1 here)
    std::vector<T> ones(cn, one<R>());
    CK(cudaMemcpyAsync(Ecur, ones.data(), sizeof(T) * cn, cudaMemcpyHostToDevice, st));
    for (int s = 0; s < N; ++s) {
      const int dl = h->bond[s], k = h->kd[s], dr = h->bond[s + 1];
      const T* A = static_cast<const T*>(h->site(s));
      const long cols = 3L * k * dr, plane = (long)dl * k * dr;
      // F_q = E_q^T A  (dl x cols), packed per sample (stride dl*cols = 3*plane)
      CK(pgemm<R>(h, OP_T, OP_N, dl, (int)cols, dl, Ecur, dl, (long)dl * dl, A, cols, 0, Ef,
                  cols, 3 * plane, cn));
      // Fp_q[v][l'][k][r] and Ap[v][l'][k][r] (into Y)
      PO(swap12<T>(st, cn, dl, 3, (long)k * dr, Ef, Fp));
      PO(swap12<T>(st, 1, dl, 3, (long)k * dr, A, Y));
      for (int v = 0; v < 3; ++v)
        CK(pgemm<R>(h, OP_T, OP_R, dr, dr, dl * k, Fp + v * plane, dr, 3 * plane, Y + v * plane,
                    dr, 0, Ev + v * (long)dr * dr, dr, 3L * dr * dr, cn));
      PO(sample_pick<R>(st, cn, dr, Ev, renv + (long)(s + 1) * env, seed, s, s, N, Enext,
                        dbits + (size_t)c0 * N, dprob + c0, s == N - 1 ? 1 : 0));
      std::swap(Ecur, Enext);
    }
  }
  if (bits) CK(cudaMemcpyAsync(bits, dbits, (size_t)ns * N, cudaMemcpyDeviceToHost, st));
  if (probs) CK(cudaMemcpyAsync(probs, dprob, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_drain(h);
  return MPDO_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int mpdo_create(const mpdo_config* cfg, const double* init_site_vec, mpdo_t* out) {
  if (!cfg || !out) return fail(nullptr, MPDO_ERR_ARG, "null config or output");
  if (cfg->n_sites < 2) return fail(nullptr, MPDO_ERR_ARG, "n_sites must be >= 2");
  if (cfg->d != 3) return fail(nullptr, MPDO_ERR_ARG, "d must be 3");
  if (cfg->chi_max < 1 || cfg->chi_max > 1024) return fail(nullptr, MPDO_ERR_ARG, "chi_max out of 1..1024");
  if (cfg->k_max < 1 || cfg->k_max > 1024) return fail(nullptr, MPDO_ERR_ARG, "k_max out of 1..1024");
  if (cfg->m_max < 1 || (long)cfg->m_max * cfg->k_max > 1024)
    return fail(nullptr, MPDO_ERR_ARG, "m_max*k_max must be in 1..1024");
  if (cfg->prec < MPDO_FP64 || cfg->prec > MPDO_BF16X3)
    return fail(nullptr, MPDO_ERR_ARG, "unknown precision mode");
  if (cfg->order != 0 && cfg->order != 1)
    return fail(nullptr, MPDO_ERR_ARG, "order must be 0 (left to right) or 1 (snake)");
  if (cfg->alloc && !cfg->free)
    return fail(nullptr, MPDO_ERR_ARG, "an alloc hook needs a free hook");
  // a failed create releases what it allocated (through the hooks) and keeps the message
  struct CtxDel {
    void operator()(mpdo_ctx* p) const {
      if (!p->err.empty()) g_err = p->err;
      mpdo_destroy(p);
    }
  };
  std::unique_ptr<mpdo_ctx, CtxDel> h(new (std::nothrow) mpdo_ctx());
  if (!h) return fail(nullptr, MPDO_ERR_OOM, "host allocation");
  mpdo_ctx* hp = h.get();
  h->cfg = *cfg;
  cudaGetDevice(&h->device);
  if (cfg->cuda_stream) {
    h->st = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(nullptr, MPDO_ERR_CUDA, "stream creation failed");
    }
    h->own_stream = true;
  }
  h->n = h->n_cap = cfg->n_sites;
  h->chi = h->chi_cap = cfg->chi_max;
  h->kmax = h->kmax_cap = cfg->k_max;
  h->use_ppt = cfg->use_ppt;
  h->mmax = cfg->m_max;
  h->dbl = (cfg->prec == MPDO_FP64);
  h->elt = h->dbl ? 16 : 8;
  h->mixed = !h->dbl && cfg->gram_fp64;
  h->eltm = (h->dbl || h->mixed) ? 16 : 8;
  h->tcmode = cfg->prec == MPDO_TF32X3 ? TC_TF32X3 : cfg->prec == MPDO_BF16X3 ? TC_BF16X3 : -1;
  h->tc_min_macs = kTcMinMacs;
  if (const char* tm = std::getenv("MPDO_TC_MIN_MACS")) h->tc_min_macs = std::atof(tm);
  // Numerical-zero cuts.  Gram eigenvalues resolve only down to ~eps * max, so the cuts
  // are applied there: bond lambda = s^2 > htol*lambda_0, inner w > kcut^2 * w_0.  With
  // FP64 Grams of FP32 tensors the floor is the rounding of the tensors themselves
  // (relative 6e-8 per entry, i.e. ~4e-15 on lambda), taken as eps = 1e-14.
  // Tensor-core products of FP32 Grams: TF32x3 keeps ~22 significand bits per operand
  // (2^-22), BF16x3 ~16 (2^-16); the mixed form's Grams stay FP64 whatever the product engine.
  const double eps = h->dbl     ? 1e-16
                     : h->mixed ? 1e-14
                     : h->tcmode == TC_TF32X3 ? 2.4e-7
                     : h->tcmode == TC_BF16X3 ? 1.5e-5
                                              : 6e-8;
  double sv = cfg->sv_cutoff > 0 ? cfg->sv_cutoff : 1e-14;
  h->htol = std::max(sv * sv, 10 * eps);
  // The left factor's rank cut: directions of G_i below gtol carry less than gtol of the
  // block's weight each; in mixed mode they need not be resolved below 1% of the bond cut.
  h->gtol = h->mixed ? std::max(10 * eps, 0.01 * h->htol) : 10 * eps;
  double kc = cfg->kraus_cutoff > 0 ? cfg->kraus_cutoff : 1e-14;
  h->kcut = std::max(kc, std::sqrt(10 * eps));
  h->max_sweeps = (h->dbl || h->mixed) ? 30 : 20;
  h->bond.assign(h->n + 1, 1);
  h->kd.assign(h->n, 1);
  const long D = h->chi, K = h->kmax, M = h->mmax;
  const long n3 = 3 * D, n9 = 9 * D, KM = K * M;
  h->site_cap = (size_t)D * 3 * K * D;
  int rc;
  if ((rc = alloc_dev(hp, &h->sites, h->site_cap * h->elt * h->n))) return rc;
  const size_t e = h->elt, em = h->eltm;
  // A: storage precision (site tensors, large contractions); B: Gram-derived matrices
  auto A = [&](void** p, size_t count) { return alloc_dev(hp, p, count * e); };
  auto B = [&](void** p, size_t count) { return alloc_dev(hp, p, count * em); };
  if ((rc = A(&h->wM, D * K * n3)) || (rc = B(&h->wGi, n3 * n3)) || (rc = B(&h->wGj, n3 * n3)) ||
      (rc = B(&h->wVg, n3 * n3)) || (rc = B(&h->wR, n3 * n3)) || (rc = B(&h->wVs, n3 * n3)) ||
      (rc = B(&h->wVr, n3 * n3)) || (rc = B(&h->wPhi, n9 * n9)) || (rc = B(&h->wX, n9 * n9)) ||
      (rc = B(&h->wH, n9 * n9)) || (rc = B(&h->wU, n9 * n9)) || (rc = B(&h->wVgen, n9 * D)) ||
      (rc = A(&h->wW, n9 * D)) || (rc = B(&h->wTmp, D * K * 3 * D)) ||
      (rc = A(&h->wQ, D * 3 * M * n3)) || (rc = A(&h->wWB, D * 3 * M * K * D)) ||
      (rc = A(&h->wBp, D * 3 * M * K * D)) || (rc = B(&h->wWK, KM * KM)) ||
      (rc = B(&h->wVk, KM * KM)) || (rc = A(&h->wVks, KM * K)) || (rc = A(&h->wCn, K * D * 3 * D)))
    return rc;
  // the left factor and its polar step run in the Gram precision in mixed mode
  if ((rc = B(&h->wPol, D * D)) || (rc = B(&h->wQol, D * D)) || (rc = B(&h->wGa, D * D)))
    return rc;
  if (h->mixed && (rc = B(&h->wAcM, D * K * 3 * D))) return rc;
  const size_t rsz = em / 2;
  if ((rc = alloc_dev(hp, &h->wRs, n3 * rsz)) || (rc = alloc_dev(hp, &h->wIrs, n3 * rsz)) ||
      (rc = alloc_dev(hp, (void**)&h->wSig, n3 * 8)) || (rc = alloc_dev(hp, (void**)&h->wLam, n9 * 8)) ||
      (rc = alloc_dev(hp, (void**)&h->wWv, KM * 8)) ||
      (rc = alloc_dev(hp, (void**)&h->wF, (1024 + 2 * 64) * 8)))
    return rc;
  const int ncap = (int)std::max(n9, KM);
  size_t eb = em == 16 ? eig_work_bytes<double>(ncap) : eig_work_bytes<float>(ncap);
  if ((rc = alloc_dev(hp, &h->eigmem, eb))) return rc;
  if (em == 16) eig_work_bind<double>(h->eig64, h->eigmem, ncap);
  else eig_work_bind<float>(h->eig32, h->eigmem, ncap);
  if ((rc = alloc_dev(hp, &h->wLg, (size_t)std::max(n9, KM) * kInnerRmax * em)) ||
      (rc = alloc_dev(hp, &h->wL, (size_t)KM * kInnerRmax * em)) ||
      (rc = B(&h->wGs, (size_t)kInnerRmax * kInnerRmax)) ||
      (rc = B(&h->wZ, (size_t)kInnerRmax * kInnerRmax)) ||
      (rc = alloc_dev(hp, (void**)&h->dpc, sizeof(mpdo_ctx::PcOut))))
    return rc;
  if (cudaEventCreateWithFlags(&h->bev, cudaEventBlockingSync | cudaEventDisableTiming) !=
      cudaSuccess) {
    cudaGetLastError();
    h->bev = nullptr;
  }
  if (cudaMallocHost((void**)&h->hpc, sizeof(mpdo_ctx::PcOut)) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MPDO_ERR_OOM, "pinned host allocation");
  }
  if (h->mixed) {
    // the mixed solver serves every Gram of the update (bond H up to 9 chi, inner W up to
    // m_max k_max), so its workspace is sized for the largest
    const int mcap = ncap;
    if ((rc = alloc_dev(hp, &h->mixmem, mix_work_bytes(mcap)))) return rc;
    mix_work_bind(h->mixw, h->mixmem, mcap);
    // MPDO_NO_GRAPHS=1: launch the mixed eigensolver's levels directly (no CUDA graphs)
    const char* ng = std::getenv("MPDO_NO_GRAPHS");
    if (ng && ng[0] == '1') h->mixw.use_graphs = false;
  }
  if ((rc = alloc_dev(hp, (void**)&h->dtrace, sizeof(double))) ||
      (rc = alloc_dev(hp, (void**)&h->dsc, sizeof(StepScalars))) ||
      (rc = alloc_dev(hp, (void**)&h->dstats, sizeof(DevStats))))
    return rc;
  if (cudaMallocHost((void**)&h->hsc, sizeof(StepScalars)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hstats, sizeof(DevStats)) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MPDO_ERR_OOM, "pinned host allocation");
  }
  if (h->tcmode >= 0) {
    // packed operands of the tensor-core products: long K loops are processed in chunks
    // that fit (tc_cgemm), so the workspace only needs to hold a few k-blocks of the
    // largest packed pair
    const size_t want = (size_t)(D <= 64 ? 64 : 256) << 20;
    if ((rc = alloc_dev(hp, &h->tcws, want))) return rc;
    h->tcws_bytes = want;
    if ((rc = alloc_dev(hp, (void**)&h->tcerr, sizeof(int)))) return rc;
    if (cudaMallocHost((void**)&h->htcerr, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(nullptr, MPDO_ERR_OOM, "pinned host allocation");
    }
    *h->htcerr = 0;
  }
  if (h->mixed && h->tcmode >= 0) {
    // the mixed eigensolver's FP64 products take the same exact-slice tensor-core route
    // (MPDO_EIG_TC=0 keeps them on the CUDA cores)
    const char* et = std::getenv("MPDO_EIG_TC");
    if (!(et && et[0] == '0')) {
      h->mixw.tcws = h->tcws;
      h->mixw.tcws_bytes = h->tcws_bytes;
      h->mixw.tcerr = h->tcerr;
      h->mixw.tc_min_macs = h->tc_min_macs;
    }
  }
  {
    // identity channel for the left-to-right order's centre moves
    std::vector<double> idop(2 * 81, 0.0);
    for (int a = 0; a < 9; ++a) idop[2 * (a * 9 + a)] = 1.0;
    mpdo_op op{2, 0, 1, idop.data()};
    mpdo_layer L{1, &op};
    if ((rc = prepare_layer(hp, &L, &h->ident, false))) return rc;
  }
  rc = init_state(hp, init_site_vec);
  if (rc) return rc;
  *out = h.release();
  return MPDO_OK;
}

int mpdo_reset(mpdo_t h, const double* v) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  return init_state(h, v);
}

int mpdo_apply_layer(mpdo_t h, const mpdo_layer* layer, mpdo_trunc_stats* stats) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  int rc = prepare_layer(h, layer, &h->staged, true);
  if (rc) return rc;
  return run_ops(h, h->staged.ops, stats, h->chi, h->kmax, h->use_ppt);
}

int mpdo_layer_upload(mpdo_t h, const mpdo_layer* layer, mpdo_dlayer* out) {
  if (!h || !out) return fail(h, MPDO_ERR_ARG, "null handle or output");
  std::unique_ptr<mpdo_dlayer_s> dl(new (std::nothrow) mpdo_dlayer_s());
  if (!dl) return fail(h, MPDO_ERR_OOM, "host allocation");
  int rc = prepare_layer(h, layer, dl.get(), false);
  if (rc) return rc;
  *out = dl.release();
  return MPDO_OK;
}

int mpdo_apply_dlayer(mpdo_t h, mpdo_dlayer dl, mpdo_trunc_stats* stats) {
  if (!h || !dl) return fail(h, MPDO_ERR_ARG, "null handle or layer");
  return run_ops(h, dl->ops, stats, h->chi, h->kmax, h->use_ppt);
}

int mpdo_layer_free(mpdo_t h, mpdo_dlayer dl) {
  if (!dl) return MPDO_OK;
  if (dl->mem) {
    if (h) {
      cudaStreamSynchronize(h->st);
      dfree(h, dl->mem);
    } else {
      cudaDeviceSynchronize();
      cudaFree(dl->mem);
    }
  }
  delete dl;
  return MPDO_OK;
}

int mpdo_truncate(mpdo_t h, int chi_max, int k_max, int use_ppt, mpdo_trunc_stats* stats) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  if (chi_max < 1 || chi_max > h->chi || k_max < 1 || k_max > h->kmax)
    return fail(h, MPDO_ERR_ARG, "truncate limits must be within the handle's capacity");
  // identity channel, one Kraus operator
  std::vector<double> idop(2 * 81, 0.0);
  for (int a = 0; a < 9; ++a) idop[2 * (a * 9 + a)] = 1.0;
  std::vector<mpdo_op> ops;
  int c = h->centre;
  for (int i = c; i < h->n - 1; ++i) ops.push_back(mpdo_op{2, i, 1, idop.data()});
  for (int i = h->n - 2; i >= 0; --i) ops.push_back(mpdo_op{2, i, 1, idop.data()});
  mpdo_layer L{(int)ops.size(), ops.data()};
  int rc = prepare_layer(h, &L, &h->staged, true);
  if (rc) return rc;
  return run_ops(h, h->staged.ops, stats, chi_max, k_max, use_ppt);
}

int mpdo_expect_energy(mpdo_t h, double J, double hx, double b, double* e_raw, double* e_success,
                       double* success_prob, double* trace) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  double r[7];
  int rc = h->dbl ? energy<double>(h, J, hx, b, r) : energy<float>(h, J, hx, b, r);
  if (rc) return rc;
  // r: [0] tr(Pi rho) [2] tr(Pi H Pi rho) [3] tr(rho) [5] tr(H rho) [6] carried trace
  if (!(r[3] > 0) || !std::isfinite(r[3])) return fail(h, MPDO_ERR_NUMERIC, "zero trace");
  // The contracted trace of FP32-stored sites differs from the state's trace by the rounding
  // of the stored isometries (~1e-7 per site); the trace the updates keep is carried in FP64
  // (kraus_select), so the unnormalised outputs are rescaled to it.  The energies are
  // ratios of contractions and need no rescale.
  const double tr = r[6];
  if (!(tr > 0) || !std::isfinite(tr)) return fail(h, MPDO_ERR_NUMERIC, "zero trace");
  if (e_raw) *e_raw = r[5] / r[3];
  if (e_success) *e_success = r[0] > 0 ? r[2] / r[0] : NAN;
  if (success_prob) *success_prob = r[0] / r[3] * tr;
  if (trace) *trace = tr;
  return MPDO_OK;
}

int mpdo_sample_probs(mpdo_t h, int n_samples, uint64_t seed, uint8_t* bits, double* probs) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  if (n_samples < 0) return fail(h, MPDO_ERR_ARG, "n_samples < 0");
  if (n_samples == 0) return MPDO_OK;
  return h->dbl ? sample<double>(h, n_samples, seed, bits, probs)
                : sample<float>(h, n_samples, seed, bits, probs);
}

int mpdo_expect_second_order(mpdo_t h, int cut, double* xi, double* collision, double* s2_left,
                             double* s2_right, double* i2) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  if (cut < 1 || cut > h->n - 1) return fail(h, MPDO_ERR_ARG, "cut must be within 1..N-1");
  // storage coordinates: a mirrored chain swaps the halves
  const int sc = h->rev ? h->n - cut : cut;
  double r[5];
  int rc = h->dbl ? second_order<double>(h, sc, r) : second_order<float>(h, sc, r);
  if (rc) return rc;
  const double tr2 = r[3] * r[3];
  if (!(tr2 > 0) || !std::isfinite(tr2) || !(r[0] > 0) || !(r[1] > 0) || !(r[2] > 0))
    return fail(h, MPDO_ERR_NUMERIC, "non-positive second-order contraction");
  const double pl = h->rev ? r[2] : r[1], pr = h->rev ? r[1] : r[2];
  const double s2 = -std::log(r[0] / tr2), sl = -std::log(pl / tr2), sr = -std::log(pr / tr2);
  if (xi) *xi = r[0] / tr2;
  if (collision) *collision = r[4] / tr2;
  if (s2_left) *s2_left = sl;
  if (s2_right) *s2_right = sr;
  if (i2) *i2 = sl + sr - s2;
  return MPDO_OK;
}

int mpdo_reconfigure(mpdo_t h, int n_sites, int chi_max, int k_max, int use_ppt,
                     const double* init_site_vec) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  if (n_sites < 2 || n_sites > h->n_cap || chi_max < 1 || chi_max > h->chi_cap || k_max < 1 ||
      k_max > h->kmax_cap)
    return fail(h, MPDO_ERR_ARG, "reconfigure limits exceed the handle's capacity");
  CK(cudaStreamSynchronize(h->st));
  h->n = n_sites;
  h->chi = chi_max;
  h->kmax = k_max;
  h->use_ppt = use_ppt;
  h->bond.assign(h->n + 1, 1);
  h->kd.assign(h->n, 1);
  return init_state(h, init_site_vec);
}

namespace {
int run_circuit(mpdo_t h, const mpdo_circuit& c, double* out) {
  int rc = mpdo_reconfigure(h, c.n_sites, c.chi_max, c.k_max, c.use_ppt, nullptr);
  if (rc) return rc;
  for (int l = 0; l < c.n_layers; ++l) {
    if (!c.layers[l]) return fail(h, MPDO_ERR_ARG, "null layer in circuit");
    rc = run_ops(h, c.layers[l]->ops, nullptr, h->chi, h->kmax, h->use_ppt);
    if (rc) return rc;
  }
  return mpdo_expect_energy(h, c.J, c.hx, c.b, out, out + 1, out + 2, out + 3);
}

// The host-layer form: each layer is prepared (converted, channel partial traces formed)
// and copied into the handle's staging buffer on its own stream, so the uploads of one
// circuit overlap the kernels of the others.
int run_circuit_host(mpdo_t h, const mpdo_circuit_host& c, double* out) {
  int rc = mpdo_reconfigure(h, c.n_sites, c.chi_max, c.k_max, c.use_ppt, nullptr);
  if (rc) return rc;
  if (c.n_layers > 0 && !c.layers) return fail(h, MPDO_ERR_ARG, "null layer list in circuit");
  for (int l = 0; l < c.n_layers; ++l) {
    rc = prepare_layer(h, &c.layers[l], &h->staged, true);
    if (rc) return rc;
    rc = run_ops(h, h->staged.ops, nullptr, h->chi, h->kmax, h->use_ppt);
    if (rc) return rc;
  }
  return mpdo_expect_energy(h, c.J, c.hx, c.b, out, out + 1, out + 2, out + 3);
}

// Shared driver of the batch executors: one host thread per pool handle, circuits taken
// from a shared queue in index order.
}  // namespace
}  // extern "C"
namespace {
template <typename Circ, typename Run>
int batch_drive(int n_handles, mpdo_t* handles, int n_circuits, const Circ* circuits,
                double* out, int* status, Run run) {
  if (n_handles < 1 || !handles || n_circuits < 0 || (n_circuits > 0 && (!circuits || !out)))
    return fail(nullptr, MPDO_ERR_ARG, "bad batch arguments");
  for (int k = 0; k < n_handles; ++k)
    if (!handles[k]) return fail(nullptr, MPDO_ERR_ARG, "null handle in pool");
  for (int k = 0; k < n_handles; ++k)
    for (int j = k + 1; j < n_handles; ++j)
      if (handles[k] == handles[j]) return fail(nullptr, MPDO_ERR_ARG, "handle repeated in pool");
  std::atomic<int> next{0};
  std::vector<int> st(n_circuits, MPDO_OK);
  std::vector<std::string> msg(n_circuits);
  // MPDO_SPIN_SYNC=1 keeps spinning waits in the executor too
  const char* spin = std::getenv("MPDO_SPIN_SYNC");
  const bool blocking = n_handles > 2 && !(spin && spin[0] == '1');
  auto worker = [&](int k) {
    mpdo_t h = handles[k];
    cudaSetDevice(h->device);
    h->block_sync = blocking;
    h->mixw.block_ev = blocking ? h->bev : nullptr;
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= n_circuits) break;
      st[i] = run(h, circuits[i], out + 4 * (size_t)i);
      if (st[i]) msg[i] = h->err;
    }
    h->block_sync = false;
    h->mixw.block_ev = nullptr;
  };
  const int nt = std::min(n_handles, std::max(1, n_circuits));
  std::vector<std::thread> pool;
  for (int k = 1; k < nt; ++k) pool.emplace_back(worker, k);
  worker(0);
  for (auto& t : pool) t.join();
  int first = MPDO_OK;
  for (int i = 0; i < n_circuits; ++i) {
    if (status) status[i] = st[i];
    if (st[i] && first == MPDO_OK) first = st[i];
  }
  if (first) {
    for (int i = 0; i < n_circuits; ++i)
      if (st[i]) { g_err = "batch: circuit " + std::to_string(i) + ": " + msg[i]; break; }
  }
  return first;
}
}  // namespace
extern "C" {

int mpdo_batch_run(int n_handles, mpdo_t* handles, int n_circuits, const mpdo_circuit* circuits,
                   double* out, int* status) {
  return batch_drive(n_handles, handles, n_circuits, circuits, out, status, run_circuit);
}

int mpdo_batch_run_host(int n_handles, mpdo_t* handles, int n_circuits,
                        const mpdo_circuit_host* circuits, double* out, int* status) {
  return batch_drive(n_handles, handles, n_circuits, circuits, out, status, run_circuit_host);
}

int mpdo_get_dims(mpdo_t h, int* bond_dims, int* kraus_dims, int* centre) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  for (int u = 0; u < h->n; ++u) {
    int s = h->rev ? h->n - 1 - u : u;
    if (kraus_dims) kraus_dims[u] = h->kd[s];
    if (bond_dims && u < h->n - 1) bond_dims[u] = h->rev ? h->bond[s] : h->bond[s + 1];
  }
  if (centre) *centre = h->centre;
  return MPDO_OK;
}

int mpdo_get_site(mpdo_t h, int n, double* out, size_t cap, int* dims) {
  if (!h || !out || !dims) return fail(h, MPDO_ERR_ARG, "null argument");
  if (n < 0 || n >= h->n) return fail(h, MPDO_ERR_ARG, "site out of range");
  int s = h->rev ? h->n - 1 - n : n;
  int dl = h->bond[s], k = h->kd[s], dr = h->bond[s + 1];
  size_t cnt = (size_t)dl * 3 * k * dr;
  if (cap < cnt) return fail(h, MPDO_ERR_ARG, "output capacity too small");
  std::vector<double> tmp(2 * cnt);
  if (h->dbl) {
    CK(cudaMemcpyAsync(tmp.data(), h->site(s), cnt * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  } else {
    std::vector<float> f(2 * cnt);
    CK(cudaMemcpyAsync(f.data(), h->site(s), cnt * 8, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (size_t a = 0; a < 2 * cnt; ++a) tmp[a] = f[a];
  }
  if (!h->rev) {
    std::memcpy(out, tmp.data(), cnt * 16);
    dims[0] = dl; dims[1] = 3; dims[2] = k; dims[3] = dr;
  } else {
    // storage [r_u][s][k][l_u] -> user [l_u][s][k][r_u]
    for (int a = 0; a < dl; ++a)
      for (int q = 0; q < 3; ++q)
        for (int kk = 0; kk < k; ++kk)
          for (int b = 0; b < dr; ++b) {
            size_t src = (((size_t)a * 3 + q) * k + kk) * dr + b;
            size_t dst = (((size_t)b * 3 + q) * k + kk) * dl + a;
            out[2 * dst] = tmp[2 * src];
            out[2 * dst + 1] = tmp[2 * src + 1];
          }
    dims[0] = dr; dims[1] = 3; dims[2] = k; dims[3] = dl;
  }
  return MPDO_OK;
}

int mpdo_destroy(mpdo_t h) {
  if (!h) return MPDO_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  mix_work_release(h->mixw);
  if (h->bev) cudaEventDestroy(h->bev);
  for (void* p : h->allocs) dfree(h, p);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  if (h->prof_counts) cudaFreeHost(h->prof_counts);
  if (h->staged.mem) dfree(h, h->staged.mem);
  if (h->ident.mem) dfree(h, h->ident.mem);
  if (h->hstage) cudaFreeHost(h->hstage);
  if (h->obs) dfree(h, h->obs);
  if (h->hsc) cudaFreeHost(h->hsc);
  if (h->hstats) cudaFreeHost(h->hstats);
  if (h->hpc) cudaFreeHost(h->hpc);
  if (h->htcerr) cudaFreeHost(h->htcerr);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
  return MPDO_OK;
}

const char* mpdo_last_error(mpdo_t h) { return h ? h->err.c_str() : g_err.c_str(); }

long long mpdo_kernel_launches(void) { return mpdo::g_launches.load(); }

int mpdo_profile(mpdo_t h, int class_mask) {
  if (!h) return fail(nullptr, MPDO_ERR_ARG, "null handle");
  if (class_mask & ~7) return fail(h, MPDO_ERR_ARG, "class mask must be within 0..7");
  if (class_mask && h->prof_ev.empty()) {
    h->prof_ev.resize(8192);
    for (auto& e : h->prof_ev) CK(cudaEventCreate(&e));
    h->prof_nslots = 4096;
    CK(cudaMallocHost((void**)&h->prof_counts, sizeof(int) * h->prof_nslots));
  }
  CK(cudaStreamSynchronize(h->st));
  prof_drain(h);
  h->prof_mask = class_mask;
  for (int c = 0; c < 3; ++c) { h->prof_ms[c] = 0; h->prof_cnt[c] = 0; h->prof_flops[c] = 0; }
  return MPDO_OK;
}

int mpdo_profile_read(mpdo_t h, int cls, double* ms, long long* launches, double* flops) {
  if (!h || cls < 0 || cls > 2) return fail(h, MPDO_ERR_ARG, "bad profile class");
  CK(cudaStreamSynchronize(h->st));
  prof_drain(h);
  if (ms) *ms = h->prof_ms[cls];
  if (launches) *launches = h->prof_cnt[cls];
  if (flops) *flops = h->prof_flops[cls];
  return MPDO_OK;
}

int mpdo_kernel_cgemm(int prec, int opa, int opb, int m, int n, int k, const void* a, long lda,
                      long sa, const void* b, long ldb, long sb, void* c, long ldc, long sc,
                      int batch, void* stream) {
  if (opa < 0 || opa > 3 || opb < 0 || opb > 3 || m < 0 || n < 0 || k < 0 || batch < 0)
    return fail(nullptr, MPDO_ERR_ARG, "bad gemm arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prec == 0)
    e = cgemm<double>(st, opa, opb, m, n, k, (const double2*)a, lda, sa, (const double2*)b, ldb,
                      sb, (double2*)c, ldc, sc, batch, one<double>(), zero<double>());
  else
    e = cgemm<float>(st, opa, opb, m, n, k, (const float2*)a, lda, sa, (const float2*)b, ldb, sb,
                     (float2*)c, ldc, sc, batch, one<float>(), zero<float>());
  if (e != cudaSuccess) return fail(nullptr, MPDO_ERR_CUDA, cudaGetErrorString(e));
  return MPDO_OK;
}

int mpdo_kernel_heig(int prec, int n, void* a, void* v, double* w, int* sweeps, void* stream) {
  if (n < 1 || n > 4096 || !a || !v || !w) return fail(nullptr, MPDO_ERR_ARG, "bad heig arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* mem = nullptr;
  if (prec == 2 || prec == 3) {
    // mixed-precision solver on an FP64 matrix (resolved down to 1e-14 of the largest);
    // prec 3: its FP64 products as exact slice products on the tensor cores
    void* mm = nullptr;
    if (cudaMalloc(&mm, mix_work_bytes(n)) != cudaSuccess) { cudaGetLastError(); return fail(nullptr, MPDO_ERR_OOM, "heig work"); }
    void* tw = nullptr;
    const size_t tw_bytes = (size_t)256 << 20;
    if (prec == 3 && cudaMalloc(&tw, tw_bytes + 256) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(mm);
      return fail(nullptr, MPDO_ERR_OOM, "heig tensor-core workspace");
    }
    // the solver's CTA ticket starts at zero
    if (cudaMemsetAsync(mm, 0, mix_work_bytes(n), st) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(mm);
      return fail(nullptr, MPDO_ERR_CUDA, "heig work clear");
    }
    MixWork mw;
    mix_work_bind(mw, mm, n);
    int herr = 0;
    cudaError_t e2 = cudaSuccess;
    if (tw) {
      mw.tcws = static_cast<char*>(tw) + 256;
      mw.tcws_bytes = tw_bytes;
      mw.tcerr = static_cast<int*>(tw);
      mw.tc_min_macs = kTcMinMacs;
      e2 = cudaMemsetAsync(tw, 0, sizeof(int), st);
    }
    int lv = 0;
    if (e2 == cudaSuccess)
      e2 = heig_mixed(st, n, (const double2*)a, n, (double2*)v, n, w, 1e-14, mw, &lv);
    if (e2 == cudaSuccess && tw) e2 = cudaMemcpyAsync(&herr, tw, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    mix_work_release(mw);
    cudaFree(mm);
    if (tw) cudaFree(tw);
    if (e2 != cudaSuccess) return fail(nullptr, MPDO_ERR_CUDA, cudaGetErrorString(e2));
    if (herr) return fail(nullptr, MPDO_ERR_TIMEOUT, "heig: a tensor-core pipeline wait gave up");
    if (sweeps) *sweeps = lv;
    return MPDO_OK;
  }
  size_t bytes = prec == 0 ? eig_work_bytes<double>(n) : eig_work_bytes<float>(n);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) { cudaGetLastError(); return fail(nullptr, MPDO_ERR_OOM, "heig work"); }
  cudaError_t e;
  int* counters;
  if (prec == 0) {
    EigWork<double> wk;
    eig_work_bind<double>(wk, mem, n);
    counters = wk.counters;
    e = heig<double>(st, n, (const double2*)a, n, (double2*)v, n, w, wk, 30);
  } else {
    EigWork<float> wk;
    eig_work_bind<float>(wk, mem, n);
    counters = wk.counters;
    e = heig<float>(st, n, (const float2*)a, n, (float2*)v, n, w, wk, 20);
  }
  int sw = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sw, counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (e != cudaSuccess) return fail(nullptr, MPDO_ERR_CUDA, cudaGetErrorString(e));
  if (sweeps) *sweeps = sw;
  return MPDO_OK;
}

}  // extern "C"
