// Launchers of the small kernels in kernels.cu (internal).
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace mpdo {
// out (rows x cols, row stride ldo) = in converted from precision Ri to Ro.
template <typename Ri, typename Ro>
cudaError_t convert(cudaStream_t st, int rows, int cols, const cx<Ri>* in, long ldi, cx<Ro>* out,
                    long ldo);
template <typename T>
cudaError_t swap12(cudaStream_t st, long n0, long n1, long n2, long n3, const T* in, T* out);
template <typename T>
cudaError_t reverse_site(cudaStream_t st, int dl, int d, int k, int dr, const T* in, T* out);
template <typename R>
cudaError_t one_site(cudaStream_t st, int dl, int k, int dr, const cx<R>* u, cx<R>* a);
template <typename R>
cudaError_t product_state(cudaStream_t st, const double* v, cx<R>* base, long stride, int n);
template <typename R>
cudaError_t gram_mask(cudaStream_t st, int n, const double* sig, double gtol, R* rs, R* irs,
                      StepScalars* sc);
template <typename R>
cudaError_t gram_factor(cudaStream_t st, int n, const cx<R>* v, const R* rs, const R* irs,
                        cx<R>* rmat, cx<R>* vs, cx<R>* vr);
template <typename R>
cudaError_t build_phi(cudaStream_t st, int dm, const cx<R>* ct, const cx<R>* gj, cx<R>* phi);
template <typename R>
cudaError_t bond_select(cudaStream_t st, int n, const double* lam, const cx<R>* hm, long ldh,
                        double htol, int chi, StepScalars* sc, DevStats* ds);
template <typename R>
cudaError_t make_q(cudaStream_t st, int dm, int keep, int m_ops, const cx<R>* w, const cx<R>* e,
                   const StepScalars* sc, cx<R>* q);
template <typename R, typename RO>
cudaError_t dual_rows(cudaStream_t st, int kk, int cols, const cx<R>* y, long ldy, const double* f,
                      const double* w, cx<RO>* out);
template <typename R>
cudaError_t polar_factors(cudaStream_t st, int n, const cx<R>* g, cx<R>* pm, cx<R>* qm);
// n eigenvalues w (descending); the total weight is the trace of wm (ntr x ntr)
// trace (device FP64, may be NULL): the carried trace of the state, multiplied by the
// block's tr(theta')/tr(theta) = sc->tot / sc->trpre; the kept weights are rescaled to it.
// f holds 1024 + 128 doubles (scale factors, then partial sums of tr W and ||W||_F^2).
template <typename R>
cudaError_t kraus_select(cudaStream_t st, int n, const double* w, const cx<R>* wm, int ntr,
                         double kcut, int kmax, int use_ppt, double* f, StepScalars* sc,
                         DevStats* ds, double* trace);
// sc->trpre = ||theta||^2 of the block from its Gram matrices G_i, G_j (3 dm x 3 dm)
template <typename R>
cudaError_t trace_pre(cudaStream_t st, int dm, const cx<R>* gi, const cx<R>* gj, StepScalars* sc);
// Pivoted Cholesky W ~ L L^+ of a Hermitian PSD matrix (n <= 1024, rmax <= 128); device
// outputs: L (n x r, row stride lr), *rout = r, *resid = remaining diag max / tr W.
template <typename R>
cudaError_t pchol(cudaStream_t st, int n, const cx<R>* w, int rmax, double tol, cx<R>* L, int lr,
                  int* rout, double* resid);
// zs = z diag(s^-1/2) (r x r)
template <typename R>
cudaError_t lift(cudaStream_t st, int r, const cx<R>* z, const double* s, cx<R>* zs);
// out = in with its 6 axes reordered (out axis i = in axis p[i]; in dims d[0..5], host arrays)
template <typename T>
cudaError_t permute6(cudaStream_t st, const int* d, const int* p, const T* in, T* out);
// r = R[(a,b)][s][s'][(r,r')] of one site: mode 1 zeroes the s != s' blocks; mode 2 writes
// sum_s R[(a,b)][s][s][(r,r')] into tr
template <typename R>
cudaError_t rho_site(cudaStream_t st, long dl2, long dr2, cx<R>* r, cx<R>* tr, int mode);
// *out (device) = sum Re(x y) over n2 entries (mode 0), or sum_{i,j} Re(x[i][j] y[i] y[j])
// over n2 x n2 (mode 1), in FP64 with a fixed summation order; parts: 64 doubles of scratch
template <typename R>
cudaError_t env_dot(cudaStream_t st, long n2, const cx<R>* x, const cx<R>* y, int mode,
                    double* parts, double* out);
// out (device double) = sum of |a|^2 over n complex entries, accumulated in FP64
template <typename R>
cudaError_t sumsq(cudaStream_t st, long n, const cx<R>* a, double* out);
template <typename R, typename RO>
cudaError_t scale_vk(cudaStream_t st, int n, int kk, const cx<R>* v, long ldv, const double* f,
                     cx<RO>* out);
template <typename R>
cudaError_t energy_mix(cudaStream_t st, int dl, int plane, const cx<R>* f, long fstride,
                       cx<R>* g, long gstride, double J, double hx, double bz);
template <typename R>
cudaError_t sample_pick(cudaStream_t st, int n_samples, int dr, const cx<R>* ev, const cx<R>* rt,
                        uint64_t seed, int site, int site_user, int n_sites, cx<R>* env_out,
                        uint8_t* bits, double* probs, int last);
}  // namespace mpdo
