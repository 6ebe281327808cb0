// Host channel builder (FP64, off the hot path): the noisy ZZ block of the QAOA layer in
// the gate-level model and the layer's ordered op list.
//
// Local basis 0 = |0>, 1 = |1>, 2 = |r>.  Two-site operators are 9x9 on s_i*3 + s_j.
//  * ZZ block (Sec. IV, Eq. HZ_block_representation): CNOT (I (x) exp(-i a S^z)) CNOT,
//    CNOT = (I (x) Had) CZ (I (x) Had); Had and S^z act on the qubit levels, CZ flips the
//    sign of |11>.
//  * Crosstalk (Sec. III.B, reduced to the active pair): exp(-i phi n_r (x) n_r) first.
//  * Post-promotion (Sec. IV.A): exp(-i dPP (|1><r| + |r><1|)) on both atoms after the block.
//  * Noise: one unit of the single-atom Lindblad evolution with the jump operators of
//    Sec. II, L_j = sqrt(g b_j)|j><r| and dephasing sqrt(gp/2)(|0><0| - |1><1|) (linear-rate
//    reading), solved in closed form: r-population e^{-g}, qubit-Rydberg coherences
//    e^{-g/2 - gp/4}, rho_01 e^{-gp}, b_j (1 - e^{-g}) of the r-population moved to |j>
//    (the dark share b_d leaves the simulated space).
//  * The Kraus set is read off the Choi matrix of the composed superoperator by a cyclic
//    Jacobi eigendecomposition (eigenvalues below eta * lambda_max dropped).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/mpdo.h"

namespace {

using zc = std::complex<double>;
using Mat = std::vector<zc>;  // row-major square

Mat eye(int n) {
  Mat m(n * n, 0.0);
  for (int i = 0; i < n; ++i) m[i * n + i] = 1.0;
  return m;
}
Mat matmul(const Mat& a, const Mat& b, int n) {
  Mat c(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      zc aik = a[i * n + k];
      if (aik == 0.0) continue;
      for (int j = 0; j < n; ++j) c[i * n + j] += aik * b[k * n + j];
    }
  return c;
}
Mat kron(const Mat& a, int na, const Mat& b, int nb) {
  int n = na * nb;
  Mat c(n * n);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < na; ++j)
      for (int k = 0; k < nb; ++k)
        for (int l = 0; l < nb; ++l) c[(i * nb + k) * n + j * nb + l] = a[i * na + j] * b[k * nb + l];
  return c;
}
Mat dagger(const Mat& a, int n) {
  Mat c(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) c[j * n + i] = std::conj(a[i * n + j]);
  return c;
}
Mat conjm(const Mat& a) {
  Mat c(a.size());
  for (size_t i = 0; i < a.size(); ++i) c[i] = std::conj(a[i]);
  return c;
}

// Cyclic two-sided Jacobi for a Hermitian matrix: a = V diag(w) V^+.
void jacobi_herm(Mat a, int n, std::vector<double>& w, Mat& v) {
  v = eye(n);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, diag = 0;
    for (int i = 0; i < n; ++i) {
      diag += std::norm(a[i * n + i]);
      for (int j = i + 1; j < n; ++j) off += std::norm(a[i * n + j]);
    }
    if (off <= 1e-32 * (diag + off) || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        zc g = a[p * n + q];
        double ag = std::abs(g);
        if (ag < 1e-300) continue;
        double al = a[p * n + p].real(), be = a[q * n + q].real();
        double tau = (be - al) / (2 * ag);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double c = 1 / std::sqrt(1 + t * t), s = t * c;
        zc e = g / ag;
        // columns: a <- a U, U = [[c, s e], [-s conj(e), c]] on (p, q)
        for (int r = 0; r < n; ++r) {
          zc x = a[r * n + p], y = a[r * n + q];
          a[r * n + p] = c * x - s * std::conj(e) * y;
          a[r * n + q] = s * e * x + c * y;
          zc vx = v[r * n + p], vy = v[r * n + q];
          v[r * n + p] = c * vx - s * std::conj(e) * vy;
          v[r * n + q] = s * e * vx + c * vy;
        }
        // rows: a <- U^+ a
        for (int col = 0; col < n; ++col) {
          zc x = a[p * n + col], y = a[q * n + col];
          a[p * n + col] = c * x - s * e * y;
          a[q * n + col] = s * std::conj(e) * x + c * y;
        }
        a[p * n + q] = 0.0;
        a[q * n + p] = 0.0;
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i].real();
}

// exp(-i theta h), h Hermitian
Mat expmh(double theta, const Mat& h, int n) {
  std::vector<double> w;
  Mat v;
  jacobi_herm(h, n, w, v);
  Mat d(n * n, 0.0);
  for (int i = 0; i < n; ++i) d[i * n + i] = std::exp(zc(0, -theta * w[i]));
  return matmul(matmul(v, d, n), dagger(v, n), n);
}

Mat op3(std::initializer_list<zc> vals) { return Mat(vals); }

Mat zq() { return op3({1, 0, 0, 0, -1, 0, 0, 0, 0}); }
Mat xq() { return op3({0, 1, 0, 1, 0, 0, 0, 0, 0}); }
Mat nr() { return op3({0, 0, 0, 0, 0, 0, 0, 0, 1}); }
Mat hadq() {
  double r = 1 / std::sqrt(2.0);
  return op3({r, r, 0, r, -r, 0, 0, 0, 1});
}

// superoperator of rho -> U rho U^+ on row-major vec: U (x) conj(U)
Mat unitary_superop(const Mat& u, int n) { return kron(u, n, conjm(u), n); }

// closed-form single-atom noise superoperator (9x9 on row-major vec of a 3x3 rho)
Mat noise_superop(double g, double gp, double b0, double b1) {
  Mat s(81, 0.0);
  auto idx = [](int a, int b) { return a * 3 + b; };
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double f;
      if ((a == 2) != (b == 2)) f = std::exp(-g / 2 - gp / 4);
      else if (a == 2 && b == 2) f = std::exp(-g);
      else if (a != b) f = std::exp(-gp);
      else f = 1.0;
      s[idx(a, b) * 9 + idx(a, b)] = f;
    }
  s[idx(0, 0) * 9 + idx(2, 2)] += b0 * (1 - std::exp(-g));
  s[idx(1, 1) * 9 + idx(2, 2)] += b1 * (1 - std::exp(-g));
  return s;
}

// two-site superoperator of n1 (x) n1: rows/cols of the product are (a,a',b,b'),
// two-site row-major vec is ((a,b),(a',b')).
Mat two_site_product(const Mat& n1) {
  Mat p = kron(n1, 9, n1, 9);  // 81 x 81 on (a,a')(b,b')
  Mat out(81 * 81);
  for (int a = 0; a < 3; ++a)
    for (int ap = 0; ap < 3; ++ap)
      for (int b = 0; b < 3; ++b)
        for (int bp = 0; bp < 3; ++bp)
          for (int c = 0; c < 3; ++c)
            for (int cp = 0; cp < 3; ++cp)
              for (int e = 0; e < 3; ++e)
                for (int ep = 0; ep < 3; ++ep) {
                  int rin = ((a * 3 + ap) * 3 + b) * 3 + bp;
                  int cin = ((c * 3 + cp) * 3 + e) * 3 + ep;
                  int rout = ((a * 3 + b) * 3 + ap) * 3 + bp;
                  int cout = ((c * 3 + e) * 3 + cp) * 3 + ep;
                  out[rout * 81 + cout] = p[rin * 81 + cin];
                }
  return out;
}

// Kraus set from a superoperator on n-dim rho (row-major vec), via the Choi reshuffle
// C[(a,b),(a',b')] = S[(a,a'),(b,b')].
int kraus_from_superop(const Mat& s, int n, double eta, std::vector<Mat>& out) {
  int n2 = n * n;
  Mat c(n2 * n2);
  for (int a = 0; a < n; ++a)
    for (int ap = 0; ap < n; ++ap)
      for (int b = 0; b < n; ++b)
        for (int bp = 0; bp < n; ++bp)
          c[(a * n + b) * n2 + ap * n + bp] = s[(a * n + ap) * n2 + b * n + bp];
  // Hermitian part
  for (int i = 0; i < n2; ++i)
    for (int j = i; j < n2; ++j) {
      zc m = 0.5 * (c[i * n2 + j] + std::conj(c[j * n2 + i]));
      c[i * n2 + j] = m;
      c[j * n2 + i] = std::conj(m);
    }
  std::vector<double> w;
  Mat v;
  jacobi_herm(c, n2, w, v);
  std::vector<int> ord(n2);
  for (int i = 0; i < n2; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return w[x] > w[y]; });
  double wmax = w[ord[0]];
  if (!(wmax > 0)) return MPDO_ERR_NUMERIC;
  out.clear();
  for (int k : ord) {
    if (w[k] <= eta * wmax) break;
    double sq = std::sqrt(w[k]);
    Mat e(n2);
    for (int i = 0; i < n2; ++i) e[i] = sq * v[i * n2 + k];
    out.push_back(e);
  }
  return MPDO_OK;
}

Mat zz_block(double angle) {
  Mat had2 = kron(eye(3), 3, hadq(), 3);
  Mat cz = eye(9);
  cz[4 * 9 + 4] = -1.0;
  Mat cnot = matmul(matmul(had2, cz, 9), had2, 9);
  Mat rz = kron(eye(3), 3, expmh(angle, zq(), 3), 3);
  return matmul(matmul(cnot, rz, 9), cnot, 9);
}

int block_channel(double angle_zz, double gd, double gp, double phi, double dpp, double b0,
                  double b1, double bd, const Mat* post_l, const Mat* post_r, double eta,
                  std::vector<Mat>& kraus, const Mat* shift = nullptr) {
  (void)bd;
  Mat u = zz_block(angle_zz);
  if (phi != 0.0) u = matmul(u, expmh(phi, kron(nr(), 3, nr(), 3), 9), 9);
  if (dpp != 0.0) {
    Mat gen = op3({0, 0, 0, 0, 0, 1, 0, 1, 0});
    Mat pp = expmh(dpp, gen, 3);
    u = matmul(kron(pp, 3, pp, 3), u, 9);
  }
  Mat s = matmul(two_site_product(noise_superop(gd, gp, b0, b1)), unitary_superop(u, 9), 81);
  if (shift) s = matmul(unitary_superop(*shift, 9), s, 81);
  if (post_l || post_r) {
    Mat v = kron(post_l ? *post_l : eye(3), 3, post_r ? *post_r : eye(3), 3);
    s = matmul(unitary_superop(v, 9), s, 81);
  }
  return kraus_from_superop(s, 9, eta, kraus);
}

// ------------------------------------------------------------------ App. E coherent part
// Rydberg dissipation gamma (per pulse) damps the pulse's two-atom coherences by
// alpha = e^{-0.012291 gamma} (one atom through |r>) and beta = e^{-0.0185454 gamma} (both),
// which shows up in the Ising phase gate as the extra phases
//   d1 = ((1 - alpha) / (1 + alpha))^2 on S^z_i + S^z_j,  d2 = ((alpha - beta) / (alpha + beta))^2
// on S^z_i S^z_j (App. E).  With S^z the Pauli matrix on the qubit levels and zero on |r>
// (the workload's reading of S^z), the shift after a block of angle a is the diagonal
// exp(-i sign a (d2 z_i z_j + d1 (z_i + z_j))), z = (1, -1, 0) on (|0>, |1>, |r>).
void appe_shifts(double gamma, double* d1, double* d2) {
  const double al = std::exp(-0.012291 * gamma), be = std::exp(-0.0185454 * gamma);
  *d1 = ((1.0 - al) / (1.0 + al)) * ((1.0 - al) / (1.0 + al));
  *d2 = ((al - be) / (al + be)) * ((al - be) / (al + be));
}

Mat appe_shift(double angle, double d1, double d2, double sign) {
  const double z[3] = {1.0, -1.0, 0.0};
  Mat u(81, zc(0, 0));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double ph = -sign * angle * (d2 * z[a] * z[b] + d1 * (z[a] + z[b]));
      u[(a * 3 + b) * 9 + (a * 3 + b)] = zc(std::cos(ph), std::sin(ph));
    }
  return u;
}

// ------------------------------------------------------------------ gate model G1
// Pulse-level CZ (Sec. II): two atoms under H_p(t) = H_1 (x) I + I (x) H_2 + B |rr><rr|,
// H_i = Omega(t)/2 (|r><1| + h.c.) + Delta |r><r|, Gaussian Omega of Fig. 1 (offset to start
// and end at 0), with the one-atom dissipators of Eq. LME at rates gamma / T (gamma per
// pulse).  The pulse is integrated into one channel (Sec. III.A) by n equal steps, each
//   N(tau/2) (U_k (x) conj U_k) N(tau/2),  U_k = exp(-i tau H_p(t_k)), t_k the midpoint,
// with N the closed-form one-atom noise on both atoms (exact for a constant generator)
// and H_p exponentiated whole (Jacobi eigendecomposition of the 9 x 9 matrix).  Each atom
// then gets diag(1, e^{-i phi_1}, 1), phi_1 the |01> phase of the noiseless pulse, which
// turns the pulse into a CZ when phi_11 - 2 phi_1 = pi.
double gaussian_omega(double t, const mpdo_pulse& p) {
  const double u = p.width * p.T, t0 = 0.5 * p.T;
  const double a = std::exp(-(t0 / u) * (t0 / u));
  const double x = (t - t0) / u;
  return p.omega_max * (std::exp(-x * x) - a) / (1.0 - a);
}

Mat pulse_hamiltonian(double om, const mpdo_pulse& p) {
  Mat h1 = op3({0, 0, 0, 0, 0, 0.5 * om, 0, 0.5 * om, p.delta});
  Mat h = kron(h1, 3, eye(3), 3);
  Mat h2 = kron(eye(3), 3, h1, 3);
  for (int i = 0; i < 81; ++i) h[i] += h2[i];
  h[8 * 9 + 8] += p.blockade;   // |rr><rr|
  return h;
}

// s <- (u (x) conj u) s on two-atom superoperators: every column is a 9 x 9 matrix X over
// ((a,b),(a',b')) and becomes u X u^+.
void apply_unitary(Mat& s, const Mat& u) {
  Mat x(81), y(81);
  for (int c = 0; c < 81; ++c) {
    for (int i = 0; i < 81; ++i) x[i] = s[i * 81 + c];
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) {
        zc acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += u[i * 9 + k] * x[k * 9 + j];
        y[i * 9 + j] = acc;
      }
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) {
        zc acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += y[i * 9 + k] * std::conj(u[j * 9 + k]);
        s[(i * 9 + j) * 81 + c] = acc;
      }
  }
}

// s <- (n1 on atom `site`) s, n1 a one-atom superoperator (9 x 9 on (a,a')), applied through
// its nonzero entries.
void apply_one_atom(Mat& s, const Mat& n1, int site) {
  struct Nz { int r, c; zc v; };
  std::vector<Nz> nz;
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c)
      if (n1[r * 9 + c] != 0.0) nz.push_back({r, c, n1[r * 9 + c]});
  Mat out(81 * 81, 0.0);
  for (const Nz& e : nz) {
    const int a = e.r / 3, ap = e.r % 3, c = e.c / 3, cp = e.c % 3;
    for (int o = 0; o < 3; ++o)
      for (int op = 0; op < 3; ++op) {
        // the other atom's indices o (ket) and op (bra) are untouched
        const int rin = site == 0 ? (c * 3 + o) * 9 + (cp * 3 + op) : (o * 3 + c) * 9 + (op * 3 + cp);
        const int rout = site == 0 ? (a * 3 + o) * 9 + (ap * 3 + op) : (o * 3 + a) * 9 + (op * 3 + ap);
        for (int col = 0; col < 81; ++col) out[rout * 81 + col] += e.v * s[rin * 81 + col];
      }
  }
  s.swap(out);
}

int cz_pulse(const mpdo_pulse& p, double gd, double gp, double b0, double b1, int n_steps,
             Mat& s, double& phi1, double& infid) {
  const double tau = p.T / n_steps;
  auto step = [&](int k) {
    return expmh(tau, pulse_hamiltonian(gaussian_omega((k + 0.5) * tau, p), p), 9);
  };
  // noiseless pulse and its phase correction (the step exponentials are recomputed in the
  // second pass rather than stored: n_steps may be large)
  Mat u = eye(9);
  for (int k = 0; k < n_steps; ++k) u = matmul(step(k), u, 9);
  phi1 = std::arg(u[1 * 9 + 1]) - std::arg(u[0]);
  Mat c1 = op3({1, 0, 0, 0, std::exp(zc(0, -phi1)), 0, 0, 0, 1});
  Mat cc = kron(c1, 3, c1, 3);
  Mat uc = matmul(cc, u, 9);
  const int q[4] = {0, 1, 3, 4};
  zc tr = 0.0;
  for (int i = 0; i < 4; ++i) tr += (i == 3 ? -1.0 : 1.0) * uc[q[i] * 9 + q[i]];
  infid = 1.0 - (std::norm(tr) + 4.0) / 20.0;
  // the noisy channel
  const Mat nh = noise_superop(gd * 0.5 * tau / p.T, gp * 0.5 * tau / p.T, b0, b1);
  s = eye(81);
  for (int k = 0; k < n_steps; ++k) {
    apply_one_atom(s, nh, 0);
    apply_one_atom(s, nh, 1);
    apply_unitary(s, step(k));
    apply_one_atom(s, nh, 0);
    apply_one_atom(s, nh, 1);
  }
  apply_unitary(s, cc);
  for (zc v : s)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return MPDO_ERR_NUMERIC;
  return MPDO_OK;
}

// The ZZ block with each CZ replaced by the channel s_cz (81 x 81): superoperator products
// of (I (x) Had) s_cz (I (x) Had Rz Had) s_cz (I (x) Had), crosstalk phase first, optional
// one-site unitaries after; Kraus set from the Choi matrix.
int block_channel_cz(double angle_zz, const Mat& s_cz, double phi, const Mat* post_l,
                     const Mat* post_r, double eta, std::vector<Mat>& kraus) {
  Mat had2 = kron(eye(3), 3, hadq(), 3);
  Mat rz = kron(eye(3), 3, expmh(angle_zz, zq(), 3), 3);
  Mat mid = matmul(matmul(had2, rz, 9), had2, 9);
  Mat s = unitary_superop(had2, 9);
  s = matmul(s_cz, s, 81);
  s = matmul(unitary_superop(mid, 9), s, 81);
  s = matmul(s_cz, s, 81);
  s = matmul(unitary_superop(had2, 9), s, 81);
  if (phi != 0.0) s = matmul(s, unitary_superop(expmh(phi, kron(nr(), 3, nr(), 3), 9), 9), 81);
  if (post_l || post_r) {
    Mat v = kron(post_l ? *post_l : eye(3), 3, post_r ? *post_r : eye(3), 3);
    s = matmul(unitary_superop(v, 9), s, 81);
  }
  return kraus_from_superop(s, 9, eta, kraus);
}

bool finite_all(std::initializer_list<double> xs) {
  for (double x : xs)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace

extern "C" int mpdo_build_block_channel(double angle_zz, double gamma_diss, double gamma_deph,
                                        double xtalk_phase, double delta_pp, double b0, double b1,
                                        double bd, const double* post_left,
                                        const double* post_right, double eta, double* out,
                                        int cap, int* n_kraus) {
  if (!out || !n_kraus || cap < 1) return MPDO_ERR_ARG;
  if (!finite_all({angle_zz, gamma_diss, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd, eta}))
    return MPDO_ERR_NUMERIC;
  if (gamma_diss < 0 || gamma_deph < 0 || b0 < 0 || b1 < 0 || bd < 0) return MPDO_ERR_ARG;
  // a negative eta would keep negative Choi eigenvalues (square roots of them are NaN)
  if (eta < 0) return MPDO_ERR_ARG;
  Mat pl, pr;
  if (post_left) {
    pl.resize(9);
    for (int i = 0; i < 9; ++i) pl[i] = zc(post_left[2 * i], post_left[2 * i + 1]);
  }
  if (post_right) {
    pr.resize(9);
    for (int i = 0; i < 9; ++i) pr[i] = zc(post_right[2 * i], post_right[2 * i + 1]);
  }
  std::vector<Mat> k;
  int rc = block_channel(angle_zz, gamma_diss, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd,
                         post_left ? &pl : nullptr, post_right ? &pr : nullptr, eta, k);
  if (rc) return rc;
  *n_kraus = (int)k.size();
  if ((int)k.size() > cap) return MPDO_ERR_ARG;
  for (size_t m = 0; m < k.size(); ++m)
    for (int i = 0; i < 81; ++i) {
      out[(m * 81 + i) * 2] = k[m][i].real();
      out[(m * 81 + i) * 2 + 1] = k[m][i].imag();
    }
  return MPDO_OK;
}

// QAOA layer k in gate model G0; part = -1 the full block, 0 its App. E coherent part alone
// (no dissipation, the shift of gamma_diss applied), 1 the block with that shift reversed.
int qaoa_layer(int n_sites, int k, double alpha, double beta, double J, double bz,
               double gamma_diss, double gamma_deph, double xtalk_phase, double delta_pp,
               double b0, double b1, double bd, double eta, int part, int* sites, int* ms,
               double* out, size_t cap) {
  if (n_sites < 2 || k < 0 || !sites || !ms || !out || part < -1 || part > 1) return MPDO_ERR_ARG;
  if (!finite_all({alpha, beta, J, bz, eta})) return MPDO_ERR_NUMERIC;
  if (eta < 0) return MPDO_ERR_ARG;
  if (part >= 0 && (!std::isfinite(gamma_diss) || gamma_diss < 0)) return MPDO_ERR_ARG;
  // one-site gate exp(-i beta S^x) exp(-i b J alpha S^z), folded after the last block
  Mat v = matmul(expmh(beta, xq(), 3), expmh(bz * J * alpha, zq(), 3), 3);
  Mat shift;
  double gd = gamma_diss;
  if (part >= 0) {
    double d1, d2;
    appe_shifts(gamma_diss, &d1, &d2);
    shift = appe_shift(J * alpha, d1, d2, part == 0 ? 1.0 : -1.0);
    if (part == 0) gd = 0.0;
  }
  const Mat* sh = part >= 0 ? &shift : nullptr;
  std::vector<Mat> both, mid;
  int rc = block_channel(J * alpha, gd, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd, &v, &v,
                         eta, both, sh);
  if (rc) return rc;
  const bool ltr = (k % 2 == 0);
  rc = block_channel(J * alpha, gd, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd,
                     ltr ? &v : nullptr, ltr ? nullptr : &v, eta, mid, sh);
  if (rc) return rc;
  size_t off = 0;
  for (int q = 0; q < n_sites - 1; ++q) {
    int i = ltr ? q : n_sites - 2 - q;
    bool last = ltr ? (i == n_sites - 2) : (i == 0);
    const std::vector<Mat>& ch = last ? both : mid;
    sites[q] = i;
    ms[q] = (int)ch.size();
    if (off + ch.size() * 81 > cap) return MPDO_ERR_ARG;
    for (const Mat& e : ch)
      for (int a = 0; a < 81; ++a) {
        out[2 * off] = e[a].real();
        out[2 * off + 1] = e[a].imag();
        ++off;
      }
  }
  return MPDO_OK;
}

extern "C" int mpdo_build_qaoa_layer(int n_sites, int k, double alpha, double beta, double J,
                                     double bz, double gamma_diss, double gamma_deph,
                                     double xtalk_phase, double delta_pp, double b0, double b1,
                                     double bd, double eta, int* sites, int* ms, double* out,
                                     size_t cap) {
  return qaoa_layer(n_sites, k, alpha, beta, J, bz, gamma_diss, gamma_deph, xtalk_phase,
                    delta_pp, b0, b1, bd, eta, -1, sites, ms, out, cap);
}

extern "C" int mpdo_build_qaoa_layer_appe(int n_sites, int k, double alpha, double beta,
                                          double J, double bz, double gamma_diss,
                                          double gamma_deph, double xtalk_phase,
                                          double delta_pp, double b0, double b1, double bd,
                                          int part, double eta, int* sites, int* ms,
                                          double* out, size_t cap) {
  if (part != 0 && part != 1) return MPDO_ERR_ARG;
  return qaoa_layer(n_sites, k, alpha, beta, J, bz, gamma_diss, gamma_deph, xtalk_phase,
                    delta_pp, b0, b1, bd, eta, part, sites, ms, out, cap);
}

// Random-circuit layer (the paper's RCS workload, Sec. IV / Figs. 4-5): one sweep over the
// bonds (left to right for even k, right to left for odd k); bond i carries a noisy CZ when
// i = k mod 2 (gate model G0: crosstalk phase, ideal CZ, post-promotion, one unit of decay and
// dephasing on both atoms), otherwise only one-atom gates; every atom's Haar gate (2 x 2 on the
// qubit levels, |r> untouched) is folded into the first op of the sweep that touches it.
extern "C" int mpdo_build_rcs_layer(int n_sites, int k, const double* haar, double gamma_diss,
                                    double gamma_deph, double xtalk_phase, double delta_pp,
                                    double b0, double b1, double bd, double eta, int* sites,
                                    int* ms, double* out, size_t cap) {
  if (n_sites < 2 || k < 0 || !haar || !sites || !ms || !out) return MPDO_ERR_ARG;
  if (!finite_all({gamma_diss, gamma_deph, xtalk_phase, delta_pp, b0, b1, bd, eta}))
    return MPDO_ERR_NUMERIC;
  if (gamma_diss < 0 || gamma_deph < 0 || b0 < 0 || b1 < 0 || bd < 0 || eta < 0)
    return MPDO_ERR_ARG;
  std::vector<Mat> gates(n_sites);
  for (int j = 0; j < n_sites; ++j) {
    Mat g = eye(3);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double* p = haar + 2 * (4 * j + 2 * a + b);
        if (!std::isfinite(p[0]) || !std::isfinite(p[1])) return MPDO_ERR_NUMERIC;
        g[a * 3 + b] = zc(p[0], p[1]);
      }
    gates[j] = g;
  }
  const bool ltr = (k % 2 == 0);
  std::vector<bool> seen(n_sites, false);
  Mat cz = eye(9);
  cz[4 * 9 + 4] = -1.0;
  size_t off = 0;
  for (int q = 0; q < n_sites - 1; ++q) {
    const int i = ltr ? q : n_sites - 2 - q;
    Mat pl = seen[i] ? eye(3) : gates[i];
    Mat pr = seen[i + 1] ? eye(3) : gates[i + 1];
    seen[i] = seen[i + 1] = true;
    Mat pre = kron(pl, 3, pr, 3);
    std::vector<Mat> ch;
    if (i % 2 == k % 2) {
      Mat u = cz;
      if (xtalk_phase != 0.0) u = matmul(u, expmh(xtalk_phase, kron(nr(), 3, nr(), 3), 9), 9);
      u = matmul(u, pre, 9);
      if (delta_pp != 0.0) {
        Mat pp = expmh(delta_pp, op3({0, 0, 0, 0, 0, 1, 0, 1, 0}), 3);
        u = matmul(kron(pp, 3, pp, 3), u, 9);
      }
      Mat s = matmul(two_site_product(noise_superop(gamma_diss, gamma_deph, b0, b1)),
                     unitary_superop(u, 9), 81);
      int rc = kraus_from_superop(s, 9, eta, ch);
      if (rc) return rc;
    } else {
      ch.push_back(pre);
    }
    sites[q] = i;
    ms[q] = (int)ch.size();
    if (off + ch.size() * 81 > cap) return MPDO_ERR_ARG;
    for (const Mat& e : ch)
      for (int a = 0; a < 81; ++a) {
        out[2 * off] = e[a].real();
        out[2 * off + 1] = e[a].imag();
        ++off;
      }
  }
  return MPDO_OK;
}

extern "C" int mpdo_build_cz_pulse(const mpdo_pulse* pulse, double gamma_diss,
                                   double gamma_deph, double b0, double b1, int n_steps,
                                   double* superop, double* phi1, double* infidelity) {
  if (!pulse || !superop || n_steps < 1 || n_steps > 1000000) return MPDO_ERR_ARG;
  if (!finite_all({pulse->T, pulse->omega_max, pulse->delta, pulse->blockade, pulse->width,
                   gamma_diss, gamma_deph, b0, b1}))
    return MPDO_ERR_NUMERIC;
  if (!(pulse->T > 0) || !(pulse->width > 0) || gamma_diss < 0 || gamma_deph < 0 || b0 < 0 ||
      b1 < 0)
    return MPDO_ERR_ARG;
  Mat s;
  double ph = 0, inf = 0;
  int rc = cz_pulse(*pulse, gamma_diss, gamma_deph, b0, b1, n_steps, s, ph, inf);
  if (rc) return rc;
  for (int i = 0; i < 81 * 81; ++i) {
    superop[2 * i] = s[i].real();
    superop[2 * i + 1] = s[i].imag();
  }
  if (phi1) *phi1 = ph;
  if (infidelity) *infidelity = inf;
  return MPDO_OK;
}

// Crosstalk CZ (Sec. III.B): the noiseless pulse with the atoms' detunings shifted by
// s1, s2 (a Rydberg neighbour next to an active atom shifts its detuning by the neighbour
// blockade), then the controlled combination over the non-active neighbours' Rydberg
// projectors.  The phase correction is the unshifted pulse's.
Mat pulse_unitary_shifted(const mpdo_pulse& p, int n_steps, double s1, double s2) {
  const double tau = p.T / n_steps;
  Mat u = eye(9);
  for (int k = 0; k < n_steps; ++k) {
    const double om = gaussian_omega((k + 0.5) * tau, p);
    Mat h1 = op3({0, 0, 0, 0, 0, 0.5 * om, 0, 0.5 * om, p.delta + s1});
    Mat h2 = op3({0, 0, 0, 0, 0, 0.5 * om, 0, 0.5 * om, p.delta + s2});
    Mat h = kron(h1, 3, eye(3), 3);
    Mat hb = kron(eye(3), 3, h2, 3);
    for (int i = 0; i < 81; ++i) h[i] += hb[i];
    h[8 * 9 + 8] += p.blockade;   // |rr><rr|
    u = matmul(expmh(tau, h, 9), u, 9);
  }
  return u;
}

extern "C" int mpdo_build_crosstalk_cz(const mpdo_pulse* pulse, double b_x, int n_steps,
                                       double* out) {
  if (!pulse || !out || n_steps < 1 || n_steps > 1000000) return MPDO_ERR_ARG;
  if (!finite_all({pulse->T, pulse->omega_max, pulse->delta, pulse->blockade, pulse->width,
                   b_x}))
    return MPDO_ERR_NUMERIC;
  if (!(pulse->T > 0) || !(pulse->width > 0)) return MPDO_ERR_ARG;
  const Mat u0 = pulse_unitary_shifted(*pulse, n_steps, 0.0, 0.0);
  const double phi1 = std::arg(u0[1 * 9 + 1]) - std::arg(u0[0]);
  const Mat c1 = op3({1, 0, 0, 0, std::exp(zc(0, -phi1)), 0, 0, 0, 1});
  const Mat cc = kron(c1, 3, c1, 3);
  const Mat pr = op3({0, 0, 0, 0, 0, 0, 0, 0, 1});
  const Mat pn = op3({1, 0, 0, 0, 1, 0, 0, 0, 0});
  Mat acc(81 * 81, zc(0, 0));
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const Mat ua = (a == 0 && b == 0) ? u0
                                        : pulse_unitary_shifted(*pulse, n_steps, a * b_x, b * b_x);
      const Mat g = matmul(cc, ua, 9);
      const Mat term = kron(kron(a ? pr : pn, 3, g, 9), 27, b ? pr : pn, 3);
      for (int i = 0; i < 81 * 81; ++i) acc[i] += term[i];
    }
  for (int i = 0; i < 81 * 81; ++i) {
    out[2 * i] = acc[i].real();
    out[2 * i + 1] = acc[i].imag();
  }
  return MPDO_OK;
}

extern "C" int mpdo_build_qaoa_layer_cz(int n_sites, int k, double alpha, double beta, double J,
                                        double bz, const double* cz_superop, double xtalk_phase,
                                        double eta, int* sites, int* ms, double* out,
                                        size_t cap) {
  if (n_sites < 2 || k < 0 || !cz_superop || !sites || !ms || !out) return MPDO_ERR_ARG;
  if (!finite_all({alpha, beta, J, bz, xtalk_phase, eta})) return MPDO_ERR_NUMERIC;
  if (eta < 0) return MPDO_ERR_ARG;
  Mat scz(81 * 81);
  for (int i = 0; i < 81 * 81; ++i) {
    scz[i] = zc(cz_superop[2 * i], cz_superop[2 * i + 1]);
    if (!std::isfinite(scz[i].real()) || !std::isfinite(scz[i].imag())) return MPDO_ERR_NUMERIC;
  }
  // one-site gate exp(-i beta S^x) exp(-i b J alpha S^z), folded after the last block
  Mat v = matmul(expmh(beta, xq(), 3), expmh(bz * J * alpha, zq(), 3), 3);
  std::vector<Mat> both, mid;
  int rc = block_channel_cz(J * alpha, scz, xtalk_phase, &v, &v, eta, both);
  if (rc) return rc;
  const bool ltr = (k % 2 == 0);
  rc = block_channel_cz(J * alpha, scz, xtalk_phase, ltr ? &v : nullptr, ltr ? nullptr : &v,
                        eta, mid);
  if (rc) return rc;
  size_t off = 0;
  for (int q = 0; q < n_sites - 1; ++q) {
    int i = ltr ? q : n_sites - 2 - q;
    bool last = ltr ? (i == n_sites - 2) : (i == 0);
    const std::vector<Mat>& ch = last ? both : mid;
    sites[q] = i;
    ms[q] = (int)ch.size();
    if (off + ch.size() * 81 > cap) return MPDO_ERR_ARG;
    for (const Mat& e : ch)
      for (int a = 0; a < 81; ++a) {
        out[2 * off] = e[a].real();
        out[2 * off + 1] = e[a].imag();
        ++off;
      }
  }
  return MPDO_OK;
}
