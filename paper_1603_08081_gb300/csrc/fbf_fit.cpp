// Host-side FP64 parts of the C ABI: Algorithm 2 (coefficient fit), window
// resolution, spatial weights, status strings.
#include <cmath>
#include <cstring>
#include <vector>

#include "fbf.h"
#include "fbf_internal.h"

namespace fbf {

// Range kernel phi: Gaussian eq. (3); exponential exp(-|t|/sigma_r) (Sec. I).
static double range_kernel(fbf_range_kernel k, double sigma_r, double t) {
  if (k == FBF_RANGE_EXPONENTIAL) return std::exp(-std::fabs(t) / sigma_r);
  return std::exp(-(t * t) / (2.0 * sigma_r * sigma_r));
}

int resolve_window(fbf_spatial_kernel spatial, double sigma_s, int W) {
  if (W > 0) return W;
  if (spatial != FBF_SPATIAL_GAUSSIAN || !(sigma_s > 0.0) || !std::isfinite(sigma_s)) return -1;
  // Sec. I: Omega = [-W, W]^2 with W = 3 sigma_s; rounded up for fractional sigma_s.
  double w = std::ceil(3.0 * sigma_s - 1e-12);
  if (w > 1e6) return -1;
  return (int)w;
}

// Recursive Gaussian (the constant-time Gaussian filtering cited in Sec. II,
// after eq. (5): Deriche 1993).  Deriche writes exp(-x^2 / (2 s^2)), x >= 0, as
// two damped sinusoids (a_i cos(w_i x/s) + b_i sin(w_i x/s)) exp(-l_i x/s) with
// the published constants below.  Each term, sampled at k >= 0, is the impulse
// response of a second-order section: its z-transform is
//   (a + e^{-l}(b sin w - a cos w) z^-1) / (1 - 2 e^{-l} cos w z^-1 + e^{-2l} z^-2)
// (w, l divided by s); its mirror k <= -1 is the anticausal section with
// numerator N(1/z) - a D(1/z) on z, z^2.  The two sections run in parallel and
// their sum is scaled to unit gain.
void recursive_coeffs(double sigma_s, FilterArgs *a) {
  static const double ka[2] = {1.680, -0.6803}, kb[2] = {3.735, -0.2598};
  static const double kw[2] = {0.6318, 1.997}, kl[2] = {1.783, 1.723};
  double n[2][2], m[2][2], p[2][2], gain = 0.0;
  for (int i = 0; i < 2; ++i) {
    const double w = kw[i] / sigma_s, e = std::exp(-kl[i] / sigma_s);
    n[i][0] = ka[i];
    n[i][1] = e * (kb[i] * std::sin(w) - ka[i] * std::cos(w));
    p[i][0] = -2.0 * e * std::cos(w);
    p[i][1] = e * e;
    m[i][0] = n[i][1] - n[i][0] * p[i][0];
    m[i][1] = -n[i][0] * p[i][1];
    gain += (n[i][0] + n[i][1] + m[i][0] + m[i][1]) / (1.0 + p[i][0] + p[i][1]);
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      a->rn[i][j] = (float)(n[i][j] / gain);
      a->rm[i][j] = (float)(m[i][j] / gain);
      a->rp[i][j] = (float)p[i][j];
    }
  a->rE = (int)std::ceil(8.0 * sigma_s);
}

// Normalised 1-D weights w1[j + W], j = -W..W, sum 1; the 2-D kernel of eq. (2)
// is w1(j_y) w1(j_x) and sums to 1 (Sec. IV assumes unit sum).
void spatial_weights(fbf_spatial_kernel spatial, double sigma_s, int W, float *w1) {
  std::vector<double> w(2 * W + 1);
  double s = 0.0;
  for (int j = -W; j <= W; ++j) {
    double v = spatial == FBF_SPATIAL_BOX ? 1.0 : std::exp(-(double)j * j / (2.0 * sigma_s * sigma_s));
    w[j + W] = v;
    s += v;
  }
  for (int j = 0; j < 2 * W + 1; ++j) w1[j] = (float)(w[j] / s);
}

}  // namespace fbf

using namespace fbf;

extern "C" int fbf_resolve_window(const fbf_params *p) {
  if (!p) return -1;
  return resolve_window(p->spatial, p->sigma_s, p->W);
}

// Algorithm 2: Progressive Fourier Approximation with a recursive modified
// Gram-Schmidt QR.  Column k of A is cos(k omega t) (k = 0 is the all-ones
// start vector); each new column is orthogonalised against the previous q's
// one at a time (MGS), normalised, appended to Q, and Q^T b and R grow by one
// entry / column; R d = p is solved by back-substitution and the residual
// E = ||b - A d|| decides whether to continue (Sec. III).  b holds the samples
// phi(t_l) on the grid t (L points), however they were obtained.
namespace {

fbf_status progressive_fit(const std::vector<double> &t, const std::vector<double> &b, int L, double T,
                           double eps, int K_fixed, fbf_coeffs *out) {
  const int Kcap = L < FBF_KMAX ? L : FBF_KMAX;
  if (K_fixed > Kcap) return FBF_ERR_RANGE;

  const double omega = M_PI / T;
  std::vector<double> a(L);
  std::vector<double> Qm((size_t)L * Kcap);  // orthonormal columns q_1..q_N
  std::vector<double> R((size_t)Kcap * Kcap, 0.0);  // R[row * Kcap + col]
  std::vector<double> p(Kcap), d(Kcap);

  auto residual = [&](int N, double *l2, double *linf) {
    double e2 = 0.0, em = 0.0;
    for (int l = 0; l < L; ++l) {
      double r = b[l];
      for (int k = 0; k < N; ++k) r -= std::cos((double)k * omega * t[l]) * d[k];
      e2 += r * r;
      em = std::fmax(em, std::fabs(r));
    }
    *l2 = std::sqrt(e2);
    *linf = em;
  };
  auto back_substitute = [&](int N) {
    for (int i = N - 1; i >= 0; --i) {
      double s = p[i];
      for (int c = i + 1; c < N; ++c) s -= R[(size_t)i * Kcap + c] * d[c];
      d[i] = s / R[(size_t)i * Kcap + i];
    }
  };

  // Initialise with the all-ones column: R = ||a||, Q = a / R, p = Q^T b.
  int N = 1;
  double nrm = std::sqrt((double)L);
  R[0] = nrm;
  for (int l = 0; l < L; ++l) Qm[l] = 1.0 / nrm;
  double s = 0.0;
  for (int l = 0; l < L; ++l) s += Qm[l] * b[l];
  p[0] = s;
  back_substitute(1);
  double E, Einf;
  residual(1, &E, &Einf);

  auto done = [&]() { return K_fixed > 0 ? N >= K_fixed : E <= eps; };
  while (!done() && N < Kcap) {
    // New column: the next harmonic, cos(N omega t) for 0-based column index N.
    for (int l = 0; l < L; ++l) a[l] = std::cos((double)N * omega * t[l]);
    for (int k = 0; k < N; ++k) {  // modified Gram-Schmidt sweep
      const double *qk = &Qm[(size_t)k * L];
      double r = 0.0;
      for (int l = 0; l < L; ++l) r += a[l] * qk[l];
      R[(size_t)k * Kcap + N] = r;
      for (int l = 0; l < L; ++l) a[l] -= r * qk[l];
    }
    double rn = 0.0;
    for (int l = 0; l < L; ++l) rn += a[l] * a[l];
    rn = std::sqrt(rn);
    if (!(rn > 0.0)) break;  // basis exhausted (cannot happen for N < L)
    R[(size_t)N * Kcap + N] = rn;
    double *qn = &Qm[(size_t)N * L];
    double pb = 0.0;
    for (int l = 0; l < L; ++l) {
      qn[l] = a[l] / rn;
      pb += qn[l] * b[l];
    }
    p[N] = pb;
    ++N;
    back_substitute(N);
    residual(N, &E, &Einf);
  }

  std::memset(out, 0, sizeof(*out));
  out->K = N;
  out->levels = L;
  out->T = T;
  out->omega = omega;
  out->resid_l2 = E;
  out->resid_linf = Einf;
  for (int k = 0; k < N; ++k) out->d[k] = d[k];
  return done() ? FBF_OK : FBF_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" fbf_status fbf_fit_coeffs(fbf_range_kernel kernel, double sigma_r, double T,
                                     double eps, int K_fixed, int levels, fbf_coeffs *out) {
  if (!out) return FBF_ERR_INVALID_ARGUMENT;
  if (kernel != FBF_RANGE_GAUSSIAN && kernel != FBF_RANGE_EXPONENTIAL) return FBF_ERR_INVALID_ARGUMENT;
  if (!(sigma_r > 0.0) || !std::isfinite(sigma_r)) return FBF_ERR_INVALID_ARGUMENT;
  if (!(T > 0.0) || !std::isfinite(T)) return FBF_ERR_INVALID_ARGUMENT;
  if (K_fixed < 0 || levels < 0 || levels == 1) return FBF_ERR_INVALID_ARGUMENT;
  if (K_fixed == 0 && !(eps > 0.0)) return FBF_ERR_INVALID_ARGUMENT;
  int L;
  if (levels == 0) {
    if (T != std::floor(T) || T > 1e6) return FBF_ERR_INVALID_ARGUMENT;
    L = (int)T + 1;
  } else {
    L = levels;
  }
  std::vector<double> t(L), b(L);
  for (int l = 0; l < L; ++l) {
    t[l] = levels == 0 ? (double)l : (double)l * T / (double)(levels - 1);
    b[l] = range_kernel(kernel, sigma_r, t[l]);
  }
  return progressive_fit(t, b, L, T, eps, K_fixed, out);
}

// Any range kernel given by its samples (Sec. III: every kernel whose Fourier
// series converges pointwise qualifies): phi[l] = phi(t_l) on the equispaced
// grid t_l = l T / (L - 1), l = 0..L-1 (for integer T and L = T + 1, the grid
// {0, 1, ..., T} of Algorithm 2).
extern "C" fbf_status fbf_fit_coeffs_samples(const double *phi, int L, double T, double eps, int K_fixed,
                                             fbf_coeffs *out) {
  if (!out || !phi) return FBF_ERR_INVALID_ARGUMENT;
  if (L < 2 || L > (1 << 20)) return FBF_ERR_INVALID_ARGUMENT;
  if (!(T > 0.0) || !std::isfinite(T)) return FBF_ERR_INVALID_ARGUMENT;
  if (K_fixed < 0) return FBF_ERR_INVALID_ARGUMENT;
  if (K_fixed == 0 && !(eps > 0.0)) return FBF_ERR_INVALID_ARGUMENT;
  std::vector<double> t(L), b(L);
  for (int l = 0; l < L; ++l) {
    if (!std::isfinite(phi[l])) return FBF_ERR_INVALID_ARGUMENT;
    t[l] = (double)l * T / (double)(L - 1);
    b[l] = phi[l];
  }
  return progressive_fit(t, b, L, T, eps, K_fixed, out);
}

extern "C" const char *fbf_status_string(fbf_status s) {
  switch (s) {
    case FBF_OK: return "FBF_OK";
    case FBF_ERR_INVALID_ARGUMENT: return "FBF_ERR_INVALID_ARGUMENT: invalid argument";
    case FBF_ERR_NOT_CONVERGED: return "FBF_ERR_NOT_CONVERGED: tolerance not reached";
    case FBF_ERR_RANGE: return "FBF_ERR_RANGE: beyond the compiled limits";
    case FBF_ERR_UNSUPPORTED: return "FBF_ERR_UNSUPPORTED: not implemented for this request";
    case FBF_ERR_CUDA: return "FBF_ERR_CUDA: CUDA runtime or launch failure";
    case FBF_ERR_TIMEOUT: return "FBF_ERR_TIMEOUT: bounded device wait expired";
  }
  return "unknown fbf_status";
}

extern "C" int fbf_version(void) { return 100; }
