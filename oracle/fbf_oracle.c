/*
 * fbf_oracle.c -- plain, slow, FP64 CPU oracle for the shiftable Fourier-kernel
 * bilateral filter of Ghosh & Chaudhury, "On Fast Bilateral Filtering using
 * Fourier Kernels" (arXiv 1603.08081).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA library, and neither side includes the other.
 *
 * What is here, each function citing the passage it follows:
 *   orc_phi            range kernels: Gaussian eq. (3); exponential (Sec. I)
 *   orc_fit_samples    least-squares fit of the cosine series eq. (6) to samples,
 *                      eqs. (7)-(8), smallest order with residual <= eps (Sec. III)
 *   orc_fit            the same on the grid Lambda_T of Sec. III / Algorithm 2
 *   orc_weights_1d     spatial kernel eq. (2) on Omega = [-W, W]^2, sum w = 1
 *                      (Sec. IV); box kernel (Sec. I)
 *   orc_direct         direct O(W^2)-per-pixel filter: eq. (1) with the exact
 *                      range kernel, or eq. (9) with phi_N
 *   orc_alg1           Algorithm 1 in the paper's complex notation, eqs. (4)-(5)
 *   orc_grad_direct    d/df(m) of sum_i g(i) fhat(i), fhat from eq. (9)
 *   orc_grad_at        the same derivative at sampled pixels only
 *   orc_local_range    the dynamic range T of the image over the window Omega,
 *                      the definition that opens Sec. III
 *   orc_rec_kernel,    the recursive Gaussian that Sec. II cites for constant-
 *   orc_rec_coeffs,    time filtering (Deriche): its kernel, its recursion
 *   orc_rec_filter_line  coefficients and one line through it
 *   orc_alg1_rec       Algorithm 1 with that recursive filter as the convolution
 *
 * The fit uses Householder QR, deliberately not the modified Gram-Schmidt
 * recursion of Algorithm 2, so the two are independent: the least-squares
 * solution is unique, and both must reach it.
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *   * basis columns are cos(k*omega*t), k = 0..K-1, omega = pi/T; K counts
 *     coefficients d_0..d_{K-1} (the order "N" of Tables 3-4);
 *   * the fit stops at the first K with ||b - A d||_2 <= eps;
 *   * borders: REFLECT is half-sample symmetric (index -1 -> 0, period 2n);
 *     TRUNCATE sums only over neighbours inside the image;
 *   * Gaussian W defaults to ceil(3 sigma_s) (Sec. I gives W = 3 sigma_s); the
 *     box kernel is uniform over [-W, W]^2.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_RANGE_GAUSSIAN 0
#define ORC_RANGE_EXPONENTIAL 1
#define ORC_SPATIAL_GAUSSIAN 0
#define ORC_SPATIAL_BOX 1
#define ORC_BORDER_REFLECT 0
#define ORC_BORDER_TRUNCATE 1

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel loops (timing on one core or all). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Range kernel.  Gaussian: eq. (3).  Exponential: exp(-|t|/sigma_r), the kernel
 * of the works cited in Sec. I (the paper names it without printing it). */
double orc_phi(int kernel, double sigma_r, double t) {
  if (kernel == ORC_RANGE_EXPONENTIAL) return exp(-fabs(t) / sigma_r);
  return exp(-(t * t) / (2.0 * sigma_r * sigma_r));
}

/* phi_N(t) = d_0 + sum_{k>=1} d_k cos(k omega t), omega = pi / T  (eq. (6)). */
double orc_phi_n(const double *d, int K, double T, double t) {
  double omega = M_PI / T, s = 0.0;
  for (int k = 0; k < K; ++k) s += d[k] * cos((double)k * omega * t);
  return s;
}

/* Least squares over the columns a_k = [cos(k omega t_l)]_l, k = 0..K-1
 * (eqs. (7)-(8)).  For K = 1, 2, ... solve min_d ||b - A_K d||_2 and stop at the
 * first K with E_K = ||b - A_K d||_2 <= eps (Sec. III, the loop of Algorithm 2).
 * K_fixed > 0 solves at exactly that K instead.
 *
 * Householder QR: after reflection j the leading (j+1)x(j+1) block of R and the
 * first j+1 entries of Q^T b are those of the (j+1)-column problem, so each K
 * costs one back-substitution plus a residual evaluated directly as b - A d.
 *
 * Returns 0 (converged / fixed K reached), 1 (eps not reached by Kmax columns),
 * -1 (bad argument).  d_out gets K_out coefficients. */
int orc_fit_samples(const double *t, const double *b, int L, double T, double eps,
                    int K_fixed, int Kmax, double *d_out, int *K_out, double *E_out,
                    double *linf_out) {
  if (L < 1 || !(T > 0.0) || Kmax < 1) return -1;
  int Kcap = K_fixed > 0 ? K_fixed : Kmax;
  if (Kcap > L) {
    if (K_fixed > 0) return -1;
    Kcap = L;
  }
  double omega = M_PI / T;
  double *A = malloc(sizeof(double) * (size_t)L * Kcap); /* column-major, untouched */
  double *M = malloc(sizeof(double) * (size_t)L * Kcap); /* reduced in place to R */
  double *y = malloc(sizeof(double) * (size_t)L);
  double *v = malloc(sizeof(double) * (size_t)L);
  double *d = malloc(sizeof(double) * (size_t)Kcap);
  for (int k = 0; k < Kcap; ++k)
    for (int l = 0; l < L; ++l) A[(size_t)k * L + l] = cos((double)k * omega * t[l]);
  memcpy(M, A, sizeof(double) * (size_t)L * Kcap);
  memcpy(y, b, sizeof(double) * (size_t)L);

  int status = 1, K = Kcap;
  double E = INFINITY, linf = INFINITY;
  for (int j = 0; j < Kcap; ++j) {
    double *cj = M + (size_t)j * L;
    double nrm = 0.0;
    for (int l = j; l < L; ++l) nrm += cj[l] * cj[l];
    nrm = sqrt(nrm);
    double alpha = cj[j] > 0.0 ? -nrm : nrm;
    double vv = 0.0;
    for (int l = j; l < L; ++l) v[l] = cj[l];
    v[j] -= alpha;
    for (int l = j; l < L; ++l) vv += v[l] * v[l];
    if (vv > 0.0) {
      for (int c = j + 1; c < Kcap; ++c) {
        double *cc = M + (size_t)c * L, s = 0.0;
        for (int l = j; l < L; ++l) s += v[l] * cc[l];
        s = 2.0 * s / vv;
        for (int l = j; l < L; ++l) cc[l] -= s * v[l];
      }
      double s = 0.0;
      for (int l = j; l < L; ++l) s += v[l] * y[l];
      s = 2.0 * s / vv;
      for (int l = j; l < L; ++l) y[l] -= s * v[l];
    }
    cj[j] = alpha;
    for (int l = j + 1; l < L; ++l) cj[l] = 0.0;

    /* Solve R d = (Q^T b) for the first j+1 unknowns (back-substitution). */
    int n = j + 1;
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int c = i + 1; c < n; ++c) s -= M[(size_t)c * L + i] * d[c];
      d[i] = s / M[(size_t)i * L + i];
    }
    /* Residual evaluated directly: E = ||b - A d||, plus its max norm. */
    double e2 = 0.0, emax = 0.0;
    for (int l = 0; l < L; ++l) {
      double r = b[l];
      for (int c = 0; c < n; ++c) r -= A[(size_t)c * L + l] * d[c];
      e2 += r * r;
      if (fabs(r) > emax) emax = fabs(r);
    }
    E = sqrt(e2);
    linf = emax;
    if (K_fixed == 0 && E <= eps) {
      status = 0;
      K = n;
      break;
    }
    if (K_fixed > 0 && n == K_fixed) {
      status = 0;
      K = n;
      break;
    }
  }
  for (int k = 0; k < K; ++k) d_out[k] = d[k];
  *K_out = K;
  *E_out = E;
  *linf_out = linf;
  free(A);
  free(M);
  free(y);
  free(v);
  free(d);
  return status;
}

/* The fit on the sampling grid of Sec. III: Lambda_T = {0, 1, ..., T} when
 * levels == 0 (T a positive integer), else `levels` equispaced points on [0, T]
 * (a reading for non-integer T, e.g. T = 1 with 256 quantisation levels).
 * b = [phi(t)]_t (the first sampling step of Algorithm 2).  Kmax caps K. */
int orc_fit(int kernel, double sigma_r, double T, double eps, int K_fixed, int levels,
            int Kmax, double *d_out, int *K_out, double *E_out, double *linf_out) {
  if (!(T > 0.0) || !(sigma_r > 0.0)) return -1;
  int L;
  if (levels == 0) {
    if (T != floor(T) || T > 1e6) return -1;
    L = (int)T + 1;
  } else {
    if (levels < 2) return -1;
    L = levels;
  }
  double *t = malloc(sizeof(double) * (size_t)L), *b = malloc(sizeof(double) * (size_t)L);
  for (int l = 0; l < L; ++l) {
    t[l] = levels == 0 ? (double)l : (double)l * T / (double)(levels - 1);
    b[l] = orc_phi(kernel, sigma_r, t[l]);
  }
  int kmax = Kmax < L ? Kmax : L;
  int st = orc_fit_samples(t, b, L, T, eps, K_fixed, kmax, d_out, K_out, E_out, linf_out);
  free(t);
  free(b);
  return st;
}

/* 1-D spatial weights on [-W, W] (w1[j + W] = weight of offset j), normalised
 * to sum 1 so that the 2-D weights w(j) = w1(j_y) w1(j_x) sum to 1 (Sec. IV).
 * Gaussian: eq. (2), separable as exp(-j_y^2/2s^2) exp(-j_x^2/2s^2).  Box:
 * uniform.  Returns the tap count 2W + 1, or -1. */
int orc_weights_1d(int spatial, double sigma_s, int W, double *w1) {
  if (W < 0) return -1;
  double s = 0.0;
  for (int j = -W; j <= W; ++j) {
    double v = spatial == ORC_SPATIAL_BOX ? 1.0
                                          : exp(-(double)(j * j) / (2.0 * sigma_s * sigma_s));
    w1[j + W] = v;
    s += v;
  }
  for (int j = 0; j < 2 * W + 1; ++j) w1[j] /= s;
  return 2 * W + 1;
}

/* Half-sample symmetric reflection into [0, n): ... 1 0 | 0 1 ... n-1 | n-1 ... */
static long orc_reflect(long i, long n) {
  long p = 2 * n;
  long m = i % p;
  if (m < 0) m += p;
  return m < n ? m : p - 1 - m;
}

/* Direct evaluation of eq. (1) (use_phi_n == 0, exact range kernel) or of eq.
 * (9) (use_phi_n != 0, phi replaced by phi_N of eq. (6)) at every pixel, or at
 * the npts pixels (ys[p], xs[p]) when ys != NULL.  The sum runs over j in
 * Omega = [-W, W]^2 with neighbour f(i - j); out = P / Q with P, Q the
 * numerator and denominator (the P_1, Q_1 / P_2, Q_2 of the Appendix). */
void orc_direct(const double *f, int H, int Wd, const double *w1, int W, int border,
                int use_phi_n, int kernel, double sigma_r, const double *d, int K, double T,
                const int *ys, const int *xs, long npts, double *out, double *P, double *Q) {
  long n = ys ? npts : (long)H * Wd;
#pragma omp parallel for schedule(dynamic, 16)
  for (long p = 0; p < n; ++p) {
    long iy = ys ? ys[p] : p / Wd, ix = ys ? xs[p] : p % Wd;
    double fc = f[iy * Wd + ix], num = 0.0, den = 0.0;
    for (int jy = -W; jy <= W; ++jy) {
      long sy = iy - jy;
      if (border == ORC_BORDER_REFLECT) sy = orc_reflect(sy, H);
      else if (sy < 0 || sy >= H) continue;
      for (int jx = -W; jx <= W; ++jx) {
        long sx = ix - jx;
        if (border == ORC_BORDER_REFLECT) sx = orc_reflect(sx, Wd);
        else if (sx < 0 || sx >= Wd) continue;
        double fn = f[sy * Wd + sx];
        double t = fn - fc;
        double ph = use_phi_n ? orc_phi_n(d, K, T, t) : orc_phi(kernel, sigma_r, t);
        double wj = w1[jy + W] * w1[jx + W];
        num += wj * ph * fn;
        den += wj * ph;
      }
    }
    out[p] = num / den;
    if (P) P[p] = num;
    if (Q) Q[p] = den;
  }
}

/* Separable 2-D convolution Y = X * w on output rows [r0, r1): Y(i) =
 * sum_j w1(j_y) w1(j_x) X(i - j), X extended by the border rule.  X holds the
 * image rows [xr0, xr1) (enough for the outputs requested). */
static void orc_conv2(const double complex *X, int xr0, int xr1, int H, int Wd,
                      const double *w1, int W, int border, int r0, int r1, double complex *Y,
                      double complex *tmp) {
  int he = r1 - r0 + 2 * W;
  (void)xr1;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < he; ++k) {
    long e = (long)r0 - W + k; /* extended row index */
    double complex *trow = tmp + (size_t)k * Wd;
    if (border == ORC_BORDER_TRUNCATE && (e < 0 || e >= H)) {
      for (int x = 0; x < Wd; ++x) trow[x] = 0.0;
      continue;
    }
    long s = border == ORC_BORDER_REFLECT ? orc_reflect(e, H) : e;
    const double complex *xrow = X + (size_t)(s - xr0) * Wd;
    for (int x = 0; x < Wd; ++x) {
      double complex acc = 0.0;
      for (int j = -W; j <= W; ++j) {
        long sx = (long)x - j;
        if (border == ORC_BORDER_REFLECT) sx = orc_reflect(sx, Wd);
        else if (sx < 0 || sx >= Wd) continue;
        acc += w1[j + W] * xrow[sx];
      }
      trow[x] = acc;
    }
  }
#pragma omp parallel for schedule(static)
  for (int y = r0; y < r1; ++y) {
    for (int x = 0; x < Wd; ++x) {
      double complex acc = 0.0;
      for (int j = -W; j <= W; ++j) acc += w1[j + W] * tmp[(size_t)(y - j - r0 + W) * Wd + x];
      Y[(size_t)(y - r0) * Wd + x] = acc;
    }
  }
}

/* Algorithm 1 (Shiftable Bilateral Filtering) in the paper's complex notation,
 * for output rows [r0, r1).  With N = K - 1 and c_0 = d_0, c_{+-n} = d_n / 2
 * (Sec. III, below eq. (6)):
 *   for n = -N..N:  G = exp(i n omega f),  F = G f,  H = c_n conj(G),
 *                   Fbar = F * w,  Gbar = G * w   (eq. (5) and its analogue),
 *                   P += H Fbar,  Q += H Gbar;
 *   out = P / Q.
 * (The paper's line computing the convolutions prints "Gbar" twice; the first is
 * Fbar = F * w, which the next line uses.)  P and Q are real up to rounding;
 * their imaginary parts are returned for checking.  Arrays are (r1-r0) x Wd. */
int orc_alg1(const double *f, int H, int Wd, const double *w1, int W, int border,
             const double *d, int K, double T, int r0, int r1, double *out, double *P,
             double *Q, double *Pim, double *Qim) {
  if (r0 < 0 || r1 > H || r0 >= r1 || K < 1 || !(T > 0.0)) return -1;
  /* Source rows [xr0, xr1) that the window of rows [r0, r1) reaches. */
  int xr0 = H, xr1 = 0;
  for (long e = (long)r0 - W; e < (long)r1 + W; ++e) {
    long s = e;
    if (border == ORC_BORDER_REFLECT) s = orc_reflect(e, H);
    else if (e < 0 || e >= H) continue;
    if (s < xr0) xr0 = (int)s;
    if (s + 1 > xr1) xr1 = (int)s + 1;
  }
  size_t nx = (size_t)(xr1 - xr0) * Wd, ny = (size_t)(r1 - r0) * Wd;
  size_t nt = (size_t)(r1 - r0 + 2 * W) * Wd;
  double complex *G = malloc(sizeof(double complex) * nx);
  double complex *F = malloc(sizeof(double complex) * nx);
  double complex *Fb = malloc(sizeof(double complex) * ny);
  double complex *Gb = malloc(sizeof(double complex) * ny);
  double complex *Pc = calloc(ny, sizeof(double complex));
  double complex *Qc = calloc(ny, sizeof(double complex));
  double complex *tmp = malloc(sizeof(double complex) * nt);
  double omega = M_PI / T;
  int N = K - 1;
  for (int n = -N; n <= N; ++n) {
    int an = n < 0 ? -n : n;
    double cn = n == 0 ? d[0] : 0.5 * d[an];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)nx; ++p) {
      double fv = f[(size_t)xr0 * Wd + p];
      G[p] = cexp(I * ((double)n * omega * fv));
      F[p] = G[p] * fv;
    }
    orc_conv2(F, xr0, xr1, H, Wd, w1, W, border, r0, r1, Fb, tmp);
    orc_conv2(G, xr0, xr1, H, Wd, w1, W, border, r0, r1, Gb, tmp);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)ny; ++p) {
      double fv = f[(size_t)r0 * Wd + p];
      double complex Hc = cn * conj(cexp(I * ((double)n * omega * fv)));
      Pc[p] += Hc * Fb[p];
      Qc[p] += Hc * Gb[p];
    }
  }
  for (size_t p = 0; p < ny; ++p) {
    out[p] = creal(Pc[p]) / creal(Qc[p]);
    if (P) P[p] = creal(Pc[p]);
    if (Q) Q[p] = creal(Qc[p]);
    if (Pim) Pim[p] = cimag(Pc[p]);
    if (Qim) Qim[p] = cimag(Qc[p]);
  }
  free(G);
  free(F);
  free(Fb);
  free(Gb);
  free(Pc);
  free(Qc);
  free(tmp);
  return 0;
}

/* Derivative of phi_N: phi_N'(t) = -sum_k k omega d_k sin(k omega t). */
static double orc_dphi_n(const double *d, int K, double T, double t) {
  double omega = M_PI / T, s = 0.0;
  for (int k = 1; k < K; ++k) s -= (double)k * omega * d[k] * sin((double)k * omega * t);
  return s;
}

/* Gradient of L = sum_i g(i) fhat(i), fhat = P_2 / Q_2 of eq. (9), with respect
 * to every input pixel f(m), by direct differentiation of the window sums:
 *   dL/df(m) = sum_i g(i)/Q(i) [dP(i)/df(m) - fhat(i) dQ(i)/df(m)].
 * f(m) enters P(i), Q(i) as a neighbour (every (i, j) whose mapped source
 * index i - j is m) and as the centre (i = m).  For one pair (i, j) with
 * neighbour value u = f(i-j), centre c = f(i), t = u - c:
 *   P term  w phi_N(t) u :  d/du = w (phi_N(t) + u phi_N'(t)),  d/dc = -w u phi_N'(t)
 *   Q term  w phi_N(t)   :  d/du = w phi_N'(t),                  d/dc = -w phi_N'(t)
 * Under REFLECT a mirrored neighbour index that maps onto m contributes to m;
 * under TRUNCATE neighbours outside the image are absent.  T, omega and d are
 * constants.  Evaluated by looping over every output pixel and scattering,
 * serial over rows of i to keep the scatter race-free. */
void orc_grad_direct(const double *f, const double *g, int H, int Wd, const double *w1, int W,
                     int border, const double *d, int K, double T, double *grad) {
  size_t np = (size_t)H * Wd;
  double *a = malloc(sizeof(double) * np), *bb = malloc(sizeof(double) * np);
  double *P = malloc(sizeof(double) * np), *Q = malloc(sizeof(double) * np);
  double *out = malloc(sizeof(double) * np);
  orc_direct(f, H, Wd, w1, W, border, 1, 0, 1.0, d, K, T, NULL, NULL, 0, out, P, Q);
  for (size_t p = 0; p < np; ++p) {
    a[p] = g[p] / Q[p];        /* weight of dP */
    bb[p] = g[p] * out[p] / Q[p]; /* weight of dQ */
    grad[p] = 0.0;
  }
  for (long iy = 0; iy < H; ++iy) {
    for (long ix = 0; ix < Wd; ++ix) {
      size_t i = (size_t)iy * Wd + ix;
      double c = f[i];
      double centre = 0.0;
      for (int jy = -W; jy <= W; ++jy) {
        long sy = iy - jy;
        if (border == ORC_BORDER_REFLECT) sy = orc_reflect(sy, H);
        else if (sy < 0 || sy >= H) continue;
        for (int jx = -W; jx <= W; ++jx) {
          long sx = ix - jx;
          if (border == ORC_BORDER_REFLECT) sx = orc_reflect(sx, Wd);
          else if (sx < 0 || sx >= Wd) continue;
          size_t m = (size_t)sy * Wd + sx;
          double u = f[m], t = u - c;
          double wj = w1[jy + W] * w1[jx + W];
          double ph = orc_phi_n(d, K, T, t), dph = orc_dphi_n(d, K, T, t);
          grad[m] += wj * (a[i] * (ph + u * dph) - bb[i] * dph);
          centre += wj * (-a[i] * u * dph + bb[i] * dph);
        }
      }
      grad[i] += centre;
    }
  }
  free(a);
  free(bb);
  free(P);
  free(Q);
  free(out);
}

/* The same derivative as orc_grad_direct, evaluated only at the npts pixels
 * (ys[p], xs[p]), for images too large for the full computation.  For a
 * sampled m it enumerates the pairs (i, j) whose (mapped) neighbour index
 * i - j is m: under REFLECT every extended position q in [-W, H+W) x [-W, Wd+W)
 * that reflects onto m and every i in the image with i - q in [-W, W]^2; under
 * TRUNCATE q = m only.  a(i) = g(i)/Q(i), b(i) = g(i) fhat(i)/Q(i) come from
 * eq. (9) evaluated directly at each i.  Adds the centre term of i = m. */
static void orc_pq_at(const double *f, int H, int Wd, const double *w1, int W, int border, const double *d,
                      int K, double T, long iy, long ix, double *P, double *Q) {
  double fc = f[iy * Wd + ix], num = 0.0, den = 0.0;
  for (int jy = -W; jy <= W; ++jy) {
    long sy = iy - jy;
    if (border == ORC_BORDER_REFLECT) sy = orc_reflect(sy, H);
    else if (sy < 0 || sy >= H) continue;
    for (int jx = -W; jx <= W; ++jx) {
      long sx = ix - jx;
      if (border == ORC_BORDER_REFLECT) sx = orc_reflect(sx, Wd);
      else if (sx < 0 || sx >= Wd) continue;
      double u = f[sy * Wd + sx], ph = orc_phi_n(d, K, T, u - fc), wj = w1[jy + W] * w1[jx + W];
      num += wj * ph * u;
      den += wj * ph;
    }
  }
  *P = num;
  *Q = den;
}

int orc_grad_at(const double *f, const double *g, int H, int Wd, const double *w1, int W, int border,
                const double *d, int K, double T, const int *ys, const int *xs, long npts, double *out) {
  /* Each 1-D preimage list holds at most every extended position of its axis
   * (H + 2W rows, Wd + 2W columns); the lists are sized for that, so no
   * preimage is ever dropped.  Returns 0, or -1 when the lists cannot be
   * allocated (then `out` is not filled). */
  const long cap_y = (long)H + 2L * W, cap_x = (long)Wd + 2L * W;
  int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
  for (long p = 0; p < npts; ++p) {
    long my = ys[p], mx = xs[p];
    double fm = f[my * Wd + mx], acc = 0.0;
    /* 1-D preimages of my / mx among the extended positions */
    long *qy = malloc(sizeof(long) * (size_t)cap_y), *qx = malloc(sizeof(long) * (size_t)cap_x);
    if (!qy || !qx) {
      free(qy);
      free(qx);
      failed = 1;
      continue;
    }
    int ny = 0, nx = 0;
    if (border == ORC_BORDER_REFLECT) {
      for (long q = -W; q < H + W; ++q)
        if (orc_reflect(q, H) == my) qy[ny++] = q;
      for (long q = -W; q < Wd + W; ++q)
        if (orc_reflect(q, Wd) == mx) qx[nx++] = q;
    } else {
      qy[ny++] = my;
      qx[nx++] = mx;
    }
    for (int a1 = 0; a1 < ny; ++a1)
      for (int a2 = 0; a2 < nx; ++a2)
        for (int jy = -W; jy <= W; ++jy)
          for (int jx = -W; jx <= W; ++jx) {
            long iy = qy[a1] + jy, ix = qx[a2] + jx; /* i - j = q */
            if (iy < 0 || iy >= H || ix < 0 || ix >= Wd) continue;
            double Pi, Qi;
            orc_pq_at(f, H, Wd, w1, W, border, d, K, T, iy, ix, &Pi, &Qi);
            double gi = g[iy * Wd + ix], ai = gi / Qi, bi = gi * (Pi / Qi) / Qi;
            double t = fm - f[iy * Wd + ix], wj = w1[jy + W] * w1[jx + W];
            double ph = orc_phi_n(d, K, T, t), dph = orc_dphi_n(d, K, T, t);
            acc += wj * (ai * (ph + fm * dph) - bi * dph);
          }
    /* centre term, i = m */
    double Pm, Qm;
    orc_pq_at(f, H, Wd, w1, W, border, d, K, T, my, mx, &Pm, &Qm);
    double gm = g[my * Wd + mx], am = gm / Qm, bm = gm * (Pm / Qm) / Qm;
    for (int jy = -W; jy <= W; ++jy) {
      long sy = my - jy;
      if (border == ORC_BORDER_REFLECT) sy = orc_reflect(sy, H);
      else if (sy < 0 || sy >= H) continue;
      for (int jx = -W; jx <= W; ++jx) {
        long sx = mx - jx;
        if (border == ORC_BORDER_REFLECT) sx = orc_reflect(sx, Wd);
        else if (sx < 0 || sx >= Wd) continue;
        double u = f[sy * Wd + sx], t = u - fm, wj = w1[jy + W] * w1[jx + W];
        double dph = orc_dphi_n(d, K, T, t);
        acc += wj * (-am * u * dph + bm * dph);
      }
    }
    out[p] = acc;
    free(qy);
    free(qx);
  }
  return failed ? -1 : 0;
}

/*
 * Dynamic range of f over the window (the definition of T at the start of
 * Sec. III): the largest |f(i - j) - f(i)| over every pixel i and every offset
 * j in Omega = [-W, W]^2, read with f(i) as the centre (the paper's f(j) there
 * is taken as a misprint).  Neighbours outside the image are skipped
 * (TRUNCATE) or mirrored (REFLECT).  Written out directly: O(W^2) per pixel.
 */
double orc_local_range(const double *f, int H, int Wd, int W, int border) {
  double T = 0.0;
#pragma omp parallel for reduction(max : T) schedule(static)
  for (long y = 0; y < H; ++y) {
    for (long x = 0; x < Wd; ++x) {
      const double c = f[y * Wd + x];
      for (long dy = -W; dy <= W; ++dy) {
        long sy = y - dy;
        if (border == ORC_BORDER_REFLECT) {
          sy = orc_reflect(sy, H);
        } else if (sy < 0 || sy >= H) {
          continue;
        }
        for (long dx = -W; dx <= W; ++dx) {
          long sx = x - dx;
          if (border == ORC_BORDER_REFLECT) {
            sx = orc_reflect(sx, Wd);
          } else if (sx < 0 || sx >= Wd) {
            continue;
          }
          const double t = fabs(f[sy * Wd + sx] - c);
          if (t > T) T = t;
        }
      }
    }
  }
  return T;
}

/*
 * Recursive Gaussian (the constant-time Gaussian filtering that Sec. II cites,
 * after eq. (5): R. Deriche, "Recursively implementing the Gaussian and its
 * derivatives", 1993).  Deriche approximates exp(-x^2 / (2 s^2)), x >= 0, by
 * two damped sinusoids,
 *   g(x) = (a1 cos(w1 x/s) + b1 sin(w1 x/s)) exp(-l1 x/s)
 *        + (a2 cos(w2 x/s) + b2 sin(w2 x/s)) exp(-l2 x/s),
 * with his published constants (a1, b1, w1, l1) = (1.680, 3.735, 0.6318, 1.783)
 * and (a2, b2, w2, l2) = (-0.6803, -0.2598, 1.997, 1.723), and g(-x) = g(x).
 * The samples g(k), k >= 0, are the impulse response of a causal recursion
 * whose transfer function is the sum of the z-transforms of the two terms
 * (each a first-degree numerator over a second-degree denominator); the
 * samples g(k), k <= -1, that of the mirrored anticausal recursion.  The sum of
 * the two is scaled to unit gain.
 *
 * Readings taken here (the paper prints no formula for the recursive filter):
 *   * Deriche's fourth-order approximation with the constants above;
 *   * the 1-D kernel is scaled so that sum_k g(k) = 1 (the FIR kernel's Sec. IV
 *     normalisation; the scale cancels in P / Q anyway);
 *   * borders: TRUNCATE is zero outside the image (the infinite-support kernel
 *     restricted to the image); REFLECT extends each line by E = ceil(8 s)
 *     half-sample-symmetric samples on each side (repeated for E longer than
 *     the line) and is zero beyond them;
 *   * the 2-D filter is the rows' recursion followed by the columns'.
 */
static const double orc_der_a[2] = {1.680, -0.6803}, orc_der_b[2] = {3.735, -0.2598};
static const double orc_der_w[2] = {0.6318, 1.997}, orc_der_l[2] = {1.783, 1.723};

/* g(k) of the approximation above, unscaled. */
double orc_rec_kernel(double s, long k) {
  double x = fabs((double)k) / s, g = 0.0;
  for (int i = 0; i < 2; ++i)
    g += (orc_der_a[i] * cos(orc_der_w[i] * x) + orc_der_b[i] * sin(orc_der_w[i] * x)) * exp(-orc_der_l[i] * x);
  return g;
}

/* Recursion coefficients for scale s: causal numerator nc[0..3], common
 * denominator 1 + dd[1] z^-1 + ... + dd[4] z^-4, anticausal numerator
 * na[1..4] (na[0] = 0), all scaled to unit total gain.  Term i contributes
 *   sum_{k>=0} (a cos(wk) + b sin(wk)) e^{-lk} z^-k
 *     = (a + e^{-l}(b sin w - a cos w) z^-1) / (1 - 2 e^{-l} cos w z^-1 + e^{-2l} z^-2)
 * (w, l already divided by s). */
void orc_rec_coeffs(double s, double nc[4], double dd[5], double na[5]) {
  double num[2][2], den[2][3];
  for (int i = 0; i < 2; ++i) {
    const double w = orc_der_w[i] / s, l = orc_der_l[i] / s, e = exp(-l);
    num[i][0] = orc_der_a[i];
    num[i][1] = e * (orc_der_b[i] * sin(w) - orc_der_a[i] * cos(w));
    den[i][0] = 1.0;
    den[i][1] = -2.0 * e * cos(w);
    den[i][2] = e * e;
  }
  for (int k = 0; k < 5; ++k) dd[k] = 0.0;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) dd[p + q] += den[0][p] * den[1][q];
  for (int k = 0; k < 4; ++k) nc[k] = 0.0;
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 3; ++q) nc[p + q] += num[0][p] * den[1][q] + num[1][p] * den[0][q];
  /* anticausal: sum_{k>=1} g(k) z^k = N(1/z)/D(1/z) - g(0) */
  na[0] = 0.0;
  for (int k = 1; k < 4; ++k) na[k] = nc[k] - nc[0] * dd[k];
  na[4] = -nc[0] * dd[4];
  /* unit gain: (N(1) + Na(1)) / D(1) */
  double sn = 0.0, sa = 0.0, sd = 0.0;
  for (int k = 0; k < 4; ++k) sn += nc[k];
  for (int k = 1; k < 5; ++k) sa += na[k];
  for (int k = 0; k < 5; ++k) sd += dd[k];
  const double gain = (sn + sa) / sd;
  for (int k = 0; k < 4; ++k) nc[k] /= gain;
  for (int k = 1; k < 5; ++k) na[k] /= gain;
}

/* One line x[0..L) through both recursions (zero before 0 and after L - 1):
 * y = causal + anticausal.  Complex samples, real coefficients. */
static void orc_rec_line(const double complex *x, long L, const double nc[4], const double dd[5],
                         const double na[5], double complex *y, double complex *tmp) {
  for (long i = 0; i < L; ++i) {
    double complex acc = 0.0;
    for (int k = 0; k < 4; ++k)
      if (i - k >= 0) acc += nc[k] * x[i - k];
    for (int k = 1; k < 5; ++k)
      if (i - k >= 0) acc -= dd[k] * tmp[i - k];
    tmp[i] = acc;
  }
  for (long i = L - 1; i >= 0; --i) {
    double complex acc = 0.0;
    for (int k = 1; k < 5; ++k)
      if (i + k < L) acc += na[k] * x[i + k] - dd[k] * y[i + k];
    y[i] = acc;
  }
  for (long i = 0; i < L; ++i) y[i] += tmp[i];
}

/* 1-D recursive filter of a real line (exported for the tests' impulse
 * responses): x[0..L) -> y[0..L), zero outside. */
void orc_rec_filter_line(const double *x, long L, double s, double *y) {
  double nc[4], dd[5], na[5];
  orc_rec_coeffs(s, nc, dd, na);
  double complex *xc = malloc(sizeof(double complex) * L), *yc = malloc(sizeof(double complex) * L),
                 *tc = malloc(sizeof(double complex) * L);
  for (long i = 0; i < L; ++i) xc[i] = x[i];
  orc_rec_line(xc, L, nc, dd, na, yc, tc);
  for (long i = 0; i < L; ++i) y[i] = creal(yc[i]);
  free(xc);
  free(yc);
  free(tc);
}

/* Separable recursive filter of an H x Wd complex image in place: each row,
 * then each column, extended per the border reading above. */
static void orc_rec2(double complex *X, int H, int Wd, double s, int border) {
  double nc[4], dd[5], na[5];
  orc_rec_coeffs(s, nc, dd, na);
  const long E = border == ORC_BORDER_REFLECT ? (long)ceil(8.0 * s) : 0;
  for (int pass = 0; pass < 2; ++pass) {
    const long n = pass == 0 ? Wd : H, lines = pass == 0 ? H : Wd, L = n + 2 * E;
#pragma omp parallel
    {
      double complex *xe = malloc(sizeof(double complex) * L), *ye = malloc(sizeof(double complex) * L),
                     *te = malloc(sizeof(double complex) * L);
#pragma omp for schedule(static)
      for (long ln = 0; ln < lines; ++ln) {
        for (long i = 0; i < L; ++i) {
          const long j = border == ORC_BORDER_REFLECT ? orc_reflect(i - E, n) : i;
          xe[i] = pass == 0 ? X[ln * Wd + j] : X[j * Wd + ln];
        }
        orc_rec_line(xe, L, nc, dd, na, ye, te);
        for (long i = 0; i < n; ++i) {
          if (pass == 0)
            X[ln * Wd + i] = ye[i + E];
          else
            X[i * Wd + ln] = ye[i + E];
        }
      }
      free(xe);
      free(ye);
      free(te);
    }
  }
}

/* Algorithm 1 with the recursive Gaussian in place of the FIR convolution
 * (the constant-time variant of Sec. II): the same modulation, demodulation
 * and c_{+-n} = d_n / 2 as orc_alg1, each channel filtered by orc_rec2.  Whole
 * image; out, P, Q are H x Wd. */
int orc_alg1_rec(const double *f, int H, int Wd, double sigma_s, int border, const double *d, int K,
                 double T, double *out, double *P, double *Q) {
  if (H < 1 || Wd < 1 || K < 1 || !(T > 0.0) || !(sigma_s > 0.0)) return -1;
  const size_t np = (size_t)H * Wd;
  double complex *G = malloc(sizeof(double complex) * np), *F = malloc(sizeof(double complex) * np);
  double complex *Pc = calloc(np, sizeof(double complex)), *Qc = calloc(np, sizeof(double complex));
  const double omega = M_PI / T;
  const int N = K - 1;
  for (int n = -N; n <= N; ++n) {
    const int an = n < 0 ? -n : n;
    const double cn = n == 0 ? d[0] : 0.5 * d[an];
    for (size_t p = 0; p < np; ++p) {
      G[p] = cexp(I * ((double)n * omega * f[p]));
      F[p] = G[p] * f[p];
    }
    orc_rec2(F, H, Wd, sigma_s, border);
    orc_rec2(G, H, Wd, sigma_s, border);
    for (size_t p = 0; p < np; ++p) {
      const double complex Hc = cn * conj(cexp(I * ((double)n * omega * f[p])));
      Pc[p] += Hc * F[p];
      Qc[p] += Hc * G[p];
    }
  }
  for (size_t p = 0; p < np; ++p) {
    out[p] = creal(Pc[p]) / creal(Qc[p]);
    if (P) P[p] = creal(Pc[p]);
    if (Q) Q[p] = creal(Qc[p]);
  }
  free(G);
  free(F);
  free(Pc);
  free(Qc);
  return 0;
}
