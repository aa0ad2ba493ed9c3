/*
 * mdi_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU implementation in FP64 of what the MDI-LR
 * hot path computes (Zhong & Feng, "An efficient implementation algorithm for
 * quasi-Monte Carlo approximations of high-dimensional integrals").  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * this file's library.  The product path (the CUDA library) shares no code,
 * header, table or constant with it, and neither includes the other.
 *
 * Every function names the passage of the paper it follows.  No blocking, no
 * fusion, no reordering beyond what the definition states: sums run in index
 * order, in double precision, with unsigned __int128 for lattice indices.
 *
 * Integrand families (oracle-local numbering).  Product-form ones carry per-axis
 * parameters c[0..d) and w[0..d):
 *   OR_EXP   f(x) = exp(sum_j c_j x_j)                phi_j(x) = exp(c_j x)
 *   OR_OSC   f(x) = cos(2 pi u + sum_j c_j x_j)       phi_j(x) = exp(i c_j x), u = w[0],
 *            f = Re(exp(2 pi i u) prod_j phi_j)
 *   OR_GAUSS f(x) = exp(-sum_j c_j^2 (x_j - w_j)^2)   phi_j(x) = exp(-c_j^2 (x - w_j)^2)
 *   OR_PEAK  f(x) = prod_j (c_j^-2 + (x_j - w_j)^2)^-1
 * Non-product integrands of the paper's tests (brute-force rules only):
 *   OR_T1    f(x) = x_2 exp(x_1 x_2) / (e - 2)        (Test 1, d = 2)
 *   OR_SINSQ f(x) = sin(2 pi + sum_j x_j^2)           (Tests 1-2)
 *   OR_ALTSQ f(x) = exp(sum_j (-1)^(j+1) x_j^2)       (Test 7, f_5)
 *   OR_RIDGE f(x) = (1 + sum_j x_j)^-(d+1)            (Test 7, f_6)
 *
 * Parity status.  Every function is pinned by tests/test_oracle_pins.py against
 * values the paper prints, closed forms, identities the paper states, or brute
 * force; see the pin list in that file.  The node-state sweep or_mdi_nodes is an
 * approximation the paper does not spell out (it leaves the representation of
 * its "symbolic functions" open); it is pinned against the exact sweep on cases
 * small enough to enumerate and against closed forms, and beyond those sizes only
 * through invariants.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum {
  OR_EXP = 0, OR_OSC = 1, OR_GAUSS = 2, OR_PEAK = 3,
  OR_T1 = 10, OR_SINSQ = 11, OR_ALTSQ = 12, OR_RIDGE = 13
};

typedef unsigned __int128 u128;
typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Integer lattice arithmetic                                                 */
/* ------------------------------------------------------------------------- */

static uint64_t mulmod(uint64_t x, uint64_t y, uint64_t n) {
  return (uint64_t)(((u128)x * (u128)y) % (u128)n);
}

/* Korobov generating vector z(a) = (1, a, a^2, ..., a^(d-1)) mod n
 * (Section 2.2, Example 2 "Korobov lattice"). */
int or_korobov_z(int d, uint64_t a, uint64_t n, uint64_t *z) {
  if (d < 1 || n < 1) return -1;
  uint64_t v = 1 % n;
  for (int i = 0; i < d; ++i) {
    z[i] = v;
    v = mulmod(v, a % n, n);
  }
  return 0;
}

/* Lattice indices r_{j,i} = j z_i mod n for j = j0 .. j0+count-1, row-major
 * (count, d): the integer numerators of x_j = {j z / n}, eq. (2.1). */
int or_lattice_indices(int d, uint64_t n, const uint64_t *z, uint64_t j0, uint64_t count,
                       uint64_t *r_out) {
  if (d < 1 || n < 1) return -1;
  for (uint64_t t = 0; t < count; ++t)
    for (int i = 0; i < d; ++i) r_out[t * (uint64_t)d + i] = mulmod((j0 + t) % n, z[i] % n, n);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Integrands, evaluated directly from their definitions                      */
/* ------------------------------------------------------------------------- */

static double f_eval(int fam, int d, const double *x, const double *c, const double *w) {
  double s = 0.0, p = 1.0;
  switch (fam) {
    case OR_EXP:
      for (int j = 0; j < d; ++j) s += c[j] * x[j];
      return exp(s);
    case OR_OSC:
      for (int j = 0; j < d; ++j) s += c[j] * x[j];
      return cos(2.0 * M_PI * w[0] + s);
    case OR_GAUSS:
      for (int j = 0; j < d; ++j) s += c[j] * c[j] * (x[j] - w[j]) * (x[j] - w[j]);
      return exp(-s);
    case OR_PEAK:
      for (int j = 0; j < d; ++j) p *= 1.0 / (1.0 / (c[j] * c[j]) + (x[j] - w[j]) * (x[j] - w[j]));
      return p;
    case OR_T1:
      return x[1] * exp(x[0] * x[1]) / (M_E - 2.0);
    case OR_SINSQ:
      for (int j = 0; j < d; ++j) s += x[j] * x[j];
      return sin(2.0 * M_PI + s);
    case OR_ALTSQ:
      for (int j = 0; j < d; ++j) s += ((j % 2 == 0) ? 1.0 : -1.0) * x[j] * x[j];
      return exp(s);
    case OR_RIDGE:
      for (int j = 0; j < d; ++j) s += x[j];
      return pow(1.0 + s, -(double)(d + 1));
  }
  return NAN;
}

/* One-dimensional factor phi_j of a product-form integrand (complex for OR_OSC). */
static cplx phi(int fam, int j, double x, const double *c, const double *w) {
  switch (fam) {
    case OR_EXP: return exp(c[j] * x);
    case OR_OSC: return cexp(I * c[j] * x);
    case OR_GAUSS: return exp(-c[j] * c[j] * (x - w[j]) * (x - w[j]));
    case OR_PEAK: return 1.0 / (1.0 / (c[j] * c[j]) + (x - w[j]) * (x - w[j]));
  }
  return NAN;
}

/* Derivatives of phi_j with respect to c_j (which = 0) and w_j (which = 1). */
static cplx dphi(int fam, int j, int which, double x, const double *c, const double *w) {
  double cj = c[j], dx = x - w[j];
  switch (fam) {
    case OR_EXP: return which == 0 ? x * exp(cj * x) : 0.0;
    case OR_OSC: return which == 0 ? I * x * cexp(I * cj * x) : 0.0;
    case OR_GAUSS: {
      double e = exp(-cj * cj * dx * dx);
      return which == 0 ? -2.0 * cj * dx * dx * e : 2.0 * cj * cj * dx * e;
    }
    case OR_PEAK: {
      double D = 1.0 / (cj * cj) + dx * dx;
      return which == 0 ? (2.0 / (cj * cj * cj)) / (D * D) : (2.0 * dx) / (D * D);
    }
  }
  return NAN;
}

static int is_product(int fam) { return fam >= OR_EXP && fam <= OR_PEAK; }

/* Constant factor in front of the product: exp(2 pi i u) for OR_OSC, else 1. */
static cplx front(int fam, const double *w) {
  return fam == OR_OSC ? cexp(I * 2.0 * M_PI * w[0]) : 1.0;
}

/* ------------------------------------------------------------------------- */
/* Standard lattice rule, eq. (1.2) with the points of eq. (2.1)              */
/* ------------------------------------------------------------------------- */

/* Q = (1/n) sum_{j<n} f({j z / n}); coordinates are (j z_i mod n) / n computed in
 * exact 128-bit integer arithmetic and one FP64 division each. */
double or_slr(int fam, int d, uint64_t n, const uint64_t *z, const double *c, const double *w) {
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  double sum = 0.0;
  for (uint64_t j = 0; j < n; ++j) {
    for (int i = 0; i < d; ++i) x[i] = (double)mulmod(j, z[i] % n, n) / (double)n;
    sum += f_eval(fam, d, x, c, w);
  }
  free(x);
  return sum / (double)n;
}

/* Derivative of the rule with respect to c_k (grad[k]) and w_k (grad[d+k]) for the
 * product-form families; for OR_OSC grad[d] is d/du.  Plain definition:
 * (1/n) sum_j df(x_j)/dtheta, with the analytic derivative of the integrand. */
int or_slr_grad(int fam, int d, uint64_t n, const uint64_t *z, const double *c, const double *w,
                double *grad) {
  if (!is_product(fam)) return -1;
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  for (int k = 0; k < 2 * d; ++k) grad[k] = 0.0;
  for (uint64_t j = 0; j < n; ++j) {
    for (int i = 0; i < d; ++i) x[i] = (double)mulmod(j, z[i] % n, n) / (double)n;
    double f = f_eval(fam, d, x, c, w);
    if (fam == OR_OSC) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += c[i] * x[i];
      double sn = sin(2.0 * M_PI * w[0] + s);
      for (int k = 0; k < d; ++k) grad[k] += -sn * x[k];
      grad[d] += -2.0 * M_PI * sn;
    } else {
      for (int k = 0; k < d; ++k) {
        double dx = x[k] - w[k], ck = c[k];
        if (fam == OR_EXP) {
          grad[k] += f * x[k];
        } else if (fam == OR_GAUSS) {
          grad[k] += f * (-2.0 * ck * dx * dx);
          grad[d + k] += f * (2.0 * ck * ck * dx);
        } else { /* OR_PEAK: f / D_k * (-dD_k/dtheta) */
          double D = 1.0 / (ck * ck) + dx * dx;
          grad[k] += f * (2.0 / (ck * ck * ck)) / D;
          grad[d + k] += f * (2.0 * dx) / D;
        }
      }
    }
  }
  for (int k = 0; k < 2 * d; ++k) grad[k] /= (double)n;
  free(x);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Affine transformation of Theorem 3.1 and grid sizes of eq. (3.5)           */
/* ------------------------------------------------------------------------- */

static uint64_t gcd_u64(uint64_t x, uint64_t y) {
  while (y) { uint64_t t = x % y; x = y; y = t; }
  return x;
}

/* n_i = lcm(z_i, z_{i+1}) / min(z_i, z_{i+1}) for i < d, n_d = ceil(n / z_d), eq. (3.5). */
int or_grid_sizes(int d, uint64_t n, const uint64_t *z, uint64_t *Nd) {
  for (int i = 0; i + 1 < d; ++i) {
    uint64_t lo = z[i] < z[i + 1] ? z[i] : z[i + 1];
    uint64_t l = (z[i] / gcd_u64(z[i], z[i + 1])) * z[i + 1];
    Nd[i] = l / lo;
  }
  Nd[d - 1] = (n + z[d - 1] - 1) / z[d - 1];
  return 0;
}

/* y_j = abs(A x_j + b) for the points j = 0..n-1, eq. (3.1): row i < d gives
 * x_i / z_i - x_{i+1} / z_{i+1}; the last row gives x_d + b_d with
 * b_d = -{n x_d / z_d} z_d / n, evaluated from the exact integer r_d = j z_d mod n. */
int or_affine_y(int d, uint64_t n, const uint64_t *z, double *y_out) {
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  for (uint64_t j = 0; j < n; ++j) {
    for (int i = 0; i < d; ++i) x[i] = (double)mulmod(j, z[i] % n, n) / (double)n;
    for (int i = 0; i + 1 < d; ++i)
      y_out[j * (uint64_t)d + i] = fabs(x[i] / (double)z[i] - x[i + 1] / (double)z[i + 1]);
    uint64_t rd = mulmod(j, z[d - 1] % n, n);
    double bd = -(double)(rd % z[d - 1]) / (double)n;
    y_out[j * (uint64_t)d + d - 1] = fabs(x[d - 1] + bd);
  }
  free(x);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The improved rule on the transformed grid, brute force (Lemma 3.2, eq. 4.3) */
/* ------------------------------------------------------------------------- */

/* For the Korobov vector z = (1, a, ..., a^(d-1)) and n = nd a^(d-1), Lemma 3.2
 * gives the axis sets y_i in {0, 1/a^i, ..., (a-1)/a^i} (i < d) and
 * y_d in {0, a^(d-1)/n, ..., (n - a^(d-1))/n}.  Every grid point is mapped back by
 * x = A^{-1}(y - b) (b = 0 on this grid), i.e. x_d = y_d and
 * x_i = z_i (y_i + x_{i+1} / z_{i+1}), and the rule averages f over the
 * prod n_i = n grid points with weight 1 / prod n_i.  Requires n <= 2^40. */
double or_grid_korobov(int fam, int d, uint64_t a, uint64_t nd, const double *c, const double *w) {
  uint64_t npts = nd;
  for (int i = 1; i < d; ++i) npts *= a;
  double *zf = (double *)malloc(sizeof(double) * (size_t)d);
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  uint64_t *s = (uint64_t *)calloc((size_t)d, sizeof(uint64_t));
  double ai = 1.0, n = (double)npts, sum = 0.0;
  for (int i = 0; i < d; ++i) { zf[i] = ai; ai *= (double)a; }
  for (uint64_t t = 0; t < npts; ++t) {
    /* digits: s[0..d-2] in [0,a), s[d-1] in [0,nd); s[0] fastest */
    uint64_t rem = t;
    for (int i = 0; i + 1 < d; ++i) { s[i] = rem % a; rem /= a; }
    s[d - 1] = rem;
    x[d - 1] = (double)s[d - 1] * zf[d - 1] / n;
    for (int i = d - 2; i >= 0; --i) {
      double yi = (double)s[i] / (zf[i] * (double)a); /* s_i / a^(i+1) in 1-based terms */
      x[i] = zf[i] * (yi + x[i + 1] / zf[i + 1]);
    }
    sum += f_eval(fam, d, x, c, w);
  }
  free(zf); free(x); free(s);
  return sum / n;
}

/* ------------------------------------------------------------------------- */
/* MDI sweeps (Algorithm 1 with m = 1 inside Algorithm 2)                     */
/* ------------------------------------------------------------------------- */
/*
 * Notation.  Level k = 1..d contracts transformed coordinate k (the first
 * remaining one, Algorithm 1 deletes the first m = 1 components per pass).  The
 * cluster of level k around a parent value x (the original coordinate x_{k+1})
 * is u = (q + x) / r_k, q = 0..r_k-1, with r_k = a for k < d and r_d = nd (the
 * last axis, whose parent is x_{d+1} = 0).  The state after level k is
 *     G_k(x) = (1/r_k) sum_q phi_k(u) G_{k-1}(u),   G_0 = 1,
 * which is eq. (4.4) with equal weights; the rule is front * G_d.
 */

/* (E) Exact level tables: G_k is kept at every parent the lattice needs,
 * x = m / M_k, M_k = M_{k-1} / r_k, M_0 = n.  Requires n <= 2^32. */
double or_mdi_exact(int fam, int d, uint64_t a, uint64_t nd, const double *c, const double *w) {
  if (!is_product(fam)) return NAN;
  uint64_t M = nd;
  for (int i = 1; i < d; ++i) M *= a;
  cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)M);
  for (uint64_t m = 0; m < M; ++m) G[m] = 1.0;
  for (int k = 1; k <= d; ++k) {
    uint64_t r = (k < d) ? a : nd, Mk = M / r;
    cplx *H = (cplx *)malloc(sizeof(cplx) * (size_t)Mk);
    for (uint64_t m = 0; m < Mk; ++m) {
      cplx acc = 0.0;
      for (uint64_t q = 0; q < r; ++q) {
        uint64_t idx = q * Mk + m;
        acc += phi(fam, k - 1, (double)idx / (double)M, c, w) * G[idx];
      }
      H[m] = acc / (double)r;
    }
    free(G);
    G = H;
    M = Mk;
  }
  double out = creal(front(fam, w) * G[0]);
  free(G);
  return out;
}

/* (C) Closed state for the exponential families: G_k(x) = K_k exp(beta_k x).
 * Substituting into the level recursion gives gamma_k = beta_{k-1} + c_k (times i
 * for OR_OSC), K_k = K_{k-1} (1/r_k) sum_q exp(gamma_k q / r_k), beta_k = gamma_k / r_k. */
double or_mdi_closed(int fam, int d, uint64_t a, uint64_t nd, const double *c, const double *w) {
  if (fam != OR_EXP && fam != OR_OSC) return NAN;
  cplx beta = 0.0, K = 1.0;
  for (int k = 1; k <= d; ++k) {
    double r = (double)((k < d) ? a : nd);
    cplx ck = (fam == OR_OSC) ? I * c[k - 1] : c[k - 1];
    cplx gamma = beta + ck, S = 0.0;
    for (uint64_t q = 0; q < (uint64_t)r; ++q) S += cexp(gamma * (double)q / r);
    K *= S / r;
    beta = gamma / r;
  }
  return creal(front(fam, w) * K);
}

/* Forward-mode derivative of the closed-state sweep: grad[k] = dQ/dc_k, and for
 * OR_OSC grad[d] = dQ/du.  Each tangent is carried through the same recursion. */
int or_mdi_closed_grad(int fam, int d, uint64_t a, uint64_t nd, const double *c, const double *w,
                       double *grad) {
  if (fam != OR_EXP && fam != OR_OSC) return -1;
  for (int k = 0; k < 2 * d; ++k) grad[k] = 0.0;
  for (int t = 0; t < d; ++t) {
    cplx beta = 0.0, K = 1.0, dbeta = 0.0, dK = 0.0;
    for (int k = 1; k <= d; ++k) {
      double r = (double)((k < d) ? a : nd);
      cplx ck = (fam == OR_OSC) ? I * c[k - 1] : c[k - 1];
      cplx dck = (k - 1 == t) ? ((fam == OR_OSC) ? I : 1.0) : 0.0;
      cplx gamma = beta + ck, dgamma = dbeta + dck, S = 0.0, dS = 0.0;
      for (uint64_t q = 0; q < (uint64_t)r; ++q) {
        cplx e = cexp(gamma * (double)q / r);
        S += e;
        dS += e * dgamma * (double)q / r;
      }
      dK = dK * (S / r) + K * (dS / r);
      K *= S / r;
      beta = gamma / r;
      dbeta = dgamma / r;
    }
    grad[t] = creal(front(fam, w) * dK);
    if (fam == OR_OSC && t == 0) grad[d] = creal(2.0 * M_PI * I * front(fam, w) * K);
  }
  return 0;
}

/* (S) Node state: G_k is kept at P Chebyshev points of the first kind on [0,1],
 * xi_p = (1 + cos(pi (2p+1) / (2P))) / 2, and read between them by the barycentric
 * formula of the second kind with weights (-1)^p sin(pi (2p+1) / (2P))
 * (Berrut & Trefethen, SIAM Review 46 (2004), eq. 4.2 and Sec. 5). */
static void cheb_nodes(int P, double *xi, double *bw) {
  for (int p = 0; p < P; ++p) {
    double th = M_PI * (2.0 * p + 1.0) / (2.0 * P);
    xi[p] = 0.5 * (1.0 + cos(th));
    bw[p] = ((p % 2 == 0) ? 1.0 : -1.0) * sin(th);
  }
}

static cplx bary(int P, const double *xi, const double *bw, const cplx *G, double u) {
  cplx num = 0.0;
  double den = 0.0;
  for (int p = 0; p < P; ++p) {
    if (u == xi[p]) return G[p];
    double t = bw[p] / (u - xi[p]);
    num += t * G[p];
    den += t;
  }
  return num / den;
}

/* Barycentric basis value l_p(u) (the weight of node p when reading at u). */
static double bary_basis(int P, const double *xi, const double *bw, int p, double u) {
  double den = 0.0;
  for (int t = 0; t < P; ++t) {
    if (u == xi[t]) return t == p ? 1.0 : 0.0;
    den += bw[t] / (u - xi[t]);
  }
  return (bw[p] / (u - xi[p])) / den;
}

/* Node-state sweep; states_out (optional, (d+1) x P complex as 2 doubles) receives
 * G_0 .. G_{d-1} at the nodes and G_d in slot [d][0]. */
static cplx mdi_nodes_core(int fam, int d, uint64_t a, uint64_t nd, int P, const double *c,
                           const double *w, double *states_out) {
  double *xi = (double *)malloc(sizeof(double) * (size_t)P);
  double *bw = (double *)malloc(sizeof(double) * (size_t)P);
  cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cplx *H = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cheb_nodes(P, xi, bw);
  for (int p = 0; p < P; ++p) G[p] = 1.0;
  for (int k = 1; k < d; ++k) {
    if (states_out)
      for (int p = 0; p < P; ++p) {
        states_out[2 * ((size_t)(k - 1) * P + p)] = creal(G[p]);
        states_out[2 * ((size_t)(k - 1) * P + p) + 1] = cimag(G[p]);
      }
    for (int p = 0; p < P; ++p) {
      cplx acc = 0.0;
      for (uint64_t q = 0; q < a; ++q) {
        double u = ((double)q + xi[p]) / (double)a;
        acc += phi(fam, k - 1, u, c, w) * bary(P, xi, bw, G, u);
      }
      H[p] = acc / (double)a;
    }
    memcpy(G, H, sizeof(cplx) * (size_t)P);
  }
  if (states_out)
    for (int p = 0; p < P; ++p) {
      states_out[2 * ((size_t)(d - 1) * P + p)] = creal(G[p]);
      states_out[2 * ((size_t)(d - 1) * P + p) + 1] = cimag(G[p]);
    }
  cplx acc = 0.0;
  for (uint64_t s = 0; s < nd; ++s) {
    double u = (double)s / (double)nd;
    acc += phi(fam, d - 1, u, c, w) * (d > 1 ? bary(P, xi, bw, G, u) : 1.0);
  }
  acc /= (double)nd;
  if (states_out) {
    states_out[2 * (size_t)d * P] = creal(acc);
    states_out[2 * (size_t)d * P + 1] = cimag(acc);
  }
  free(xi); free(bw); free(G); free(H);
  return acc;
}

double or_mdi_nodes(int fam, int d, uint64_t a, uint64_t nd, int P, const double *c,
                    const double *w) {
  if (!is_product(fam) || P < 2) return NAN;
  return creal(front(fam, w) * mdi_nodes_core(fam, d, a, nd, P, c, w, NULL));
}

/* States of the node sweep, for checking the device's level states and checkpoints. */
int or_mdi_nodes_states(int fam, int d, uint64_t a, uint64_t nd, int P, const double *c,
                        const double *w, double *states_out) {
  if (!is_product(fam) || P < 2) return -1;
  mdi_nodes_core(fam, d, a, nd, P, c, w, states_out);
  return 0;
}

/* Node state with step size m (Algorithm 1 with m = 1, 2, 3; eq. 2.14c): every
 * iteration contracts m transformed axes at once instead of one.  The symbolic
 * function after the iteration, g_{k-m}, is kept at the P nodes like the m = 1
 * state; its value at node xi_p is the weighted sum over the a^m digit tuples
 * (q_i, ..., q_{i+m-1}) of the contracted axes of the product of their factors,
 * the coordinates generated outermost first by the affine recurrence of
 * Theorem 3.1 / Lemma 3.2 (x_{i+m} = xi_p, x_j = (q_j + x_{j+1}) / a), times the
 * previous iteration's function read at the innermost coordinate x_i.  Each tuple
 * weighs 1/a^m (w_{i_1} ... w_{i_m} with w = 1/a).  The d-1 cluster axes are taken
 * in order, the first m first (the paper deletes the first m components); when
 * m does not divide d-1 the last iteration takes the remaining axes.  The last
 * axis (n_d points s/n_d) is summed as in the m = 1 sweep.  m = 1 is
 * or_mdi_nodes. */
static cplx mdi_nodes_step_core(int fam, int d, uint64_t a, uint64_t nd, int P, int m, const double *c,
                                const double *w) {
  double *xi = (double *)malloc(sizeof(double) * (size_t)P);
  double *bw = (double *)malloc(sizeof(double) * (size_t)P);
  cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cplx *H = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cheb_nodes(P, xi, bw);
  for (int p = 0; p < P; ++p) G[p] = 1.0;
  for (int i = 1; i < d; i += m) {           /* contract axes i .. i+mi-1 (1-based) */
    int mi = (d - i < m) ? d - i : m;
    uint64_t tuples = 1;  /* a^mi: every tuple weighs 1/a^mi */
    for (int j = 0; j < mi; ++j) tuples *= a;
    for (int p = 0; p < P; ++p) {
      cplx acc = 0.0;
      for (uint64_t t = 0; t < tuples; ++t) {
        /* digit of axis i+j is (t / a^j) mod a */
        double x = xi[p];
        cplx prod = 1.0;
        for (int j = mi - 1; j >= 0; --j) {
          uint64_t aj = 1;
          for (int l = 0; l < j; ++l) aj *= a;
          uint64_t q = (t / aj) % a;
          x = ((double)q + x) / (double)a;  /* x_{i+j} */
          prod *= phi(fam, i + j - 1, x, c, w);
        }
        acc += prod * bary(P, xi, bw, G, x);
      }
      H[p] = acc / (double)tuples;
    }
    memcpy(G, H, sizeof(cplx) * (size_t)P);
  }
  cplx acc = 0.0;
  for (uint64_t s = 0; s < nd; ++s) {
    double u = (double)s / (double)nd;
    acc += phi(fam, d - 1, u, c, w) * (d > 1 ? bary(P, xi, bw, G, u) : 1.0);
  }
  acc /= (double)nd;
  free(xi); free(bw); free(G); free(H);
  return acc;
}

double or_mdi_nodes_step(int fam, int d, uint64_t a, uint64_t nd, int P, int m, const double *c,
                         const double *w) {
  if (!is_product(fam) || P < 2 || m < 1 || m > 3) return NAN;
  return creal(front(fam, w) * mdi_nodes_step_core(fam, d, a, nd, P, m, c, w));
}

/* Forward-mode derivative of the step-m node-state sweep (or_mdi_nodes_step) with
 * respect to the parameters t listed in which[0..nwhich) (indices as in
 * or_mdi_nodes_grad).  The tangent Gd is carried through each iteration by the
 * same weighted tuple sum as G; in the iteration that contracts the parameter's
 * axis, the tuple's factor of that axis is replaced by its derivative (the
 * product rule over the tuple's factors) and multiplied by G read at the same
 * innermost coordinate.  A parameter of the last axis enters the last sum. */
int or_mdi_nodes_step_grad(int fam, int d, uint64_t a, uint64_t nd, int P, int m, const double *c,
                           const double *w, const int *which, int nwhich, double *grad_out) {
  if (!is_product(fam) || P < 2 || m < 1 || m > 3) return -1;
  double *xi = (double *)malloc(sizeof(double) * (size_t)P);
  double *bw = (double *)malloc(sizeof(double) * (size_t)P);
  cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)P), *H = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cplx *Gd = (cplx *)malloc(sizeof(cplx) * (size_t)P), *Hd = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cheb_nodes(P, xi, bw);
  for (int iw = 0; iw < nwhich; ++iw) {
    int t = which[iw];
    if (fam == OR_OSC && t == d) {  /* Q = Re(exp(2 pi i u) q): dQ/du = Re(2 pi i exp(2 pi i u) q) */
      cplx q = mdi_nodes_step_core(fam, d, a, nd, P, m, c, w);
      grad_out[iw] = creal(2.0 * M_PI * I * front(fam, w) * q);
      continue;
    }
    int lev = (t < d) ? t : t - d;  /* 0-based axis of the parameter */
    int kind = (t < d) ? 0 : 1;     /* 0: c, 1: w */
    if (kind == 1 && (fam == OR_EXP || fam == OR_OSC)) { grad_out[iw] = 0.0; continue; }
    for (int p = 0; p < P; ++p) { G[p] = 1.0; Gd[p] = 0.0; }
    for (int i = 1; i < d; i += m) {  /* axes i .. i+mi-1 (1-based), as or_mdi_nodes_step */
      int mi = (d - i < m) ? d - i : m;
      uint64_t tuples = 1;
      for (int j = 0; j < mi; ++j) tuples *= a;
      int here = lev >= i - 1 && lev < i - 1 + mi;  /* the parameter's axis is contracted now */
      for (int p = 0; p < P; ++p) {
        cplx acc = 0.0, accd = 0.0;
        for (uint64_t tu = 0; tu < tuples; ++tu) {
          double x = xi[p];
          cplx prod = 1.0, dprod = 1.0;
          for (int j = mi - 1; j >= 0; --j) {
            uint64_t aj = 1;
            for (int l = 0; l < j; ++l) aj *= a;
            uint64_t q = (tu / aj) % a;
            x = ((double)q + x) / (double)a;  /* x_{i+j} */
            cplx f = phi(fam, i + j - 1, x, c, w);
            prod *= f;
            dprod *= (i + j - 1 == lev) ? dphi(fam, i + j - 1, kind, x, c, w) : f;
          }
          cplx g = bary(P, xi, bw, G, x), gd = bary(P, xi, bw, Gd, x);
          acc += prod * g;
          accd += prod * gd;
          if (here) accd += dprod * g;
        }
        H[p] = acc / (double)tuples;
        Hd[p] = accd / (double)tuples;
      }
      memcpy(G, H, sizeof(cplx) * (size_t)P);
      memcpy(Gd, Hd, sizeof(cplx) * (size_t)P);
    }
    cplx accd = 0.0;
    for (uint64_t s = 0; s < nd; ++s) {
      double u = (double)s / (double)nd;
      cplx g = d > 1 ? bary(P, xi, bw, G, u) : 1.0;
      cplx gd = d > 1 ? bary(P, xi, bw, Gd, u) : 0.0;
      accd += phi(fam, d - 1, u, c, w) * gd;
      if (d - 1 == lev) accd += dphi(fam, d - 1, kind, u, c, w) * g;
    }
    grad_out[iw] = creal(front(fam, w) * accd / (double)nd);
  }
  free(xi); free(bw); free(G); free(H); free(Gd); free(Hd);
  return 0;
}

/* Forward-mode derivative of the node-state sweep with respect to c_t and w_t for
 * the parameters t listed in which[0..nwhich) (indices into the 2d-long gradient:
 * t < d is c_t, t >= d is w_{t-d}; for OR_OSC index d is u).  The tangent Gdot is
 * zero below the level of the parameter, picks up the derivative of phi there,
 * and is carried through the later levels by the same (linear) recursion. */
int or_mdi_nodes_grad(int fam, int d, uint64_t a, uint64_t nd, int P, const double *c,
                      const double *w, const int *which, int nwhich, double *grad_out) {
  if (!is_product(fam) || P < 2) return -1;
  double *xi = (double *)malloc(sizeof(double) * (size_t)P);
  double *bw = (double *)malloc(sizeof(double) * (size_t)P);
  cplx *G = (cplx *)malloc(sizeof(cplx) * (size_t)P), *H = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cplx *Gd = (cplx *)malloc(sizeof(cplx) * (size_t)P), *Hd = (cplx *)malloc(sizeof(cplx) * (size_t)P);
  cheb_nodes(P, xi, bw);
  for (int iw = 0; iw < nwhich; ++iw) {
    int t = which[iw];
    if (fam == OR_OSC && t == d) {
      cplx Q = mdi_nodes_core(fam, d, a, nd, P, c, w, NULL);
      grad_out[iw] = creal(2.0 * M_PI * I * front(fam, w) * Q);
      continue;
    }
    int lev = (t < d) ? t : t - d;        /* 0-based axis of the parameter */
    int kind = (t < d) ? 0 : 1;           /* 0: c, 1: w */
    if (kind == 1 && (fam == OR_EXP || fam == OR_OSC)) { grad_out[iw] = 0.0; continue; }
    for (int p = 0; p < P; ++p) { G[p] = 1.0; Gd[p] = 0.0; }
    for (int k = 1; k < d; ++k) {
      for (int p = 0; p < P; ++p) {
        cplx acc = 0.0, accd = 0.0;
        for (uint64_t q = 0; q < a; ++q) {
          double u = ((double)q + xi[p]) / (double)a;
          cplx g = bary(P, xi, bw, G, u), gd = bary(P, xi, bw, Gd, u);
          acc += phi(fam, k - 1, u, c, w) * g;
          accd += phi(fam, k - 1, u, c, w) * gd;
          if (k - 1 == lev) accd += dphi(fam, k - 1, kind, u, c, w) * g;
        }
        H[p] = acc / (double)a;
        Hd[p] = accd / (double)a;
      }
      memcpy(G, H, sizeof(cplx) * (size_t)P);
      memcpy(Gd, Hd, sizeof(cplx) * (size_t)P);
    }
    cplx accd = 0.0;
    for (uint64_t s = 0; s < nd; ++s) {
      double u = (double)s / (double)nd;
      cplx g = d > 1 ? bary(P, xi, bw, G, u) : 1.0;
      cplx gd = d > 1 ? bary(P, xi, bw, Gd, u) : 0.0;
      accd += phi(fam, d - 1, u, c, w) * gd;
      if (d - 1 == lev) accd += dphi(fam, d - 1, kind, u, c, w) * g;
    }
    grad_out[iw] = creal(front(fam, w) * accd / (double)nd);
  }
  free(xi); free(bw); free(G); free(H); free(Gd); free(Hd);
  return 0;
}

/* Barycentric basis matrix L[(q,p), t] = l_t((q + xi_p)/a), for checking the
 * device's interpolation table. */
int or_bary_matrix(int P, uint64_t a, double *L) {
  double *xi = (double *)malloc(sizeof(double) * (size_t)P);
  double *bw = (double *)malloc(sizeof(double) * (size_t)P);
  cheb_nodes(P, xi, bw);
  for (uint64_t q = 0; q < a; ++q)
    for (int p = 0; p < P; ++p)
      for (int t = 0; t < P; ++t)
        L[(q * (uint64_t)P + p) * (uint64_t)P + t] =
            bary_basis(P, xi, bw, t, ((double)q + xi[p]) / (double)a);
  free(xi); free(bw);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* The tensor midpoint rule that reproduces the paper's printed MDI-LR columns */
/* ------------------------------------------------------------------------- */

/* Brute force over the grid of eq. (3.5): points ((k_i + 1/2) / n_i)_i, equal weight. */
double or_midpoint_grid(int fam, int d, const uint64_t *Nd, const double *c, const double *w) {
  uint64_t npts = 1;
  for (int i = 0; i < d; ++i) npts *= Nd[i];
  double *x = (double *)malloc(sizeof(double) * (size_t)d), sum = 0.0;
  for (uint64_t t = 0; t < npts; ++t) {
    uint64_t rem = t;
    for (int i = 0; i < d; ++i) { x[i] = ((double)(rem % Nd[i]) + 0.5) / (double)Nd[i]; rem /= Nd[i]; }
    sum += f_eval(fam, d, x, c, w);
  }
  free(x);
  return sum / (double)npts;
}

/* The same rule for product-form integrands: product of one-dimensional means. */
double or_midpoint_product(int fam, int d, const uint64_t *Nd, const double *c, const double *w) {
  if (!is_product(fam)) return NAN;
  cplx prod = 1.0;
  for (int i = 0; i < d; ++i) {
    cplx s = 0.0;
    for (uint64_t k = 0; k < Nd[i]; ++k) s += phi(fam, i, ((double)k + 0.5) / (double)Nd[i], c, w);
    prod *= s / (double)Nd[i];
  }
  return creal(front(fam, w) * prod);
}

/* The same rule for a ridge integrand f(x) = (c0 + sum_i x_i)^(-p) on the grid
 * n_1 = ... = n_{d-1} = N, n_d = n_last, by the dimension iteration of Algorithm 1
 * (m = 1, eq. 2.14c): after the first i axes are summed out, the symbolic function
 * depends on them only through the digit sum S = k_1 + ... + k_i, so its state is
 * the weight H_i[S] of each S, H_i[S] = (1/N) sum_{k<N} H_{i-1}[S - k], H_0 = [1].
 * Then Q = sum_S H_{d-1}[S] (1/n_last) sum_{k<n_last} f at the coordinate sum
 * (S + (d-1)/2)/N + (k + 1/2)/n_last.  Test 7's f_6 is c0 = 1, p = d + 1. */
double or_midpoint_ridge(int d, uint64_t N, uint64_t n_last, double c0, double p) {
  if (d < 1 || N < 1 || n_last < 1) return NAN;
  const uint64_t L = (uint64_t)(d - 1) * (N - 1) + 1;
  double *h = (double *)calloc((size_t)L, sizeof(double)), *g = (double *)calloc((size_t)L, sizeof(double));
  h[0] = 1.0;
  uint64_t len = 1;
  for (int i = 1; i < d; ++i) {
    const uint64_t nlen = len + N - 1;
    for (uint64_t S = 0; S < nlen; ++S) {
      double acc = 0.0;
      for (uint64_t k = 0; k < N; ++k)
        if (S >= k && S - k < len) acc += h[S - k];
      g[S] = acc / (double)N;
    }
    double *t = h;
    h = g;
    g = t;
    len = nlen;
  }
  double q = 0.0;
  for (uint64_t S = 0; S < len; ++S) {
    double inner = 0.0;
    const double base = ((double)S + 0.5 * (double)(d - 1)) / (double)N;
    for (uint64_t k = 0; k < n_last; ++k) inner += pow(c0 + base + ((double)k + 0.5) / (double)n_last, -p);
    q += h[S] * inner / (double)n_last;
  }
  free(h);
  free(g);
  return q;
}

/* ------------------------------------------------------------------------- */
/* Exact integrals over [0,1]^d (textbook antiderivatives per axis)           */
/* ------------------------------------------------------------------------- */

static cplx axis_integral(int fam, int j, const double *c, const double *w) {
  double cj = c[j];
  switch (fam) {
    case OR_EXP: return cj == 0.0 ? 1.0 : expm1(cj) / cj;
    case OR_OSC: return cj == 0.0 ? 1.0 : (cexp(I * cj) - 1.0) / (I * cj);
    case OR_GAUSS: return sqrt(M_PI) / (2.0 * cj) * (erf(cj * (1.0 - w[j])) + erf(cj * w[j]));
    case OR_PEAK: return cj * (atan(cj * (1.0 - w[j])) + atan(cj * w[j]));
  }
  return NAN;
}

static cplx axis_integral_d(int fam, int j, int kind, const double *c, const double *w) {
  double cj = c[j], wj = w[j];
  switch (fam) {
    case OR_EXP: /* d/dc (e^c - 1)/c */
      if (kind) return 0.0;
      return cj == 0.0 ? 0.5 : (cj * exp(cj) - expm1(cj)) / (cj * cj);
    case OR_OSC: { /* d/dc int_0^1 e^{icx} dx = i int_0^1 x e^{icx} dx */
      if (kind) return 0.0;
      if (cj == 0.0) return 0.5 * I;
      cplx ic = I * cj, e = cexp(ic);
      return I * (e / ic - (e - 1.0) / (ic * ic));
    }
    case OR_GAUSS: {
      double F = sqrt(M_PI) / (2.0 * cj) * (erf(cj * (1.0 - wj)) + erf(cj * wj));
      double e1 = exp(-cj * cj * (1.0 - wj) * (1.0 - wj)), e0 = exp(-cj * cj * wj * wj);
      if (kind == 0) return -F / cj + ((1.0 - wj) * e1 + wj * e0) / cj;
      return e0 - e1;
    }
    case OR_PEAK: {
      double F = cj * (atan(cj * (1.0 - wj)) + atan(cj * wj));
      double A1 = 1.0 + cj * cj * (1.0 - wj) * (1.0 - wj), A0 = 1.0 + cj * cj * wj * wj;
      if (kind == 0) return F / cj + cj * ((1.0 - wj) / A1 + wj / A0);
      return cj * (-cj / A1 + cj / A0);
    }
  }
  return NAN;
}

double or_closed_form(int fam, int d, const double *c, const double *w) {
  if (!is_product(fam)) return NAN;
  cplx p = 1.0;
  for (int j = 0; j < d; ++j) p *= axis_integral(fam, j, c, w);
  return creal(front(fam, w) * p);
}

/* Exact gradient of the integral: grad[k] = dI/dc_k, grad[d+k] = dI/dw_k
 * (OR_OSC: grad[d] = dI/du). */
int or_closed_form_grad(int fam, int d, const double *c, const double *w, double *grad) {
  if (!is_product(fam)) return -1;
  for (int k = 0; k < 2 * d; ++k) grad[k] = 0.0;
  for (int kind = 0; kind < 2; ++kind) {
    if (kind == 1 && (fam == OR_EXP || fam == OR_OSC)) continue;
    for (int k = 0; k < d; ++k) {
      cplx p = 1.0;
      for (int j = 0; j < d; ++j)
        p *= (j == k) ? axis_integral_d(fam, j, kind, c, w) : axis_integral(fam, j, c, w);
      grad[kind * d + k] = creal(front(fam, w) * p);
    }
  }
  if (fam == OR_OSC) {
    cplx p = 1.0;
    for (int j = 0; j < d; ++j) p *= axis_integral(fam, j, c, w);
    grad[d] = creal(2.0 * M_PI * I * front(fam, w) * p);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Randomly shifted lattice rule (Section 2.1): P + Delta = {{t + Delta} : t in P} */
/* ------------------------------------------------------------------------- */

/* (1/n) sum_{j<n} f({j z / n + Delta}), {x} = x - floor(x) componentwise. */
double or_slr_shifted(int fam, int d, uint64_t n, const uint64_t *z, const double *c, const double *w,
                      const double *shift) {
  double *x = (double *)malloc(sizeof(double) * (size_t)d), sum = 0.0;
  for (uint64_t j = 0; j < n; ++j) {
    for (int i = 0; i < d; ++i) {
      const double v = (double)mulmod(j, z[i] % n, n) / (double)n + shift[i];
      x[i] = v - floor(v);
    }
    sum += f_eval(fam, d, x, c, w);
  }
  free(x);
  return sum / (double)n;
}

/* ------------------------------------------------------------------------- */
/* Generating-vector criteria and searches (Section 2.2)                      */
/* ------------------------------------------------------------------------- */

/* Bernoulli polynomials on [0, 1] for the even alpha the criteria use. */
static double bernoulli_poly(int alpha, double x) {
  if (alpha == 2) return x * x - x + 1.0 / 6.0;
  if (alpha == 4) return x * x * x * x - 2.0 * x * x * x + x * x - 1.0 / 30.0;
  return NAN;
}

/* (-1)^(alpha/2 + 1) (2 pi)^alpha / alpha!, the coefficient of B_alpha in eq. (2.4). */
static double p_alpha_coef(int alpha) {
  double fact = 1.0;
  for (int i = 2; i <= alpha; ++i) fact *= (double)i;
  const double sign = ((alpha / 2 + 1) % 2 == 0) ? 1.0 : -1.0;
  return sign * pow(2.0 * M_PI, (double)alpha) / fact;
}

/* P_alpha(z) by the finite form of eq. (2.4),
 *   -1 + (1/n) sum_{k<n} prod_j (1 + C_alpha B_alpha({k z_j / n})),
 * for alpha = 2 or 4.  The paper writes the k = 0 term apart as
 * (1/n) prod_j (1 + 2 zeta(alpha)); it is the same term, C_alpha B_alpha(0) = 2 zeta(alpha). */
double or_p_alpha(int alpha, int d, uint64_t n, const uint64_t *z) {
  if ((alpha != 2 && alpha != 4) || d < 1 || n < 1) return NAN;
  const double C = p_alpha_coef(alpha);
  double sum = 0.0;
  for (uint64_t k = 0; k < n; ++k) {
    double prod = 1.0;
    for (int j = 0; j < d; ++j)
      prod *= 1.0 + C * bernoulli_poly(alpha, (double)mulmod(k, z[j] % n, n) / (double)n);
    sum += prod;
  }
  return -1.0 + sum / (double)n;
}

/* Example 2's search: values[t] = P_alpha(z(a)) for a = a_first + t, t < count.  A
 * candidate outside 1 <= a <= n-1 or with gcd(a, n) != 1 is not admissible and gets
 * +inf.  *best_a = the first a attaining the smallest value (0 if none is admissible). */
int or_korobov_search(int alpha, int d, uint64_t n, uint64_t a_first, uint64_t count, double *values,
                      uint64_t *best_a) {
  if (d < 1 || n < 1) return -1;
  uint64_t *z = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)d);
  double best = INFINITY;
  *best_a = 0;
  for (uint64_t t = 0; t < count; ++t) {
    const uint64_t a = a_first + t;
    if (a < 1 || a >= n || gcd_u64(a, n) != 1) {
      values[t] = INFINITY;
      continue;
    }
    or_korobov_z(d, a, n, z);
    values[t] = or_p_alpha(alpha, d, n, z);
    if (values[t] < best) {
      best = values[t];
      *best_a = a;
    }
  }
  free(z);
  return 0;
}

/* Squared shift-averaged worst-case error of a rank-1 lattice, eq. (2.12) in its
 * second (product-weight) form,
 *   -prod_j (1 + gamma_j beta) + (1/n) sum_{k<n} prod_j (1 + gamma_j [B_2({k z_j / n}) + beta]),
 * beta = 0 for the unanchored Sobolev space, c^2 - c + 1/3 for the one anchored at c. */
double or_wce2_shift(int d, uint64_t n, const uint64_t *z, const double *gamma, double beta) {
  if (d < 1 || n < 1) return NAN;
  double prod0 = 1.0, sum = 0.0;
  for (int j = 0; j < d; ++j) prod0 *= 1.0 + gamma[j] * beta;
  for (uint64_t k = 0; k < n; ++k) {
    double prod = 1.0;
    for (int j = 0; j < d; ++j)
      prod *= 1.0 + gamma[j] * (bernoulli_poly(2, (double)mulmod(k, z[j] % n, n) / (double)n) + beta);
    sum += prod;
  }
  return -prod0 + sum / (double)n;
}

/* Component-by-component construction of Example 3 with product weights: z_1 = 1; for
 * s = 2..d, with z_1..z_{s-1} held fixed, z_s is the z in N_n = {1 <= z <= n-1,
 * gcd(z, n) = 1} minimising the s-dimensional [E^(sh)]^2 of eq. (2.12) (the first such z
 * on ties).  e2[s-1] receives that minimum; e2[0] is the value of z_1 = 1 alone. */
int or_cbc(int d, uint64_t n, const double *gamma, double beta, uint64_t *z, double *e2) {
  if (d < 1 || n < 2) return -1;
  z[0] = 1;
  e2[0] = or_wce2_shift(1, n, z, gamma, beta);
  for (int s = 1; s < d; ++s) {
    double best = INFINITY;
    uint64_t best_z = 0;
    for (uint64_t c = 1; c < n; ++c) {
      if (gcd_u64(c, n) != 1) continue;
      z[s] = c;
      const double v = or_wce2_shift(s + 1, n, z, gamma, beta);
      if (v < best) {
        best = v;
        best_z = c;
      }
    }
    z[s] = best_z;
    e2[s] = best;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Improved lattice rule, Definition 3.3 (Section 2.2.2), Korobov z = (1,a,..)  */
/* ------------------------------------------------------------------------- */

/* The n points {j z / n} with z = (1, a, ..., a^(d-1)) lie on the lines of the
 * transformed grid of Theorem 3.1: the first d-1 transformed coordinates of point j
 * are the base-a digits of L(j) = floor(j a^(d-1) / n) (eq. 3.7), and eq. (3.5)
 * gives n_d = ceil(n / a^(d-1)) positions along the last axis.  A line holding
 * fewer than n_d points is completed by the points that continue its arithmetic
 * progression: the last point of the line plus k z / n, NOT reduced mod 1 (the
 * unwrapped reading of the ghost points).  The rule is the equal-weight mean over
 * the n lattice points and the n* added ones, 1/(n + n*) (Section 3).  Brute force:
 * every point is generated, grouped by line and evaluated.  Returns NAN when
 * a^(d-1) n does not fit in 63 bits or a^(d-1) exceeds 2^26 (the line table). */
double or_improved(int fam, int d, uint64_t n, uint64_t a, const double *c, const double *w, uint64_t *nstar) {
  uint64_t M = 1;
  for (int i = 1; i < d; ++i) {
    if (M > (1ull << 26) / a) return NAN;
    M *= a;
  }
  if (n > (1ull << 62) / M) return NAN;
  const uint64_t nd = (n + M - 1) / M;
  uint64_t *count = (uint64_t *)calloc(M, sizeof(uint64_t));
  uint64_t *last = (uint64_t *)calloc(M, sizeof(uint64_t));
  uint64_t *z = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)d);
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  z[0] = 1 % n;
  for (int i = 1; i < d; ++i) z[i] = mulmod(z[i - 1], a % n, n);
  double sum = 0.0;
  for (uint64_t j = 0; j < n; ++j) {
    const uint64_t L = j * M / n;
    count[L] += 1;
    last[L] = j;
    for (int i = 0; i < d; ++i) x[i] = (double)mulmod(j, z[i], n) / (double)n;
    sum += f_eval(fam, d, x, c, w);
  }
  uint64_t added = 0;
  for (uint64_t L = 0; L < M; ++L) {
    if (count[L] == 0) continue;  /* lines without a lattice point have no progression */
    for (uint64_t k = 1; count[L] + k <= nd; ++k) {
      for (int i = 0; i < d; ++i)
        x[i] = (double)mulmod(last[L], z[i], n) / (double)n + (double)k * (double)z[i] / (double)n;
      sum += f_eval(fam, d, x, c, w);
      added += 1;
    }
  }
  free(count);
  free(last);
  free(z);
  free(x);
  if (nstar) *nstar = added;
  return sum / (double)(n + added);
}
