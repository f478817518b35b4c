/*
 * FP64 CPU oracle for the spherical harmonic transform pair and the
 * per-degree spectral filter of FourCastNet 3's global spectral blocks.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may build, load or
 * call it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every function follows the paper's definitions directly:
 *   - grids and quadrature weights: Sec. B.1, Eq. (latlon_grid),
 *     Eq. (latlon_quad_weights) and its footnote (Clenshaw-Curtis), and the
 *     Gauss-Legendre paragraph after it;
 *   - orthonormal spherical harmonics Y_l^m = Phat_l^m(cos t) e^{i m p}:
 *     Sec. B.3, Eq. (spherical_harmonics);
 *   - forward transform: Eq. (sht), realised as a longitude DFT followed by
 *     a quadrature-weighted Legendre sum (Sec. B.3, last paragraph; Sec.
 *     F.2.2, Algorithm 1, where the quadrature weights multiply L);
 *   - inverse transform: Eq. (isht) for a real field (coefficients stored for
 *     m >= 0 only);
 *   - spectral filter: the convolution theorem, Eq. (s2_spectral_conv),
 *     generalised to a complex channel-mixing weight W[l][o][i] per degree;
 *   - adjoints of all three under the real inner product Re sum conj(a) b.
 *
 * Conventions (readings of the paper, listed with reasons in the design
 * notes of the repository):
 *   - lmax, mmax are counts: 0 <= l < lmax, 0 <= m < mmax.
 *   - latitude row k = 0 is the northernmost (theta smallest).
 *   - equiangular latitudes include both poles: theta_k = pi k / (nlat - 1).
 *   - the full 2-D quadrature weight is w_k * (2 pi / nlon), with w_k the
 *     weight of the integral over x = cos(theta) in [-1, 1].
 *   - the longitude DFT uses integer-reduced phases 2 pi ((j m) mod nlon)/nlon
 *     so that every phase is exact.
 *   - inverse: m = 0 and the Nyquist mode m = nlon/2 enter with weight 1 and
 *     only their real part; every other m enters as 2 Re(.).
 *
 * Spectral arrays are complex128 stored as interleaved (re, im) doubles in
 * the dense layout [field][l][m] (l-major), entries with l < m set to zero.
 * Spatial arrays are [field][k][j] doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GRID_GAUSS 0
#define ORC_GRID_EQUIANGULAR_CC 1
#define ORC_GRID_EQUIANGULAR_TRAPZ 2

static const double ORC_PI = 3.14159265358979323846264338327950288;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Grids and weights (Sec. B.1)                                              */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(z) and P_{n-1}(z) by the three-term (Bonnet)
 * recurrence (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}. */
static void legendre_pn(int n, double z, double *pn, double *pnm1) {
  double p0 = 1.0, p1 = z;
  if (n == 0) {
    *pn = 1.0;
    *pnm1 = 0.0;
    return;
  }
  for (int j = 2; j <= n; j++) {
    double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / (double)j;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

/* Gauss-Legendre nodes x_k = cos(theta_k) (roots of P_n, ordered north to
 * south, i.e. descending x) and weights 2 / ((1 - x^2) P_n'(x)^2).  Newton
 * iteration from the classical initial guess cos(pi (k + 3/4) / (n + 1/2)).
 * sin(theta_k) is returned as sqrt((1 - x)(1 + x)). */
void orc_gauss_legendre(int n, double *x, double *s, double *w) {
  for (int k = 0; k < n; k++) {
    double z = cos(ORC_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double pn, pnm1;
      legendre_pn(n, z, &pn, &pnm1);
      double dp = n * (pnm1 - z * pn) / ((1.0 - z) * (1.0 + z));
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) <= 1e-16) break;
    }
    double pn, pnm1;
    legendre_pn(n, z, &pn, &pnm1);
    double omz2 = (1.0 - z) * (1.0 + z);
    double dp = n * (pnm1 - z * pn) / omz2;
    x[k] = z;
    s[k] = sqrt(omz2);
    w[k] = 2.0 / (omz2 * dp * dp);
  }
}

/* Equiangular latitudes including both poles, theta_k = pi k / (n - 1). */
void orc_equiangular(int n, double *theta, double *x, double *s) {
  for (int k = 0; k < n; k++) {
    double t = ORC_PI * (double)k / (double)(n - 1);
    theta[k] = t;
    x[k] = cos(t);
    s[k] = sin(t);
  }
}

/* Clenshaw-Curtis weights on theta_k = pi k / N, N = n - 1 (footnote of
 * Eq. latlon_quad_weights):
 *   w_k = (c_k / N) * (1 - sum_{j=1}^{floor(N/2)} b_j cos(2 j theta_k) / (4 j^2 - 1))
 * with c_k = 1 at the poles and 2 elsewhere, b_j = 1 when 2 j = N, else 2. */
void orc_cc_weights(int n, double *w) {
  int N = n - 1;
  for (int k = 0; k < n; k++) {
    double t = ORC_PI * (double)k / (double)N;
    double acc = 1.0;
    for (int j = 1; 2 * j <= N; j++) {
      double b = (2 * j == N) ? 1.0 : 2.0;
      acc -= b * cos(2.0 * j * t) / (4.0 * j * j - 1.0);
    }
    double c = (k == 0 || k == N) ? 1.0 : 2.0;
    w[k] = c * acc / (double)N;
  }
}

/* Trapezoid-type weights of Eq. (latlon_quad_weights), sin(theta) dtheta,
 * with the pole-inclusive spacing dtheta = pi / (n - 1). */
void orc_trapz_weights(int n, double *w) {
  for (int k = 0; k < n; k++) {
    double t = ORC_PI * (double)k / (double)(n - 1);
    w[k] = ORC_PI / (double)(n - 1) * sin(t);
  }
}

/* Nodes and latitude weights for a grid type; returns 0 on success. */
int orc_grid(int grid, int nlat, double *x, double *s, double *w) {
  if (nlat < 1) return -1;
  if (grid == ORC_GRID_GAUSS) {
    orc_gauss_legendre(nlat, x, s, w);
    return 0;
  }
  if (nlat < 2) return -1;
  double *theta = (double *)malloc(sizeof(double) * nlat);
  if (!theta) return -2;
  orc_equiangular(nlat, theta, x, s);
  free(theta);
  if (grid == ORC_GRID_EQUIANGULAR_CC) {
    orc_cc_weights(nlat, w);
    return 0;
  }
  if (grid == ORC_GRID_EQUIANGULAR_TRAPZ) {
    orc_trapz_weights(nlat, w);
    return 0;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Normalised associated Legendre functions (Eq. spherical_harmonics)        */
/* ------------------------------------------------------------------------ */

/* Recurrence coefficients for the normalised functions below:
 *   a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)),
 *   b_lm = sqrt(((l - 1)^2 - m^2) / (4 (l - 1)^2 - 1)),
 * stored at [l * M + m] for l >= m + 2 (zero elsewhere). */
static void legendre_coeffs(int L, int M, double *a, double *b) {
  memset(a, 0, sizeof(double) * (size_t)L * (size_t)M);
  memset(b, 0, sizeof(double) * (size_t)L * (size_t)M);
  for (int m = 0; m < M; m++)
    for (int l = m + 2; l < L; l++) {
      double dl = (double)l, dm = (double)m;
      a[(size_t)l * M + m] = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
      b[(size_t)l * M + m] = sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) /
                                  (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
    }
}

/* Phat_l^m(x) = (-1)^m c_l^m P_l^m(x), for 0 <= m < M, m <= l < L, written
 * to out[l * M + m] (zero for l < m).  s = sqrt(1 - x^2) is passed in.
 * Recurrences (standard, from the definition):
 *   Phat_0^0 = 1 / sqrt(4 pi)
 *   Phat_m^m = -sqrt((2m + 1) / (2m)) s Phat_{m-1}^{m-1}
 *   Phat_{m+1}^m = sqrt(2m + 3) x Phat_m^m
 *   Phat_l^m = a_lm (x Phat_{l-1}^m - b_lm Phat_{l-2}^m)
 * with a_lm, b_lm from legendre_coeffs. */
static void legendre_with(int L, int M, double x, double s, const double *a,
                          const double *b, double *out) {
  memset(out, 0, sizeof(double) * (size_t)L * (size_t)M);
  double pmm = 1.0 / sqrt(4.0 * ORC_PI);
  for (int m = 0; m < M && m < L; m++) {
    if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;
    out[(size_t)m * M + m] = pmm;
    if (m + 1 >= L) continue;
    double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
    out[(size_t)(m + 1) * M + m] = p1;
    double p0 = pmm;
    for (int l = m + 2; l < L; l++) {
      size_t i = (size_t)l * M + m;
      double p2 = a[i] * (x * p1 - b[i] * p0);
      out[i] = p2;
      p0 = p1;
      p1 = p2;
    }
  }
}

/* Stand-alone form of legendre_with (computes its own coefficients). */
void orc_legendre(int L, int M, double x, double s, double *out) {
  double *a = (double *)malloc(sizeof(double) * (size_t)L * M);
  double *b = (double *)malloc(sizeof(double) * (size_t)L * M);
  legendre_coeffs(L, M, a, b);
  legendre_with(L, M, x, s, a, b, out);
  free(a);
  free(b);
}

/* Phat_l^m(x) for one (l, m), same recurrence. */
double orc_legendre_one(int l, int m, double x, double s) {
  double pmm = 1.0 / sqrt(4.0 * ORC_PI);
  for (int i = 1; i <= m; i++) pmm = -sqrt((2.0 * i + 1.0) / (2.0 * i)) * s * pmm;
  if (l == m) return pmm;
  double p0 = pmm;
  double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
  for (int ll = m + 2; ll <= l; ll++) {
    double dl = (double)ll, dm = (double)m;
    double a = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
    double b = sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) /
                    (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
    double p2 = a * (x * p1 - b * p0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* ------------------------------------------------------------------------ */
/* Longitude DFT                                                             */
/* ------------------------------------------------------------------------ */

/* Exact-phase table: cs[2 r] = cos(2 pi r / n), cs[2 r + 1] = sin(2 pi r / n),
 * r = 0 .. n-1.  The phase of (j, m) is looked up at r = (j m) mod n. */
static double *phase_table(int n) {
  double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  if (!cs) return NULL;
  for (int r = 0; r < n; r++) {
    double ph = 2.0 * ORC_PI * (double)r / (double)n;
    cs[2 * r] = cos(ph);
    cs[2 * r + 1] = sin(ph);
  }
  return cs;
}

/* F(m) = sum_j u_j exp(-2 pi i j m / n), m < M. */
static void dft_forward(int n, int M, const double *cs, const double *u,
                        double *F) {
  for (int m = 0; m < M; m++) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < n; j++) {
      size_t r = (size_t)(((int64_t)j * (int64_t)m) % n);
      re += u[j] * cs[2 * r];
      im -= u[j] * cs[2 * r + 1];
    }
    F[2 * m] = re;
    F[2 * m + 1] = im;
  }
}

/* weight of mode m in the real inverse: 1 for m = 0 and for the Nyquist
 * mode m = n/2 (n even), 2 otherwise */
static double mode_weight(int m, int n) {
  if (m == 0) return 1.0;
  if ((n % 2 == 0) && (2 * m == n)) return 1.0;
  return 2.0;
}

/* u_j = sum_m c_m Re(G(m) e^{2 pi i j m / n}) with caller-provided c_m. */
static void dft_real_synthesis(int n, int M, const double *cs, const double *G,
                               const double *c, double *u) {
  for (int j = 0; j < n; j++) {
    double acc = 0.0;
    for (int m = 0; m < M; m++) {
      size_t r = (size_t)(((int64_t)j * (int64_t)m) % n);
      acc += c[m] * (G[2 * m] * cs[2 * r] - G[2 * m + 1] * cs[2 * r + 1]);
    }
    u[j] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* Forward / inverse SHT and their adjoints                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nlat, nlon, L, M;
  double *x, *s, *w; /* nodes, sin(theta), latitude weights */
  double *cs;        /* exact-phase table */
  double *a, *b;     /* recurrence coefficients */
} orc_geom;

static int geom_init(orc_geom *g, int nlat, int nlon, int grid, int L, int M) {
  memset(g, 0, sizeof(*g));
  g->nlat = nlat;
  g->nlon = nlon;
  g->L = L;
  g->M = M;
  g->x = (double *)malloc(sizeof(double) * nlat);
  g->s = (double *)malloc(sizeof(double) * nlat);
  g->w = (double *)malloc(sizeof(double) * nlat);
  g->cs = phase_table(nlon);
  g->a = (double *)malloc(sizeof(double) * (size_t)L * M);
  g->b = (double *)malloc(sizeof(double) * (size_t)L * M);
  if (!g->x || !g->s || !g->w || !g->cs || !g->a || !g->b) return -2;
  legendre_coeffs(L, M, g->a, g->b);
  return orc_grid(grid, nlat, g->x, g->s, g->w);
}

static void geom_free(orc_geom *g) {
  free(g->x);
  free(g->s);
  free(g->w);
  free(g->cs);
  free(g->a);
  free(g->b);
}

static int check_sizes(int nlat, int nlon, int L, int M) {
  if (nlat < 1 || nlon < 1 || L < 1 || M < 1) return -1;
  if (M > L) return -1;
  if (M > nlon / 2 + 1) return -1;
  return 0;
}

/* Shared body of the forward SHT and of the inverse-SHT adjoint (analysis):
 *   out_lm = sum_k q_k Phat_l^m(x_k) c_m F_k(m),  F_k(m) = sum_j u_kj e^{-i m phi_j}
 * forward: q_k = w_k 2 pi / nlon, c_m = 1;
 * inverse adjoint: q_k = 1, c_m = mode weight of the real inverse. */
static int analysis(int nlat, int nlon, int grid, int L, int M, int B,
                    const double *x, double *xhat, int adjoint, int k0, int k1) {
  if (check_sizes(nlat, nlon, L, M)) return -1;
  if (k0 < 0 || k1 > nlat || k0 > k1) return -1;
  orc_geom g;
  int rc = geom_init(&g, nlat, nlon, grid, L, M);
  if (rc) {
    geom_free(&g);
    return rc;
  }
  const double dphi = 2.0 * ORC_PI / (double)nlon;
  size_t plm = (size_t)L * M;
  int fail = 0;
#pragma omp parallel
  {
    double *P = (double *)malloc(sizeof(double) * plm);
    double *F = (double *)malloc(sizeof(double) * 2 * (size_t)M);
    if (!P || !F) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int b = 0; b < B; b++) {
      if (!P || !F) continue;
      double *out = xhat + (size_t)b * plm * 2;
      memset(out, 0, sizeof(double) * plm * 2);
      for (int k = k0; k < k1; k++) {
        dft_forward(nlon, M, g.cs, x + ((size_t)b * nlat + k) * nlon, F);
        legendre_with(L, M, g.x[k], g.s[k], g.a, g.b, P);
        for (int m = 0; m < M; m++) {
          double q = adjoint ? mode_weight(m, nlon) : g.w[k] * dphi;
          double fr = q * F[2 * m], fi = q * F[2 * m + 1];
          for (int l = m; l < L; l++) {
            double p = P[(size_t)l * M + m];
            out[2 * ((size_t)l * M + m)] += p * fr;
            out[2 * ((size_t)l * M + m) + 1] += p * fi;
          }
        }
      }
    }
    free(P);
    free(F);
  }
  geom_free(&g);
  return fail ? -2 : 0;
}

/* Forward SHT, Eq. (sht) with the grid quadrature:
 *   xhat_lm = sum_k w_k (2 pi / nlon) Phat_l^m(x_k) F_k(m),
 *   F_k(m)  = sum_j u_kj exp(-i m phi_j).
 * x: [B][nlat][nlon], xhat: [B][L][M] complex (interleaved). */
int orc_sht_forward(int nlat, int nlon, int grid, int L, int M, int B,
                    const double *x, double *xhat) {
  return analysis(nlat, nlon, grid, L, M, B, x, xhat, 0, 0, nlat);
}

/* The forward sum restricted to latitude rows k0 <= k < k1 (a partial
 * quadrature; the full transform is the range [0, nlat)).  Used to time
 * bounded samples of the oracle. */
int orc_sht_forward_rows(int nlat, int nlon, int grid, int L, int M, int B,
                         const double *x, double *xhat, int k0, int k1) {
  return analysis(nlat, nlon, grid, L, M, B, x, xhat, 0, k0, k1);
}

/* Adjoint of the inverse SHT:
 *   Gbar_k(m) = c_m sum_j gx_kj e^{-i m phi_j},
 *   gy_lm     = sum_k Phat_l^m(x_k) Gbar_k(m)   (l >= m; zero for l < m). */
int orc_sht_inverse_adjoint(int nlat, int nlon, int grid, int L, int M, int B,
                            const double *gx, double *gy) {
  return analysis(nlat, nlon, grid, L, M, B, gx, gy, 1, 0, nlat);
}

/* Shared body of the inverse SHT and of the forward-SHT adjoint (synthesis):
 *   G_k(m) = sum_{l=m}^{L-1} Phat_l^m(x_k) yhat_lm
 *   u_kj   = r_k * sum_m c_m Re(G_k(m) e^{i m phi_j})
 * inverse: r_k = 1, c_m = mode weight; forward adjoint: r_k = w_k 2 pi / nlon,
 * c_m = 1. */
static int synthesis(int nlat, int nlon, int grid, int L, int M, int B,
                     const double *yhat, double *u, int adjoint, int k0, int k1) {
  if (check_sizes(nlat, nlon, L, M)) return -1;
  if (k0 < 0 || k1 > nlat || k0 > k1) return -1;
  orc_geom g;
  int rc = geom_init(&g, nlat, nlon, grid, L, M);
  if (rc) {
    geom_free(&g);
    return rc;
  }
  double *c = (double *)malloc(sizeof(double) * M);
  for (int m = 0; m < M; m++) c[m] = adjoint ? 1.0 : mode_weight(m, nlon);
  const double dphi = 2.0 * ORC_PI / (double)nlon;
  size_t plm = (size_t)L * M;
  int fail = 0;
#pragma omp parallel
  {
    double *P = (double *)malloc(sizeof(double) * plm);
    double *G = (double *)malloc(sizeof(double) * 2 * (size_t)M);
    if (!P || !G) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int b = 0; b < B; b++) {
      if (!P || !G) continue;
      const double *in = yhat + (size_t)b * plm * 2;
      for (int k = k0; k < k1; k++) {
        legendre_with(L, M, g.x[k], g.s[k], g.a, g.b, P);
        for (int m = 0; m < M; m++) {
          double re = 0.0, im = 0.0;
          for (int l = m; l < L; l++) {
            double p = P[(size_t)l * M + m];
            re += p * in[2 * ((size_t)l * M + m)];
            im += p * in[2 * ((size_t)l * M + m) + 1];
          }
          G[2 * m] = re;
          G[2 * m + 1] = im;
        }
        double *row = u + ((size_t)b * nlat + k) * nlon;
        dft_real_synthesis(nlon, M, g.cs, G, c, row);
        if (adjoint) {
          double q = g.w[k] * dphi;
          for (int j = 0; j < nlon; j++) row[j] *= q;
        }
      }
    }
    free(P);
    free(G);
  }
  free(c);
  geom_free(&g);
  return fail ? -2 : 0;
}

/* Inverse SHT, Eq. (isht) for a real field:
 *   u_kj = sum_m c_m Re(G_k(m) e^{i m phi_j}),
 * c_0 = 1, c_{nlon/2} = 1, c_m = 2 otherwise; Im of m = 0 (and of the
 * Nyquist mode) does not enter. */
int orc_sht_inverse(int nlat, int nlon, int grid, int L, int M, int B,
                    const double *yhat, double *u) {
  return synthesis(nlat, nlon, grid, L, M, B, yhat, u, 0, 0, nlat);
}

/* The inverse evaluated only on latitude rows k0 <= k < k1 (other rows of
 * u are left untouched). */
int orc_sht_inverse_rows(int nlat, int nlon, int grid, int L, int M, int B,
                         const double *yhat, double *u, int k0, int k1) {
  return synthesis(nlat, nlon, grid, L, M, B, yhat, u, 0, k0, k1);
}

/* Adjoint of the forward SHT under <a, b> = Re sum conj(a) b:
 *   gx_kj = w_k (2 pi / nlon) Re sum_m e^{i m phi_j} G_k(m),
 *   G_k(m) = sum_l Phat_l^m(x_k) gy_lm   (every m with weight 1). */
int orc_sht_forward_adjoint(int nlat, int nlon, int grid, int L, int M, int B,
                            const double *gy, double *gx) {
  return synthesis(nlat, nlon, grid, L, M, B, gy, gx, 1, 0, nlat);
}

/* ------------------------------------------------------------------------ */
/* Sampled evaluation (one output at a time, for full-size spot checks)     */
/* ------------------------------------------------------------------------ */

/* One forward coefficient xhat_lm of one field x[nlat][nlon]. */
int orc_sht_forward_at(int nlat, int nlon, int grid, const double *x, int l,
                       int m, double *out_re, double *out_im) {
  if (l < 0 || m < 0 || m > l || m > nlon / 2) return -1;
  orc_geom g;
  int rc = geom_init(&g, nlat, nlon, grid, l + 1, m + 1);
  if (rc) {
    geom_free(&g);
    return rc;
  }
  const double dphi = 2.0 * ORC_PI / (double)nlon;
  double re = 0.0, im = 0.0;
  double F[2];
  for (int k = 0; k < nlat; k++) {
    /* single-mode DFT of ring k */
    double fr = 0.0, fi = 0.0;
    const double *row = x + (size_t)k * nlon;
    for (int j = 0; j < nlon; j++) {
      int64_t r = ((int64_t)j * (int64_t)m) % nlon;
      double ph = 2.0 * ORC_PI * (double)r / (double)nlon;
      fr += row[j] * cos(ph);
      fi -= row[j] * sin(ph);
    }
    F[0] = fr;
    F[1] = fi;
    double p = g.w[k] * dphi * orc_legendre_one(l, m, g.x[k], g.s[k]);
    re += p * F[0];
    im += p * F[1];
  }
  geom_free(&g);
  *out_re = re;
  *out_im = im;
  return 0;
}

/* One inverse value u(k, j) from one coefficient array yhat[L][M]. */
int orc_sht_inverse_at(int nlat, int nlon, int grid, int L, int M,
                       const double *yhat, int k, int j, double *out) {
  if (check_sizes(nlat, nlon, L, M)) return -1;
  if (k < 0 || k >= nlat || j < 0 || j >= nlon) return -1;
  orc_geom g;
  int rc = geom_init(&g, nlat, nlon, grid, L, M);
  if (rc) {
    geom_free(&g);
    return rc;
  }
  double *P = (double *)malloc(sizeof(double) * (size_t)L * M);
  legendre_with(L, M, g.x[k], g.s[k], g.a, g.b, P);
  double acc = 0.0;
  for (int m = 0; m < M; m++) {
    double re = 0.0, im = 0.0;
    for (int l = m; l < L; l++) {
      double p = P[(size_t)l * M + m];
      re += p * yhat[2 * ((size_t)l * M + m)];
      im += p * yhat[2 * ((size_t)l * M + m) + 1];
    }
    int64_t r = ((int64_t)j * (int64_t)m) % nlon;
    double ph = 2.0 * ORC_PI * (double)r / (double)nlon;
    acc += mode_weight(m, nlon) * (re * cos(ph) - im * sin(ph));
  }
  free(P);
  geom_free(&g);
  *out = acc;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Unfactored quadrature (tiny grids): no DFT, no integer phase reduction    */
/* ------------------------------------------------------------------------ */

/* xhat_lm = sum_{k,j} u_kj conj(Y_lm(theta_k, phi_j)) w_k (2 pi / nlon),
 * Y_lm evaluated as Phat_l^m(x_k) (cos(m phi_j) + i sin(m phi_j)). */
int orc_sht_forward_bruteforce(int nlat, int nlon, int grid, int L, int M,
                               const double *x, double *xhat) {
  if (check_sizes(nlat, nlon, L, M)) return -1;
  orc_geom g;
  int rc = geom_init(&g, nlat, nlon, grid, L, M);
  if (rc) {
    geom_free(&g);
    return rc;
  }
  double *P = (double *)malloc(sizeof(double) * (size_t)L * M);
  memset(xhat, 0, sizeof(double) * 2 * (size_t)L * M);
  for (int k = 0; k < nlat; k++) {
    legendre_with(L, M, g.x[k], g.s[k], g.a, g.b, P);
    for (int j = 0; j < nlon; j++) {
      double phi = 2.0 * ORC_PI * (double)j / (double)nlon;
      double q = x[(size_t)k * nlon + j] * g.w[k] * (2.0 * ORC_PI / nlon);
      for (int l = 0; l < L; l++)
        for (int m = 0; m <= l && m < M; m++) {
          double y = P[(size_t)l * M + m];
          xhat[2 * ((size_t)l * M + m)] += q * y * cos(m * phi);
          xhat[2 * ((size_t)l * M + m) + 1] -= q * y * sin(m * phi);
        }
    }
  }
  free(P);
  geom_free(&g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Spectral filter and its adjoint (Eq. s2_spectral_conv, channel mixing)    */
/* ------------------------------------------------------------------------ */

/* yhat[b][o][l][m] = sum_i W[l][o][i] xhat[b][i][l][m] for m <= l (zero
 * otherwise).  Complex arrays interleaved; W: [L][Cout][Cin]. */
static int filter_range(int L, int M, int Bm, int Cin, int Cout,
                        const double *xhat, const double *W, double *yhat,
                        int l0, int l1) {
  if (L < 1 || M < 1 || Bm < 0 || Cin < 1 || Cout < 1) return -1;
  if (l0 < 0 || l1 > L || l0 > l1) return -1;
  size_t plm = (size_t)L * M;
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < Bm; b++)
    for (int o = 0; o < Cout; o++) {
      double *out = yhat + ((size_t)b * Cout + o) * plm * 2;
      for (int l = l0; l < l1; l++)
        for (int m = 0; m < M; m++) {
          double re = 0.0, im = 0.0;
          if (m <= l) {
            for (int i = 0; i < Cin; i++) {
              const double *w = W + 2 * (((size_t)l * Cout + o) * Cin + i);
              const double *xi =
                  xhat + 2 * (((size_t)b * Cin + i) * plm + (size_t)l * M + m);
              re += w[0] * xi[0] - w[1] * xi[1];
              im += w[0] * xi[1] + w[1] * xi[0];
            }
          }
          out[2 * ((size_t)l * M + m)] = re;
          out[2 * ((size_t)l * M + m) + 1] = im;
        }
    }
  return 0;
}

int orc_spectral_filter(int L, int M, int Bm, int Cin, int Cout,
                        const double *xhat, const double *W, double *yhat) {
  return filter_range(L, M, Bm, Cin, Cout, xhat, W, yhat, 0, L);
}

/* The filter evaluated only for degrees l0 <= l < l1 (other rows of yhat
 * are left untouched). */
int orc_spectral_filter_degrees(int L, int M, int Bm, int Cin, int Cout,
                                const double *xhat, const double *W,
                                double *yhat, int l0, int l1) {
  return filter_range(L, M, Bm, Cin, Cout, xhat, W, yhat, l0, l1);
}

/* Adjoint of the filter in both arguments:
 *   gx[b][i][l][m] = sum_o conj(W[l][o][i]) gy[b][o][l][m]     (m <= l)
 *   gW[l][o][i]    = sum_{b, m <= l} gy[b][o][l][m] conj(xhat[b][i][l][m])
 * Either output may be NULL. */
int orc_spectral_filter_adjoint(int L, int M, int Bm, int Cin, int Cout,
                                const double *gy, const double *W,
                                const double *xhat, double *gx, double *gW) {
  if (L < 1 || M < 1 || Bm < 0 || Cin < 1 || Cout < 1) return -1;
  size_t plm = (size_t)L * M;
  if (gx) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < Bm; b++)
      for (int i = 0; i < Cin; i++) {
        double *out = gx + ((size_t)b * Cin + i) * plm * 2;
        for (int l = 0; l < L; l++)
          for (int m = 0; m < M; m++) {
            double re = 0.0, im = 0.0;
            if (m <= l) {
              for (int o = 0; o < Cout; o++) {
                const double *w = W + 2 * (((size_t)l * Cout + o) * Cin + i);
                const double *g =
                    gy + 2 * (((size_t)b * Cout + o) * plm + (size_t)l * M + m);
                /* conj(w) * g */
                re += w[0] * g[0] + w[1] * g[1];
                im += w[0] * g[1] - w[1] * g[0];
              }
            }
            out[2 * ((size_t)l * M + m)] = re;
            out[2 * ((size_t)l * M + m) + 1] = im;
          }
      }
  }
  if (gW) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int l = 0; l < L; l++)
      for (int o = 0; o < Cout; o++)
        for (int i = 0; i < Cin; i++) {
          double re = 0.0, im = 0.0;
          for (int b = 0; b < Bm; b++)
            for (int m = 0; m <= l && m < M; m++) {
              const double *g =
                  gy + 2 * (((size_t)b * Cout + o) * plm + (size_t)l * M + m);
              const double *xi =
                  xhat + 2 * (((size_t)b * Cin + i) * plm + (size_t)l * M + m);
              /* g * conj(x) */
              re += g[0] * xi[0] + g[1] * xi[1];
              im += g[1] * xi[0] - g[0] * xi[1];
            }
          gW[2 * (((size_t)l * Cout + o) * Cin + i)] = re;
          gW[2 * (((size_t)l * Cout + o) * Cin + i) + 1] = im;
        }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported for the pin tests                                                */
/* ------------------------------------------------------------------------ */

/* Longitude DFT of one ring, F(m) = sum_j u_j e^{-2 pi i j m / n}, m < M. */
int orc_dft(int n, int M, const double *u, double *F) {
  double *cs = phase_table(n);
  if (!cs) return -2;
  dft_forward(n, M, cs, u, F);
  free(cs);
  return 0;
}
