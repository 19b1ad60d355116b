/*
 * lens_oracle.c -- plain, slow FP64 CPU oracle for the parametric lens model.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant table with
 * the CUDA path.
 *
 * What it computes (Schaefer, Fourestey & Kneib, "Lenstool-HPC"):
 *   - lens equation beta = theta - alpha(theta)                 (Sec. 2.1, Eq. 1)
 *   - alpha = grad psi, kappa = (psi_xx + psi_yy)/2              (Sec. 2.1; Sec. 2.4 Eq. 7)
 *   - Jacobian A^-1 = [[1-k-g1, -g2], [-g2, 1-k+g1]], mu = 1/det (Sec. 2.1, Eqs. 4-5)
 *   - gamma1 = (psi_xx - psi_yy)/2, gamma2 = psi_xy           (Sec. 2.1 Eq. 4; Sec. 2.4 Eq. 8,
 *                                                                read as gamma^2 = g1^2 + g2^2)
 *   - the total gradient is the sum of the per-potential gradients (Sec. 4.1, Eq. 10)
 *   - chi2 = sum_i sum_j |c_ij - x_ij|^2 / sigma_ij^2          (Sec. 2.2, Eq. 6)
 *   - source estimate = barycentre of the back-traced images   (Sec. 2.2, Fig. 3)
 *   - brute-force image search: ray-shoot a triangulated image-plane grid to
 *     the source plane, test each triangle for the source and refine a hit by
 *     subdividing it                                             (Sec. 2.3, Fig. 4;
 *     Sec. 4.2, Fig. 8)
 *
 * The paper gives no profile formulas; it cites Eliasdottir et al. (2007) for
 * the parametric sub-halos (Sec. 2.2).  The dPIE used here is that profile,
 *   kappa = (b0/2) [ (rc^2 + rho^2)^-1/2 - (rt^2 + rho^2)^-1/2 ],
 *   rho^2 = x^2/(1+e)^2 + y^2/(1-e)^2   (halo frame, x on the major axis),
 * written as the difference of two pseudo-isothermal elliptical mass
 * distributions PIEMD(b, q, s) with kappa = (b/2)/sqrt(s^2 + x^2 + y^2/q^2)
 * (Kassiola & Kovner 1993), b = b0(1+e), q = (1-e)/(1+e), s = rc(1+e) and
 * s = rt(1+e).  PIEMD deflection, Hessian and potential follow the
 * softened-isothermal-ellipsoid expressions of Keeton (2001,
 * astro-ph/0102341), with u = sqrt(1-q^2) = 2 sqrt(e)/(1+e):
 *   alpha_x = (b q/u) atan (u x/(psi + s)),
 *   alpha_y = (b q/u) atanh(u y/(psi + q^2 s)),  psi^2 = q^2(s^2 + x^2) + y^2,
 *   psi_xx = b q (q^2 s^2 + y^2 + s psi)/(psi D),
 *   psi_yy = b q (s^2 + x^2 + s psi)/(psi D),
 *   psi_xy = -b q x y/(psi D),  D = (1+q^2) s^2 + 2 psi s + x^2 + y^2,
 *   phi    = x alpha_x + y alpha_y - b q s ln sqrt((psi + s)^2 + u^2 x^2).
 * SIS: alpha = b theta/|theta|.  Point mass: alpha = b^2 theta/|theta|^2
 * (b = Einstein radius).  At the exact centre of an SIS or point mass the
 * oracle returns zero deflection and Hessian.
 *
 * Precision: every quantity in double; sums are taken in halo order with no
 * compensation.  No blocking or reordering beyond the formulas above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_DPIE = 0, OR_SIS = 1, OR_POINT = 2 };

/* Image search: subdivisions of a hit triangle before Newton, how far
 * outside every sub-triangle (in barycentric weight) the source may be
 * before the refinement stops, and how far (in cell sizes) a root may lie
 * from the hit triangle's centroid. */
#define SUBDIV_LEVELS 6
#define SUBDIV_TOL 1e-3
#define LOCAL_CELLS 2.0

/* One potential, same field order as the halo table rows. */
typedef struct {
  int32_t type;
  double x0, y0, theta, eps, rcore, rcut, b0;
} or_halo;

/* Constraint table: source i owns images off[i] .. off[i+1]-1. */
typedef struct {
  int32_t nsrc;
  const int32_t *off;
  const double *x, *y, *sigma, *dls_ds;
} or_constraints;

typedef struct {
  double xmin, xmax, ymin, ymax;
  int32_t nx, ny;
} or_grid;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads used by later calls (timing a single core); n < 1 is ignored. */
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* atan(u t)/u and atanh(u t)/u; for tiny u the quotient is 0/0 in floating
 * point, so use the Taylor series (|u t| < u < 1e-4: the first dropped term is
 * below 1e-24 relative). */
static double atan_over_u(double u, double t) {
  if (u < 1e-4) {
    double z2 = (u * t) * (u * t);
    return t * (1.0 - z2 / 3.0 + z2 * z2 / 5.0);
  }
  return atan(u * t) / u;
}
static double atanh_over_u(double u, double t) {
  if (u < 1e-4) {
    double z2 = (u * t) * (u * t);
    return t * (1.0 + z2 / 3.0 + z2 * z2 / 5.0);
  }
  return atanh(u * t) / u;
}

/* One PIEMD(b, q, s) in its own frame: out = {ax, ay, hxx, hyy, hxy}. */
static void piemd_eval(double b, double q, double u, double s, double x, double y, double out[5]) {
  double psi = sqrt(q * q * (s * s + x * x) + y * y);
  out[0] = b * q * atan_over_u(u, x / (psi + s));
  out[1] = b * q * atanh_over_u(u, y / (psi + q * q * s));
  double D = (1.0 + q * q) * s * s + 2.0 * psi * s + x * x + y * y;
  double f = b * q / (psi * D);
  out[2] = f * (q * q * s * s + y * y + s * psi);
  out[3] = f * (s * s + x * x + s * psi);
  out[4] = -f * x * y;
}

static double piemd_potential(double b, double q, double u, double s, double x, double y) {
  double psi = sqrt(q * q * (s * s + x * x) + y * y);
  double ax = b * q * atan_over_u(u, x / (psi + s));
  double ay = b * q * atanh_over_u(u, y / (psi + q * q * s));
  double w = (psi + s) * (psi + s) + u * u * x * x;
  return x * ax + y * ay - b * q * s * 0.5 * log(w);
}

/* dPIE shape constants from the user parameters. */
static void dpie_shape(const or_halo *h, double *b, double *q, double *u, double *sc, double *st) {
  double e = h->eps;
  *q = (1.0 - e) / (1.0 + e);
  *u = 2.0 * sqrt(e) / (1.0 + e); /* = sqrt(1 - q^2) without cancellation */
  *b = h->b0 * (1.0 + e);
  *sc = h->rcore * (1.0 + e);
  *st = h->rcut * (1.0 + e);
}

/* Deflection and Hessian of one potential at (X, Y) for D_ls/D_s = 1, in the
 * sky frame: out = {ax, ay, hxx, hyy, hxy}. */
void or_halo_eval(const or_halo *h, double X, double Y, double out[5]) {
  double dX = X - h->x0, dY = Y - h->y0;
  if (h->type == OR_SIS || h->type == OR_POINT) {
    double r2 = dX * dX + dY * dY;
    if (r2 == 0.0) {
      memset(out, 0, 5 * sizeof(double));
      return;
    }
    double r = sqrt(r2);
    if (h->type == OR_SIS) {
      double b = h->b0, r3 = r2 * r;
      out[0] = b * dX / r;
      out[1] = b * dY / r;
      out[2] = b * dY * dY / r3;
      out[3] = b * dX * dX / r3;
      out[4] = -b * dX * dY / r3;
    } else {
      double te2 = h->b0 * h->b0, r4 = r2 * r2;
      out[0] = te2 * dX / r2;
      out[1] = te2 * dY / r2;
      out[2] = te2 * (dY * dY - dX * dX) / r4;
      out[3] = te2 * (dX * dX - dY * dY) / r4;
      out[4] = -2.0 * te2 * dX * dY / r4;
    }
    return;
  }
  double c = cos(h->theta), s = sin(h->theta);
  double x = c * dX + s * dY, y = -s * dX + c * dY; /* halo frame */
  double b, q, u, sc, st, core[5], cut[5], p[5];
  dpie_shape(h, &b, &q, &u, &sc, &st);
  piemd_eval(b, q, u, sc, x, y, core);
  piemd_eval(b, q, u, st, x, y, cut);
  for (int k = 0; k < 5; ++k) p[k] = core[k] - cut[k];
  /* back to the sky frame: alpha = R^T alpha', H = R^T H' R */
  out[0] = c * p[0] - s * p[1];
  out[1] = s * p[0] + c * p[1];
  out[2] = c * c * p[2] - 2.0 * c * s * p[4] + s * s * p[3];
  out[3] = s * s * p[2] + 2.0 * c * s * p[4] + c * c * p[3];
  out[4] = c * s * (p[2] - p[3]) + (c * c - s * s) * p[4];
}

/* Lensing potential of one potential at (X, Y), D_ls/D_s = 1, up to a constant. */
double or_halo_potential(const or_halo *h, double X, double Y) {
  double dX = X - h->x0, dY = Y - h->y0;
  double r2 = dX * dX + dY * dY;
  if (h->type == OR_SIS) return h->b0 * sqrt(r2);
  if (h->type == OR_POINT) return r2 > 0.0 ? h->b0 * h->b0 * 0.5 * log(r2) : 0.0;
  double c = cos(h->theta), s = sin(h->theta);
  double x = c * dX + s * dY, y = -s * dX + c * dY;
  double b, q, u, sc, st;
  dpie_shape(h, &b, &q, &u, &sc, &st);
  return piemd_potential(b, q, u, sc, x, y) - piemd_potential(b, q, u, st, x, y);
}

/* Surface density straight from the profile definitions (not via the
 * Hessian): dPIE item above, SIS b/(2r), point mass 0 away from the centre. */
double or_halo_kappa(const or_halo *h, double X, double Y) {
  double dX = X - h->x0, dY = Y - h->y0;
  if (h->type == OR_SIS) return 0.5 * h->b0 / sqrt(dX * dX + dY * dY);
  if (h->type == OR_POINT) return 0.0;
  double c = cos(h->theta), s = sin(h->theta);
  double x = c * dX + s * dY, y = -s * dX + c * dY;
  double e = h->eps;
  double rho2 = x * x / ((1 + e) * (1 + e)) + y * y / ((1 - e) * (1 - e));
  return 0.5 * h->b0 * (1.0 / sqrt(h->rcore * h->rcore + rho2) - 1.0 / sqrt(h->rcut * h->rcut + rho2));
}

/* Sum over all potentials, in halo order, scaled by D_ls/D_s (Sec. 4.1 Eq. 10). */
void or_model_eval(const or_halo *h, int32_t n, double X, double Y, double dls_ds, double out[5]) {
  double acc[5] = {0, 0, 0, 0, 0}, t[5];
  for (int32_t i = 0; i < n; ++i) {
    or_halo_eval(&h[i], X, Y, t);
    for (int k = 0; k < 5; ++k) acc[k] += t[k];
  }
  for (int k = 0; k < 5; ++k) out[k] = dls_ds * acc[k];
}

/* Vectorised helpers over arbitrary point lists (out: [npt][5] or [npt]). */
void or_model_eval_points(const or_halo *h, int32_t n, const double *X, const double *Y, int64_t npt,
                          double dls_ds, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < npt; ++p) or_model_eval(h, n, X[p], Y[p], dls_ds, out + 5 * p);
}

void or_model_potential_points(const or_halo *h, int32_t n, const double *X, const double *Y, int64_t npt,
                               double dls_ds, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < npt; ++p) {
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) acc += or_halo_potential(&h[i], X[p], Y[p]);
    out[p] = dls_ds * acc;
  }
}

void or_model_kappa_points(const or_halo *h, int32_t n, const double *X, const double *Y, int64_t npt,
                           double dls_ds, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < npt; ++p) {
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) acc += or_halo_kappa(&h[i], X[p], Y[p]);
    out[p] = dls_ds * acc;
  }
}

static double grid_x(const or_grid *g, int32_t i) {
  return g->nx > 1 ? g->xmin + i * ((g->xmax - g->xmin) / (g->nx - 1)) : g->xmin;
}
static double grid_y(const or_grid *g, int32_t j) {
  return g->ny > 1 ? g->ymin + j * ((g->ymax - g->ymin) / (g->ny - 1)) : g->ymin;
}

/* Maps over a rectangular grid with inclusive corners (Sec. 2.4; Sec. 4.1).
 * Planes [ny][nx]: nplanes = 2 -> ax, ay;  nplanes = 6 -> ax, ay, kappa,
 * gamma1, gamma2, mu with kappa/gamma from the summed Hessian (Sec. 2.4
 * Eqs. 7-9) and mu = 1/det A^-1 (Sec. 2.1 Eq. 5). */
void or_maps(const or_halo *h, int32_t n, const or_grid *g, double dls_ds, int32_t nplanes, double *out) {
  int64_t plane = (int64_t)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < g->ny; ++j) {
    for (int32_t i = 0; i < g->nx; ++i) {
      double v[5];
      or_model_eval(h, n, grid_x(g, i), grid_y(g, j), dls_ds, v);
      int64_t p = (int64_t)j * g->nx + i;
      out[p] = v[0];
      out[plane + p] = v[1];
      if (nplanes == 6) {
        double kappa = 0.5 * (v[2] + v[3]);
        double g1 = 0.5 * (v[2] - v[3]);
        double g2 = v[4];
        double det = (1.0 - kappa) * (1.0 - kappa) - g1 * g1 - g2 * g2;
        out[2 * plane + p] = kappa;
        out[3 * plane + p] = g1;
        out[4 * plane + p] = g2;
        out[5 * plane + p] = 1.0 / det;
      }
    }
  }
}

/* Parameter set -> model: halos var[0], var[1] take the 14 numbers
 * (x0, y0, eps, theta, rcore, rcut, b0) x 2; all other halos unchanged. */
void or_apply_params(const or_halo *base, int32_t n, const int32_t var[2], const double *p14, or_halo *out) {
  memcpy(out, base, (size_t)n * sizeof(or_halo));
  for (int k = 0; k < 2; ++k) {
    or_halo *h = &out[var[k]];
    const double *p = p14 + 7 * k;
    h->x0 = p[0];
    h->y0 = p[1];
    h->eps = p[2];
    h->theta = p[3];
    h->rcore = p[4];
    h->rcut = p[5];
    h->b0 = p[6];
  }
}

/* Back-trace every constraint (Sec. 2.1 Eq. 1) and form each source's
 * barycentre (Sec. 2.2, Fig. 3).  beta: [nimg][2]; bary: [nsrc][2]. */
void or_backtrace(const or_halo *h, int32_t n, const or_constraints *c, double *beta, double *bary) {
  for (int32_t i = 0; i < c->nsrc; ++i) {
    double sx = 0.0, sy = 0.0;
    int32_t m = c->off[i + 1] - c->off[i];
    for (int32_t j = c->off[i]; j < c->off[i + 1]; ++j) {
      double v[5];
      or_model_eval(h, n, c->x[j], c->y[j], c->dls_ds[i], v);
      beta[2 * j] = c->x[j] - v[0];
      beta[2 * j + 1] = c->y[j] - v[1];
      sx += beta[2 * j];
      sy += beta[2 * j + 1];
    }
    bary[2 * i] = m > 0 ? sx / m : 0.0;
    bary[2 * i + 1] = m > 0 ? sy / m : 0.0;
  }
}

/* Source-plane chi2 of one model.
 * variant 0: sum |A (bary - beta)|^2 / sigma^2 with A = (A^-1)^-1 at the
 *            image (the residual mapped to the image plane to first order);
 * variant 1: sum |bary - beta|^2 |mu| / sigma^2;
 * variant 2: sum |bary - beta|^2 / sigma^2. */
double or_chi2_source(const or_halo *h, int32_t n, const or_constraints *c, int32_t variant) {
  int32_t nimg = c->off[c->nsrc];
  double *beta = (double *)malloc(sizeof(double) * 2 * (nimg > 0 ? nimg : 1));
  double *bary = (double *)malloc(sizeof(double) * 2 * (c->nsrc > 0 ? c->nsrc : 1));
  or_backtrace(h, n, c, beta, bary);
  double chi2 = 0.0;
  for (int32_t i = 0; i < c->nsrc; ++i) {
    for (int32_t j = c->off[i]; j < c->off[i + 1]; ++j) {
      double dbx = bary[2 * i] - beta[2 * j], dby = bary[2 * i + 1] - beta[2 * j + 1];
      double s2 = c->sigma[j] * c->sigma[j];
      if (variant == 2) {
        chi2 += (dbx * dbx + dby * dby) / s2;
        continue;
      }
      double v[5];
      or_model_eval(h, n, c->x[j], c->y[j], c->dls_ds[i], v);
      /* A^-1 = I - H (Sec. 2.1 Eq. 4) */
      double a11 = 1.0 - v[2], a22 = 1.0 - v[3], a12 = -v[4];
      double det = a11 * a22 - a12 * a12;
      if (variant == 1) {
        chi2 += (dbx * dbx + dby * dby) * fabs(1.0 / det) / s2;
      } else {
        double rx = (a22 * dbx - a12 * dby) / det;
        double ry = (-a12 * dbx + a11 * dby) / det;
        chi2 += (rx * rx + ry * ry) / s2;
      }
    }
  }
  free(beta);
  free(bary);
  return chi2;
}

void or_chi2_source_batch(const or_halo *base, int32_t n, const or_constraints *c, const int32_t var[2],
                          const double *params, int32_t P, int32_t variant, double *chi2) {
#pragma omp parallel
  {
    or_halo *m = (or_halo *)malloc(sizeof(or_halo) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
    for (int32_t p = 0; p < P; ++p) {
      or_apply_params(base, n, var, params + 14 * (int64_t)p, m);
      chi2[p] = or_chi2_source(m, n, c, variant);
    }
    free(m);
  }
}

/* ---------------- brute-force image finding (Sec. 2.3, Fig. 4) ----------- */

/* Newton iteration on the lens equation with the full model:
 * theta <- theta + A(theta) (beta_s - theta + r alpha(theta)), A = (I - r H)^-1,
 * each step shortened to at most step_max (no limit if step_max <= 0).
 * Returns the iteration count on convergence (|step| < tol), -1 otherwise. */
int32_t or_newton(const or_halo *h, int32_t n, double r, double bx, double by, double *tx, double *ty,
                  int32_t maxit, double tol, double step_max) {
  double x = *tx, y = *ty;
  for (int32_t it = 1; it <= maxit; ++it) {
    double v[5];
    or_model_eval(h, n, x, y, r, v);
    double fx = bx - (x - v[0]), fy = by - (y - v[1]);
    double a11 = 1.0 - v[2], a22 = 1.0 - v[3], a12 = -v[4];
    double det = a11 * a22 - a12 * a12;
    if (det == 0.0 || !isfinite(det)) return -1;
    double dx = (a22 * fx - a12 * fy) / det;
    double dy = (-a12 * fx + a11 * fy) / det;
    double len = sqrt(dx * dx + dy * dy);
    if (step_max > 0.0 && len > step_max) { /* trust region: at most step_max per step */
      dx *= step_max / len;
      dy *= step_max / len;
    }
    x += dx;
    y += dy;
    *tx = x;
    *ty = y;
    if (sqrt(dx * dx + dy * dy) < tol) return it;
  }
  return -1;
}

/* Is p inside triangle (a, b, c)?  Signed areas taken relative to the
 * triangle's own orientation, so folded (inverted) triangles work too;
 * boundaries count as inside.  Degenerate triangles (|2 area| <= tiny) never
 * contain anything.  On a hit, w = barycentric weights of a, b, c. */
static int in_triangle(const double a[2], const double b[2], const double c[2], const double p[2], double tiny,
                       double w[3]) {
  double area2 = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
  if (fabs(area2) <= tiny) return 0;
  double wa = ((b[0] - p[0]) * (c[1] - p[1]) - (b[1] - p[1]) * (c[0] - p[0])) / area2;
  double wb = ((c[0] - p[0]) * (a[1] - p[1]) - (c[1] - p[1]) * (a[0] - p[0])) / area2;
  double wc = ((a[0] - p[0]) * (b[1] - p[1]) - (a[1] - p[1]) * (b[0] - p[0])) / area2;
  if (wa < 0.0 || wb < 0.0 || wc < 0.0) return 0;
  w[0] = wa;
  w[1] = wb;
  w[2] = wc;
  return 1;
}

/* Refine a hit (Sec. 2.3 and Sec. 4.2: the triangle holding the source is
 * subdivided): `levels` times, split the triangle into its four midpoint
 * sub-triangles (corners 0, 1, 2, then the middle one), map the three new
 * vertices to the source plane with the full model, and keep the sub-triangle
 * whose smallest barycentric weight of the source is largest (the first on a
 * tie; degenerate sub-triangles are never kept).  When no sub-triangle holds
 * the source the refinement stops at the current triangle.  th/be: image- and
 * source-plane vertices, updated in place; w: the source's barycentric
 * weights in the final triangle.  Returns the number of levels refined. */
static void tri_weights(double be[3][2], const double p[2], double tiny, double w[3]) {
  double area2 = (be[1][0] - be[0][0]) * (be[2][1] - be[0][1]) - (be[1][1] - be[0][1]) * (be[2][0] - be[0][0]);
  if (fabs(area2) <= tiny) {
    w[0] = w[1] = w[2] = 1.0 / 3.0;
    return;
  }
  w[0] = ((be[1][0] - p[0]) * (be[2][1] - p[1]) - (be[1][1] - p[1]) * (be[2][0] - p[0])) / area2;
  w[1] = ((be[2][0] - p[0]) * (be[0][1] - p[1]) - (be[2][1] - p[1]) * (be[0][0] - p[0])) / area2;
  w[2] = 1.0 - w[0] - w[1];
}

static int subdivide(const or_halo *h, int32_t n, double r, const double p[2], double th[3][2], double be[3][2],
                     int32_t levels, double tiny, double w[3]) {
  static const int sub[4][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}, {3, 4, 5}};
  static const int mid[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int32_t lev = 0;; ++lev) {
    if (lev == levels) {
      tri_weights(be, p, tiny, w);
      return lev;
    }
    double t6[6][2], b6[6][2];
    for (int k = 0; k < 3; ++k) {
      double v[5];
      t6[k][0] = th[k][0];
      t6[k][1] = th[k][1];
      b6[k][0] = be[k][0];
      b6[k][1] = be[k][1];
      t6[3 + k][0] = 0.5 * (th[mid[k][0]][0] + th[mid[k][1]][0]);
      t6[3 + k][1] = 0.5 * (th[mid[k][0]][1] + th[mid[k][1]][1]);
      or_model_eval(h, n, t6[3 + k][0], t6[3 + k][1], r, v);
      b6[3 + k][0] = t6[3 + k][0] - v[0];
      b6[3 + k][1] = t6[3 + k][1] - v[1];
    }
    const double tiny_sub = 0.25 * tiny;
    int best = -1;
    double best_score = -INFINITY;
    for (int s = 0; s < 4; ++s) {
      const double *a = b6[sub[s][0]], *b = b6[sub[s][1]], *c = b6[sub[s][2]];
      double area2 = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
      if (fabs(area2) <= tiny_sub) continue;
      double wa = ((b[0] - p[0]) * (c[1] - p[1]) - (b[1] - p[1]) * (c[0] - p[0])) / area2;
      double wb = ((c[0] - p[0]) * (a[1] - p[1]) - (c[1] - p[1]) * (a[0] - p[0])) / area2;
      double wc = 1.0 - wa - wb;
      double score = fmin(wa, fmin(wb, wc));
      if (score > best_score) {
        best_score = score;
        best = s;
      }
    }
    if (best < 0 || best_score < -SUBDIV_TOL) {
      /* no sub-triangle holds the source: the map is far from linear on this
       * triangle (a galaxy core or a fold inside); stop refining here */
      tri_weights(be, p, tiny, w);
      return lev;
    }
    for (int k = 0; k < 3; ++k) {
      th[k][0] = t6[sub[best][k]][0];
      th[k][1] = t6[sub[best][k]][1];
      be[k][0] = b6[sub[best][k]][0];
      be[k][1] = b6[sub[best][k]][1];
    }
    tiny = tiny_sub;
  }
}

/* Predicted images of one source at beta_s for distance ratio r.
 * alpha_grid: [ny][nx][2] deflection at the grid nodes for D_ls/D_s = 1.
 * Each grid cell (i, j) splits into triangles {(i,j),(i+1,j),(i+1,j+1)} and
 * {(i,j),(i+1,j+1),(i,j+1)}, visited in (j, i, k) order.  A triangle holding
 * the source is refined by SUBDIV_LEVELS subdivisions; Newton starts at the
 * source's barycentric position in the final sub-triangle.  A converged root
 * counts only if it lies within LOCAL_CELLS cell sizes of the hit triangle's
 * centroid (a root further away belongs to another triangle's search), and
 * images closer than dedup to an earlier one are dropped.  Newton steps are
 * limited to one cell size.  difficulty (may be NULL) receives per image the
 * smallest, over the candidates that reached it, of 100 x (refinement cut
 * short) + Newton iterations.
 * Returns the number of images written to img (capacity cap), or the number
 * found if it exceeds cap (the caller treats that as an overflow). */
int32_t or_find_images(const or_halo *h, int32_t n, const or_grid *g, const double *alpha_grid, double r,
                       double bx, double by, int32_t maxit, double tol, double dedup, double *img, int32_t cap,
                       int32_t *difficulty) {
  int32_t found = 0;
  double dx = (g->xmax - g->xmin) / (g->nx - 1), dy = (g->ymax - g->ymin) / (g->ny - 1);
  double tiny = 1e-14 * fabs(dx * dy);
  double p[2] = {bx, by};
  for (int32_t j = 0; j + 1 < g->ny; ++j) {
    for (int32_t i = 0; i + 1 < g->nx; ++i) {
      int32_t vi[4] = {i, i + 1, i + 1, i}, vj[4] = {j, j, j + 1, j + 1};
      double th[4][2], be[4][2];
      for (int k = 0; k < 4; ++k) {
        th[k][0] = grid_x(g, vi[k]);
        th[k][1] = grid_y(g, vj[k]);
        const double *al = alpha_grid + 2 * ((int64_t)vj[k] * g->nx + vi[k]);
        be[k][0] = th[k][0] - r * al[0];
        be[k][1] = th[k][1] - r * al[1];
      }
      static const int tri[2][3] = {{0, 1, 2}, {0, 2, 3}};
      for (int t = 0; t < 2; ++t) {
        const int *v = tri[t];
        double w[3];
        if (!in_triangle(be[v[0]], be[v[1]], be[v[2]], p, tiny, w)) continue;
        double tt[3][2], bb[3][2];
        for (int k = 0; k < 3; ++k) {
          tt[k][0] = th[v[k]][0];
          tt[k][1] = th[v[k]][1];
          bb[k][0] = be[v[k]][0];
          bb[k][1] = be[v[k]][1];
        }
        double cx = (tt[0][0] + tt[1][0] + tt[2][0]) / 3.0, cy = (tt[0][1] + tt[1][1] + tt[2][1]) / 3.0;
        const int32_t lev = subdivide(h, n, r, p, tt, bb, SUBDIV_LEVELS, tiny, w);
        double tx = w[0] * tt[0][0] + w[1] * tt[1][0] + w[2] * tt[2][0];
        double ty = w[0] * tt[0][1] + w[1] * tt[1][1] + w[2] * tt[2][1];
        const int32_t it = or_newton(h, n, r, bx, by, &tx, &ty, maxit, tol, fmax(dx, dy));
        if (it < 0) continue;
        if (hypot(tx - cx, ty - cy) > LOCAL_CELLS * fmax(dx, dy)) continue;
        /* how hard this candidate was: refinement cut short, Newton iterations */
        const int32_t diff = (lev < SUBDIV_LEVELS ? 100 : 0) + it;
        int dup = -1;
        for (int32_t k = 0; k < found && k < cap; ++k) {
          double ex = img[2 * k] - tx, ey = img[2 * k + 1] - ty;
          if (sqrt(ex * ex + ey * ey) < dedup) {
            dup = k;
            break;
          }
        }
        if (dup >= 0) {
          if (difficulty && diff < difficulty[dup]) difficulty[dup] = diff;
          continue;
        }
        if (found < cap) {
          img[2 * found] = tx;
          img[2 * found + 1] = ty;
          if (difficulty) difficulty[found] = diff;
        }
        ++found;
      }
    }
  }
  return found;
}

/* Deflection at every grid node for D_ls/D_s = 1: out [ny][nx][2]. */
void or_alpha_grid(const or_halo *h, int32_t n, const or_grid *g, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < g->ny; ++j)
    for (int32_t i = 0; i < g->nx; ++i) {
      double v[5];
      or_model_eval(h, n, grid_x(g, i), grid_y(g, j), 1.0, v);
      int64_t p = (int64_t)j * g->nx + i;
      out[2 * p] = v[0];
      out[2 * p + 1] = v[1];
    }
}

/* Image-plane chi2 of one model (Sec. 2.2 Eq. 6 with the brute-force search
 * of Sec. 2.3 / Sec. 4.2): barycentre source per constraint set, predicted
 * images by grid search + Newton, each constraint matched to the nearest
 * predicted image of its own source (ties: lower y, then lower x).
 * nfound[i] receives each source's image count; a source with no image makes
 * the chi2 NaN.  alpha_grid may be NULL (computed here). */
double or_chi2_image(const or_halo *h, int32_t n, const or_constraints *c, const or_grid *g,
                     const double *alpha_grid, int32_t maxit, double tol, double dedup, int32_t cap,
                     int32_t *nfound) {
  int32_t nimg = c->off[c->nsrc];
  double *ag = NULL;
  if (!alpha_grid) {
    ag = (double *)malloc(sizeof(double) * 2 * (size_t)g->nx * g->ny);
    or_alpha_grid(h, n, g, ag);
    alpha_grid = ag;
  }
  double *beta = (double *)malloc(sizeof(double) * 2 * (nimg > 0 ? nimg : 1));
  double *bary = (double *)malloc(sizeof(double) * 2 * (c->nsrc > 0 ? c->nsrc : 1));
  or_backtrace(h, n, c, beta, bary);
  double *chi2_i = (double *)malloc(sizeof(double) * (c->nsrc > 0 ? c->nsrc : 1));
#pragma omp parallel
  {
    double *img = (double *)malloc(sizeof(double) * 2 * (size_t)(cap > 0 ? cap : 1));
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < c->nsrc; ++i) {
      int32_t nf = or_find_images(h, n, g, alpha_grid, c->dls_ds[i], bary[2 * i], bary[2 * i + 1], maxit, tol,
                                  dedup, img, cap, NULL);
      if (nfound) nfound[i] = nf;
      double ci = 0.0;
      if (nf > cap || (nf == 0 && c->off[i + 1] > c->off[i])) ci = NAN;
      for (int32_t j = c->off[i]; j < c->off[i + 1] && nf > 0 && nf <= cap; ++j) {
        int32_t best = 0;
        double bd = INFINITY;
        for (int32_t k = 0; k < nf; ++k) {
          double ex = c->x[j] - img[2 * k], ey = c->y[j] - img[2 * k + 1];
          double d2 = ex * ex + ey * ey;
          if (d2 < bd || (d2 == bd && (img[2 * k + 1] < img[2 * best + 1] ||
                                       (img[2 * k + 1] == img[2 * best + 1] && img[2 * k] < img[2 * best])))) {
            bd = d2;
            best = k;
          }
        }
        ci += bd / (c->sigma[j] * c->sigma[j]);
      }
      chi2_i[i] = ci;
    }
    free(img);
  }
  double chi2 = 0.0;
  for (int32_t i = 0; i < c->nsrc; ++i) chi2 += chi2_i[i];
  free(chi2_i);
  free(beta);
  free(bary);
  free(ag);
  return chi2;
}

void or_chi2_image_batch(const or_halo *base, int32_t n, const or_constraints *c, const or_grid *g,
                         const int32_t var[2], const double *params, int32_t P, int32_t maxit, double tol,
                         double dedup, int32_t cap, double *chi2, int32_t *nfound) {
  or_halo *m = (or_halo *)malloc(sizeof(or_halo) * (size_t)n);
  for (int32_t p = 0; p < P; ++p) {
    or_apply_params(base, n, var, params + 14 * (int64_t)p, m);
    chi2[p] = or_chi2_image(m, n, c, g, NULL, maxit, tol, dedup, cap, nfound ? nfound + (int64_t)p * c->nsrc : NULL);
  }
  free(m);
}
