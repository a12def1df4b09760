/*
 * FP64 CPU oracle for the PA-SFM differentiable acoustic radiation operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (paper, Appendix A and Section 2 "Differentiable Acoustic
 * Radiation"):
 *
 *  - Each voxel k is a uniform sphere of radius a0 and amplitude P_c^(k).  Seen
 *    from an observation point at distance r > a0 it radiates the N-shaped pulse
 *    of the uniform-spherical-source closed form (Appendix A, "Uniform Spherical
 *    Source"):  p = P_c (r - v_s t) / (2 r)  for  r - a0 <= v_s t <= r + a0,
 *    else 0.  For this source the far-field form (Appendix A, Eq. far_field_general)
 *    is exact, and the discrete model (Appendix A, Eq. gpu_forward_model) sums it
 *    over all voxels.
 *  - Written in the distance variable tau = c t and w = tau - d, the pulse is
 *    P(d, tau) = -w / (2 d) for |w| <= a0.  Sample n of an element's trace is
 *    that pulse averaged over the sample interval [tau_n - h/2, tau_n + h/2],
 *    h = c / fs, tau_n = c (t0 + n / fs).  Integrating the linear pulse gives
 *        W(d, n) = (w_lo^2 - w_hi^2) / (4 d h),
 *    w_lo = clamp(tau_n - h/2 - d, -a0, a0), w_hi = clamp(tau_n + h/2 - d, -a0, a0).
 *    (Reading: the paper samples on a (detector, time) grid without saying how;
 *    point samples of a discontinuous pulse are ill-posed for gradients, so
 *    samples are interval averages.  A point-sample flag is kept for comparison.)
 *  - Gaussian kernel (Eq. 1 and Appendix A, Eq. gaussian_far_field with the
 *    kernel K_G of Eq. gpu_forward_model): each voxel radiates the outgoing
 *    Gaussian pulse P(d, tau) = -w / (2 d) exp(-w^2 / (2 sigma^2)), w = tau - d,
 *    truncated to |w| <= rho = 4 sigma (reading: the paper states no support).
 *    Averaged over a sample interval, with E(w) = exp(-w^2 / (2 sigma^2)) and
 *    wl, wh clamped to [-rho, rho] as above (the antiderivative of
 *    -w E(w) / (2 d) is sigma^2 E(w) / (2 d)):
 *        W(d, n) = sigma^2 (E(wh) - E(wl)) / (2 d h).
 *    The uniform sphere is the same formula with the antiderivative -w^2/(4 d)
 *    and rho = a0.
 *  - Element j of frame f sits at x_fj = R_f e_j + t_f (rigid model, Stage 4).
 *    Voxel centres are r_i = Rv (o + D (ix, iy, iz)) + tv; (Rv, tv) is identity
 *    in normal use and exists only for the rigid-invariance check.
 *  - forward:   s[f][j][n] = sum_i p0_i W(|x_fj - r_i|, n)            (Eq. 1)
 *  - adjoint:   v_i        = sum_{f,j,n} g[f][j][n] W(|x_fj - r_i|, n)
 *  - pose grad: G_fj = sum_i p0_i sum_n g[f][j][n] dW/dd (x_fj - r_i)/d,
 *               dL/dv_f = sum_j G_fj, dL/dw_f = sum_j x_fj x G_fj
 *    for the left perturbation x -> Exp(w) x + v about the world origin
 *    (reading of the Stage 4 rigid parameters as an se(3) twist).
 *  - loss head: g = mask (s - S), L = 1/2 sum g^2 (data term of Eq. 2).
 *
 * Every sum is a plain FP64 loop; pairs are visited in the obvious order.  The
 * sample loop visits a superset of the support and lets the clamps produce
 * exact zeros outside it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t nx, ny, nz;
  int32_t n_elem, n_frames, n_samples;
  double dx, dy, dz;
  double ox, oy, oz;
  double fs, t0, c, a0;
  int32_t point_sampling; /* 0: interval averages (default); 1: point samples */
  int32_t kernel;         /* 0: uniform sphere of radius a0; 1: Gaussian of width sigma */
  double vol_pose[12];    /* [Rv | tv] row-major; identity for normal use      */
  double sigma;           /* Gaussian width (mm), kernel 1 only                */
} oracle_geom;

static double clampd(double w, double a) { return w < -a ? -a : (w > a ? a : w); }

/* Half-width of a voxel's pulse in the distance variable: a0, or 4 sigma. */
double oracle_support(const oracle_geom* g) { return g->kernel == 1 ? 4.0 * g->sigma : g->a0; }

/* Unit-amplitude pulse at w = tau - d (zero outside the support). */
static double point_pulse(const oracle_geom* g, double d, double w) {
  const double rho = oracle_support(g);
  if (fabs(w) > rho) return 0.0;
  if (g->kernel == 1) return -w / (2.0 * d) * exp(-w * w / (2.0 * g->sigma * g->sigma));
  return -w / (2.0 * d);
}

/* Antiderivative in w of the pulse times 2 d, at a clamped w:
 * sphere -w^2 / 2, Gaussian sigma^2 E(w). */
static double prim(const oracle_geom* g, double w) {
  if (g->kernel == 1) return g->sigma * g->sigma * exp(-w * w / (2.0 * g->sigma * g->sigma));
  return -0.5 * w * w;
}

/* Its w-derivative, -w for the sphere and -w E(w) for the Gaussian. */
static double prim_dw(const oracle_geom* g, double w) {
  if (g->kernel == 1) return -w * exp(-w * w / (2.0 * g->sigma * g->sigma));
  return -w;
}

/* Sample n of the pulse of a unit-amplitude voxel observed at distance d. */
double oracle_pulse(const oracle_geom* g, double d, int n) {
  const double h = g->c / g->fs;
  const double tau = g->c * (g->t0 + (double)n / g->fs);
  if (g->point_sampling) return point_pulse(g, d, tau - d);
  const double rho = oracle_support(g);
  const double wl = clampd(tau - 0.5 * h - d, rho);
  const double wh = clampd(tau + 0.5 * h - d, rho);
  return (prim(g, wh) - prim(g, wl)) / (2.0 * d * h);
}

/* d/dd of oracle_pulse (interval averages).  A clamped end contributes nothing;
 * an end strictly inside the support moves with d (dw/dd = -1). */
double oracle_pulse_dd(const oracle_geom* g, double d, int n) {
  const double h = g->c / g->fs;
  const double tau = g->c * (g->t0 + (double)n / g->fs);
  const double rho = oracle_support(g);
  const double rl = tau - 0.5 * h - d, rh = tau + 0.5 * h - d;
  const double wl = clampd(rl, rho), wh = clampd(rh, rho);
  const double W = (prim(g, wh) - prim(g, wl)) / (2.0 * d * h);
  const double dl = fabs(rl) < rho ? -prim_dw(g, wl) : 0.0; /* d prim(wl) / dd */
  const double dh = fabs(rh) < rho ? -prim_dw(g, wh) : 0.0; /* d prim(wh) / dd */
  return (dh - dl) / (2.0 * d * h) - W / d;
}

/* Superset [*lo, *hi] of the samples whose interval meets [d - rho, d + rho]. */
static int sample_range(const oracle_geom* g, double d, int* lo, int* hi) {
  const double h = g->c / g->fs, tau0 = g->c * g->t0, rho = oracle_support(g);
  double a = floor((d - rho - tau0) / h - 0.5) - 1.0;
  double b = ceil((d + rho - tau0) / h + 0.5) + 1.0;
  if (a < 0) a = 0;
  if (b > g->n_samples - 1) b = g->n_samples - 1;
  if (a > b) return 0;
  *lo = (int)a;
  *hi = (int)b;
  return 1;
}

static void voxel_centre(const oracle_geom* g, int ix, int iy, int iz, double r[3]) {
  const double p[3] = {g->ox + g->dx * ix, g->oy + g->dy * iy, g->oz + g->dz * iz};
  const double* V = g->vol_pose;
  for (int a = 0; a < 3; ++a) r[a] = V[4 * a] * p[0] + V[4 * a + 1] * p[1] + V[4 * a + 2] * p[2] + V[4 * a + 3];
}

static double dist3(const double x[3], const double r[3]) {
  const double a = x[0] - r[0], b = x[1] - r[1], c = x[2] - r[2];
  return sqrt(a * a + b * b + c * c);
}

/* x[f][j][3] = R_f e_j + t_f. */
void oracle_element_positions(const oracle_geom* g, const double* elem, const double* pose, double* xw) {
  for (int f = 0; f < g->n_frames; ++f)
    for (int j = 0; j < g->n_elem; ++j) {
      const double* P = pose + 12 * f;
      const double* e = elem + 3 * j;
      double* x = xw + 3 * ((int64_t)f * g->n_elem + j);
      for (int a = 0; a < 3; ++a) x[a] = P[4 * a] * e[0] + P[4 * a + 1] * e[1] + P[4 * a + 2] * e[2] + P[4 * a + 3];
    }
}

/* Returns the number of pairs with d <= rho (observation point inside a voxel's
 * support, where the exterior / far-field form does not hold). */
static int64_t count_inside(const oracle_geom* g, const double* xw, int64_t fj0, int64_t fj1) {
  int64_t bad = 0;
  for (int64_t fj = fj0; fj < fj1; ++fj)
    for (int iz = 0; iz < g->nz; ++iz)
      for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
          double r[3];
          voxel_centre(g, ix, iy, iz, r);
          if (dist3(xw + 3 * fj, r) <= oracle_support(g)) ++bad;
        }
  return bad;
}

int64_t oracle_check_geometry(const oracle_geom* g, const double* xw) {
  return count_inside(g, xw, 0, (int64_t)g->n_frames * g->n_elem);
}

/* Forward for the (frame, element) rows listed in rows[0..n_rows) (all rows if
 * rows == NULL); sig is [n_rows][Nt] in the listed order. */
void oracle_forward_rows(const oracle_geom* g, const float* p0, const double* xw,
                         const int64_t* rows, int64_t n_rows, double* sig) {
  const int64_t nrow = rows ? n_rows : (int64_t)g->n_frames * g->n_elem;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < nrow; ++k) {
    const int64_t fj = rows ? rows[k] : k;
    const double* x = xw + 3 * fj;
    double* s = sig + k * g->n_samples;
    memset(s, 0, sizeof(double) * g->n_samples);
    for (int iz = 0; iz < g->nz; ++iz)
      for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
          const double p = p0[((int64_t)iz * g->ny + iy) * g->nx + ix];
          if (p == 0.0) continue;
          double r[3];
          voxel_centre(g, ix, iy, iz, r);
          const double d = dist3(x, r);
          int lo, hi;
          if (!sample_range(g, d, &lo, &hi)) continue;
          for (int n = lo; n <= hi; ++n) s[n] += p * oracle_pulse(g, d, n);
        }
  }
}

void oracle_forward(const oracle_geom* g, const float* p0, const double* xw, double* sig) {
  oracle_forward_rows(g, p0, xw, NULL, 0, sig);
}

/* Adjoint for the voxels listed in vox[0..n_vox) (all voxels if vox == NULL). */
void oracle_adjoint_voxels(const oracle_geom* g, const double* gsig, const double* xw,
                           const int64_t* vox, int64_t n_vox, double* out) {
  const int64_t nv = vox ? n_vox : (int64_t)g->nx * g->ny * g->nz;
  const int64_t nfj = (int64_t)g->n_frames * g->n_elem;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < nv; ++k) {
    const int64_t i = vox ? vox[k] : k;
    const int ix = (int)(i % g->nx), iy = (int)((i / g->nx) % g->ny), iz = (int)(i / ((int64_t)g->nx * g->ny));
    double r[3];
    voxel_centre(g, ix, iy, iz, r);
    double acc = 0.0;
    for (int64_t fj = 0; fj < nfj; ++fj) {
      const double d = dist3(xw + 3 * fj, r);
      int lo, hi;
      if (!sample_range(g, d, &lo, &hi)) continue;
      const double* gs = gsig + fj * g->n_samples;
      for (int n = lo; n <= hi; ++n) acc += gs[n] * oracle_pulse(g, d, n);
    }
    out[k] = acc;
  }
}

void oracle_adjoint(const oracle_geom* g, const double* gsig, const double* xw, double* vol) {
  oracle_adjoint_voxels(g, gsig, xw, NULL, 0, vol);
}

/* Element-position gradient of one (frame, element) trace:
 * G = sum_i p0_i sum_n g[n] dW/dd (x - r_i) / d. */
static void element_gradient(const oracle_geom* g, const float* p0, const double* gs, const double* x,
                             double G[3]) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int iz = 0; iz < g->nz; ++iz)
    for (int iy = 0; iy < g->ny; ++iy)
      for (int ix = 0; ix < g->nx; ++ix) {
        const double p = p0[((int64_t)iz * g->ny + iy) * g->nx + ix];
        if (p == 0.0) continue;
        double r[3];
        voxel_centre(g, ix, iy, iz, r);
        const double d = dist3(x, r);
        int lo, hi;
        if (!sample_range(g, d, &lo, &hi)) continue;
        double s = 0.0;
        for (int n = lo; n <= hi; ++n) s += gs[n] * oracle_pulse_dd(g, d, n);
        for (int a = 0; a < 3; ++a) acc[a] += p * s * (x[a] - r[a]) / d;
      }
  for (int a = 0; a < 3; ++a) G[a] = acc[a];
}

/* Element gradients for the (frame, element) rows listed in rows[0..n_rows);
 * gsig holds the full [F][E][Nt] residual; G is [n_rows][3]. */
void oracle_element_gradient_rows(const oracle_geom* g, const float* p0, const double* gsig, const double* xw,
                                  const int64_t* rows, int64_t n_rows, double* G) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n_rows; ++k)
    element_gradient(g, p0, gsig + rows[k] * g->n_samples, xw + 3 * rows[k], G + 3 * k);
}

/* Element gradients with their one-sided ambiguity at the support edges.
 * dW/dd jumps where a sample-interval boundary w_b = tau_b - h/2 - d crosses
 * +-rho (the strict rule counts a boundary as moving with d only if |w_b| < rho).
 * For boundaries within eps (mm) of +-rho both one-sided values are admissible:
 * boundary b then adds c_b = (g_b - g_{b-1}) F'(clamp(w_b)) / (2 d h) to
 * (F' the w-derivative of the pulse antiderivative: -w, or -w E(w))
 * sum_n g_n dW_n/dd, or nothing.  Gmid takes half of every such c_b and Ghalf
 * their half-magnitudes (componentwise, times |x - r| / d), so every choice of
 * sides lies in [Gmid - Ghalf, Gmid + Ghalf].  With eps = 0, Gmid equals the
 * strict gradient and Ghalf is 0.  namb (may be NULL) receives per row the number
 * of such boundaries whose c_b is not zero: a row with none has a single
 * admissible gradient, the strict one. */
void oracle_element_gradient_bounds(const oracle_geom* g, const float* p0, const double* gsig,
                                    const double* xw, const int64_t* rows, int64_t n_rows, double eps,
                                    double* Gmid, double* Ghalf, int64_t* namb) {
  const double h = g->c / g->fs, rho = oracle_support(g);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < n_rows; ++k) {
    const double* x = xw + 3 * rows[k];
    const double* gs = gsig + rows[k] * g->n_samples;
    double mid[3] = {0, 0, 0}, half[3] = {0, 0, 0};
    int64_t count = 0;
    for (int iz = 0; iz < g->nz; ++iz)
      for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
          const double p = p0[((int64_t)iz * g->ny + iy) * g->nx + ix];
          if (p == 0.0) continue;
          double r[3];
          voxel_centre(g, ix, iy, iz, r);
          const double d = dist3(x, r);
          int lo, hi;
          if (!sample_range(g, d, &lo, &hi)) continue;
          double s = 0.0, amb = 0.0;
          for (int n = lo; n <= hi; ++n) s += gs[n] * oracle_pulse_dd(g, d, n);
          for (int b = lo; b <= hi + 1; ++b) {
            const double wb = g->c * (g->t0 + (double)b / g->fs) - 0.5 * h - d;
            if (fabs(fabs(wb) - rho) >= eps) continue;
            const double gb = b <= hi ? gs[b] : 0.0, gbm = b - 1 >= lo ? gs[b - 1] : 0.0;
            const double cb = (gb - gbm) * prim_dw(g, clampd(wb, rho)) / (2.0 * d * h);
            const double strict = fabs(wb) < rho ? cb : 0.0;
            s += 0.5 * cb - strict;
            amb += 0.5 * fabs(cb);
            if (cb != 0.0) ++count;
          }
          for (int a = 0; a < 3; ++a) {
            mid[a] += p * s * (x[a] - r[a]) / d;
            half[a] += fabs(p) * amb * fabs(x[a] - r[a]) / d;
          }
        }
    for (int a = 0; a < 3; ++a) {
      Gmid[3 * k + a] = mid[a];
      Ghalf[3 * k + a] = half[a];
    }
    if (namb) namb[k] = count;
  }
}

/* Element-position gradient G[f][j][3] and twist gradient grad6[f][6] = (w, v).
 * mask (may be NULL) zeroes whole (frame, element) traces of g. */
void oracle_pose_grad(const oracle_geom* g, const float* p0, const double* gsig, const double* xw,
                      const uint8_t* mask, double* grad6, double* gelem) {
  const int64_t nfj = (int64_t)g->n_frames * g->n_elem;
  double* G = gelem ? gelem : (double*)malloc(sizeof(double) * 3 * (size_t)(nfj > 0 ? nfj : 1));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t fj = 0; fj < nfj; ++fj) {
    if (!mask || mask[fj]) {
      element_gradient(g, p0, gsig + fj * g->n_samples, xw + 3 * fj, G + 3 * fj);
    } else {
      G[3 * fj] = G[3 * fj + 1] = G[3 * fj + 2] = 0.0;
    }
  }
  for (int f = 0; f < g->n_frames; ++f) {
    double w[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    for (int j = 0; j < g->n_elem; ++j) {
      const double* x = xw + 3 * ((int64_t)f * g->n_elem + j);
      const double* Gj = G + 3 * ((int64_t)f * g->n_elem + j);
      w[0] += x[1] * Gj[2] - x[2] * Gj[1];
      w[1] += x[2] * Gj[0] - x[0] * Gj[2];
      w[2] += x[0] * Gj[1] - x[1] * Gj[0];
      for (int a = 0; a < 3; ++a) v[a] += Gj[a];
    }
    for (int a = 0; a < 3; ++a) {
      grad6[6 * f + a] = w[a];
      grad6[6 * f + 3 + a] = v[a];
    }
  }
  if (!gelem) free(G);
}

/* g = mask (s - S); returns L = 1/2 sum g^2. */
double oracle_loss(const oracle_geom* g, const double* sig, const double* meas, const uint8_t* mask, double* gout) {
  const int64_t nfj = (int64_t)g->n_frames * g->n_elem;
  double L = 0.0;
  for (int64_t fj = 0; fj < nfj; ++fj)
    for (int n = 0; n < g->n_samples; ++n) {
      const int64_t k = fj * g->n_samples + n;
      const double r = (!mask || mask[fj]) ? sig[k] - meas[k] : 0.0;
      gout[k] = r;
      L += 0.5 * r * r;
    }
  return L;
}

int oracle_abi_version(void) { return 2; }
