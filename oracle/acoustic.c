/*
 * acoustic.c - FP64 CPU oracle of the acoustic forward map and its exact
 * discrete adjoint. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper passages followed:
 *   - explicit recursion U_k = A(theta) U_{k-1} + F_{k-1}: Method, Eq. forward
 *   - misfit J = 1/2 sum_k |U_k - U_k^obs|^2 restricted to the receivers:
 *     Method (after Eq. forward) and Full-waveform Inversion (L2 loss)
 *   - adjoint recursion lambda_k = A^T lambda_{k+1} + (U_k - U_k^obs):
 *     Eq. adjoint-backward (equivalently Eq. ad-backward, by the Theorem)
 *   - gradient sum_k lambda_k^T (dA/dtheta) U_{k-1}: Eq. adjoint-gradient
 *   - acoustic equation u_tt = div(c^2 grad u) + f: Implementation, Eq. acoustic
 *   - Gaussian point-source re-parameterisation with sigma = dx/2:
 *     Earthquake Location and Source Time Function Retrieval
 *
 * The adjoint is written by hand, statement by statement in reverse order of
 * the forward step in acoustic_fwd_body.h.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Staggered first-derivative weights: the N odd moments of the stencil must
 * reproduce the first derivative exactly, sum_k a_k (2k-1)^(2j-1) = delta_j1
 * for j = 1..N (Taylor expansion of u(x + (2k-1)h/2) - u(x - (2k-1)h/2)).
 * Solved by Gaussian elimination with partial pivoting. */
int or_fd_coeffs(int order, double *a) {
  if (order != 2 && order != 4 && order != 6 && order != 8) return -1;
  int N = order / 2;
  double M[4][5];
  for (int j = 0; j < N; j++) {
    for (int k = 0; k < N; k++) M[j][k] = pow(2.0 * (k + 1) - 1.0, 2.0 * (j + 1) - 1.0);
    M[j][N] = (j == 0) ? 1.0 : 0.0;
  }
  for (int col = 0; col < N; col++) {
    int piv = col;
    for (int r = col + 1; r < N; r++)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    for (int k = 0; k <= N; k++) {
      double t = M[col][k];
      M[col][k] = M[piv][k];
      M[piv][k] = t;
    }
    for (int r = 0; r < N; r++) {
      if (r == col) continue;
      double f = M[r][col] / M[col][col];
      for (int k = col; k <= N; k++) M[r][k] -= f * M[col][k];
    }
  }
  for (int k = 0; k < N; k++) a[k] = M[k][N] / M[k][k];
  return 0;
}

/* Convolutional PML of Komatitsch & Martin (2007), cited in Implementation,
 * with kappa = 1, quadratic damping d(l) = d0 (l/L)^2,
 * d0 = -3 vmax ln(R) / (2 L), alpha(l) = pi f0 (1 - l/L), and recursive
 * convolution coefficients b = exp(-(d + alpha) dt), a = d (b - 1)/(d + alpha).
 * l is the distance into the layer from its inner edge (the outermost
 * physical node); outside the layer a = 0 and b = 1. */
void or_cpml_profile(int n_phys, int npml, double h, double dt, double R,
                     double vmax, double f0, int half, int n_out, double *a,
                     double *b) {
  double L = npml * h;
  for (int k = 0; k < n_out; k++) {
    a[k] = 0.0;
    b[k] = 1.0;
    if (npml <= 0) continue;
    double x = k + (half ? 0.5 : 0.0);
    double l = 0.0;
    if (npml - x > l) l = npml - x;
    if (x - (npml + n_phys - 1) > l) l = x - (npml + n_phys - 1);
    l *= h;
    if (l <= 0.0) continue;
    double d0 = -3.0 * vmax * log(R) / (2.0 * L);
    double d = d0 * (l / L) * (l / L);
    double al = M_PI * f0 * (1.0 - l / L);
    b[k] = exp(-(d + al) * dt);
    a[k] = d * (b[k] - 1.0) / (d + al);
  }
}

/* ---- real instantiation ---- */
#define REAL double
#define FN(name) name##_r
#define CEXP(x) exp(x)
#define RE(x) (x)
#include "acoustic_fwd_body.h"
#undef REAL
#undef FN
#undef CEXP
#undef RE

/* ---- complex instantiation (complex-step derivatives) ---- */
#define REAL double complex
#define FN(name) name##_c
#define CEXP(x) cexp(x)
#define RE(x) creal(x)
#include "acoustic_fwd_body.h"
#undef REAL
#undef FN
#undef CEXP
#undef RE

static int check_cfg(const or_acoustic_cfg *cfg) {
  if (cfg->nz < 1 || cfg->nx < 1 || cfg->nt < 1 || cfg->nshots < 0 || cfg->npml < 0) return -1;
  if (cfg->order != 4 && cfg->order != 8 && cfg->order != 2 && cfg->order != 6) return -1;
  if (cfg->src_kind != 0 && cfg->src_kind != 1 && cfg->src_kind != 3) return -1;
  if (cfg->src_kind == 3 && cfg->line_len < 1) return -1;
  if (cfg->op != 0 && cfg->op != 1) return -1;
  for (int r = 0; r < cfg->nrec; r++)
    if (cfg->rec_iz[r] < 0 || cfg->rec_iz[r] >= cfg->nz || cfg->rec_ix[r] < 0 || cfg->rec_ix[r] >= cfg->nx)
      return -1;
  return 0;
}

int or_acoustic_forward(const or_acoustic_cfg *cfg, const double *c,
                        const double *stf, const double *x0, double *seis) {
  if (check_cfg(cfg)) return -1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < cfg->nshots; s++)
    err |= acoustic_shot_r(cfg, c, stf + (size_t)s * OR_STF_STRIDE(cfg), x0 + 2 * s,
                           seis + (size_t)s * cfg->nrec * cfg->nt, NULL, NULL) != 0;
  return err ? -1 : 0;
}

int or_acoustic_forward_cplx(const or_acoustic_cfg *cfg, const void *c_,
                             const void *stf_, const void *x0_, void *seis_) {
  if (check_cfg(cfg)) return -1;
  const double complex *c = c_, *stf = stf_, *x0 = x0_;
  double complex *seis = seis_;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < cfg->nshots; s++)
    err |= acoustic_shot_c(cfg, c, stf + (size_t)s * OR_STF_STRIDE(cfg), x0 + 2 * s,
                           seis + (size_t)s * cfg->nrec * cfg->nt, NULL, NULL) != 0;
  return err ? -1 : 0;
}

/* Reverse sweep of one shot. lam1 is the adjoint of u^{n+1}, lam0 the part of
 * the adjoint of u^n collected so far; zx, zz, px_, pz_ are the adjoints of
 * the CPML memory variables carried backwards; gmx, gmz accumulate the
 * gradient with respect to the half-point coefficients (Eq. adjoint-gradient:
 * lambda^T (dA/dm) U). */
static int acoustic_shot_adjoint(const or_acoustic_cfg *cfg, const double *c,
                                 const double *stf, const double *x0s,
                                 const double *res, double *gm_pad,
                                 double *gstf, double *gx0) {
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np, N = cfg->order / 2, nt = cfg->nt;
  const double dx = cfg->dx, dz = cfg->dz, dt = cfg->dt;
  const size_t NN = (size_t)Nz * Nx;
  double a[8];
  or_fd_coeffs(cfg->order, a);

  /* Forward pass keeping p_x^n and p_z^n of every step. */
  double *pxs = malloc(sizeof(double) * NN * nt);
  double *pzs = malloc(sizeof(double) * NN * nt);
  double *seis = malloc(sizeof(double) * (size_t)cfg->nrec * nt);
  if (!pxs || !pzs || !seis) {
    free(pxs); free(pzs); free(seis);
    return -1;
  }
  int rc = acoustic_shot_r(cfg, c, stf, x0s, seis, pxs, pzs);
  free(seis);
  if (rc) {
    free(pxs); free(pzs);
    return rc;
  }

  double *ax = malloc(sizeof(double) * Nx), *bx = malloc(sizeof(double) * Nx);
  double *axh = malloc(sizeof(double) * Nx), *bxh = malloc(sizeof(double) * Nx);
  double *az = malloc(sizeof(double) * Nz), *bz = malloc(sizeof(double) * Nz);
  double *azh = malloc(sizeof(double) * Nz), *bzh = malloc(sizeof(double) * Nz);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nx, ax, bx);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nx, axh, bxh);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nz, az, bz);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nz, azh, bzh);

  double *m = calloc(NN, sizeof(double));
  double *mhx = calloc(NN, sizeof(double)), *mhz = calloc(NN, sizeof(double));
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int jX = 0; jX < Nx; jX++) {
      int i = iZ - np, j = jX - np;
      if (i < 0) i = 0;
      if (i > nz - 1) i = nz - 1;
      if (j < 0) j = 0;
      if (j > nx - 1) j = nx - 1;
      m[(size_t)iZ * Nx + jX] = c[(size_t)i * nx + j] * c[(size_t)i * nx + j];
    }
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int h = 0; h < Nx - 1; h++)
      mhx[(size_t)iZ * Nx + h] = 0.5 * (m[(size_t)iZ * Nx + h] + m[(size_t)iZ * Nx + h + 1]);
  for (int h = 0; h < Nz - 1; h++)
    for (int jX = 0; jX < Nx; jX++)
      mhz[(size_t)h * Nx + jX] = 0.5 * (m[(size_t)h * Nx + jX] + m[(size_t)(h + 1) * Nx + jX]);

  double *lam1 = calloc(NN, sizeof(double)), *lam0 = calloc(NN, sizeof(double));
  double *zx = calloc(NN, sizeof(double)), *zz = calloc(NN, sizeof(double));
  double *px_ = calloc(NN, sizeof(double)), *pz_ = calloc(NN, sizeof(double));
  double *hbx = calloc(NN, sizeof(double)), *hbz = calloc(NN, sizeof(double));
  double *gbx = calloc(NN, sizeof(double)), *gbz = calloc(NN, sizeof(double));
  double *gmx = calloc(NN, sizeof(double)), *gmz = calloc(NN, sizeof(double));
  double *gmc = calloc(NN, sizeof(double));  /* op 1: dJ/dm at the cells */
  const int op = cfg->op;

  const int cap = OR_MAX_SUPPORT(cfg);
  int *ci = malloc(sizeof(int) * cap), *cj = malloc(sizeof(int) * cap), nsup = 0;
  double *w = malloc(sizeof(double) * cap);
  source_support_r(cfg, x0s, ci, cj, &nsup, w);
  const int line = cfg->src_kind == 3;
  double sg = 0.5 * dx;

#define AT(arr, iZ, jX) (((iZ) >= 0 && (iZ) < Nz && (jX) >= 0 && (jX) < Nx) ? (arr)[(size_t)(iZ) * Nx + (jX)] : 0.0)
#define GX_AT(iZ, jX) (((jX) >= 0 && (jX) < Nx - 1) ? gbx[(size_t)(iZ) * Nx + (jX)] : 0.0)
#define GZ_AT(iZ, jX) (((iZ) >= 0 && (iZ) < Nz - 1) ? gbz[(size_t)(iZ) * Nx + (jX)] : 0.0)

  for (int n = nt - 1; n >= 0; n--) {
    /* the sample recorded from u^{n+1} contributes its residual */
    for (int r = 0; r < cfg->nrec; r++) {
      int iZ = cfg->rec_iz[r] + np, jX = cfg->rec_ix[r] + np;
      lam1[(size_t)iZ * Nx + jX] += res[(size_t)r * nt + n];
    }
    /* lam1 is now complete: source terms F_n = dt^2 w g(t_n) */
    for (int q = 0; q < nsup; q++) {
      double l = lam1[(size_t)ci[q] * Nx + cj[q]];
      if (gstf) gstf[line ? (size_t)n * nsup + q : (size_t)n] += dt * dt * w[q] * l;
      if (gx0 && cfg->src_kind == 1) {
        double xi = (cj[q] - np) * dx - x0s[0], zi = (ci[q] - np) * dz - x0s[1];
        gx0[0] += stf[n] * dt * dt * l * w[q] * xi / (sg * sg);
        gx0[1] += stf[n] * dt * dt * l * w[q] * zi / (sg * sg);
      }
    }
    /* reverse of: r = h + zeta_new, zeta_new = b zeta + a h, h = D-(q) */
    for (int iZ = 0; iZ < Nz; iZ++)
      for (int jX = 0; jX < Nx; jX++) {
        size_t id = (size_t)iZ * Nx + jX;
        /* op 1: u^{n+1} += dt^2 m r, so dJ/dm += dt^2 lam r and rbar = dt^2 m lam */
        if (op) gmc[id] += dt * dt * lam1[id] * pxs[(size_t)n * NN + id];
        double rb = dt * dt * (op ? m[id] : 1.0) * lam1[id];
        double t = zx[id] + rb;
        hbx[id] = rb + ax[jX] * t;
        zx[id] = bx[jX] * t;
        t = zz[id] + rb;
        hbz[id] = rb + az[iZ] * t;
        zz[id] = bz[iZ] * t;
      }
    /* reverse of: q = m p, p = g + psi_new, psi_new = b psi + a g, g = D+(u) */
    for (int iZ = 0; iZ < Nz; iZ++)
      for (int h = 0; h < Nx - 1; h++) {
        size_t id = (size_t)iZ * Nx + h;
        double qb = 0;
        for (int k = 1; k <= N; k++) qb += a[k - 1] * (AT(hbx, iZ, h - k + 1) - AT(hbx, iZ, h + k));
        qb /= dx;
        if (!op) gmx[id] += qb * pxs[(size_t)n * NN + id];
        double pb = op ? qb : mhx[id] * qb;
        double t = px_[id] + pb;
        gbx[id] = pb + axh[h] * t;
        px_[id] = bxh[h] * t;
      }
    for (int h = 0; h < Nz - 1; h++)
      for (int jX = 0; jX < Nx; jX++) {
        size_t id = (size_t)h * Nx + jX;
        double qb = 0;
        for (int k = 1; k <= N; k++) qb += a[k - 1] * (AT(hbz, h - k + 1, jX) - AT(hbz, h + k, jX));
        qb /= dz;
        if (!op) gmz[id] += qb * pzs[(size_t)n * NN + id];
        double pb = op ? qb : mhz[id] * qb;
        double t = pz_[id] + pb;
        gbz[id] = pb + azh[h] * t;
        pz_[id] = bzh[h] * t;
      }
    /* adjoint of u^n: 2 lam_{n+1} from the leapfrog plus D+^T of gbar */
    for (int iZ = 0; iZ < Nz; iZ++)
      for (int jX = 0; jX < Nx; jX++) {
        double s = 0;
        for (int k = 1; k <= N; k++) {
          s += a[k - 1] * (GX_AT(iZ, jX - k) - GX_AT(iZ, jX + k - 1)) / dx;
          s += a[k - 1] * (GZ_AT(iZ - k, jX) - GZ_AT(iZ + k - 1, jX)) / dz;
        }
        size_t id = (size_t)iZ * Nx + jX;
        lam0[id] += 2.0 * lam1[id] + s;
      }
    /* shift: u^n becomes the newest state, u^{n-1} receives -lam_{n+1} */
    double *t = lam1;
    lam1 = lam0;
    lam0 = t;
    for (size_t id = 0; id < NN; id++) lam0[id] = -lam0[id];
  }
#undef AT
#undef GX_AT
#undef GZ_AT

  /* chain rule from half points to cells: each half-point value is the mean
   * of its two neighbours */
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int jX = 0; jX < Nx; jX++) {
      double g = 0;
      if (jX - 1 >= 0) g += 0.5 * gmx[(size_t)iZ * Nx + jX - 1];
      if (jX < Nx - 1) g += 0.5 * gmx[(size_t)iZ * Nx + jX];
      if (iZ - 1 >= 0) g += 0.5 * gmz[(size_t)(iZ - 1) * Nx + jX];
      if (iZ < Nz - 1) g += 0.5 * gmz[(size_t)iZ * Nx + jX];
      gm_pad[(size_t)iZ * Nx + jX] = op ? gmc[(size_t)iZ * Nx + jX] : g;
    }

  free(pxs); free(pzs);
  free(ax); free(bx); free(axh); free(bxh); free(az); free(bz); free(azh); free(bzh);
  free(m); free(mhx); free(mhz); free(lam1); free(lam0); free(zx); free(zz);
  free(px_); free(pz_); free(hbx); free(hbz); free(gbx); free(gbz); free(gmx); free(gmz); free(gmc);
  free(ci); free(cj); free(w);
  return 0;
}

int or_acoustic_adjoint(const or_acoustic_cfg *cfg, const double *c,
                        const double *stf, const double *x0, const double *res,
                        double *grad_c, double *grad_stf, double *grad_x0) {
  if (check_cfg(cfg)) return -1;
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np;
  const size_t NN = (size_t)Nz * Nx;
  double *gm_all = calloc(NN * (size_t)cfg->nshots, sizeof(double));
  double *gstf = calloc((size_t)cfg->nshots * OR_STF_STRIDE(cfg), sizeof(double));
  double *gx0 = calloc((size_t)cfg->nshots * 2, sizeof(double));
  if (!gm_all || !gstf || !gx0) {
    free(gm_all); free(gstf); free(gx0);
    return -1;
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < cfg->nshots; s++)
    err |= acoustic_shot_adjoint(cfg, c, stf + (size_t)s * OR_STF_STRIDE(cfg), x0 + 2 * s,
                                 res + (size_t)s * cfg->nrec * cfg->nt, gm_all + NN * s,
                                 gstf + (size_t)s * OR_STF_STRIDE(cfg), gx0 + 2 * s) != 0;
  if (!err) {
    if (grad_c) {
      /* sum over shots, transpose of the edge replication into the CPML,
       * then dJ/dc = 2 c dJ/dm */
      memset(grad_c, 0, sizeof(double) * (size_t)nz * nx);
      for (int s = 0; s < cfg->nshots; s++)
        for (int iZ = 0; iZ < Nz; iZ++)
          for (int jX = 0; jX < Nx; jX++) {
            int i = iZ - np, j = jX - np;
            if (i < 0) i = 0;
            if (i > nz - 1) i = nz - 1;
            if (j < 0) j = 0;
            if (j > nx - 1) j = nx - 1;
            grad_c[(size_t)i * nx + j] += gm_all[NN * s + (size_t)iZ * Nx + jX];
          }
      for (size_t k = 0; k < (size_t)nz * nx; k++) grad_c[k] *= 2.0 * c[k];
    }
    if (grad_stf) memcpy(grad_stf, gstf, sizeof(double) * (size_t)cfg->nshots * OR_STF_STRIDE(cfg));
    if (grad_x0) memcpy(grad_x0, gx0, sizeof(double) * 2 * (size_t)cfg->nshots);
  }
  free(gm_all); free(gstf); free(gx0);
  return err ? -1 : 0;
}
