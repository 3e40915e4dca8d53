/*
 * elastic.c - FP64 CPU oracle of the elastic velocity-stress forward map and
 * its exact discrete adjoint. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper passages followed: the elastic equations (Implementation, Eq.
 * elastic; the lambda term is read with its Kronecker delta, the standard
 * isotropic law), the explicit recursion (Eq. forward), the misfit, the
 * adjoint recursion (Eq. adjoint-backward) and the gradient with respect to
 * lambda, mu, rho (Eq. adjoint-gradient). The adjoint below reverses the
 * statements of elastic_body.h one by one.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define REAL double
#define FN(name) name##_r
#define CEXP(x) exp(x)
#define RE(x) (x)
#include "elastic_body.h"
#undef REAL
#undef FN
#undef CEXP
#undef RE

#define REAL double complex
#define FN(name) name##_c
#define CEXP(x) cexp(x)
#define RE(x) creal(x)
#include "elastic_body.h"
#undef REAL
#undef FN
#undef CEXP
#undef RE

static int el_check(const or_acoustic_cfg *cfg) {
  if (cfg->nz < 1 || cfg->nx < 1 || cfg->nt < 1 || cfg->nshots < 0 || cfg->npml < 0) return -1;
  if (cfg->order != 4 && cfg->order != 8) return -1;
  if (cfg->src_kind != 0 && cfg->src_kind != 1) return -1;  /* point or Gaussian moment tensors only */
  for (int r = 0; r < cfg->nrec; r++)
    if (cfg->rec_iz[r] < 0 || cfg->rec_iz[r] >= cfg->nz || cfg->rec_ix[r] < 0 || cfg->rec_ix[r] >= cfg->nx)
      return -1;
  return 0;
}

int or_elastic_forward(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                       const double *stf, const double *x0, const double *mt, double *seis) {
  if (el_check(cfg)) return -1;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < cfg->nshots; s++)
    err |= elastic_shot_r(cfg, vp, vs, rho, stf + (size_t)s * cfg->nt, x0 + 2 * s, mt + 3 * s,
                          seis + (size_t)s * 2 * cfg->nrec * cfg->nt, NULL, NULL, 0) != 0;
  return err ? -1 : 0;
}

int or_elastic_forward_cplx(const or_acoustic_cfg *cfg, const void *vp_, const void *vs_, const void *rho_,
                            const void *stf_, const void *x0_, const void *mt_, void *seis_) {
  if (el_check(cfg)) return -1;
  const double complex *vp = vp_, *vs = vs_, *rho = rho_, *stf = stf_, *x0 = x0_, *mt = mt_;
  double complex *seis = seis_;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < cfg->nshots; s++)
    err |= elastic_shot_c(cfg, vp, vs, rho, stf + (size_t)s * cfg->nt, x0 + 2 * s, mt + 3 * s,
                          seis + (size_t)s * 2 * cfg->nrec * cfg->nt, NULL, NULL, 0) != 0;
  return err ? -1 : 0;
}

/* State (vx, vz, sxx, szz, sxz) of shot 0 after `step` steps, i.e.
 * (v^{step-1/2}, sigma^{step}), each [Nz][Nx]. */
int or_elastic_snapshot(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                        const double *stf, const double *x0, const double *mt, int step, double *fields) {
  if (el_check(cfg) || step < 0 || step > cfg->nt) return -1;
  double *seis = malloc(sizeof(double) * 2 * (size_t)(cfg->nrec + 1) * cfg->nt);
  int rc = elastic_shot_r(cfg, vp, vs, rho, stf, x0, mt, seis, NULL, fields, step);
  free(seis);
  return rc;
}

static int elastic_shot_adjoint(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rh,
                                const double *stf, const double *x0s, const double *mt, const double *res,
                                double *glam_pad, double *gmu_pad, double *grho_pad, double *gstf, double *gx0) {
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np, N = cfg->order / 2, nt = cfg->nt;
  const double dx = cfg->dx, dz = cfg->dz, dt = cfg->dt;
  const size_t NN = (size_t)Nz * Nx;
  double a[8];
  or_fd_coeffs(cfg->order, a);

  double *store = malloc(sizeof(double) * 5 * NN * (size_t)nt);
  double *seis = malloc(sizeof(double) * 2 * (size_t)(cfg->nrec + 1) * nt);
  if (!store || !seis) {
    free(store); free(seis);
    return -1;
  }
  int rc = elastic_shot_r(cfg, vp, vs, rh, stf, x0s, mt, seis, store, NULL, 0);
  free(seis);
  if (rc) {
    free(store);
    return rc;
  }

  double *ax = malloc(sizeof(double) * Nx), *bxt = malloc(sizeof(double) * Nx);
  double *axh = malloc(sizeof(double) * Nx), *bxh = malloc(sizeof(double) * Nx);
  double *az = malloc(sizeof(double) * Nz), *bzt = malloc(sizeof(double) * Nz);
  double *azh = malloc(sizeof(double) * Nz), *bzh = malloc(sizeof(double) * Nz);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nx, ax, bxt);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nx, axh, bxh);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nz, az, bzt);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nz, azh, bzh);

  double *lam = calloc(NN, 8), *mu = calloc(NN, 8), *rho = calloc(NN, 8);
  double *bx = calloc(NN, 8), *bz = calloc(NN, 8), *mxz = calloc(NN, 8);
  el_medium_r(cfg, vp, vs, rh, lam, mu, rho, bx, bz, mxz);
  el_box_r bn, bs;
  el_src_box_r(cfg, x0s, 0.0, 0.0, Nz, Nx, &bn);
  el_src_box_r(cfg, x0s, 0.5, 0.5, Nz - 1, Nx - 1, &bs);

  /* adjoint state and work arrays */
  double *Vx = calloc(NN, 8), *Vz = calloc(NN, 8), *Sxx = calloc(NN, 8), *Szz = calloc(NN, 8), *Sxz = calloc(NN, 8);
  double *M[8];
  for (int k = 0; k < 8; k++) M[k] = calloc(NN, 8);
  double *bdvx = calloc(NN, 8), *bdvz = calloc(NN, 8), *bdvxz = calloc(NN, 8), *bdvzx = calloc(NN, 8);
  double *bdsxx = calloc(NN, 8), *bdsxz = calloc(NN, 8), *bdsxzx = calloc(NN, 8), *bdszz = calloc(NN, 8);
  double *glam = calloc(NN, 8), *gmu = calloc(NN, 8), *gmxz = calloc(NN, 8), *gbx = calloc(NN, 8), *gbz = calloc(NN, 8);
  const double sg2 = 0.25 * dx * dx;

#define NRM(arr, iR, jR) (((iR) >= 0 && (iR) < Nz && (jR) >= 0 && (jR) < Nx) ? (arr)[(size_t)(iR) * Nx + (jR)] : 0.0)
#define SHR(arr, iR, jR) (((iR) >= 0 && (iR) < Nz - 1 && (jR) >= 0 && (jR) < Nx - 1) ? (arr)[(size_t)(iR) * Nx + (jR)] : 0.0)
#define VXN(arr, iR, jR) (((iR) >= 0 && (iR) < Nz && (jR) >= 0 && (jR) < Nx - 1) ? (arr)[(size_t)(iR) * Nx + (jR)] : 0.0)
#define VZN(arr, iR, jR) (((iR) >= 0 && (iR) < Nz - 1 && (jR) >= 0 && (jR) < Nx) ? (arr)[(size_t)(iR) * Nx + (jR)] : 0.0)

  for (int n = nt - 1; n >= 0; n--) {
    const double *st = store + (size_t)n * 5 * NN;
    /* reverse of the source term sigma^{n+1} -= dt g_n M w */
    for (int di = 0; di < bn.n; di++)
      for (int dj = 0; dj < bn.n; dj++) {
        int iR = bn.i0 + di, jR = bn.j0 + dj;
        size_t id = (size_t)iR * Nx + jR;
        double w = bn.w[di * bn.n + dj];
        double s = -dt * (mt[0] * Sxx[id] + mt[1] * Szz[id]);
        if (gstf) gstf[n] += s * w;
        if (gx0 && cfg->src_kind == 1) {
          gx0[0] += stf[n] * s * w * ((jR - np) * dx - x0s[0]) / sg2;
          gx0[1] += stf[n] * s * w * ((iR - np) * dz - x0s[1]) / sg2;
        }
      }
    for (int di = 0; di < bs.n; di++)
      for (int dj = 0; dj < bs.n; dj++) {
        int iR = bs.i0 + di, jR = bs.j0 + dj;
        size_t id = (size_t)iR * Nx + jR;
        double w = bs.w[di * bs.n + dj];
        double s = -dt * mt[2] * Sxz[id];
        if (gstf) gstf[n] += s * w;
        if (gx0 && cfg->src_kind == 1) {
          gx0[0] += stf[n] * s * w * ((jR - np + 0.5) * dx - x0s[0]) / sg2;
          gx0[1] += stf[n] * s * w * ((iR - np + 0.5) * dz - x0s[1]) / sg2;
        }
      }
    /* reverse of the shear stress update (sxz passes its adjoint through) */
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx - 1; j++) {
        size_t id = (size_t)i * Nx + j;
        double t = dt * mxz[id] * Sxz[id];
        gmxz[id] += dt * Sxz[id] * st[4 * NN + id];
        double m7 = M[6][id] + t, m8 = M[7][id] + t;
        bdvxz[id] = t + azh[i] * m7;
        M[6][id] = bzh[i] * m7;
        bdvzx[id] = t + axh[j] * m8;
        M[7][id] = bxh[j] * m8;
      }
    /* reverse of the normal stress update */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx; j++) {
        size_t id = (size_t)i * Nx + j;
        double l = lam[id], m = mu[id];
        double ebx = dt * ((l + 2.0 * m) * Sxx[id] + l * Szz[id]);
        double ebz = dt * (l * Sxx[id] + (l + 2.0 * m) * Szz[id]);
        double ex = st[2 * NN + id], ez = st[3 * NN + id];
        glam[id] += dt * (ex + ez) * (Sxx[id] + Szz[id]);
        gmu[id] += 2.0 * dt * (ex * Sxx[id] + ez * Szz[id]);
        double m5 = M[4][id] + ebx, m6 = M[5][id] + ebz;
        bdvx[id] = ebx + ax[j] * m5;
        M[4][id] = bxt[j] * m5;
        bdvz[id] = ebz + az[i] * m6;
        M[5][id] = bzt[i] * m6;
      }
    /* adjoint of v^{n+1/2}: transposes of the strain operators */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx - 1; j++) {
        double s = 0;
        for (int k = 1; k <= N; k++) {
          s += a[k - 1] * (NRM(bdvx, i, j - k + 1) - NRM(bdvx, i, j + k)) / dx;
          s += a[k - 1] * (SHR(bdvxz, i - k, j) - SHR(bdvxz, i + k - 1, j)) / dz;
        }
        Vx[(size_t)i * Nx + j] += s;
      }
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx; j++) {
        double s = 0;
        for (int k = 1; k <= N; k++) {
          s += a[k - 1] * (NRM(bdvz, i - k + 1, j) - NRM(bdvz, i + k, j)) / dz;
          s += a[k - 1] * (SHR(bdvzx, i, j - k) - SHR(bdvzx, i, j + k - 1)) / dx;
        }
        Vz[(size_t)i * Nx + j] += s;
      }
    /* residuals of sample n (v^{n+1/2} at the receivers) */
    for (int r = 0; r < cfg->nrec; r++) {
      int iR = cfg->rec_iz[r] + np, jR = cfg->rec_ix[r] + np;
      if (jR < Nx - 1) Vx[(size_t)iR * Nx + jR] += res[(size_t)r * nt + n];
      if (iR < Nz - 1) Vz[(size_t)iR * Nx + jR] += res[((size_t)cfg->nrec + r) * nt + n];
    }
    /* reverse of the velocity update (v passes its adjoint through) */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx - 1; j++) {
        size_t id = (size_t)i * Nx + j;
        double t = dt * bx[id] * Vx[id];
        gbx[id] += dt * Vx[id] * st[id];
        double m1 = M[0][id] + t, m2 = M[1][id] + t;
        bdsxx[id] = t + axh[j] * m1;
        M[0][id] = bxh[j] * m1;
        bdsxz[id] = t + az[i] * m2;
        M[1][id] = bzt[i] * m2;
      }
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx; j++) {
        size_t id = (size_t)i * Nx + j;
        double t = dt * bz[id] * Vz[id];
        gbz[id] += dt * Vz[id] * st[NN + id];
        double m3 = M[2][id] + t, m4 = M[3][id] + t;
        bdsxzx[id] = t + ax[j] * m3;
        M[2][id] = bxt[j] * m3;
        bdszz[id] = t + azh[i] * m4;
        M[3][id] = bzh[i] * m4;
      }
    /* adjoint of sigma^n: transposes of the divergence operators */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx; j++) {
        double sx = 0, sz = 0;
        for (int k = 1; k <= N; k++) {
          sx += a[k - 1] * (VXN(bdsxx, i, j - k) - VXN(bdsxx, i, j + k - 1)) / dx;
          sz += a[k - 1] * (VZN(bdszz, i - k, j) - VZN(bdszz, i + k - 1, j)) / dz;
        }
        Sxx[(size_t)i * Nx + j] += sx;
        Szz[(size_t)i * Nx + j] += sz;
      }
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx - 1; j++) {
        double s = 0;
        for (int k = 1; k <= N; k++) {
          s += a[k - 1] * (VXN(bdsxz, i - k + 1, j) - VXN(bdsxz, i + k, j)) / dz;
          s += a[k - 1] * (VZN(bdsxzx, i, j - k + 1) - VZN(bdsxzx, i, j + k)) / dx;
        }
        Sxz[(size_t)i * Nx + j] += s;
      }
  }
#undef NRM
#undef SHR
#undef VXN
#undef VZN

  /* chain rule to the cell parameters on the padded grid */
  for (size_t id = 0; id < NN; id++) {
    glam_pad[id] = glam[id];
    gmu_pad[id] = gmu[id];
    grho_pad[id] = 0.0;
  }
  for (int i = 0; i < Nz - 1; i++)
    for (int j = 0; j < Nx - 1; j++) {
      size_t id = (size_t)i * Nx + j;
      if (mxz[id] == 0.0) continue;
      size_t c[4] = {id, id + 1, id + Nx, id + Nx + 1};
      for (int q = 0; q < 4; q++) gmu_pad[c[q]] += gmxz[id] * mxz[id] * mxz[id] / (4.0 * mu[c[q]] * mu[c[q]]);
    }
  for (int i = 0; i < Nz; i++)
    for (int j = 0; j < Nx - 1; j++) {
      size_t id = (size_t)i * Nx + j;
      double g = -0.5 * bx[id] * bx[id] * gbx[id];
      grho_pad[id] += g;
      grho_pad[id + 1] += g;
    }
  for (int i = 0; i < Nz - 1; i++)
    for (int j = 0; j < Nx; j++) {
      size_t id = (size_t)i * Nx + j;
      double g = -0.5 * bz[id] * bz[id] * gbz[id];
      grho_pad[id] += g;
      grho_pad[id + Nx] += g;
    }

  free(store);
  free(ax); free(bxt); free(axh); free(bxh); free(az); free(bzt); free(azh); free(bzh);
  free(lam); free(mu); free(rho); free(bx); free(bz); free(mxz);
  free(Vx); free(Vz); free(Sxx); free(Szz); free(Sxz);
  for (int k = 0; k < 8; k++) free(M[k]);
  free(bdvx); free(bdvz); free(bdvxz); free(bdvzx); free(bdsxx); free(bdsxz); free(bdsxzx); free(bdszz);
  free(glam); free(gmu); free(gmxz); free(gbx); free(gbz);
  return 0;
}

int or_elastic_adjoint(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                       const double *stf, const double *x0, const double *mt, const double *res, double *g_lam,
                       double *g_mu, double *g_rho, double *g_stf, double *g_x0) {
  if (el_check(cfg)) return -1;
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np;
  const size_t NN = (size_t)Nz * Nx;
  const int S = cfg->nshots;
  double *gp = calloc(3 * NN * (size_t)S, 8);
  double *gs = calloc((size_t)S * cfg->nt, 8), *gx = calloc((size_t)S * 2, 8);
  if (!gp || !gs || !gx) {
    free(gp); free(gs); free(gx);
    return -1;
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int s = 0; s < S; s++)
    err |= elastic_shot_adjoint(cfg, vp, vs, rho, stf + (size_t)s * cfg->nt, x0 + 2 * s, mt + 3 * s,
                                res + (size_t)s * 2 * cfg->nrec * cfg->nt, gp + 3 * NN * s, gp + 3 * NN * s + NN,
                                gp + 3 * NN * s + 2 * NN, gs + (size_t)s * cfg->nt, gx + 2 * s) != 0;
  if (!err) {
    double *outs[3] = {g_lam, g_mu, g_rho};
    for (int f = 0; f < 3; f++) {
      if (!outs[f]) continue;
      memset(outs[f], 0, sizeof(double) * (size_t)nz * nx);
      for (int s = 0; s < S; s++)
        for (int iZ = 0; iZ < Nz; iZ++)
          for (int jX = 0; jX < Nx; jX++) {
            int i = iZ - np, j = jX - np;
            if (i < 0) i = 0;
            if (i > nz - 1) i = nz - 1;
            if (j < 0) j = 0;
            if (j > nx - 1) j = nx - 1;
            outs[f][(size_t)i * nx + j] += gp[3 * NN * s + f * NN + (size_t)iZ * Nx + jX];
          }
    }
    if (g_stf) memcpy(g_stf, gs, sizeof(double) * (size_t)S * cfg->nt);
    if (g_x0) memcpy(g_x0, gx, sizeof(double) * 2 * (size_t)S);
  }
  free(gp); free(gs); free(gx);
  return err ? -1 : 0;
}
