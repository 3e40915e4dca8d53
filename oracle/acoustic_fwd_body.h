/*
 * acoustic_fwd_body.h - the acoustic forward recursion written once and
 * compiled twice by acoustic.c: with REAL = double and with
 * REAL = double complex (complex-step derivatives). TEST INFRASTRUCTURE ONLY.
 *
 * Needs: REAL, FN(name), CEXP(x), RE(x) defined by the includer.
 *
 * The state U_k of the explicit recursion U_k = A(theta) U_{k-1} + F_{k-1}
 * (Method, "Relationship to the Adjoint Method", Eq. forward) is
 * (u^k, u^{k-1}, psi_x, psi_z, zeta_x, zeta_z); theta is the velocity c of
 * the acoustic equation u_tt = div(c^2 grad u) + f (Implementation, Eq.
 * acoustic), discretised on a staggered grid with convolutional PML
 * (Implementation).
 */

/* Source weights of one shot on the padded grid: a point source puts
 * 1/(dx dz) on the nearest cell; the Gaussian source spreads
 * g(t)/(2 pi s^2) exp(-|x-x0|^2/(2 s^2)) with s = dx/2 over +-3 cells
 * (Earthquake Location section, Gaussian re-parameterisation); a line source
 * (the paper's plane-wave sources, FWI section: a line of sources fired with
 * delays) puts 1/(dx dz) on each of line_len cells of one row, from the cell
 * nearest x0, each cell with its own time function. The arrays hold at least
 * OR_MAX_SUPPORT(cfg) entries. */
static int FN(source_support)(const or_acoustic_cfg *cfg, const REAL *x0s,
                              int *ci, int *cj, int *nsup, REAL *w) {
  double xr = RE(x0s[0]), zr = RE(x0s[1]);
  int jc = (int)lround(xr / cfg->dx) + cfg->npml;
  int ic = (int)lround(zr / cfg->dz) + cfg->npml;
  int Nz = cfg->nz + 2 * cfg->npml, Nx = cfg->nx + 2 * cfg->npml;
  int n = 0;
  if (cfg->src_kind == 0) {
    if (ic < 0 || ic >= Nz || jc < 0 || jc >= Nx) return -1;
    ci[0] = ic; cj[0] = jc; w[0] = 1.0 / (cfg->dx * cfg->dz);
    *nsup = 1;
    return 0;
  }
  if (cfg->src_kind == 3) {
    if (cfg->line_len < 1 || ic < 0 || ic >= Nz || jc < 0 || jc + cfg->line_len > Nx) return -1;
    for (int q = 0; q < cfg->line_len; q++) {
      ci[q] = ic; cj[q] = jc + q; w[q] = 1.0 / (cfg->dx * cfg->dz);
    }
    *nsup = cfg->line_len;
    return 0;
  }
  double sg = 0.5 * cfg->dx;
  for (int di = -3; di <= 3; di++)
    for (int dj = -3; dj <= 3; dj++) {
      int i = ic + di, j = jc + dj;
      if (i < 0 || i >= Nz || j < 0 || j >= Nx) return -1;
      REAL xi = (j - cfg->npml) * cfg->dx - x0s[0];
      REAL zi = (i - cfg->npml) * cfg->dz - x0s[1];
      ci[n] = i; cj[n] = j;
      w[n] = CEXP(-(xi * xi + zi * zi) / (2.0 * sg * sg)) / (2.0 * M_PI * sg * sg);
      n++;
    }
  *nsup = n;
  return 0;
}

/* One shot of forward modelling. If px_store / pz_store are given, the
 * quantities p_x = D+x u + psi_x and p_z (the factors that multiply the
 * half-point coefficient m = c^2) of every step n are saved, nt x size; with
 * op = 1 (c^2 Laplacian form) px_store receives instead r = D-x p_x + zeta_x +
 * D-z p_z + zeta_z at the cells, the factor that multiplies m there. */
static int FN(acoustic_shot)(const or_acoustic_cfg *cfg, const REAL *c,
                             const REAL *stf, const REAL *x0s, REAL *seis,
                             REAL *px_store, REAL *pz_store) {
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np, N = cfg->order / 2;
  const double dx = cfg->dx, dz = cfg->dz, dt = cfg->dt;
  double a[8];
  if (or_fd_coeffs(cfg->order, a)) return -1;

  double *ax = malloc(sizeof(double) * Nx), *bx = malloc(sizeof(double) * Nx);
  double *axh = malloc(sizeof(double) * Nx), *bxh = malloc(sizeof(double) * Nx);
  double *az = malloc(sizeof(double) * Nz), *bz = malloc(sizeof(double) * Nz);
  double *azh = malloc(sizeof(double) * Nz), *bzh = malloc(sizeof(double) * Nz);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nx, ax, bx);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nx, axh, bxh);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nz, az, bz);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nz, azh, bzh);

  const size_t NN = (size_t)Nz * Nx;
  REAL *m = calloc(NN, sizeof(REAL));
  REAL *mhx = calloc(NN, sizeof(REAL)), *mhz = calloc(NN, sizeof(REAL));
  REAL *u = calloc(NN, sizeof(REAL)), *up = calloc(NN, sizeof(REAL));
  REAL *un = calloc(NN, sizeof(REAL));
  REAL *psix = calloc(NN, sizeof(REAL)), *psiz = calloc(NN, sizeof(REAL));
  REAL *zetx = calloc(NN, sizeof(REAL)), *zetz = calloc(NN, sizeof(REAL));
  REAL *qx = calloc(NN, sizeof(REAL)), *qz = calloc(NN, sizeof(REAL));

  /* m = c^2 on the padded grid, edge-replicated into the CPML. */
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int jX = 0; jX < Nx; jX++) {
      int i = iZ - np, j = jX - np;
      if (i < 0) i = 0;
      if (i > nz - 1) i = nz - 1;
      if (j < 0) j = 0;
      if (j > nx - 1) j = nx - 1;
      REAL cc = c[(size_t)i * nx + j];
      m[(size_t)iZ * Nx + jX] = cc * cc;
    }
  /* Half-point coefficients: arithmetic mean of the two neighbours.
   * mhx[iZ][h] sits at (iZ, h+1/2), h in [0, Nx-1); mhz[h][jX] at (h+1/2, jX). */
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int h = 0; h < Nx - 1; h++)
      mhx[(size_t)iZ * Nx + h] = 0.5 * (m[(size_t)iZ * Nx + h] + m[(size_t)iZ * Nx + h + 1]);
  for (int h = 0; h < Nz - 1; h++)
    for (int jX = 0; jX < Nx; jX++)
      mhz[(size_t)h * Nx + jX] = 0.5 * (m[(size_t)h * Nx + jX] + m[(size_t)(h + 1) * Nx + jX]);

  const int cap = OR_MAX_SUPPORT(cfg);
  int *ci = malloc(sizeof(int) * cap), *cj = malloc(sizeof(int) * cap), nsup = 0;
  REAL *w = malloc(sizeof(REAL) * cap);
  const int line = cfg->src_kind == 3;
  int rc = FN(source_support)(cfg, x0s, ci, cj, &nsup, w);

#define U_AT(arr, iZ, jX) (((iZ) >= 0 && (iZ) < Nz && (jX) >= 0 && (jX) < Nx) ? (arr)[(size_t)(iZ) * Nx + (jX)] : (REAL)0)
#define QX_AT(iZ, jX) (((jX) >= 0 && (jX) < Nx - 1) ? qx[(size_t)(iZ) * Nx + (jX)] : (REAL)0)
#define QZ_AT(iZ, jX) (((iZ) >= 0 && (iZ) < Nz - 1) ? qz[(size_t)(iZ) * Nx + (jX)] : (REAL)0)

  for (int n = 0; rc == 0 && n < cfg->nt; n++) {
    /* x: p_x = D+x u + psi_x with psi_x <- b psi_x + a D+x u; q_x = m p_x */
    for (int iZ = 0; iZ < Nz; iZ++)
      for (int h = 0; h < Nx - 1; h++) {
        REAL g = 0;
        for (int k = 1; k <= N; k++) g += a[k - 1] * (U_AT(u, iZ, h + k) - U_AT(u, iZ, h - k + 1));
        g /= dx;
        size_t id = (size_t)iZ * Nx + h;
        psix[id] = bxh[h] * psix[id] + axh[h] * g;
        REAL p = g + psix[id];
        if (px_store && !cfg->op) px_store[(size_t)n * NN + id] = p;
        qx[id] = cfg->op ? p : mhx[id] * p;
      }
    /* z: the same along the depth axis */
    for (int h = 0; h < Nz - 1; h++)
      for (int jX = 0; jX < Nx; jX++) {
        REAL g = 0;
        for (int k = 1; k <= N; k++) g += a[k - 1] * (U_AT(u, h + k, jX) - U_AT(u, h - k + 1, jX));
        g /= dz;
        size_t id = (size_t)h * Nx + jX;
        psiz[id] = bzh[h] * psiz[id] + azh[h] * g;
        REAL p = g + psiz[id];
        if (pz_store && !cfg->op) pz_store[(size_t)n * NN + id] = p;
        qz[id] = cfg->op ? p : mhz[id] * p;
      }
    /* divergence with its own memory variables, then the leapfrog update */
    for (int iZ = 0; iZ < Nz; iZ++)
      for (int jX = 0; jX < Nx; jX++) {
        REAL hx = 0, hz = 0;
        for (int k = 1; k <= N; k++) {
          hx += a[k - 1] * (QX_AT(iZ, jX + k - 1) - QX_AT(iZ, jX - k));
          hz += a[k - 1] * (QZ_AT(iZ + k - 1, jX) - QZ_AT(iZ - k, jX));
        }
        hx /= dx;
        hz /= dz;
        size_t id = (size_t)iZ * Nx + jX;
        zetx[id] = bx[jX] * zetx[id] + ax[jX] * hx;
        zetz[id] = bz[iZ] * zetz[id] + az[iZ] * hz;
        REAL r = hx + zetx[id] + hz + zetz[id];
        /* c^2 Laplacian form: the coefficient multiplies the whole operator at the
         * cell, and r (the Laplacian with its CPML terms) is what the gradient needs */
        if (cfg->op && px_store) px_store[(size_t)n * NN + id] = r;
        un[id] = 2.0 * u[id] - up[id] + dt * dt * (cfg->op ? m[id] * r : r);
      }
    /* source term F_n = dt^2 f(t_n) (a line source: each cell its own f) */
    for (int q = 0; q < nsup; q++)
      un[(size_t)ci[q] * Nx + cj[q]] += dt * dt * w[q] * (line ? stf[(size_t)n * nsup + q] : stf[n]);
    /* receivers sample u^{n+1} */
    for (int r = 0; r < cfg->nrec; r++) {
      int iZ = cfg->rec_iz[r] + np, jX = cfg->rec_ix[r] + np;
      seis[(size_t)r * cfg->nt + n] = un[(size_t)iZ * Nx + jX];
    }
    REAL *t = up;
    up = u;
    u = un;
    un = t;
  }
#undef U_AT
#undef QX_AT
#undef QZ_AT
  free(ax); free(bx); free(axh); free(bxh); free(az); free(bz); free(azh); free(bzh);
  free(m); free(mhx); free(mhz); free(u); free(up); free(un);
  free(psix); free(psiz); free(zetx); free(zetz); free(qx); free(qz);
  free(ci); free(cj); free(w);
  return rc;
}
