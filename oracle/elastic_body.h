/*
 * elastic_body.h - the elastic velocity-stress forward recursion written once
 * and compiled twice by elastic.c (REAL = double, REAL = double complex).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Needs: REAL, FN(name), CEXP(x), RE(x) defined by the includer.
 *
 * Equations (Implementation, Eq. elastic, with the isotropic Hooke law
 * sigma_ij,t = lambda delta_ij v_k,k + mu (v_i,j + v_j,i)):
 *   rho vx_t = sxx_x + sxz_z,   rho vz_t = sxz_x + szz_z,
 *   sxx_t = (lambda + 2 mu) vx_x + lambda vz_z,
 *   szz_t = lambda vx_x + (lambda + 2 mu) vz_z,   sxz_t = mu (vx_z + vz_x),
 * on the staggered grid (vx at (i, j+1/2), vz at (i+1/2, j), sxx and szz at
 * (i, j), sxz at (i+1/2, j+1/2)); leapfrog in time (v at half steps), CPML
 * memory variables on every derivative; moment-tensor source injected into
 * the stresses: sigma <- sigma - dt M g(t_n) w.
 * Arrays are [Nz][Nx]; a field on half points uses index h for position h+1/2
 * and is zero outside its valid range ([0, N-1) along a half axis).
 */

typedef struct {
  int i0, j0, n;   /* box origin and side (1 point or 7 Gaussian) */
  REAL w[49];
} FN(el_box);

/* Source weights on one staggered grid whose nodes sit at offset (oz, ox)
 * cells (0 or 1/2): nearest node, then 1/(dx dz) (point) or the Gaussian
 * g/(2 pi s^2) exp(-r^2/(2 s^2)), s = dx/2, on +-3 nodes. */
static int FN(el_src_box)(const or_acoustic_cfg *cfg, const REAL *x0s, double oz, double ox, int nmax_i,
                          int nmax_j, FN(el_box) *b) {
  double xr = RE(x0s[0]), zr = RE(x0s[1]);
  int jc = (int)lround(xr / cfg->dx - ox) + cfg->npml;
  int ic = (int)lround(zr / cfg->dz - oz) + cfg->npml;
  if (cfg->src_kind == 0) {
    if (ic < 0 || ic >= nmax_i || jc < 0 || jc >= nmax_j) return -1;
    b->i0 = ic; b->j0 = jc; b->n = 1;
    b->w[0] = 1.0 / (cfg->dx * cfg->dz);
    return 0;
  }
  if (ic - 3 < 0 || ic + 3 >= nmax_i || jc - 3 < 0 || jc + 3 >= nmax_j) return -1;
  b->i0 = ic - 3; b->j0 = jc - 3; b->n = 7;
  double sg = 0.5 * cfg->dx;
  for (int di = 0; di < 7; di++)
    for (int dj = 0; dj < 7; dj++) {
      REAL xi = (b->j0 + dj - cfg->npml + ox) * cfg->dx - x0s[0];
      REAL zi = (b->i0 + di - cfg->npml + oz) * cfg->dz - x0s[1];
      b->w[di * 7 + dj] = CEXP(-(xi * xi + zi * zi) / (2.0 * sg * sg)) / (2.0 * M_PI * sg * sg);
    }
  return 0;
}

/* Medium on the padded grid: lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2,
 * edge-replicated; buoyancy at the velocity nodes from the arithmetic mean of
 * rho; mu at the shear nodes as the harmonic mean of the four cells (0 if
 * any is 0). */
static void FN(el_medium)(const or_acoustic_cfg *cfg, const REAL *vp, const REAL *vs, const REAL *rh, REAL *lam,
                          REAL *mu, REAL *rho, REAL *bx, REAL *bz, REAL *mxz) {
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml, Nz = nz + 2 * np, Nx = nx + 2 * np;
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int jX = 0; jX < Nx; jX++) {
      int i = iZ - np, j = jX - np;
      if (i < 0) i = 0;
      if (i > nz - 1) i = nz - 1;
      if (j < 0) j = 0;
      if (j > nx - 1) j = nx - 1;
      size_t c = (size_t)i * nx + j, id = (size_t)iZ * Nx + jX;
      rho[id] = rh[c];
      mu[id] = rh[c] * vs[c] * vs[c];
      lam[id] = rh[c] * (vp[c] * vp[c] - 2.0 * vs[c] * vs[c]);
    }
  for (int iZ = 0; iZ < Nz; iZ++)
    for (int jX = 0; jX < Nx; jX++) {
      size_t id = (size_t)iZ * Nx + jX;
      bx[id] = (jX < Nx - 1) ? 2.0 / (rho[id] + rho[id + 1]) : (REAL)0;
      bz[id] = (iZ < Nz - 1) ? 2.0 / (rho[id] + rho[id + Nx]) : (REAL)0;
      mxz[id] = 0;
      if (iZ < Nz - 1 && jX < Nx - 1) {
        REAL m1 = mu[id], m2 = mu[id + 1], m3 = mu[id + Nx], m4 = mu[id + Nx + 1];
        if (RE(m1) != 0.0 && RE(m2) != 0.0 && RE(m3) != 0.0 && RE(m4) != 0.0)
          mxz[id] = 4.0 / (1.0 / m1 + 1.0 / m2 + 1.0 / m3 + 1.0 / m4);
      }
    }
}

/* One shot of elastic modelling. seis is [2][nrec][nt] (vx, vz samples of
 * v^{n+1/2}). If `store` is given (real version only), the forward values the
 * adjoint needs are kept for every step: store[n][5][NN] = (force on vx, force
 * on vz, ex, ez, exz), each including its CPML memory term. If `snap` is given,
 * the state (vx, vz, sxx, szz, sxz) after `snap_step` steps is copied to it. */
static int FN(elastic_shot)(const or_acoustic_cfg *cfg, const REAL *vp, const REAL *vs, const REAL *rh,
                            const REAL *stf, const REAL *x0s, const REAL *mt, REAL *seis, REAL *store, REAL *snap,
                            int snap_step) {
  const int nz = cfg->nz, nx = cfg->nx, np = cfg->npml;
  const int Nz = nz + 2 * np, Nx = nx + 2 * np, N = cfg->order / 2, nt = cfg->nt;
  const double dx = cfg->dx, dz = cfg->dz, dt = cfg->dt;
  double a[8];
  if (or_fd_coeffs(cfg->order, a)) return -1;
  const size_t NN = (size_t)Nz * Nx;

  double *ax = malloc(sizeof(double) * Nx), *bxt = malloc(sizeof(double) * Nx);
  double *axh = malloc(sizeof(double) * Nx), *bxh = malloc(sizeof(double) * Nx);
  double *az = malloc(sizeof(double) * Nz), *bzt = malloc(sizeof(double) * Nz);
  double *azh = malloc(sizeof(double) * Nz), *bzh = malloc(sizeof(double) * Nz);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nx, ax, bxt);
  or_cpml_profile(nx, np, dx, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nx, axh, bxh);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 0, Nz, az, bzt);
  or_cpml_profile(nz, np, dz, dt, cfg->pml_R, cfg->pml_vmax, cfg->pml_f0, 1, Nz, azh, bzh);

  REAL *lam = calloc(NN, sizeof(REAL)), *mu = calloc(NN, sizeof(REAL)), *rho = calloc(NN, sizeof(REAL));
  REAL *bx = calloc(NN, sizeof(REAL)), *bz = calloc(NN, sizeof(REAL)), *mxz = calloc(NN, sizeof(REAL));
  REAL *vx = calloc(NN, sizeof(REAL)), *vz = calloc(NN, sizeof(REAL));
  REAL *sxx = calloc(NN, sizeof(REAL)), *szz = calloc(NN, sizeof(REAL)), *sxz = calloc(NN, sizeof(REAL));
  REAL *mem[8];
  for (int k = 0; k < 8; k++) mem[k] = calloc(NN, sizeof(REAL));
  FN(el_medium)(cfg, vp, vs, rh, lam, mu, rho, bx, bz, mxz);

  FN(el_box) bn, bs;
  int rc = FN(el_src_box)(cfg, x0s, 0.0, 0.0, Nz, Nx, &bn);
  if (rc == 0) rc = FN(el_src_box)(cfg, x0s, 0.5, 0.5, Nz - 1, Nx - 1, &bs);

/* field readers with zero outside the valid index ranges */
#define IN(iR, jR) ((iR) >= 0 && (iR) < Nz && (jR) >= 0 && (jR) < Nx)
#define SXX(iR, jR) (IN(iR, jR) ? sxx[(size_t)(iR) * Nx + (jR)] : (REAL)0)
#define SZZ(iR, jR) (IN(iR, jR) ? szz[(size_t)(iR) * Nx + (jR)] : (REAL)0)
#define SXZ(iR, jR) (((iR) >= 0 && (iR) < Nz - 1 && (jR) >= 0 && (jR) < Nx - 1) ? sxz[(size_t)(iR) * Nx + (jR)] : (REAL)0)
#define VX(iR, jR) (((iR) >= 0 && (iR) < Nz && (jR) >= 0 && (jR) < Nx - 1) ? vx[(size_t)(iR) * Nx + (jR)] : (REAL)0)
#define VZ(iR, jR) (((iR) >= 0 && (iR) < Nz - 1 && (jR) >= 0 && (jR) < Nx) ? vz[(size_t)(iR) * Nx + (jR)] : (REAL)0)

  for (int n = 0; rc == 0 && n < nt; n++) {
    if (snap && n == snap_step) {
      memcpy(snap, vx, sizeof(REAL) * NN);
      memcpy(snap + NN, vz, sizeof(REAL) * NN);
      memcpy(snap + 2 * NN, sxx, sizeof(REAL) * NN);
      memcpy(snap + 3 * NN, szz, sizeof(REAL) * NN);
      memcpy(snap + 4 * NN, sxz, sizeof(REAL) * NN);
    }
    REAL *st = store ? store + (size_t)n * 5 * NN : NULL;
    /* velocity: v^{n+1/2} = v^{n-1/2} + dt b (div sigma^n + CPML) */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx - 1; j++) {
        REAL d1 = 0, d2 = 0;
        for (int k = 1; k <= N; k++) {
          d1 += a[k - 1] * (SXX(i, j + k) - SXX(i, j - k + 1));
          d2 += a[k - 1] * (SXZ(i + k - 1, j) - SXZ(i - k, j));
        }
        d1 /= dx;
        d2 /= dz;
        size_t id = (size_t)i * Nx + j;
        mem[0][id] = bxh[j] * mem[0][id] + axh[j] * d1;
        mem[1][id] = bzt[i] * mem[1][id] + az[i] * d2;
        REAL f = d1 + mem[0][id] + d2 + mem[1][id];
        if (st) st[id] = f;
        vx[id] += dt * bx[id] * f;
      }
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx; j++) {
        REAL d3 = 0, d4 = 0;
        for (int k = 1; k <= N; k++) {
          d3 += a[k - 1] * (SXZ(i, j + k - 1) - SXZ(i, j - k));
          d4 += a[k - 1] * (SZZ(i + k, j) - SZZ(i - k + 1, j));
        }
        d3 /= dx;
        d4 /= dz;
        size_t id = (size_t)i * Nx + j;
        mem[2][id] = bxt[j] * mem[2][id] + ax[j] * d3;
        mem[3][id] = bzh[i] * mem[3][id] + azh[i] * d4;
        REAL f = d3 + mem[2][id] + d4 + mem[3][id];
        if (st) st[NN + id] = f;
        vz[id] += dt * bz[id] * f;
      }
    /* receivers sample v^{n+1/2} at their cell's vx and vz nodes */
    for (int r = 0; r < cfg->nrec; r++) {
      int iR = cfg->rec_iz[r] + np, jR = cfg->rec_ix[r] + np;
      seis[(size_t)r * nt + n] = VX(iR, jR);
      seis[((size_t)cfg->nrec + r) * nt + n] = VZ(iR, jR);
    }
    /* stress: sigma^{n+1} = sigma^n + dt C (grad v^{n+1/2} + CPML) */
    for (int i = 0; i < Nz; i++)
      for (int j = 0; j < Nx; j++) {
        REAL d5 = 0, d6 = 0;
        for (int k = 1; k <= N; k++) {
          d5 += a[k - 1] * (VX(i, j + k - 1) - VX(i, j - k));
          d6 += a[k - 1] * (VZ(i + k - 1, j) - VZ(i - k, j));
        }
        d5 /= dx;
        d6 /= dz;
        size_t id = (size_t)i * Nx + j;
        mem[4][id] = bxt[j] * mem[4][id] + ax[j] * d5;
        mem[5][id] = bzt[i] * mem[5][id] + az[i] * d6;
        REAL ex = d5 + mem[4][id], ez = d6 + mem[5][id];
        if (st) {
          st[2 * NN + id] = ex;
          st[3 * NN + id] = ez;
        }
        sxx[id] += dt * ((lam[id] + 2.0 * mu[id]) * ex + lam[id] * ez);
        szz[id] += dt * (lam[id] * ex + (lam[id] + 2.0 * mu[id]) * ez);
      }
    for (int i = 0; i < Nz - 1; i++)
      for (int j = 0; j < Nx - 1; j++) {
        REAL d7 = 0, d8 = 0;
        for (int k = 1; k <= N; k++) {
          d7 += a[k - 1] * (VX(i + k, j) - VX(i - k + 1, j));
          d8 += a[k - 1] * (VZ(i, j + k) - VZ(i, j - k + 1));
        }
        d7 /= dz;
        d8 /= dx;
        size_t id = (size_t)i * Nx + j;
        mem[6][id] = bzh[i] * mem[6][id] + azh[i] * d7;
        mem[7][id] = bxh[j] * mem[7][id] + axh[j] * d8;
        REAL exz = d7 + mem[6][id] + d8 + mem[7][id];
        if (st) st[4 * NN + id] = exz;
        sxz[id] += dt * mxz[id] * exz;
      }
    /* moment-tensor source: sigma <- sigma - dt M g(t_n) w */
    for (int di = 0; di < bn.n; di++)
      for (int dj = 0; dj < bn.n; dj++) {
        size_t id = (size_t)(bn.i0 + di) * Nx + bn.j0 + dj;
        REAL amp = dt * stf[n] * bn.w[di * bn.n + dj];
        sxx[id] -= amp * mt[0];
        szz[id] -= amp * mt[1];
      }
    for (int di = 0; di < bs.n; di++)
      for (int dj = 0; dj < bs.n; dj++) {
        size_t id = (size_t)(bs.i0 + di) * Nx + bs.j0 + dj;
        sxz[id] -= dt * stf[n] * bs.w[di * bs.n + dj] * mt[2];
      }
  }
  if (snap && snap_step >= nt) {
    memcpy(snap, vx, sizeof(REAL) * NN);
    memcpy(snap + NN, vz, sizeof(REAL) * NN);
    memcpy(snap + 2 * NN, sxx, sizeof(REAL) * NN);
    memcpy(snap + 3 * NN, szz, sizeof(REAL) * NN);
    memcpy(snap + 4 * NN, sxz, sizeof(REAL) * NN);
  }
#undef IN
#undef SXX
#undef SZZ
#undef SXZ
#undef VX
#undef VZ
  free(ax); free(bxt); free(axh); free(bxh); free(az); free(bzt); free(azh); free(bzh);
  free(lam); free(mu); free(rho); free(bx); free(bz); free(mxz);
  free(vx); free(vz); free(sxx); free(szz); free(sxz);
  for (int k = 0; k < 8; k++) free(mem[k]);
  return rc;
}
