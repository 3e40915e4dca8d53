/*
 * oracle.h - plain FP64 CPU oracle of the seismic-inversion hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library includes, links or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no source with the CUDA path.
 *
 * Every routine restates the paper (Zhu, Xu, Darve & Beroza, "A General
 * Approach to Seismic Inversion with Automatic Differentiation") in the most
 * direct form: scalar loops, FP64, whole-array temporaries, no blocking or
 * fusion. Citations name the paper's section and equation.
 *
 * Grid conventions: the physical model is [nz][nx] (x fastest). It is padded
 * by npml cells of CPML on all four sides; the padded grid is Nz x Nx with
 * Nz = nz + 2 npml, Nx = nx + 2 npml. Positions given in metres are physical
 * coordinates (x = 0, z = 0 at physical cell (0,0)).
 */
#ifndef FWI_ORACLE_H
#define FWI_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Geometry and discretisation of one acoustic problem. */
typedef struct {
  int nz, nx;         /* physical grid */
  int npml;           /* CPML thickness in cells, padded outside the grid */
  int order;          /* spatial order: 4 or 8 (staggered first derivatives) */
  int nt;             /* number of time steps */
  int nshots;
  int src_kind;       /* 0 = point source on the nearest cell, 1 = Gaussian,
                         3 = line of line_len cells along one row (acoustic) */
  int nrec;
  double dz, dx, dt;
  double pml_R, pml_vmax, pml_f0;  /* CPML constants (not differentiated) */
  const int *rec_iz, *rec_ix;      /* [nrec] physical cell indices */
  int line_len;       /* src_kind 3: cells of the line; stf is then [nshots][nt][line_len] */
  int op;             /* acoustic operator: 0 = div(c^2 grad u) (the paper's Eq. acoustic, staggered
                         divergence form, c^2 at half points), 1 = c^2 (Laplacian u), c^2 at cells */
} or_acoustic_cfg;

/* Largest source support: the 7 x 7 Gaussian or a line of line_len cells. */
#define OR_MAX_SUPPORT(cfg) ((cfg)->src_kind == 3 ? ((cfg)->line_len > 49 ? (cfg)->line_len : 49) : 49)
/* Values of stf per shot: nt, or nt * line_len for a line source. */
#define OR_STF_STRIDE(cfg) ((size_t)(cfg)->nt * ((cfg)->src_kind == 3 ? (size_t)(cfg)->line_len : 1))

/* Staggered first-derivative coefficients a_1..a_N (N = order/2). */
int or_fd_coeffs(int order, double *a);

/* 1D CPML coefficients (a, b) at integer (half = 0) or half (half = 1)
 * positions k (+1/2) of a padded axis of n_phys + 2 npml cells. */
void or_cpml_profile(int n_phys, int npml, double h, double dt, double R,
                     double vmax, double f0, int half, int n_out, double *a,
                     double *b);

/* Forward modelling: seis[s][r][n] = u^{n+1}(receiver r) for shot s.
 * c [nz][nx], stf [nshots][nt] (line source: [nshots][nt][line_len], one
 * time function per cell), x0 [nshots][2] = (x, z) metres (line source: the
 * first cell of the line and its row). */
int or_acoustic_forward(const or_acoustic_cfg *cfg, const double *c,
                        const double *stf, const double *x0, double *seis);

/* Same map evaluated in complex arithmetic (for complex-step derivatives);
 * arrays are interleaved (re, im) pairs, i.e. C99 double complex. */
int or_acoustic_forward_cplx(const or_acoustic_cfg *cfg, const void *c,
                             const void *stf, const void *x0, void *seis);

/* Exact discrete adjoint: given the residual res[s][r][n] (the derivative of
 * the misfit with respect to seis), returns the gradients of the misfit with
 * respect to c (summed over shots), stf and x0. Any output may be NULL. */
int or_acoustic_adjoint(const or_acoustic_cfg *cfg, const double *c,
                        const double *stf, const double *x0, const double *res,
                        double *grad_c, double *grad_stf, double *grad_x0);

/* Elastic velocity-stress modelling (same geometry struct; src_kind 0 point,
 * 1 Gaussian spatial weights). vp, vs, rho [nz][nx]; mt [nshots][3] =
 * (Mxx, Mzz, Mxz); seis [nshots][2][nrec][nt] = (vx, vz) of v^{n+1/2}. */
int or_elastic_forward(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                       const double *stf, const double *x0, const double *mt, double *seis);
int or_elastic_forward_cplx(const or_acoustic_cfg *cfg, const void *vp, const void *vs, const void *rho,
                            const void *stf, const void *x0, const void *mt, void *seis);
/* Fields (vx, vz, sxx, szz, sxz) of shot 0 after `step` steps, [5][Nz][Nx]. */
int or_elastic_snapshot(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                        const double *stf, const double *x0, const double *mt, int step, double *fields);
/* Exact adjoint: gradients with respect to lambda, mu, rho (summed over
 * shots), the source time function and x0, for a misfit whose derivative
 * with respect to seis is res. Any output may be NULL. */
int or_elastic_adjoint(const or_acoustic_cfg *cfg, const double *vp, const double *vs, const double *rho,
                       const double *stf, const double *x0, const double *mt, const double *res, double *g_lam,
                       double *g_mu, double *g_rho, double *g_stf, double *g_x0);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
