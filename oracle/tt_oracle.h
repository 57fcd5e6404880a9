/*
 * tt_oracle.h -- FP64 CPU oracle for backward null-geodesic ray tracing
 * (TARTARUS, arXiv 2609.08989).
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA library
 * against a plain, slow, obviously correct implementation. Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is IEEE binary64, compiled with -ffp-contract=off so that x86-64
 * and aarch64 builds round identically.  Geometric units (G = c = 1); the
 * black-hole mass M and spin a are parameters.
 *
 * Section references are to the paper: Sec. 2.1 (Hamiltonian and equations
 * of motion), Sec. 2.2 (observer, ZAMO tetrad), Sec. 2.3 (Novikov-Thorne /
 * Page-Thorne flux), Sec. 2.4 (redshift, Liouville), Sec. 3.2 (integrators
 * and event functions), Sec. 4.1 (Hamiltonian-constraint monitor).
 */
#ifndef TT_ORACLE_H
#define TT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Termination codes of one ray. */
#define ORC_ESCAPED   0
#define ORC_CAPTURED  1
#define ORC_MAXSTEPS  2
#define ORC_UNDERFLOW 3
#define ORC_NONFINITE 4
#define ORC_BADPIXEL  5

#define ORC_MAXCROSS 3      /* crossings stored per ray */
#define ORC_TABLE_NF 20     /* doubles per table node: 5 fields x (f, f_r, f_th, f_rth) */

/* One scene: spacetime, observer, camera, solver and disk, all in one flat struct. */
typedef struct {
    /* spacetime */
    int    metric_kind;      /* 0 = Kerr closed form, 1 = tabulated metric */
    double M, a;             /* Kerr mass and spin (the disk model always uses these) */
    const double *table;     /* kind 1: nodes[nth][nr][20], see table layout in tt_oracle.c */
    int    nr, nth;
    double r_min, r_max;     /* log-spaced radial nodes; r_min is taken as the horizon */
    /* observer (Sec. 2.2) */
    double r_obs, theta_obs;
    /* camera: cell-centred alpha/beta grid, pixel p = j*nx + i */
    int    nx, ny;
    double alpha_min, alpha_max, beta_min, beta_max;
    /* solver (Sec. 3.2) */
    double rtol, atol;
    double h0;               /* <= 0: automatic initial step */
    double h_min;            /* <= 0: 1e-14 * max(1, |lambda|) */
    long long max_steps;     /* cap on accepted + rejected steps */
    double horizon_eps;      /* captured when r < r_h (1 + eps) */
    double escape_factor;    /* escaped when r > factor * r_obs */
    int    refine;           /* 0 = Henon exact-step, 1 = cubic-Hermite + bisection */
    int    method;           /* 0 = Dormand-Prince, 1 = Cash-Karp, 2 = Fehlberg (5(4) pairs),
                                3 = Gragg-Bulirsch-Stoer, 4 = Verlet (fixed step h0 > 0) */
    /* disk (Sec. 2.3-2.4) */
    int    disk_enabled;
    double r_in;             /* <= 0: prograde ISCO of (M, a) */
    double r_out, mdot;
    int    max_crossings;    /* <= 3 stored */
    int    doppler;          /* 1: full g factor; 0: the Omega p_phi term is dropped */
} orc_scene;

/* Per-pixel outputs (host arrays).  Crossing arrays are crossing-major:
 * element k of pixel p sits at [k * npix + p]. Unused slots hold 0. */
typedef struct {
    int8_t  *code;
    int8_t  *n_cross;
    double  *r_cross;
    double  *g;
    double  *I_cross;
    double  *intensity;
    double  *h_max;
    int32_t *steps;
    int32_t *rejects;
} orc_outputs;

/* ---- metric pieces (exported for the pins) ---- */
void   orc_kerr_lower(double M, double a, double r, double th, double g[16]);
void   orc_kerr_upper(double M, double a, double r, double th,
                      double gi[16], double dgi_r[16], double dgi_th[16]);
int    orc_metric_upper(const orc_scene *s, double r, double th,
                        double gi[16], double dgi_r[16], double dgi_th[16]);
int    orc_metric_lower(const orc_scene *s, double r, double th, double g[16]);
double orc_hamiltonian(const orc_scene *s, const double y[8]);
void   orc_rhs(const orc_scene *s, const double y[8], double dy[8]);
int    orc_initial_state(const orc_scene *s, double alpha, double beta, double y[8]);

/* ---- disk ---- */
double orc_rplus(double M, double a);
double orc_isco(double M, double a);
double orc_flux(double M, double a, double mdot, double r);
double orc_redshift(const orc_scene *s, double r, double p_t, double p_phi);

/* ---- embedded 5(4) pairs on a generic system (exported for the order pins) ---- */
typedef void (*orc_fn)(void *ctx, const double *y, double *dy);
void orc_rk_step(int method, int n, orc_fn f, void *ctx, const double *y, const double *f0,
                 double h, double *ynew, double *fnew, double *err);
int  orc_rk_tableau(int method, double c[7], double a[49], double b[7], double bhat[7]);
void orc_dp5_step(int n, orc_fn f, void *ctx, const double *y, const double *f0,
                  double h, double *ynew, double *fnew, double *err);
void orc_gbs_step(int n, orc_fn f, void *ctx, const double *y, const double *f0, double H, int k,
                  double *ynew, double *fnew, double *err);
void orc_verlet_step(int n, orc_fn f, void *ctx, const double *y, double h, double *ynew, double *fnew);
void orc_dp5_tableau(double c[7], double a[49], double b[7], double bhat[7]);

/* ---- one ray with its accepted-step trajectory (for the pins) ----
 * lam_out[k], y_out[8k..8k+7] for k < min(n_acc+1, cap); the initial state is k = 0.
 * Returns the number of states written. Crossing lambda values go to lamc_out[3]. */
int orc_trace_ray(const orc_scene *s, double alpha, double beta, int cap,
                  double *lam_out, double *y_out, double lamc_out[3],
                  int8_t *code, int8_t *n_cross, double r_cross[3], double g[3],
                  double I_cross[3], double *intensity, double *h_max,
                  int32_t *steps, int32_t *rejects);

/* ---- synthetic numerical metric: Kerr sampled onto the table format ---- */
int orc_kerr_table(double M, double a, int nr, int nth, double r_min, double r_max, double *nodes);

/* ---- whole images ---- */
/* Trace pixels [pix_begin, pix_begin + npix) of the camera into out (npix long). */
int orc_trace(const orc_scene *s, long long pix_begin, long long npix,
              const orc_outputs *out, int nthreads);
/* Trace an explicit list of pixel indices; out is n long. */
int orc_trace_list(const orc_scene *s, const int64_t *pix, long long n,
                   const orc_outputs *out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
