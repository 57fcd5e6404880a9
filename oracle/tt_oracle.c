/*
 * tt_oracle.c -- FP64 CPU oracle for backward null-geodesic ray tracing
 * (TARTARUS, arXiv 2609.08989).
 *
 * TEST INFRASTRUCTURE ONLY: the reference that the CUDA library is checked
 * against.  It is deliberately plain and slow: the literal 4x4 contraction of
 * the Hamiltonian flow, a generic Dormand-Prince 5(4) stepper over the full
 * 8-dimensional phase-space array, and no fusion or reordering beyond what the
 * definitions state.  It shares no code with the CUDA library.
 *
 * Readings of points the paper leaves open are marked "Reading:" below.
 */
#include "tt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(m, n) ((m) * 4 + (n))   /* index of a 4x4 row-major array, 0=t 1=r 2=th 3=phi */

/* ------------------------------------------------------------------------ */
/* Kerr metric in Boyer-Lindquist coordinates (textbook closed form; the     */
/* paper names the Kerr module in Sec. 3.1 but prints no formula).           */
/* ------------------------------------------------------------------------ */

void orc_kerr_lower(double M, double a, double r, double th, double g[16])
{
    double s = sin(th), c = cos(th);
    double s2 = s * s;
    double Sigma = r * r + a * a * c * c;
    double Delta = r * r - 2.0 * M * r + a * a;
    memset(g, 0, 16 * sizeof(double));
    g[IDX(0, 0)] = -(1.0 - 2.0 * M * r / Sigma);
    g[IDX(0, 3)] = -2.0 * M * a * r * s2 / Sigma;
    g[IDX(3, 0)] = g[IDX(0, 3)];
    g[IDX(1, 1)] = Sigma / Delta;
    g[IDX(2, 2)] = Sigma;
    g[IDX(3, 3)] = (r * r + a * a + 2.0 * M * a * a * r * s2 / Sigma) * s2;
}

/* derivative of n/d given the derivatives dn, dd */
static double dquot(double n, double dn, double d, double dd)
{
    return (dn * d - n * dd) / (d * d);
}

/* Inverse Kerr metric g^{mu nu} and its partial derivatives along r and theta. */
void orc_kerr_upper(double M, double a, double r, double th,
                    double gi[16], double dgi_r[16], double dgi_th[16])
{
    double s = sin(th), c = cos(th);
    double s2 = s * s, a2 = a * a, r2a2 = r * r + a * a;
    double Sigma = r * r + a2 * c * c;
    double Delta = r * r - 2.0 * M * r + a2;
    double Sig_r = 2.0 * r, Sig_th = -2.0 * a2 * s * c;
    double Del_r = 2.0 * r - 2.0 * M;
    double SD = Sigma * Delta;
    double SD_r = Sig_r * Delta + Sigma * Del_r;
    double SD_th = Sig_th * Delta;

    memset(gi, 0, 16 * sizeof(double));
    memset(dgi_r, 0, 16 * sizeof(double));
    memset(dgi_th, 0, 16 * sizeof(double));

    /* g^tt = -[(r^2+a^2)^2 - a^2 Delta sin^2] / (Sigma Delta) */
    double Ntt = r2a2 * r2a2 - a2 * Delta * s2;
    double Ntt_r = 4.0 * r * r2a2 - a2 * Del_r * s2;
    double Ntt_th = -a2 * Delta * 2.0 * s * c;
    gi[IDX(0, 0)] = -Ntt / SD;
    dgi_r[IDX(0, 0)] = -dquot(Ntt, Ntt_r, SD, SD_r);
    dgi_th[IDX(0, 0)] = -dquot(Ntt, Ntt_th, SD, SD_th);

    /* g^tphi = -2 M a r / (Sigma Delta) */
    double Ntp = -2.0 * M * a * r;
    gi[IDX(0, 3)] = Ntp / SD;
    dgi_r[IDX(0, 3)] = dquot(Ntp, -2.0 * M * a, SD, SD_r);
    dgi_th[IDX(0, 3)] = dquot(Ntp, 0.0, SD, SD_th);
    gi[IDX(3, 0)] = gi[IDX(0, 3)];
    dgi_r[IDX(3, 0)] = dgi_r[IDX(0, 3)];
    dgi_th[IDX(3, 0)] = dgi_th[IDX(0, 3)];

    /* g^rr = Delta / Sigma */
    gi[IDX(1, 1)] = Delta / Sigma;
    dgi_r[IDX(1, 1)] = dquot(Delta, Del_r, Sigma, Sig_r);
    dgi_th[IDX(1, 1)] = dquot(Delta, 0.0, Sigma, Sig_th);

    /* g^thth = 1 / Sigma */
    gi[IDX(2, 2)] = 1.0 / Sigma;
    dgi_r[IDX(2, 2)] = dquot(1.0, 0.0, Sigma, Sig_r);
    dgi_th[IDX(2, 2)] = dquot(1.0, 0.0, Sigma, Sig_th);

    /* g^phiphi = (Delta - a^2 sin^2) / (Sigma Delta sin^2) */
    double Npp = Delta - a2 * s2;
    double Dpp = SD * s2;
    gi[IDX(3, 3)] = Npp / Dpp;
    dgi_r[IDX(3, 3)] = dquot(Npp, Del_r, Dpp, SD_r * s2);
    dgi_th[IDX(3, 3)] = dquot(Npp, -2.0 * a2 * s * c, Dpp, SD_th * s2 + SD * 2.0 * s * c);
}

/* ------------------------------------------------------------------------ */
/* Tabulated metric (the paper supports numerically generated metrics,      */
/* abstract and Sec. 5, without giving a format).                            */
/*                                                                          */
/* Reading (format): nodes r_k = r_min (r_max/r_min)^(k/(nr-1)), k < nr,    */
/* theta_j = pi j/(nth-1), j < nth.  Node (j, k) holds 20 doubles at          */
/* table[(j*nr + k)*20]: for each field F in (g_tt, g_tphi, g_thth, g_phiphi, */
/* g^rr), the four numbers F, dF/dr, dF/dth, d2F/(dr dth).                     */
/* Interpolation: bicubic Hermite patches in (u = ln r, theta), using        */
/* dF/du = r dF/dr; the flow uses the interpolant's own derivatives.  Outside */
/* the node range the boundary cell's polynomial is extended (cell index     */
/* clamped, local coordinate not clamped).                                   */
/* ------------------------------------------------------------------------ */

/* cubic Hermite basis on [0,1] and its derivative */
static void hermite_basis(double t, double h[4], double dh[4])
{
    /* h[0]: value at 0, h[1]: slope at 0, h[2]: value at 1, h[3]: slope at 1 */
    h[0] = (1.0 + 2.0 * t) * (1.0 - t) * (1.0 - t);
    h[1] = t * (1.0 - t) * (1.0 - t);
    h[2] = t * t * (3.0 - 2.0 * t);
    h[3] = t * t * (t - 1.0);
    dh[0] = 6.0 * t * t - 6.0 * t;
    dh[1] = 3.0 * t * t - 4.0 * t + 1.0;
    dh[2] = -6.0 * t * t + 6.0 * t;
    dh[3] = 3.0 * t * t - 2.0 * t;
}

/* Interpolate all five fields at (r, th): value, d/dr, d/dth. */
static void table_interp(const orc_scene *s, double r, double th,
                         double f[5], double f_r[5], double f_th[5])
{
    const int nr = s->nr, nth = s->nth;
    const double u0 = log(s->r_min);
    const double du = (log(s->r_max) - u0) / (double)(nr - 1);
    const double dth = M_PI / (double)(nth - 1);
    double tu = (log(r) - u0) / du;
    double tt = th / dth;
    int k = (int)floor(tu), j = (int)floor(tt);
    if (k < 0) k = 0;
    if (k > nr - 2) k = nr - 2;
    if (j < 0) j = 0;
    if (j > nth - 2) j = nth - 2;
    double t = tu - (double)k, w = tt - (double)j;
    double A[4], dA[4], B[4], dB[4];
    hermite_basis(t, A, dA);
    hermite_basis(w, B, dB);
    /* node radii of the cell, for dF/du = r dF/dr */
    double rk[2] = { exp(u0 + (double)k * du), exp(u0 + (double)(k + 1) * du) };

    for (int fi = 0; fi < 5; ++fi) {
        double v = 0.0, vu = 0.0, vt = 0.0;
        for (int cu = 0; cu < 2; ++cu) {
            for (int ct = 0; ct < 2; ++ct) {
                const double *nd = s->table + ((size_t)(j + ct) * nr + (size_t)(k + cu)) * ORC_TABLE_NF + fi * 4;
                double F = nd[0];
                double Fu = rk[cu] * nd[1] * du;          /* slope in the local u coordinate */
                double Ft = nd[2] * dth;                  /* slope in the local theta coordinate */
                double Fut = rk[cu] * nd[3] * du * dth;   /* twist */
                double a0 = A[2 * cu], a1 = A[2 * cu + 1], da0 = dA[2 * cu], da1 = dA[2 * cu + 1];
                double b0 = B[2 * ct], b1 = B[2 * ct + 1], db0 = dB[2 * ct], db1 = dB[2 * ct + 1];
                v  += F * a0 * b0 + Fu * a1 * b0 + Ft * a0 * b1 + Fut * a1 * b1;
                vu += F * da0 * b0 + Fu * da1 * b0 + Ft * da0 * b1 + Fut * da1 * b1;
                vt += F * a0 * db0 + Fu * a1 * db0 + Ft * a0 * db1 + Fut * a1 * db1;
            }
        }
        f[fi] = v;
        f_r[fi] = vu / du / r;     /* d/dr = (d/du) / r, and d/du = (d/dt) / du */
        f_th[fi] = vt / dth;
    }
}

static void table_lower(const orc_scene *s, double r, double th, double g[16])
{
    double f[5], fr[5], ft[5];
    table_interp(s, r, th, f, fr, ft);
    memset(g, 0, 16 * sizeof(double));
    g[IDX(0, 0)] = f[0];
    g[IDX(0, 3)] = f[1];
    g[IDX(3, 0)] = f[1];
    g[IDX(2, 2)] = f[2];
    g[IDX(3, 3)] = f[3];
    g[IDX(1, 1)] = 1.0 / f[4];
}

static void table_upper(const orc_scene *s, double r, double th,
                        double gi[16], double dgi_r[16], double dgi_th[16])
{
    double f[5], fr[5], ft[5];
    table_interp(s, r, th, f, fr, ft);
    memset(gi, 0, 16 * sizeof(double));
    memset(dgi_r, 0, 16 * sizeof(double));
    memset(dgi_th, 0, 16 * sizeof(double));
    double gtt = f[0], gtp = f[1], gthth = f[2], gpp = f[3];
    /* inverse of the (t, phi) block: det D = g_tt g_phiphi - g_tphi^2 */
    double D = gtt * gpp - gtp * gtp;
    double dD[2] = { fr[0] * gpp + gtt * fr[3] - 2.0 * gtp * fr[1],
                     ft[0] * gpp + gtt * ft[3] - 2.0 * gtp * ft[1] };
    const double *d[2] = { fr, ft };
    double *out[2] = { dgi_r, dgi_th };
    gi[IDX(0, 0)] = gpp / D;
    gi[IDX(0, 3)] = -gtp / D;
    gi[IDX(3, 0)] = gi[IDX(0, 3)];
    gi[IDX(3, 3)] = gtt / D;
    gi[IDX(1, 1)] = f[4];
    gi[IDX(2, 2)] = 1.0 / gthth;
    for (int q = 0; q < 2; ++q) {
        out[q][IDX(0, 0)] = dquot(gpp, d[q][3], D, dD[q]);
        out[q][IDX(0, 3)] = -dquot(gtp, d[q][1], D, dD[q]);
        out[q][IDX(3, 0)] = out[q][IDX(0, 3)];
        out[q][IDX(3, 3)] = dquot(gtt, d[q][0], D, dD[q]);
        out[q][IDX(1, 1)] = d[q][4];
        out[q][IDX(2, 2)] = dquot(1.0, 0.0, gthth, d[q][2]);
    }
}

int orc_metric_upper(const orc_scene *s, double r, double th,
                     double gi[16], double dgi_r[16], double dgi_th[16])
{
    if (s->metric_kind == 1) table_upper(s, r, th, gi, dgi_r, dgi_th);
    else orc_kerr_upper(s->M, s->a, r, th, gi, dgi_r, dgi_th);
    return 0;
}

int orc_metric_lower(const orc_scene *s, double r, double th, double g[16])
{
    if (s->metric_kind == 1) table_lower(s, r, th, g);
    else orc_kerr_lower(s->M, s->a, r, th, g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hamiltonian and its flow, Sec. 2.1:                                        */
/*   H = 1/2 g^{mu nu} p_mu p_nu,                                             */
/*   dx^mu/dlambda = g^{mu nu} p_nu,  dp_mu/dlambda = -1/2 d_mu g^{ab} p_a p_b.   */
/* Phase-space array y = [t, r, th, phi, p_t, p_r, p_th, p_phi].             */
/* ------------------------------------------------------------------------ */

double orc_hamiltonian(const orc_scene *s, const double y[8])
{
    double gi[16], dr[16], dt[16];
    orc_metric_upper(s, y[1], y[2], gi, dr, dt);
    const double *p = y + 4;
    double H = 0.0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n)
            H += gi[IDX(m, n)] * p[m] * p[n];
    return 0.5 * H;
}

void orc_rhs(const orc_scene *s, const double y[8], double dy[8])
{
    double gi[16], dgr[16], dgt[16];
    orc_metric_upper(s, y[1], y[2], gi, dgr, dgt);
    const double *p = y + 4;
    for (int m = 0; m < 4; ++m) {
        double v = 0.0;
        for (int n = 0; n < 4; ++n) v += gi[IDX(m, n)] * p[n];
        dy[m] = v;
    }
    double qr = 0.0, qt = 0.0;
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) {
            qr += dgr[IDX(m, n)] * p[m] * p[n];
            qt += dgt[IDX(m, n)] * p[m] * p[n];
        }
    dy[4] = 0.0;            /* the metric does not depend on t */
    dy[5] = -0.5 * qr;
    dy[6] = -0.5 * qt;
    dy[7] = 0.0;            /* nor on phi */
}

static void rhs_cb(void *ctx, const double *y, double *dy)
{
    orc_rhs((const orc_scene *)ctx, y, dy);
}

/* ------------------------------------------------------------------------ */
/* Initial data from the ZAMO tetrad at (r_obs, theta_obs), Sec. 2.2.         */
/* Reading: e_(t)^phi = omega/N (the ZAMO frame the paper names; its list of  */
/* non-zero components omits it but its p^phi uses it).                      */
/* Reading (backward tracing): the physical, future-directed momentum is      */
/* reversed, p_mu -> -p_mu, and lambda increases: the time-reversed geodesic.  */
/* ------------------------------------------------------------------------ */

int orc_initial_state(const orc_scene *s, double alpha, double beta, double y[8])
{
    const double D = s->r_obs, th = s->theta_obs;
    double rho2 = alpha * alpha + beta * beta;
    if (!(rho2 < D * D)) return -1;
    double g[16];
    orc_metric_lower(s, D, th, g);
    double gtt = g[IDX(0, 0)], gtp = g[IDX(0, 3)], grr = g[IDX(1, 1)];
    double gthth = g[IDX(2, 2)], gpp = g[IDX(3, 3)];
    double omega = -gtp / gpp;
    double N = sqrt(-gtt + omega * omega * gpp);
    /* local components */
    double pl_t = 1.0;
    double pl_r = sqrt(1.0 - rho2 / (D * D));
    double pl_th = beta / D;
    double pl_ph = -alpha / D;
    /* coordinate components p^mu = e_(a)^mu p^(a) */
    double pu[4];
    pu[0] = pl_t / N;
    pu[1] = pl_r / sqrt(grr);
    pu[2] = pl_th / sqrt(gthth);
    pu[3] = omega / N * pl_t + pl_ph / sqrt(gpp);
    /* lower with g_{mu nu} */
    double pd[4];
    for (int m = 0; m < 4; ++m) {
        double v = 0.0;
        for (int n = 0; n < 4; ++n) v += g[IDX(m, n)] * pu[n];
        pd[m] = v;
    }
    y[0] = 0.0;
    y[1] = D;
    y[2] = th;
    y[3] = 0.0;
    for (int m = 0; m < 4; ++m) y[4 + m] = -pd[m];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Embedded Runge-Kutta 5(4) pairs of Sec. 3.2: Dormand-Prince (1980, seven    */
/* stages, first-same-as-last), Cash-Karp (1990) and Fehlberg (1969, six     */
/* stages each).  In all three the fifth-order weights advance the solution   */
/* (local extrapolation) and the difference to the embedded fourth-order      */
/* weights is the error estimate.                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int stages;          /* number of stages */
    int fsal;            /* the last stage sits at the new solution */
    double c[7], a[7][6], b[7], bhat[7];
} rk_tableau;

static const rk_tableau TAB_DP = {
    7, 1,
    { 0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0 },
    { { 0, 0, 0, 0, 0, 0 },
      { 1.0 / 5.0, 0, 0, 0, 0, 0 },
      { 3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0 },
      { 44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0 },
      { 19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0 },
      { 9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0 },
      { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0 } },
    { 35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0 },
    { 5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0 },
};

static const rk_tableau TAB_CK = {
    6, 0,
    { 0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0, 0.0 },
    { { 0, 0, 0, 0, 0, 0 },
      { 1.0 / 5.0, 0, 0, 0, 0, 0 },
      { 3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0 },
      { 3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0, 0 },
      { -11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0, 0 },
      { 1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0, 0 },
      { 0, 0, 0, 0, 0, 0 } },
    { 37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0, 0.0 },
    { 2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0, 1.0 / 4.0, 0.0 },
};

static const rk_tableau TAB_F = {
    6, 0,
    { 0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0, 0.0 },
    { { 0, 0, 0, 0, 0, 0 },
      { 1.0 / 4.0, 0, 0, 0, 0, 0 },
      { 3.0 / 32.0, 9.0 / 32.0, 0, 0, 0, 0 },
      { 1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0, 0 },
      { 439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0, 0 },
      { -8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0, 0 },
      { 0, 0, 0, 0, 0, 0 } },
    { 16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0, 0.0 },
    { 25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0, 0.0 },
};

/* method: 0 Dormand-Prince, 1 Cash-Karp, 2 Fehlberg */
static const rk_tableau *tableau_of(int method)
{
    return method == 1 ? &TAB_CK : (method == 2 ? &TAB_F : &TAB_DP);
}

int orc_rk_tableau(int method, double c[7], double a[49], double b[7], double bhat[7])
{
    const rk_tableau *t = tableau_of(method);
    for (int i = 0; i < 7; ++i) {
        c[i] = t->c[i];
        b[i] = t->b[i];
        bhat[i] = t->bhat[i];
        for (int j = 0; j < 7; ++j) a[i * 7 + j] = (j < 6) ? t->a[i][j] : 0.0;
    }
    return t->stages;
}

void orc_dp5_tableau(double c[7], double a[49], double b[7], double bhat[7])
{
    orc_rk_tableau(0, c, a, b, bhat);
}

#define ORC_NMAX 8

/* One step of size h from (y, f0 = f(y)).  ynew is the fifth-order solution,
 * fnew = f(ynew) (the last stage itself for Dormand-Prince, an extra
 * evaluation otherwise), err = ynew - yhat (fourth order). */
void orc_rk_step(int method, int n, orc_fn f, void *ctx, const double *y, const double *f0,
                 double h, double *ynew, double *fnew, double *err)
{
    const rk_tableau *t = tableau_of(method);
    double k[7][ORC_NMAX], ys[ORC_NMAX];
    for (int i = 0; i < n; ++i) k[0][i] = f0[i];
    for (int st = 1; st < t->stages; ++st) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < st; ++j) acc += t->a[st][j] * k[j][i];
            ys[i] = y[i] + h * acc;
        }
        f(ctx, ys, k[st]);
    }
    for (int i = 0; i < n; ++i) {
        if (t->fsal) {
            ynew[i] = ys[i];             /* the last stage sits at the fifth-order solution */
        } else {
            double acc = 0.0;
            for (int j = 0; j < t->stages; ++j) acc += t->b[j] * k[j][i];
            ynew[i] = y[i] + h * acc;
        }
        double e = 0.0;
        for (int j = 0; j < t->stages; ++j) e += (t->b[j] - t->bhat[j]) * k[j][i];
        err[i] = h * e;
    }
    if (t->fsal) {
        for (int i = 0; i < n; ++i) fnew[i] = k[t->stages - 1][i];
    } else {
        f(ctx, ynew, fnew);
    }
}

void orc_dp5_step(int n, orc_fn f, void *ctx, const double *y, const double *f0,
                  double h, double *ynew, double *fnew, double *err)
{
    orc_rk_step(0, n, f, ctx, y, f0, h, ynew, fnew, err);
}

/* ------------------------------------------------------------------------ */
/* Gragg-Bulirsch-Stoer (Sec. 3.2): over a macro-step H, Gragg's modified     */
/* midpoint rule with n_j = 2j sub-steps (j = 1..k; no smoothing step), whose  */
/* error has an expansion in even powers of H/n_j, then Aitken-Neville        */
/* extrapolation of the k results to sub-step size 0 in (H/n_j)^2.            */
/* Reading: k = 6 columns; the solution is the diagonal entry T_kk (order 2k) */
/* and the error estimate T_kk - T_k,k-1; see the step control in trace_one.  */
/* The midpoint chain and the extrapolation act on the increment z - y0, the  */
/* same values in exact arithmetic: the error estimate is a small difference  */
/* of the extrapolated values, and increments keep the rounding in it         */
/* relative to the step's change instead of to |y| (r ~ 10^3 here).           */
/* ------------------------------------------------------------------------ */

#define ORC_GBS_KMAX 8
#define ORC_GBS_K 6

void orc_gbs_step(int n, orc_fn f, void *ctx, const double *y, const double *f0, double H, int k,
                  double *ynew, double *fnew, double *err)
{
    double T[ORC_GBS_KMAX][ORC_GBS_KMAX][ORC_NMAX];   /* T[j-1][l-1] = T_{j,l} - y */
    double d0[ORC_NMAX], d1[ORC_NMAX], d2[ORC_NMAX], z[ORC_NMAX], fz[ORC_NMAX];
    if (k < 1) k = 1;
    if (k > ORC_GBS_KMAX) k = ORC_GBS_KMAX;
    for (int j = 1; j <= k; ++j) {
        int nj = 2 * j;
        double h = H / (double)nj;
        /* modified midpoint on the increment d = z - y: d_0 = 0, d_1 = h f(y),
         * d_{m+1} = d_{m-1} + 2h f(y + d_m) */
        for (int i = 0; i < n; ++i) {
            d0[i] = 0.0;
            d1[i] = h * f0[i];
        }
        for (int m = 1; m < nj; ++m) {
            for (int i = 0; i < n; ++i) z[i] = y[i] + d1[i];
            f(ctx, z, fz);
            for (int i = 0; i < n; ++i) {
                d2[i] = d0[i] + 2.0 * h * fz[i];
                d0[i] = d1[i];
                d1[i] = d2[i];
            }
        }
        for (int i = 0; i < n; ++i) T[j - 1][0][i] = d1[i];
        /* Aitken-Neville in h^2: T_{j,l+1} = T_{j,l} + (T_{j,l} - T_{j-1,l}) / ((n_j / n_{j-l})^2 - 1) */
        for (int l = 1; l < j; ++l) {
            double ratio = (double)nj / (double)(2 * (j - l));
            double den = ratio * ratio - 1.0;
            for (int i = 0; i < n; ++i)
                T[j - 1][l][i] = T[j - 1][l - 1][i] + (T[j - 1][l - 1][i] - T[j - 2][l - 1][i]) / den;
        }
    }
    for (int i = 0; i < n; ++i) {
        ynew[i] = y[i] + T[k - 1][k - 1][i];
        err[i] = (k > 1) ? T[k - 1][k - 1][i] - T[k - 1][k - 2][i] : 0.0;
    }
    f(ctx, ynew, fnew);
}

/* ------------------------------------------------------------------------ */
/* Verlet (Sec. 3.2): the Stormer-Verlet scheme for a general Hamiltonian     */
/* H(q, p) (the generalised leapfrog; Hairer, Lubich & Wanner, Geometric      */
/* Numerical Integration, Sec. VI.3), symmetric and symplectic, fixed step h: */
/*   p+ = p - h/2 dH/dq(q, p+)                     (implicit in p+)           */
/*   Q  = q + h/2 [dH/dp(q, p+) + dH/dp(Q, p+)]     (implicit in Q)           */
/*   P  = p+ - h/2 dH/dq(Q, p+)                                                */
/* The state holds q in its first n/2 and p in its last n/2 entries, and f    */
/* returns (dH/dp, -dH/dq).  Reading: both implicit equations are solved by   */
/* fixed-point iteration from the explicit guess, until no component moves    */
/* by more than 1e-15 max(1, |value|), at most 50 iterations.                  */
/* ------------------------------------------------------------------------ */

#define ORC_VERLET_ITMAX 50

static int moved(const double *a, const double *b, int m)
{
    for (int i = 0; i < m; ++i)
        if (fabs(a[i] - b[i]) > 1e-15 * fmax(1.0, fabs(b[i]))) return 1;
    return 0;
}

void orc_verlet_step(int n, orc_fn f, void *ctx, const double *y, double h, double *ynew, double *fnew)
{
    const int m = n / 2;
    double w[ORC_NMAX], g[ORC_NMAX], nxt[ORC_NMAX], a[ORC_NMAX];
    /* half kick: p+ = p + h/2 * (-dH/dq)(q, p+) */
    memcpy(w, y, sizeof(double) * n);
    f(ctx, w, g);
    for (int i = 0; i < m; ++i) w[m + i] = y[m + i] + 0.5 * h * g[m + i];
    for (int it = 0; it < ORC_VERLET_ITMAX; ++it) {
        f(ctx, w, g);
        for (int i = 0; i < m; ++i) nxt[i] = y[m + i] + 0.5 * h * g[m + i];
        int mv = moved(nxt, w + m, m);
        for (int i = 0; i < m; ++i) w[m + i] = nxt[i];
        if (!mv) break;
    }
    /* drift: Q = q + h/2 (dH/dp(q, p+) + dH/dp(Q, p+)) */
    f(ctx, w, g);                              /* w = (q, p+) */
    for (int i = 0; i < m; ++i) {
        a[i] = g[i];
        w[i] = y[i] + h * a[i];
    }
    for (int it = 0; it < ORC_VERLET_ITMAX; ++it) {
        f(ctx, w, g);
        for (int i = 0; i < m; ++i) nxt[i] = y[i] + 0.5 * h * (a[i] + g[i]);
        int mv = moved(nxt, w, m);
        for (int i = 0; i < m; ++i) w[i] = nxt[i];
        if (!mv) break;
    }
    /* second half kick, explicit */
    f(ctx, w, g);                              /* w = (Q, p+) */
    for (int i = 0; i < m; ++i) {
        ynew[i] = w[i];
        ynew[m + i] = w[m + i] + 0.5 * h * g[m + i];
    }
    f(ctx, ynew, fnew);
}

/* Reading (error norm): Hairer's mean-square norm over the dynamical
 * components r, theta, p_r, p_theta (t and phi are cyclic and never feed back;
 * p_t, p_phi are constants):
 *   err2 = (1/n) sum_i (e_i / (atol + rtol max(|y_i|, |ynew_i|)))^2,  accept if err2 <= 1. */
static const int NORM_IDX[4] = { 1, 2, 5, 6 };

static double err_norm2(const orc_scene *s, const double *y, const double *yn, const double *e,
                        const int *idx, int n)
{
    double acc = 0.0;
    for (int q = 0; q < n; ++q) {
        int i = idx[q];
        double sc = s->atol + s->rtol * fmax(fabs(y[i]), fabs(yn[i]));
        double v = e[i] / sc;
        acc += v * v;
    }
    return acc / (double)n;
}

/* Reading (initial step): the starting-step algorithm of Hairer, Norsett &
 * Wanner, Solving ODEs I, Sec. II.4, with the embedded order p = 4 and the same
 * four-component norm (scales atol + rtol |y0_i|). */
static double initial_step(const orc_scene *s, const double *y0, const double *f0)
{
    double d0 = 0.0, d1 = 0.0;
    for (int q = 0; q < 4; ++q) {
        int i = NORM_IDX[q];
        double sc = s->atol + s->rtol * fabs(y0[i]);
        d0 += (y0[i] / sc) * (y0[i] / sc);
        d1 += (f0[i] / sc) * (f0[i] / sc);
    }
    d0 = sqrt(d0 / 4.0);
    d1 = sqrt(d1 / 4.0);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    double y1[8], f1[8];
    for (int i = 0; i < 8; ++i) y1[i] = y0[i] + h0 * f0[i];
    orc_rhs(s, y1, f1);
    double d2 = 0.0;
    for (int q = 0; q < 4; ++q) {
        int i = NORM_IDX[q];
        double sc = s->atol + s->rtol * fabs(y0[i]);
        double v = (f1[i] - f0[i]) / sc;
        d2 += v * v;
    }
    d2 = sqrt(d2 / 4.0) / h0;
    double dm = fmax(d1, d2);
    double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / 5.0);
    return fmin(100.0 * h0, h1);
}

/* ------------------------------------------------------------------------ */
/* Disk: horizon, ISCO, Page-Thorne flux (Sec. 2.3), redshift (Sec. 2.4).     */
/* ------------------------------------------------------------------------ */

double orc_rplus(double M, double a)
{
    return M + sqrt(M * M - a * a);
}

/* Prograde ISCO (Bardeen, Press & Teukolsky 1972), spin a >= 0. */
double orc_isco(double M, double a)
{
    double as = a / M;
    double z1 = 1.0 + cbrt(1.0 - as * as) * (cbrt(1.0 + as) + cbrt(1.0 - as));
    double z2 = sqrt(3.0 * as * as + z1 * z1);
    return M * (3.0 + z2 - sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2)));
}

/* Page-Thorne flux as printed in Sec. 2.3, in x = sqrt(r/M), times mdot / M^2.
 * Reading: the printed prefactor 3/(2 x^4 (x^3 - 3x + 2a)) is kept as is.
 * The roots x_i of x^3 - 3x + 2a = 0 are the three trigonometric forms printed
 * there; at a = 0 the root x = 0 gives a vanishing term (its limit). */
double orc_flux(double M, double a, double mdot, double r)
{
    double as = a / M;
    double x = sqrt(r / M);
    double x0 = sqrt(orc_isco(M, a) / M);
    if (x < x0) return 0.0;
    double ac = acos(as);
    double xr[3] = { 2.0 * cos((ac - M_PI) / 3.0),
                     2.0 * cos((ac + M_PI) / 3.0),
                     -2.0 * cos(ac / 3.0) };
    double sum = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (xr[i] == 0.0) continue;
        double prod = 1.0;
        for (int j = 0; j < 3; ++j)
            if (j != i) prod *= (xr[i] - xr[j]);
        double coef = 3.0 * (xr[i] - as) * (xr[i] - as) / (xr[i] * prod);
        sum += coef * log((x - xr[i]) / (x0 - xr[i]));
    }
    double bracket = x - x0 - 1.5 * as * log(x / x0) - sum;
    double pref = 3.0 / (2.0 * x * x * x * x * (x * x * x - 3.0 * x + 2.0 * as));
    return mdot * pref * bracket / (M * M);
}

/* g = p_t / (u^t (p_t + Omega p_phi)) for an emitter on a prograde Keplerian
 * orbit, Omega = sqrt(M) / (r^{3/2} + a sqrt(M)), u^t from the normalisation
 * with the equatorial metric; the distant observer is static (Sec. 2.4).
 * Reading (Doppler off): the Omega p_phi term is dropped, g = 1/u^t. */
double orc_redshift(const orc_scene *s, double r, double p_t, double p_phi)
{
    double g[16];
    orc_metric_lower(s, r, M_PI_2, g);
    double Om = sqrt(s->M) / (pow(r, 1.5) + s->a * sqrt(s->M));
    double ut = 1.0 / sqrt(-g[IDX(0, 0)] - 2.0 * Om * g[IDX(0, 3)] - Om * Om * g[IDX(3, 3)]);
    if (!s->doppler) return 1.0 / ut;
    return p_t / (ut * (p_t + Om * p_phi));
}

/* ------------------------------------------------------------------------ */
/* Equatorial crossings, Sec. 3.2 (C_D = cos theta, non-terminal).           */
/* Reading (sign test): cos theta > 0 is evaluated as theta <= pi/2 with the  */
/* binary64 pi/2, which equals the sign of the rounded cosine on (0, pi).     */
/* ------------------------------------------------------------------------ */

static int side_of_equator(double th)
{
    return (th <= M_PI_2) ? 1 : -1;
}

typedef struct {
    const orc_scene *s;
} theta_ctx;

/* the flow re-parameterised by theta: dy/dtheta = f(y) / (dtheta/dlambda) */
static void rhs_in_theta(void *ctx, const double *y, double *dy)
{
    const theta_ctx *c = (const theta_ctx *)ctx;
    double f[8];
    orc_rhs(c->s, y, f);
    for (int i = 0; i < 8; ++i) dy[i] = f[i] / f[2];
}

/* Reading (refinement, default): Henon's exact-step method (M. Henon, Physica D
 * 5, 412, 1982).  From the start of the accepted step, integrate the system in
 * theta with the ray's own adaptive integrator (a 5(4) pair, or the
 * extrapolator; Dormand-Prince for Verlet rays) over Delta theta = pi/2 -
 * theta_k, in 2^m equal
 * sub-steps, m = 0, 1, ... up to 6, taking the first m whose largest sub-step
 * error norm (over r, p_r, p_theta) is <= 1.  The main step sequence is not
 * changed. */
static double refine_henon(const orc_scene *s, const double *y0, const double *f0)
{
    static const int idx3[3] = { 1, 5, 6 };
    theta_ctx ctx = { s };
    double dth = M_PI_2 - y0[2];
    double z[8], gz[8], zn[8], gn[8], e[8];
    for (int m = 0; m <= 6; ++m) {
        int nsub = 1 << m;
        double dl = dth / (double)nsub;
        for (int i = 0; i < 8; ++i) {
            z[i] = y0[i];
            gz[i] = f0[i] / f0[2];
        }
        double worst = 0.0;
        for (int q = 0; q < nsub; ++q) {
            if (s->method == 3)
                orc_gbs_step(8, rhs_in_theta, &ctx, z, gz, dl, ORC_GBS_K, zn, gn, e);
            else
                orc_rk_step(s->method <= 2 ? s->method : 0, 8, rhs_in_theta, &ctx, z, gz, dl, zn, gn, e);
            double e2 = err_norm2(s, z, zn, e, idx3, 3);
            if (!(e2 <= worst)) worst = e2;     /* NaN-propagating max */
            memcpy(z, zn, sizeof z);
            memcpy(gz, gn, sizeof gz);
        }
        if (worst <= 1.0 || m == 6) return z[1];
    }
    return z[1];
}

/* Paper's method (Sec. 3.2): the cubic-Hermite interpolant of the accepted step
 * in lambda, bisected on theta(lambda) - pi/2 until the bracket is <= 1e-12 in
 * lambda; r is read off the Hermite interpolant of r at the midpoint. */
static double refine_hermite(const double *y0, const double *f0,
                             const double *y1, const double *f1, double h, double *s_out)
{
    double lo = 0.0, hi = 1.0;
    int slo = side_of_equator(y0[2]);
    for (int it = 0; it < 200 && (hi - lo) * h > 1e-12; ++it) {
        double mid = 0.5 * (lo + hi);
        double B[4], dB[4];
        hermite_basis(mid, B, dB);
        double th = B[0] * y0[2] + B[1] * h * f0[2] + B[2] * y1[2] + B[3] * h * f1[2];
        if (side_of_equator(th) == slo) lo = mid;
        else hi = mid;
    }
    double sc = 0.5 * (lo + hi);
    double B[4], dB[4];
    hermite_basis(sc, B, dB);
    *s_out = sc;
    return B[0] * y0[1] + B[1] * h * f0[1] + B[2] * y1[1] + B[3] * h * f1[1];
}

/* ------------------------------------------------------------------------ */
/* One ray: Sec. 2.2 initial data, Sec. 3.2 integration and events,           */
/* Sec. 2.3-2.4 emission, Sec. 4.1 Hamiltonian monitor.                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int8_t code, n_cross;
    double r_cross[ORC_MAXCROSS], g[ORC_MAXCROSS], I_cross[ORC_MAXCROSS], lam_cross[ORC_MAXCROSS];
    double intensity, h_max;
    int32_t steps, rejects;
} ray_result;

typedef struct {
    double r_h, r_esc, r_in;
} scene_consts;

static void scene_setup(const orc_scene *s, scene_consts *c)
{
    /* Reading: the table's inner radius is its horizon. */
    c->r_h = (s->metric_kind == 1) ? s->r_min : orc_rplus(s->M, s->a);
    c->r_esc = s->escape_factor * s->r_obs;
    c->r_in = (s->r_in > 0.0) ? s->r_in : orc_isco(s->M, s->a);
}

static int all_finite(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

/* Reading (step control), the 5(4) pairs: h <- h min(facmax, max(0.2,
 * 0.9 err^(-1/5))), facmax = 10, or 1 on the step right after a rejection.
 * Gragg-Bulirsch-Stoer (with the controller constants of Hairer, Norsett &
 * Wanner's extrapolation code): H <- H min(facmax, max(0.02,
 * 0.94 (0.65 / err)^(1/(2k-1)))), facmax = 4, or 1 right after a rejection.
 * Verlet: fixed step.  err = sqrt(err2); after a rejection err > 1, so both
 * factors are below 1 there. */
static double step_factor(int method, double err2, int after_reject)
{
    if (method == 4) return 1.0;
    if (method == 3) {
        double fac = (err2 == 0.0) ? 4.0 : 0.94 * pow(err2 / (0.65 * 0.65), -0.5 / (2.0 * ORC_GBS_K - 1.0));
        return fmin(after_reject ? 1.0 : 4.0, fmax(0.02, fac));
    }
    double fac = (err2 == 0.0) ? 10.0 : 0.9 * pow(err2, -0.1);
    return fmin(after_reject ? 1.0 : 10.0, fmax(0.2, fac));
}

static void trace_one(const orc_scene *s, const scene_consts *c, double alpha, double beta,
                      ray_result *res, int cap, double *lam_out, double *y_out, int *n_out)
{
    memset(res, 0, sizeof *res);
    if (n_out) *n_out = 0;
    double y[8], f[8], yn[8], fn[8], e[8];
    if (!isfinite(alpha) || !isfinite(beta) || orc_initial_state(s, alpha, beta, y) != 0) {
        res->code = ORC_BADPIXEL;
        return;
    }
    orc_rhs(s, y, f);
    res->h_max = fabs(orc_hamiltonian(s, y));
    /* Verlet requires h0 > 0 (its fixed step); the adaptive methods start
     * from h0 if given, else from the starting-step algorithm. */
    double h = (s->h0 > 0.0) ? s->h0 : initial_step(s, y, f);
    double lam = 0.0;
    int last_rejected = 0;
    int nst = 0;
    if (cap > 0) {
        lam_out[0] = 0.0;
        memcpy(y_out, y, sizeof y);
        nst = 1;
    }
    const int maxc = s->max_crossings < ORC_MAXCROSS ? s->max_crossings : ORC_MAXCROSS;

    for (;;) {
        if ((long long)res->steps + (long long)res->rejects >= s->max_steps) {
            res->code = ORC_MAXSTEPS;
            break;
        }
        double hmin = (s->h_min > 0.0) ? s->h_min : 1e-14 * fmax(1.0, fabs(lam));
        if (h < hmin) {
            res->code = ORC_UNDERFLOW;
            break;
        }
        double err2;
        if (s->method == 4) {
            orc_verlet_step(8, rhs_cb, (void *)s, y, h, yn, fn);
            err2 = all_finite(yn, 8) ? 0.0 : NAN;          /* fixed step: always accepted */
        } else {
            if (s->method == 3)
                orc_gbs_step(8, rhs_cb, (void *)s, y, f, h, ORC_GBS_K, yn, fn, e);
            else
                orc_rk_step(s->method, 8, rhs_cb, (void *)s, y, f, h, yn, fn, e);
            err2 = err_norm2(s, y, yn, e, NORM_IDX, 4);
        }
        if (isnan(err2) || !all_finite(yn, 8)) {
            res->code = ORC_NONFINITE;
            break;
        }
        if (err2 <= 1.0) {
            res->steps++;
            /* disk event first (non-terminal), then the terminal events */
            if (s->disk_enabled && side_of_equator(y[2]) != side_of_equator(yn[2])) {
                double rc, lamc;
                if (s->refine == 1) {
                    double sc;
                    rc = refine_hermite(y, f, yn, fn, h, &sc);
                    lamc = lam + sc * h;
                } else {
                    rc = refine_henon(s, y, f);
                    lamc = lam;   /* the theta-parameterised step does not track lambda */
                }
                if (rc >= c->r_in && rc <= s->r_out) {
                    int k = res->n_cross;
                    if (k < maxc) {
                        double gf = orc_redshift(s, rc, yn[4], yn[7]);
                        double F = orc_flux(s->M, s->a, s->mdot, rc);
                        double I = gf * gf * gf * gf * F;     /* Liouville: I_obs = g^4 I_em */
                        res->r_cross[k] = rc;
                        res->g[k] = gf;
                        res->I_cross[k] = I;
                        res->lam_cross[k] = lamc;
                        res->intensity += I;
                    }
                    if (res->n_cross < 127) res->n_cross++;
                }
            }
            lam += h;
            memcpy(y, yn, sizeof y);
            memcpy(f, fn, sizeof f);
            double H = fabs(orc_hamiltonian(s, y));
            if (H > res->h_max) res->h_max = H;
            if (nst < cap) {
                lam_out[nst] = lam;
                memcpy(y_out + 8 * nst, y, sizeof y);
                nst++;
            }
            if (y[1] < c->r_h * (1.0 + s->horizon_eps)) {
                res->code = ORC_CAPTURED;
                break;
            }
            if (y[1] > c->r_esc) {
                res->code = ORC_ESCAPED;
                break;
            }
            h *= step_factor(s->method, err2, last_rejected);
            last_rejected = 0;
        } else {
            res->rejects++;
            h *= step_factor(s->method, err2, 1);
            last_rejected = 1;
        }
    }
    if (n_out) *n_out = nst;
}

static void pixel_coords(const orc_scene *s, long long p, double *alpha, double *beta)
{
    long long i = p % s->nx, j = p / s->nx;
    /* Reading: cell-centred pixels, j ascending in beta. */
    *alpha = s->alpha_min + ((double)i + 0.5) * ((s->alpha_max - s->alpha_min) / (double)s->nx);
    *beta = s->beta_min + ((double)j + 0.5) * ((s->beta_max - s->beta_min) / (double)s->ny);
}

static void store(const orc_outputs *o, long long q, long long n, const ray_result *r)
{
    o->code[q] = r->code;
    o->n_cross[q] = r->n_cross;
    for (int k = 0; k < ORC_MAXCROSS; ++k) {
        o->r_cross[k * n + q] = r->r_cross[k];
        o->g[k * n + q] = r->g[k];
        o->I_cross[k * n + q] = r->I_cross[k];
    }
    o->intensity[q] = r->intensity;
    o->h_max[q] = r->h_max;
    o->steps[q] = r->steps;
    o->rejects[q] = r->rejects;
}

int orc_trace_ray(const orc_scene *s, double alpha, double beta, int cap,
                  double *lam_out, double *y_out, double lamc_out[3],
                  int8_t *code, int8_t *n_cross, double r_cross[3], double g[3],
                  double I_cross[3], double *intensity, double *h_max,
                  int32_t *steps, int32_t *rejects)
{
    scene_consts c;
    scene_setup(s, &c);
    ray_result res;
    int n = 0;
    trace_one(s, &c, alpha, beta, &res, cap, lam_out, y_out, &n);
    *code = res.code;
    *n_cross = res.n_cross;
    for (int k = 0; k < 3; ++k) {
        r_cross[k] = res.r_cross[k];
        g[k] = res.g[k];
        I_cross[k] = res.I_cross[k];
        lamc_out[k] = res.lam_cross[k];
    }
    *intensity = res.intensity;
    *h_max = res.h_max;
    *steps = res.steps;
    *rejects = res.rejects;
    return n;
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_trace(const orc_scene *s, long long pix_begin, long long npix,
              const orc_outputs *out, int nthreads)
{
    scene_consts c;
    scene_setup(s, &c);
    int nt = set_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (long long q = 0; q < npix; ++q) {
        double alpha, beta;
        pixel_coords(s, pix_begin + q, &alpha, &beta);
        ray_result r;
        trace_one(s, &c, alpha, beta, &r, 0, NULL, NULL, NULL);
        store(out, q, npix, &r);
    }
    return 0;
}

int orc_trace_list(const orc_scene *s, const int64_t *pix, long long n,
                   const orc_outputs *out, int nthreads)
{
    scene_consts c;
    scene_setup(s, &c);
    int nt = set_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (long long q = 0; q < n; ++q) {
        double alpha, beta;
        pixel_coords(s, pix[q], &alpha, &beta);
        ray_result r;
        trace_one(s, &c, alpha, beta, &r, 0, NULL, NULL, NULL);
        store(out, q, n, &r);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Synthetic numerical metric: Kerr sampled onto the table format above.     */
/* Fields and their partial derivatives are the textbook closed forms.       */
/* ------------------------------------------------------------------------ */

int orc_kerr_table(double M, double a, int nr, int nth, double r_min, double r_max, double *nodes)
{
    if (nr < 2 || nth < 2 || !(r_min > 0.0) || !(r_max > r_min)) return -1;
    const double u0 = log(r_min);
    const double du = (log(r_max) - u0) / (double)(nr - 1);
    const double a2 = a * a;
    for (int j = 0; j < nth; ++j) {
        double th = M_PI * (double)j / (double)(nth - 1);
        double s = sin(th), c = cos(th);
        if (j == 0) { s = 0.0; c = 1.0; }
        if (j == nth - 1) { s = 0.0; c = -1.0; }
        double s2 = s * s, sc = s * c;
        for (int k = 0; k < nr; ++k) {
            double r = exp(u0 + (double)k * du);
            if (k == 0) r = r_min;
            if (k == nr - 1) r = r_max;
            double r2 = r * r;
            double Sig = r2 + a2 * c * c;
            double Sig2 = Sig * Sig, Sig3 = Sig2 * Sig;
            double Del = r2 - 2.0 * M * r + a2;
            double q = r / Sig;                             /* r / Sigma */
            double q_r = (a2 * c * c - r2) / Sig2;
            double q_t = 2.0 * r * a2 * sc / Sig2;
            double q_rt = 2.0 * a2 * sc * (a2 * c * c - 3.0 * r2) / Sig3;
            double *nd = nodes + ((size_t)j * nr + k) * ORC_TABLE_NF;
            /* g_tt = -1 + 2 M r / Sigma */
            nd[0] = -1.0 + 2.0 * M * q;
            nd[1] = 2.0 * M * q_r;
            nd[2] = 2.0 * M * q_t;
            nd[3] = 2.0 * M * q_rt;
            /* g_tphi = -2 M a sin^2 (r / Sigma) */
            nd[4] = -2.0 * M * a * s2 * q;
            nd[5] = -2.0 * M * a * s2 * q_r;
            nd[6] = -2.0 * M * a * (2.0 * sc * q + s2 * q_t);
            nd[7] = -2.0 * M * a * (2.0 * sc * q_r + s2 * q_rt);
            /* g_thth = Sigma */
            nd[8] = Sig;
            nd[9] = 2.0 * r;
            nd[10] = -2.0 * a2 * sc;
            nd[11] = 0.0;
            /* g_phiphi = (r^2 + a^2) sin^2 + 2 M a^2 sin^4 (r / Sigma) */
            double s4 = s2 * s2, s3c = s2 * sc;
            nd[12] = (r2 + a2) * s2 + 2.0 * M * a2 * s4 * q;
            nd[13] = 2.0 * r * s2 + 2.0 * M * a2 * s4 * q_r;
            nd[14] = (r2 + a2) * 2.0 * sc + 2.0 * M * a2 * (4.0 * s3c * q + s4 * q_t);
            nd[15] = 4.0 * r * sc + 2.0 * M * a2 * (4.0 * s3c * q_r + s4 * q_rt);
            /* g^rr = Delta / Sigma */
            nd[16] = Del / Sig;
            nd[17] = ((2.0 * r - 2.0 * M) * Sig - Del * 2.0 * r) / Sig2;
            nd[18] = 2.0 * a2 * sc * Del / Sig2;
            nd[19] = 2.0 * a2 * sc * ((2.0 * r - 2.0 * M) * Sig - 4.0 * r * Del) / Sig3;
        }
    }
    return 0;
}
