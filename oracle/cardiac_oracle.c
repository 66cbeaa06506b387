/*
 * Oracle for the explicit FP64 cardiac reaction-diffusion step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
 * restatement of what the paper's method computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  The CUDA
 * library never calls it, includes it or shares code, headers or tables with
 * it.  Compiled with -O2 -ffp-contract=off so every operation rounds as
 * written.
 *
 * What it computes (Marcotte & Grigoriev, "Implementation of PDE models of
 * cardiac dynamics on GPUs using OpenCL"):
 *   dz/dt = div(D grad z) + N[z]                              Eq. (rdeqn), Sect. 2
 *   no-flux boundaries, n . grad z = 0                          Eq. (BC:N)
 *   ghost points by flipping displacements back into the grid  Sect. 3, Fig. 1
 *   nine-point Laplacian with diagonal weight alpha_d           Eq. (diffusion)
 *   FitzHugh-Nagumo                                             Eq. (fhn)
 *   two-variable Karma model                                    Eq. (karma), Sect. 2
 *   Bueno-Orovio-Cherry-Fenton with cubic smoothed steps H_k    Eq. (bochfe), Sect. 2
 *   explicit Euler, Heun, classic RK4, fixed dt                 Sect. 3
 *   Rush-Larsen and implicit Euler on the Bueno-Orovio gates    Sect. 3, Table 2
 *   periodic ghosts (opposite-edge values)                      Sect. 3
 *   tanh replaced by 2 H_k - 1 (opt-in model variant)           Sect. 6
 * plus the tangent-linear and discrete adjoint of one explicit RK step (the
 * exact Jacobian of the discrete flow that the Newton-Krylov motivation of
 * Sect. 1 needs).
 *
 * Readings where the paper is silent:
 *  - stencil weights: alpha_a = 1 - 2 alpha_d (consistency), alpha_00 from
 *    the paper's balance condition; anisotropic tensors diag(Dxx, Dyy) use
 *    the form Dxx d_xx + Dyy d_yy + kappa h^2 d_xx d_yy,
 *    kappa = alpha_d (a + b) / 2;
 *  - MIRROR ghost: index -1 maps to 1 and n to n-2 (CLAMP: -1 -> 0, n -> n-1);
 *  - the s-gate of Eq. (bochfe) divides by tau_s;
 *  - the u-dependent time constants and steady states of the cited
 *    Bueno-Orovio model, with every step function replaced by H_k;
 *  - Rush-Larsen / implicit Euler: u takes an explicit Euler step, the gates
 *    v, w, s (linear in themselves) are advanced with u frozen at the start
 *    of the step;
 *  - the tanh variant replaces (1 + tanh(kk x))/2 by H_{kk/3}(x), the smooth
 *    step with the same value and slope at x = 0 (Karma: tanh(u - u_h) by
 *    2 H_{1/3}(u - u_h) - 1);
 *  - Karma: only u diffuses (gamma = D_u); v^M is pow(v, M) as written.
 * Model constants of the Bueno-Orovio epicardial set, and the Karma model's
 * tau_u, tau_v, u*, u_h, u_v, are not printed in the paper (it cites the
 * models' own papers): parity unpinned for those values; the Karma pins fix
 * the form of Eq. (karma) for any constants.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_FHN = 0, ORC_BOCF = 1, ORC_KARMA = 2, ORC_DIFFUSION = 3 };
enum { ORC_ST5 = 0, ORC_ST9 = 1 };
enum { ORC_MIRROR = 0, ORC_CLAMP = 1, ORC_PERIODIC = 2 };
enum { ORC_EULER = 0, ORC_HEUN = 1, ORC_RK4 = 2, ORC_RUSH_LARSEN = 3, ORC_IMPLICIT_EULER = 4 };
enum { ORC_AS_WRITTEN = 0, ORC_TANH_AS_HK = 1 };

#define ORC_MAXF 4
#define ORC_MAXP 32

typedef struct {
    int model, stencil, bc, scheme;
    long nx, ny;
    double dx, dy, alpha_d, dt;
    double Dxx[ORC_MAXF], Dyy[ORC_MAXF];
    double params[ORC_MAXP];
    int variant;        /* ORC_AS_WRITTEN or ORC_TANH_AS_HK (Bueno-Orovio, Karma) */
} orc_problem;

/* ------------------------------------------------------------------ models */

int orc_n_fields(int model)
{
    switch (model) {
    case ORC_FHN: return 2;
    case ORC_BOCF: return 4;
    case ORC_KARMA: return 2;
    case ORC_DIFFUSION: return 1;
    default: return -1;
    }
}

/* Bueno-Orovio parameter order (epicardial set of the model the paper cites
 * in Sect. 2; the values are not printed in the paper). */
enum {
    B_UO, B_UU, B_THV, B_THW, B_THVM, B_THO,
    B_TV1M, B_TV2M, B_TVP, B_TW1M, B_TW2M, B_KWM, B_UWM, B_TWP,
    B_TFI, B_TO1, B_TO2, B_TSO1, B_TSO2, B_KSO, B_USO,
    B_TS1, B_TS2, B_KS, B_US, B_TSI, B_TWINF, B_WINFSTAR, B_K,
    B_NPARAMS
};

/* Karma parameter order: the time constants, u*, u_h, u_v of Eq. (karma),
 * then Re, M and the H_k sharpness k. */
enum { K_TU, K_TV, K_USTAR, K_UH, K_UV, K_RE, K_M, K_K, K_NPARAMS };

int orc_n_params(int model)
{
    switch (model) {
    case ORC_FHN: return 3;           /* eps, a1, a0 */
    case ORC_BOCF: return B_NPARAMS;
    case ORC_KARMA: return K_NPARAMS;
    case ORC_DIFFUSION: return 0;
    default: return -1;
    }
}

int orc_default_params(int model, double *out)
{
    if (model == ORC_FHN) {
        /* Sect. 2: (delta, eps, a1, a0) = (1.5, 0.05, 1.5, -0.1); delta is
         * the v diffusivity and lives in Dxx/Dyy. */
        out[0] = 0.05; out[1] = 1.5; out[2] = -0.1;
        return 3;
    }
    if (model == ORC_BOCF) {
        double p[B_NPARAMS];
        p[B_UO] = 0.0;   p[B_UU] = 1.55;  p[B_THV] = 0.3;  p[B_THW] = 0.13;
        p[B_THVM] = 0.006; p[B_THO] = 0.006;
        p[B_TV1M] = 60.0; p[B_TV2M] = 1150.0; p[B_TVP] = 1.4506;
        p[B_TW1M] = 60.0; p[B_TW2M] = 15.0; p[B_KWM] = 65.0; p[B_UWM] = 0.03;
        p[B_TWP] = 200.0;
        p[B_TFI] = 0.11; p[B_TO1] = 400.0; p[B_TO2] = 6.0;
        p[B_TSO1] = 30.0181; p[B_TSO2] = 0.9957; p[B_KSO] = 2.0458; p[B_USO] = 0.65;
        p[B_TS1] = 2.7342; p[B_TS2] = 16.0; p[B_KS] = 2.0994; p[B_US] = 0.9087;
        p[B_TSI] = 1.8875; p[B_TWINF] = 0.07; p[B_WINFSTAR] = 0.94;
        p[B_K] = 28.4;   /* Sect. 2: k = 28.4 */
        memcpy(out, p, sizeof p);
        return B_NPARAMS;
    }
    if (model == ORC_KARMA) {
        /* Sect. 2 prints (Re, M, gamma) = (1, 6, 0.0011 cm^2/ms) (gamma is
         * D_u and lives in Dxx/Dyy) and k = 28.4; tau_u = 2.5 ms,
         * tau_v = 250 ms, u* = 1.5415, u_h = 3, u_v = 1 are the cited
         * model's values. */
        out[K_TU] = 2.5; out[K_TV] = 250.0; out[K_USTAR] = 1.5415; out[K_UH] = 3.0; out[K_UV] = 1.0;
        out[K_RE] = 1.0; out[K_M] = 6.0; out[K_K] = 28.4;
        return K_NPARAMS;
    }
    if (model == ORC_DIFFUSION) return 0;
    return -1;
}

/* Smoothed step of Sect. 2: 0 for kx < -1/2, 1 for kx > 1/2 and
 * (3 - 2kx - 1)(kx + 1/2)^2 in between. */
double orc_Hk(double x, double k)
{
    double kx = k * x;
    if (kx < -0.5) return 0.0;
    if (kx > 0.5) return 1.0;
    return (3.0 - 2.0 * kx - 1.0) * (kx + 0.5) * (kx + 0.5);
}

/* dH_k/dx: 6k t(1-t) with t = kx + 1/2 on the transition band, else 0. */
double orc_dHk(double x, double k)
{
    double kx = k * x;
    if (kx < -0.5 || kx > 0.5) return 0.0;
    double t = kx + 0.5;
    return 6.0 * k * t * (1.0 - t);
}

/* (1 + tanh(kk (u - cc)))/2 of the cited model, or H_{kk/3}(u - cc) under
 * the tanh variant of Sect. 6 (same value 1/2 and slope kk/2 at u = cc);
 * *d receives the derivative with respect to u. */
static double half_tanh(const orc_problem *p, double u, double kk, double cc, double *d)
{
    if (p->variant == ORC_TANH_AS_HK) {
        *d = orc_dHk(u - cc, kk / 3.0);
        return orc_Hk(u - cc, kk / 3.0);
    }
    double th = tanh(kk * (u - cc));
    *d = kk * (1.0 - th * th) / 2.0;
    return (1.0 + th) / 2.0;
}

/* tanh(u - u_h) of Eq. (karma), or 2 H_{1/3}(u - u_h) - 1 under the tanh
 * variant of Sect. 6; *d (if not NULL) receives the derivative in u. */
static double karma_tanh(const orc_problem *p, double u, double *d)
{
    double x = u - p->params[K_UH];
    if (p->variant == ORC_TANH_AS_HK) {
        if (d) *d = 2.0 * orc_dHk(x, 1.0 / 3.0);
        return 2.0 * orc_Hk(x, 1.0 / 3.0) - 1.0;
    }
    double th = tanh(x);
    if (d) *d = 1.0 - th * th;
    return th;
}

/* Eq. (bochfe) with the currents and the alpha/beta gate form: f = N[z] at
 * one cell and, when alpha is not NULL, the coefficients of the gate
 * equations dx/dt = alpha_x(u) x + beta_x(u) for x = v, w, s. */
static void bocf_eval(const orc_problem *p, const double *z, double *f, double *alpha, double *beta)
{
    const double *q = p->params;
    double d;
    double u = z[0], v = z[1], w = z[2], s = z[3];
    double k = q[B_K];
    /* u-dependent quantities of the cited model */
    double tau_vm = (1.0 - orc_Hk(u - q[B_THVM], k)) * q[B_TV1M] + orc_Hk(u - q[B_THVM], k) * q[B_TV2M];
    double v_inf = orc_Hk(q[B_THVM] - u, k);
    double tau_wm = q[B_TW1M] + (q[B_TW2M] - q[B_TW1M]) * half_tanh(p, u, q[B_KWM], q[B_UWM], &d);
    double w_inf = (1.0 - orc_Hk(u - q[B_THO], k)) * (1.0 - u / q[B_TWINF]) + orc_Hk(u - q[B_THO], k) * q[B_WINFSTAR];
    double tau_o = (1.0 - orc_Hk(u - q[B_THO], k)) * q[B_TO1] + orc_Hk(u - q[B_THO], k) * q[B_TO2];
    double tau_so = q[B_TSO1] + (q[B_TSO2] - q[B_TSO1]) * half_tanh(p, u, q[B_KSO], q[B_USO], &d);
    double tau_s = (1.0 - orc_Hk(u - q[B_THW], k)) * q[B_TS1] + orc_Hk(u - q[B_THW], k) * q[B_TS2];
    double s_inf = half_tanh(p, u, q[B_KS], q[B_US], &d);
    /* currents */
    double J_fi = -v * orc_Hk(u - q[B_THV], k) * (u - q[B_THV]) * (q[B_UU] - u) / q[B_TFI];
    double J_so = (u - q[B_UO]) * orc_Hk(q[B_THW] - u, k) / tau_o + orc_Hk(u - q[B_THW], k) / tau_so;
    double J_si = -orc_Hk(u - q[B_THW], k) * w * s / q[B_TSI];
    /* gates: d x/dt = alpha_x(u) x + beta_x(u) */
    double alpha_v = -orc_Hk(u - q[B_THV], k) / q[B_TVP] - orc_Hk(q[B_THV] - u, k) / tau_vm;
    double beta_v = orc_Hk(q[B_THV] - u, k) * v_inf / tau_vm;
    double alpha_w = -orc_Hk(u - q[B_THW], k) / q[B_TWP] - orc_Hk(q[B_THW] - u, k) / tau_wm;
    double beta_w = orc_Hk(q[B_THW] - u, k) * w_inf / tau_wm;
    f[0] = -(J_fi + J_so + J_si);
    f[1] = alpha_v * v + beta_v;
    f[2] = alpha_w * w + beta_w;
    f[3] = (s_inf - s) / tau_s;
    if (alpha) {
        alpha[0] = alpha_v; beta[0] = beta_v;
        alpha[1] = alpha_w; beta[1] = beta_w;
        alpha[2] = -1.0 / tau_s; beta[2] = s_inf / tau_s;
    }
}

/* N[z] at one cell.  z and f hold the n_v fields of that cell. */
void orc_pointwise(const orc_problem *p, const double *z, double *f)
{
    const double *q = p->params;
    if (p->model == ORC_FHN) {
        /* Eq. (fhn): u - v - u^3 and eps (u - a1 v - a0). */
        double u = z[0], v = z[1];
        f[0] = u - v - u * u * u;
        f[1] = q[0] * (u - q[1] * v - q[2]);
        return;
    }
    if (p->model == ORC_DIFFUSION) {
        f[0] = 0.0;
        return;
    }
    if (p->model == ORC_KARMA) {
        /* Eq. (karma) */
        double u = z[0], v = z[1], k = q[K_K];
        double th = karma_tanh(p, u, NULL);
        f[0] = (u * u / 2.0 * (1.0 - th) * (q[K_USTAR] - pow(v, q[K_M])) - u) / q[K_TU];
        f[1] = ((1.0 / (1.0 - exp(-q[K_RE])) - v) * orc_Hk(u - q[K_UV], k) - v * orc_Hk(q[K_UV] - u, k)) / q[K_TV];
        return;
    }
    bocf_eval(p, z, f, NULL, NULL);
}

/* Jacobian dN/dz at one cell, row-major J[i*n_v + j] = dN_i/dz_j, derived by
 * hand from the formulas of orc_pointwise. */
void orc_pointwise_jac(const orc_problem *p, const double *z, double *J)
{
    const double *q = p->params;
    if (p->model == ORC_FHN) {
        double u = z[0];
        J[0] = 1.0 - 3.0 * u * u; J[1] = -1.0;
        J[2] = q[0];              J[3] = -q[0] * q[1];
        return;
    }
    if (p->model == ORC_DIFFUSION) {
        J[0] = 0.0;
        return;
    }
    if (p->model == ORC_KARMA) {
        /* f_u = (u^2/2 (1 - th) g - u)/tau_u with g = u* - v^M,
         * f_v = ((a - v) H(u - u_v) - v H(u_v - u))/tau_v with
         * a = 1/(1 - e^-Re), differentiated term by term. */
        double u = z[0], v = z[1], k = q[K_K], M = q[K_M];
        double dth, th = karma_tanh(p, u, &dth);
        double g = q[K_USTAR] - pow(v, M);
        double a = 1.0 / (1.0 - exp(-q[K_RE]));
        J[0] = (u * (1.0 - th) * g - u * u / 2.0 * dth * g - 1.0) / q[K_TU];
        J[1] = -(u * u / 2.0) * (1.0 - th) * M * pow(v, M - 1.0) / q[K_TU];
        J[2] = ((a - v) * orc_dHk(u - q[K_UV], k) + v * orc_dHk(q[K_UV] - u, k)) / q[K_TV];
        J[3] = (-orc_Hk(u - q[K_UV], k) - orc_Hk(q[K_UV] - u, k)) / q[K_TV];
        return;
    }
    double u = z[0], v = z[1], w = z[2], s = z[3];
    double k = q[B_K];
    double H1 = orc_Hk(u - q[B_THV], k), dH1 = orc_dHk(u - q[B_THV], k);
    double H2 = orc_Hk(u - q[B_THW], k), dH2 = orc_dHk(u - q[B_THW], k);
    double H3 = orc_Hk(u - q[B_THVM], k), dH3 = orc_dHk(u - q[B_THVM], k);
    double H4 = orc_Hk(u - q[B_THO], k), dH4 = orc_dHk(u - q[B_THO], k);

    double tau_vm = (1.0 - H3) * q[B_TV1M] + H3 * q[B_TV2M];
    double dtau_vm = dH3 * (q[B_TV2M] - q[B_TV1M]);
    double v_inf = 1.0 - H3, dv_inf = -dH3;

    double dsw, sw = half_tanh(p, u, q[B_KWM], q[B_UWM], &dsw);
    double tau_wm = q[B_TW1M] + (q[B_TW2M] - q[B_TW1M]) * sw;
    double dtau_wm = (q[B_TW2M] - q[B_TW1M]) * dsw;

    double w_inf = (1.0 - H4) * (1.0 - u / q[B_TWINF]) + H4 * q[B_WINFSTAR];
    double dw_inf = -dH4 * (1.0 - u / q[B_TWINF]) - (1.0 - H4) / q[B_TWINF] + dH4 * q[B_WINFSTAR];

    double tau_o = (1.0 - H4) * q[B_TO1] + H4 * q[B_TO2];
    double dtau_o = dH4 * (q[B_TO2] - q[B_TO1]);

    double dsso, sso = half_tanh(p, u, q[B_KSO], q[B_USO], &dsso);
    double tau_so = q[B_TSO1] + (q[B_TSO2] - q[B_TSO1]) * sso;
    double dtau_so = (q[B_TSO2] - q[B_TSO1]) * dsso;

    double tau_s = (1.0 - H2) * q[B_TS1] + H2 * q[B_TS2];
    double dtau_s = dH2 * (q[B_TS2] - q[B_TS1]);
    double ds_inf, s_inf = half_tanh(p, u, q[B_KS], q[B_US], &ds_inf);

    /* J_fi = -v H1 (u - thv)(uu - u) / tfi */
    double a = (u - q[B_THV]), b = (q[B_UU] - u);
    double dJfi_du = -v / q[B_TFI] * (dH1 * a * b + H1 * b - H1 * a);
    double dJfi_dv = -H1 * a * b / q[B_TFI];
    /* J_so = (u - uo)(1 - H2)/tau_o + H2/tau_so */
    double c = u - q[B_UO];
    double dJso_du = (1.0 - H2) / tau_o - c * dH2 / tau_o - c * (1.0 - H2) * dtau_o / (tau_o * tau_o)
                     + dH2 / tau_so - H2 * dtau_so / (tau_so * tau_so);
    /* J_si = -H2 w s / tsi */
    double dJsi_du = -dH2 * w * s / q[B_TSI];
    double dJsi_dw = -H2 * s / q[B_TSI];
    double dJsi_ds = -H2 * w / q[B_TSI];

    /* row u */
    J[0] = -(dJfi_du + dJso_du + dJsi_du);
    J[1] = -dJfi_dv;
    J[2] = -dJsi_dw;
    J[3] = -dJsi_ds;
    /* row v: (1 - H1)(v_inf - v)/tau_vm - H1 v / tvp */
    J[4] = -dH1 * (v_inf - v) / tau_vm
           + (1.0 - H1) * (dv_inf / tau_vm - (v_inf - v) * dtau_vm / (tau_vm * tau_vm))
           - dH1 * v / q[B_TVP];
    J[5] = -(1.0 - H1) / tau_vm - H1 / q[B_TVP];
    J[6] = 0.0; J[7] = 0.0;
    /* row w: (1 - H2)(w_inf - w)/tau_wm - H2 w / twp */
    J[8] = -dH2 * (w_inf - w) / tau_wm
           + (1.0 - H2) * (dw_inf / tau_wm - (w_inf - w) * dtau_wm / (tau_wm * tau_wm))
           - dH2 * w / q[B_TWP];
    J[9] = 0.0;
    J[10] = -(1.0 - H2) / tau_wm - H2 / q[B_TWP];
    J[11] = 0.0;
    /* row s: (s_inf - s)/tau_s */
    J[12] = ds_inf / tau_s - (s_inf - s) * dtau_s / (tau_s * tau_s);
    J[13] = 0.0; J[14] = 0.0;
    J[15] = -1.0 / tau_s;
}

/* ------------------------------------------------------------- diffusion */

/* Neighbour index with the ghost rule of Sect. 3: MIRROR flips the
 * displacement back into the grid, CLAMP repeats the edge value, PERIODIC
 * takes the opposite edge's value. */
static long map_index(long i, long n, int bc)
{
    if (bc == ORC_PERIODIC) return ((i % n) + n) % n;
    if (i < 0) return bc == ORC_MIRROR ? -i : 0;
    if (i >= n) return bc == ORC_MIRROR ? 2 * (n - 1) - i : n - 1;
    return i;
}

/* 3x3 weights of D_f L for field f, w[(l+1)*3 + (k+1)] for displacement
 * (k in x, l in y).  Isotropic D with dx = dy = h reproduces Eq. (diffusion)
 * divided by h^2 with alpha_a = 1 - 2 alpha_d and alpha_00 = -4(alpha_a +
 * alpha_d). */
static void stencil_weights(const orc_problem *p, double Dxx, double Dyy, double *w)
{
    double a = Dxx / (p->dx * p->dx);
    double b = Dyy / (p->dy * p->dy);
    double ad = (p->stencil == ORC_ST9) ? p->alpha_d : 0.0;
    double kappa = ad * (a + b) / 2.0;
    double wx = a - 2.0 * kappa, wy = b - 2.0 * kappa, wd = kappa;
    double wc = -2.0 * a - 2.0 * b + 4.0 * kappa;
    w[0] = wd; w[1] = wy; w[2] = wd;
    w[3] = wx; w[4] = wc; w[5] = wx;
    w[6] = wd; w[7] = wy; w[8] = wd;
}

/* out = D_f L u on one plane (gather form).  Neighbours are summed in
 * mirror-image pairs (W+E, N+S, NE+SW, NW+SE) so that x-flips, y-flips and
 * the transpose map every sum onto itself bit for bit. */
void orc_apply_L(const orc_problem *p, double Dxx, double Dyy, const double *u, double *out)
{
    double w[9];
    stencil_weights(p, Dxx, Dyy, w);
    long nx = p->nx, ny = p->ny;
    for (long y = 0; y < ny; ++y) {
        long ys = map_index(y - 1, ny, p->bc), yn = map_index(y + 1, ny, p->bc);
        for (long x = 0; x < nx; ++x) {
            long xw = map_index(x - 1, nx, p->bc), xe = map_index(x + 1, nx, p->bc);
            double C = u[y * nx + x];
            double W = u[y * nx + xw], E = u[y * nx + xe];
            double S = u[ys * nx + x], N = u[yn * nx + x];
            double SW = u[ys * nx + xw], SE = u[ys * nx + xe];
            double NW = u[yn * nx + xw], NE = u[yn * nx + xe];
            out[y * nx + x] = w[3] * (W + E) + w[1] * (N + S)
                              + w[0] * ((NE + SW) + (NW + SE)) + w[4] * C;
        }
    }
}

/* out = (D_f L)^T u: the transpose of the matrix applied by orc_apply_L,
 * accumulated by scattering every stencil coefficient to the cell it reads. */
void orc_apply_LT(const orc_problem *p, double Dxx, double Dyy, const double *u, double *out)
{
    double w[9];
    stencil_weights(p, Dxx, Dyy, w);
    long nx = p->nx, ny = p->ny;
    memset(out, 0, sizeof(double) * (size_t)(nx * ny));
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x)
            for (int l = -1; l <= 1; ++l)
                for (int k = -1; k <= 1; ++k) {
                    long ty = map_index(y + l, ny, p->bc), tx = map_index(x + k, nx, p->bc);
                    out[ty * nx + tx] += w[(l + 1) * 3 + (k + 1)] * u[y * nx + x];
                }
}

/* ------------------------------------------------------------ right side */

/* f = F(z) = D L z + N[z] for the whole grid, layout [n_v][ny][nx]. */
int orc_rhs(const orc_problem *p, const double *z, double *f)
{
    int nv = orc_n_fields(p->model);
    if (nv < 0) return -1;
    long n = p->nx * p->ny;
    double zc[ORC_MAXF], fc[ORC_MAXF];
    for (long i = 0; i < n; ++i) {
        for (int c = 0; c < nv; ++c) zc[c] = z[c * n + i];
        orc_pointwise(p, zc, fc);
        for (int c = 0; c < nv; ++c) f[c * n + i] = fc[c];
    }
    double *lap = malloc(sizeof(double) * (size_t)n);
    for (int c = 0; c < nv; ++c) {
        if (p->Dxx[c] == 0.0 && p->Dyy[c] == 0.0) continue;
        orc_apply_L(p, p->Dxx[c], p->Dyy[c], z + c * n, lap);
        for (long i = 0; i < n; ++i) f[c * n + i] = lap[i] + f[c * n + i];
    }
    free(lap);
    return 0;
}

/* ------------------------------------------------------------ integrators */

/* One explicit step of Sect. 3: Euler z + dt F(z); Heun
 * z + dt/2 (F(z) + F(z + dt F(z))); classic RK4
 * z + dt/6 (k1 + 2 k2 + 2 k3 + k4). */
static void step_once(const orc_problem *p, double *z, long m,
                      double *k1, double *k2, double *k3, double *k4, double *y)
{
    double dt = p->dt;
    if (p->scheme == ORC_EULER) {
        orc_rhs(p, z, k1);
        for (long i = 0; i < m; ++i) z[i] = z[i] + dt * k1[i];
    } else if (p->scheme == ORC_HEUN) {
        orc_rhs(p, z, k1);
        for (long i = 0; i < m; ++i) y[i] = z[i] + dt * k1[i];
        orc_rhs(p, y, k2);
        for (long i = 0; i < m; ++i) z[i] = z[i] + dt / 2.0 * (k1[i] + k2[i]);
    } else if (p->scheme == ORC_RUSH_LARSEN || p->scheme == ORC_IMPLICIT_EULER) {
        /* Sect. 3 / Table 2: u takes an explicit Euler step; each gate
         * x = v, w, s obeys dx/dt = alpha x + beta with alpha, beta taken at
         * the step's starting state.  Rush-Larsen integrates that linear
         * equation exactly, x_inf + (x - x_inf) exp(alpha dt) with
         * x_inf = -beta/alpha; implicit Euler solves
         * x' = x + dt (alpha x' + beta) for x'. */
        long n = p->nx * p->ny;
        double zc[ORC_MAXF], fc[ORC_MAXF], al[3], be[3];
        orc_rhs(p, z, k1);
        for (long i = 0; i < n; ++i) {
            for (int c = 0; c < 4; ++c) zc[c] = z[c * n + i];
            bocf_eval(p, zc, fc, al, be);
            z[i] = z[i] + dt * k1[i];
            for (int g = 0; g < 3; ++g) {
                double x = zc[g + 1], x1;
                if (p->scheme == ORC_RUSH_LARSEN) {
                    double x_inf = -be[g] / al[g];
                    x1 = x_inf + (x - x_inf) * exp(al[g] * dt);
                } else {
                    x1 = (x + dt * be[g]) / (1.0 - dt * al[g]);
                }
                z[(g + 1) * n + i] = x1;
            }
        }
    } else {
        orc_rhs(p, z, k1);
        for (long i = 0; i < m; ++i) y[i] = z[i] + dt / 2.0 * k1[i];
        orc_rhs(p, y, k2);
        for (long i = 0; i < m; ++i) y[i] = z[i] + dt / 2.0 * k2[i];
        orc_rhs(p, y, k3);
        for (long i = 0; i < m; ++i) y[i] = z[i] + dt * k3[i];
        orc_rhs(p, y, k4);
        for (long i = 0; i < m; ++i)
            z[i] = z[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
}

/* Advance z (layout [n_v][ny][nx]) by n_steps in place. */
int orc_step(const orc_problem *p, double *z, long n_steps)
{
    int nv = orc_n_fields(p->model);
    if (nv < 0 || p->nx < 2 || p->ny < 2) return -1;
    if ((p->scheme == ORC_RUSH_LARSEN || p->scheme == ORC_IMPLICIT_EULER) && p->model != ORC_BOCF) return -3;
    long m = nv * p->nx * p->ny;
    double *buf = malloc(sizeof(double) * (size_t)(5 * m));
    if (!buf) return -2;
    for (long s = 0; s < n_steps; ++s)
        step_once(p, z, m, buf, buf + m, buf + 2 * m, buf + 3 * m, buf + 4 * m);
    free(buf);
    return 0;
}

/* ------------------------------------------------ tangent-linear / adjoint */

/* Butcher tableau of the three explicit schemes (same methods as step_once,
 * written as Y_i = z + dt sum_j a_ij k_j, z' = z + dt sum_i b_i k_i). */
static int tableau(int scheme, double A[4][4], double b[4])
{
    memset(A, 0, sizeof(double) * 16);
    memset(b, 0, sizeof(double) * 4);
    if (scheme == ORC_EULER) { b[0] = 1.0; return 1; }
    if (scheme == ORC_HEUN) { A[1][0] = 1.0; b[0] = 0.5; b[1] = 0.5; return 2; }
    if (scheme != ORC_RK4) return -1;   /* the gate integrators have no tableau */
    A[1][0] = 0.5; A[2][1] = 0.5; A[3][2] = 1.0;
    b[0] = 1.0 / 6.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 3.0; b[3] = 1.0 / 6.0;
    return 4;
}

/* out = J_F(Y) d = D L d + dN/dz(Y) d */
static void jvp_F(const orc_problem *p, const double *Y, const double *d, double *out, double *tmp)
{
    int nv = orc_n_fields(p->model);
    long n = p->nx * p->ny;
    double yc[ORC_MAXF], J[ORC_MAXF * ORC_MAXF];
    for (long i = 0; i < n; ++i) {
        for (int c = 0; c < nv; ++c) yc[c] = Y[c * n + i];
        orc_pointwise_jac(p, yc, J);
        for (int r = 0; r < nv; ++r) {
            double acc = 0.0;
            for (int c = 0; c < nv; ++c) acc += J[r * nv + c] * d[c * n + i];
            out[r * n + i] = acc;
        }
    }
    for (int c = 0; c < nv; ++c) {
        if (p->Dxx[c] == 0.0 && p->Dyy[c] == 0.0) continue;
        orc_apply_L(p, p->Dxx[c], p->Dyy[c], d + c * n, tmp);
        for (long i = 0; i < n; ++i) out[c * n + i] += tmp[i];
    }
}

/* out = J_F(Y)^T l = (D L)^T l + dN/dz(Y)^T l */
static void vjp_F(const orc_problem *p, const double *Y, const double *l, double *out, double *tmp)
{
    int nv = orc_n_fields(p->model);
    long n = p->nx * p->ny;
    double yc[ORC_MAXF], J[ORC_MAXF * ORC_MAXF];
    for (long i = 0; i < n; ++i) {
        for (int c = 0; c < nv; ++c) yc[c] = Y[c * n + i];
        orc_pointwise_jac(p, yc, J);
        for (int c = 0; c < nv; ++c) {
            double acc = 0.0;
            for (int r = 0; r < nv; ++r) acc += J[r * nv + c] * l[r * n + i];
            out[c * n + i] = acc;
        }
    }
    for (int c = 0; c < nv; ++c) {
        if (p->Dxx[c] == 0.0 && p->Dyy[c] == 0.0) continue;
        orc_apply_LT(p, p->Dxx[c], p->Dyy[c], l + c * n, tmp);
        for (long i = 0; i < n; ++i) out[c * n + i] += tmp[i];
    }
}

/* Tangent-linear model: advances z and one tangent dz by n_steps. */
int orc_tlm(const orc_problem *p, double *z, double *dz, long n_steps)
{
    int nv = orc_n_fields(p->model);
    if (nv < 0 || p->nx < 2 || p->ny < 2) return -1;
    long n = p->nx * p->ny, m = nv * n;
    double A[4][4], b[4];
    int ns = tableau(p->scheme, A, b);
    if (ns < 0) return -3;
    double dt = p->dt;
    double *K = malloc(sizeof(double) * (size_t)(4 * m));
    double *dK = malloc(sizeof(double) * (size_t)(4 * m));
    double *Y = malloc(sizeof(double) * (size_t)m);
    double *dY = malloc(sizeof(double) * (size_t)m);
    double *tmp = malloc(sizeof(double) * (size_t)n);
    if (!K || !dK || !Y || !dY || !tmp) return -2;
    for (long st = 0; st < n_steps; ++st) {
        for (int i = 0; i < ns; ++i) {
            for (long e = 0; e < m; ++e) {
                double y = z[e], dy = dz[e];
                for (int j = 0; j < i; ++j) {
                    y += dt * A[i][j] * K[j * m + e];
                    dy += dt * A[i][j] * dK[j * m + e];
                }
                Y[e] = y; dY[e] = dy;
            }
            orc_rhs(p, Y, K + i * m);
            jvp_F(p, Y, dY, dK + i * m, tmp);
        }
        for (long e = 0; e < m; ++e) {
            double a = 0.0, da = 0.0;
            for (int i = 0; i < ns; ++i) { a += b[i] * K[i * m + e]; da += b[i] * dK[i * m + e]; }
            z[e] = z[e] + dt * a;
            dz[e] = dz[e] + dt * da;
        }
    }
    free(K); free(dK); free(Y); free(dY); free(tmp);
    return 0;
}

/* Discrete adjoint of n_steps explicit steps from z0.  Given lamT = dL/dz_T
 * it returns lam0 = dL/dz_0 and, per field f, dLdD[f] = dL/dD_f where the
 * field's diffusion tensor is D_f diag(1, Dyy_f/Dxx_f) (the anisotropy ratio
 * held fixed; 0 for non-diffusive fields).  All states are stored. */
int orc_adjoint(const orc_problem *p, const double *z0, const double *lamT,
                double *lam0, double *dLdD, long n_steps)
{
    int nv = orc_n_fields(p->model);
    if (nv < 0 || p->nx < 2 || p->ny < 2) return -1;
    long n = p->nx * p->ny, m = nv * n;
    double A[4][4], b[4];
    int ns = tableau(p->scheme, A, b);
    if (ns < 0) return -3;
    double dt = p->dt;
    double *Z = malloc(sizeof(double) * (size_t)(m * (n_steps + 1)));
    double *Ys = malloc(sizeof(double) * (size_t)(4 * m));
    double *K = malloc(sizeof(double) * (size_t)(4 * m));
    double *Yb = malloc(sizeof(double) * (size_t)(4 * m));
    double *kb = malloc(sizeof(double) * (size_t)m);
    double *lam = malloc(sizeof(double) * (size_t)m);
    double *tmp = malloc(sizeof(double) * (size_t)n);
    double *lapY = malloc(sizeof(double) * (size_t)n);
    if (!Z || !Ys || !K || !Yb || !kb || !lam || !tmp || !lapY) return -2;
    /* forward sweep: store z_0 .. z_n */
    memcpy(Z, z0, sizeof(double) * (size_t)m);
    for (long st = 0; st < n_steps; ++st) {
        memcpy(Z + (st + 1) * m, Z + st * m, sizeof(double) * (size_t)m);
        orc_step(p, Z + (st + 1) * m, 1);
    }
    for (int c = 0; c < nv; ++c) dLdD[c] = 0.0;
    memcpy(lam, lamT, sizeof(double) * (size_t)m);
    for (long st = n_steps - 1; st >= 0; --st) {
        const double *z = Z + st * m;
        /* recompute the stage points Y_i and slopes k_i of this step */
        for (int i = 0; i < ns; ++i) {
            for (long e = 0; e < m; ++e) {
                double y = z[e];
                for (int j = 0; j < i; ++j) y += dt * A[i][j] * K[j * m + e];
                Ys[i * m + e] = y;
            }
            orc_rhs(p, Ys + i * m, K + i * m);
        }
        /* reverse sweep over stages */
        for (int i = ns - 1; i >= 0; --i) {
            for (long e = 0; e < m; ++e) {
                double a = dt * b[i] * lam[e];
                for (int j = i + 1; j < ns; ++j) a += dt * A[j][i] * Yb[j * m + e];
                kb[e] = a;
            }
            vjp_F(p, Ys + i * m, kb, Yb + i * m, tmp);
            for (int c = 0; c < nv; ++c) {
                if (p->Dxx[c] == 0.0) continue;
                orc_apply_L(p, 1.0, p->Dyy[c] / p->Dxx[c], Ys + i * m + c * n, lapY);
                double acc = 0.0;
                for (long e = 0; e < n; ++e) acc += kb[c * n + e] * lapY[e];
                dLdD[c] += acc;
            }
        }
        for (long e = 0; e < m; ++e) {
            double a = lam[e];
            for (int i = 0; i < ns; ++i) a += Yb[i * m + e];
            lam[e] = a;
        }
    }
    memcpy(lam0, lam, sizeof(double) * (size_t)m);
    free(Z); free(Ys); free(K); free(Yb); free(kb); free(lam); free(tmp); free(lapY);
    return 0;
}
