/*
 * rt_oracle.c -- plain FP64 CPU oracle for the column radiative-transfer path
 * of Deitrick et al., "The THOR+HELIOS general circulation model" (arXiv
 * 2203.02293).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may use it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * It is deliberately slow and literal.  Every quantity is evaluated the way
 * the paper writes it, in FP64, from FP32 inputs widened exactly:
 *   - coupling coefficients, transmission and chi/xi/psi: App. B, Eqs. B1-B2
 *   - Pi: Eq. B5; E fit and its switch-off: Eq. 19 (Sec. 2.2.4)
 *   - thermal source terms: Eqs. 2-3 (isothermal), Eqs. 4-9 and B4
 *     (non-isothermal, with the e_tau fallback of Sec. 2.2.1)
 *   - stellar beam and its source terms: Eqs. B6-B8 (Malik sign, mu* < 0),
 *     with the singularity check of Eq. 11 and the text after it
 *   - boundary conditions: Eq. 10 and the caption of Fig. thomas_isothermal
 *   - block-tridiagonal system and block Thomas: Eqs. 12-15 (2x2 blocks)
 *   - the iterative method that Thomas's algorithm replaces (Sec. 2.2.2):
 *     pairwise sweeps through the column, repeated N times
 *   - spectral sum, net flux (beam added to the downward flux, Sec. 2.2.1)
 *     and heating rate.
 * Planck per bin is the bin integral of the Planck function, done by
 * composite Gauss-Legendre quadrature (nodes found by Newton iteration).
 *
 * Readings where the paper is silent or ambiguous (the CUDA path takes the
 * same ones):
 *   - mu* enters G+- with the Malik sign, mu* = -cos(theta*) < 0 (App. B);
 *   - resonance (Eq. 11): when |D| < 1e-5 the paper mode sets D := 2 mu*;
 *     the limit mode keeps the exact solution (see sub_layer for |D| < 1e-7);
 *   - E := max(E_fit, 1) unless the raw fit is asked for (its hits are
 *     counted on E - 1 formed in FP32, see e_fit_m1_f32); the fit applies for
 *     w0 > 0.1f, i.e. the threshold is the FP32 value of 0.1; where the raw
 *     fit gives E < w0, k (Eq. B2) is not real and the system's fluxes are
 *     NaN (counted as non-finite);
 *   - the e_tau test is dtau_sub < 1e-4f with dtau_sub = dtau / 2; both
 *     sub-layers carry the layer's w0, g0 and half its optical depth;
 *   - F_BOA = pi B(T_int) per bin; no beam when cos(theta*) <= 0;
 *   - Q_l = (g / c_P) (F_net,bot - F_net,top) / (p_bot - p_top);
 *   - the block entries of Eq. 12 (the figures that draw them are missing)
 *     are documented in assemble();
 *   - B is the Planck function integrated over the bin;
 *   - E = w0 = 1 uses the k -> 0 limit of the relations (chi, xi, psi all
 *     divided by k) and Pi := pi.
 *
 * Level convention inside the oracle: level 0 is the bottom of the
 * atmosphere (BOA), level n the top (TOA), as in the paper.  Arrays passed
 * in and out follow the library's convention instead: layer 0 and
 * interface 0 are at the TOA.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846264338327950288
/* SI defining constants (exact) */
#define OR_H 6.62607015e-34
#define OR_C 299792458.0
#define OR_KB 1.380649e-23

typedef struct {
    int32_t improved;       /* 1: E from Eq. 19; 0: regular two-stream, E = 1 */
    int32_t isothermal;     /* 1: isothermal layers; 0: non-isothermal */
    int32_t resonance;      /* 0: paper rule (D := 2 mu*); 1: limit (exact solution) */
    int32_t e_clamp;        /* 1: E := max(E_fit, 1); 0: raw fit */
    double eps2;            /* second Eddington coefficient (Table 3: 2/3) */
    double grav, cp;        /* m s^-2, J kg^-1 K^-1 */
    double T_int;           /* K, interior temperature; 0 -> F_BOA = 0 */
    double F_toa;           /* diffuse downward flux at the TOA, W m^-2 */
    double wn_min, wn_max;  /* bin range, cm^-1, bins uniform in wavenumber */
    const double *wn_edges; /* NULL, or the NB + 1 increasing bin edges (cm^-1)
                               shared by every column; then wn_min/wn_max unused */
    int32_t n_sweeps;       /* 0: Thomas's algorithm (Eqs. 12-15); N > 0: the
                               iterative method of Sec. 2.2.2, N sweeps from zero
                               diffuse flux (see sweeps()) */
} oracle_cfg;

typedef struct {
    int64_t resonance_hits;  /* layer-systems with |D| < 1e-5 */
    int64_t etau_hits;       /* sub-layer-systems with dtau_sub < e_tau */
    int64_t eclamp_hits;     /* layer-systems with E_fit < 1 clamped */
    int64_t nonfinite;       /* systems with a non-finite flux */
} oracle_stats;

/* ------------------------------------------------------------------ */
/* Planck function integrated over a wavenumber bin.                    */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    if (!gl_ready) {
        gauss_legendre(GL_N, gl_x, gl_w);
        gl_ready = 1;
    }
}

/* B_nu in wavenumber units: 2 h c^2 nu^3 / (exp(h c nu / k T) - 1),
 * nu in m^-1, result in W m^-2 sr^-1 per m^-1. */
static double planck_wn(double nu, double T)
{
    double x = OR_H * OR_C * nu / (OR_KB * T);
    return 2.0 * OR_H * OR_C * OR_C * nu * nu * nu / expm1(x);
}

/* Bin-integrated Planck function, W m^-2 sr^-1, over [wn_lo, wn_hi] cm^-1. */
double oracle_planck_bin(double T, double wn_lo, double wn_hi)
{
    gl_init();
    if (!(T > 0.0) || !(wn_hi > wn_lo)) return 0.0;
    double a = wn_lo * 100.0, b = wn_hi * 100.0;
    /* sub-intervals no wider than one unit of x = h c nu / k T */
    double dx = OR_H * OR_C * (b - a) / (OR_KB * T);
    int nsub = (int)ceil(dx);
    if (nsub < 4) nsub = 4;
    if (nsub > 100000) nsub = 100000;
    double h = (b - a) / nsub, sum = 0.0;
    for (int s = 0; s < nsub; ++s) {
        double lo = a + s * h, mid = lo + 0.5 * h, acc = 0.0;
        for (int i = 0; i < GL_N; ++i) {
            double nu = mid + 0.5 * h * gl_x[i];
            if (nu > 0.0) acc += gl_w[i] * planck_wn(nu, T);
        }
        sum += 0.5 * h * acc;
    }
    return sum;
}

/* ------------------------------------------------------------------ */
/* Per-layer coefficients, App. B.                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    double E, k, zeta_p, zeta_m, Pi, q;  /* q = E (1 - w0 g0) */
    double Gp, Gm;                       /* G+- with 1/mu* absorbed (Eq. B8) */
    int resonance_hit, eclamp_hit;
    int limit_avg;                       /* limit mode with |D| < 1e-7 */
} layer_coef;

static double resonance_D(double w0, double g0, double E, double mus)
{
    return 4.0 * E * mus * mus * (E - w0) * (1.0 - w0 * g0) - 1.0;
}

/* G+- of Eq. B8 for a given denominator D (mus = mu* < 0, Malik sign). */
static void g_factors(double w0, double g0, double E, double mus, double eps2,
                      double D, double *Gp, double *Gm)
{
    double one_m_wg = 1.0 - w0 * g0;
    double lead = w0 * (2.0 * E * one_m_wg + g0 / eps2) / D;
    double tail = w0 * g0 / (2.0 * eps2 * E * one_m_wg);
    *Gp = 0.5 * (lead * (mus + 1.0 / (2.0 * E * one_m_wg)) + tail);
    *Gm = 0.5 * (lead * (mus - 1.0 / (2.0 * E * one_m_wg)) - tail);
}

/* E - 1 of Eq. 19 in FP32, the terms grouped as nested fused multiply-adds
 * (fmaf rounds each once):  0.2351 w0 g0 + (g0 (-0.07465 g0 - 0.1582)
 * + (w0 (-0.05582 w0 - 0.1777) + 0.225)).  The E clamp's hits are counted on
 * its sign: the paper states no precision for that decision, so it is taken
 * in the precision of the FP32 form, on the same expression. */
static float e_fit_m1_f32(float w0, float g0)
{
    float t = fmaf(w0, fmaf(-0.05582f, w0, -0.1777f), 0.225f);
    t = fmaf(g0, fmaf(-0.07465f, g0, -0.1582f), t);
    return fmaf(0.2351f, w0 * g0, t);
}

static void layer_coeffs(const oracle_cfg *cfg, double w0, double g0, double mu,
                         layer_coef *c)
{
    double E = 1.0;
    c->eclamp_hit = 0;
    c->resonance_hit = 0;
    c->limit_avg = 0;
    /* Eq. 19: the fit applies for w0 > 0.1 (threshold taken as 0.1f) */
    if (cfg->improved && w0 > (double)0.1f) {
        E = 1.225 - 0.1582 * g0 - 0.1777 * w0 - 0.07465 * g0 * g0
            + 0.2351 * w0 * g0 - 0.05582 * w0 * w0;
        if (cfg->e_clamp && E < 1.0)     /* keep E - w0 >= 1 - w0 > 0 */
            E = 1.0;
        if (cfg->e_clamp && e_fit_m1_f32((float)w0, (float)g0) < 0.0f)
            c->eclamp_hit = 1;
    }
    c->E = E;
    c->q = E * (1.0 - w0 * g0);
    /* Eq. B2 */
    c->k = sqrt((E - w0) / (E * (1.0 - w0 * g0)));
    c->zeta_p = 0.5 * (1.0 + c->k);
    c->zeta_m = 0.5 * (1.0 - c->k);
    /* Eq. B5; Pi := pi when E = w0 = 1 (its limit along E = 1) */
    c->Pi = (E == w0) ? OR_PI : OR_PI * (1.0 - w0) / (E - w0);
    c->Gp = c->Gm = 0.0;
    if (mu > 0.0) {
        double mus = -mu;   /* Malik sign: mu* < 0 in Eq. B8 */
        double D = resonance_D(w0, g0, E, mus);
        if (fabs(D) < 1e-5) {
            c->resonance_hit = 1;
            if (cfg->resonance == 0) {
                /* Sec. 2.2.1 after Eq. 11: switch to the reduced form 2 mu* */
                g_factors(w0, g0, E, mus, cfg->eps2, 2.0 * mus, &c->Gp, &c->Gm);
                return;
            }
            /* limit mode: the literal form at the true D is accurate in FP64
             * down to |D| ~ 1e-7; below that the caller averages two
             * consistent evaluations on either side of the singularity. */
            if (fabs(D) < 1e-7) c->limit_avg = 1;
        }
        g_factors(w0, g0, E, mus, cfg->eps2, D, &c->Gp, &c->Gm);
    }
}

/* ------------------------------------------------------------------ */
/* One sub-layer: chi, xi, psi and the right-hand sides S_up, S_dn in    */
/* the form   chi F_up,top - psi F_up,bot + xi F_dn,top = S_up          */
/*            chi F_dn,bot - psi F_dn,top + xi F_up,bot = S_dn          */
/* (Eqs. 2-9 with the flux terms moved to the left).                    */
/* ------------------------------------------------------------------ */

typedef struct {
    double chi, xi, psi, S_up, S_dn;
} sub_rel;

static void beam_terms(double chi, double xi, double psi, double Gp, double Gm,
                       double Fb_top, double Fb_bot, double *bu, double *bd)
{
    /* Eq. B7 (times chi) */
    *bu = psi * Gp * Fb_bot - (xi * Gm + chi * Gp) * Fb_top;
    *bd = psi * Gm * Fb_top - (xi * Gp + chi * Gm) * Fb_bot;
}

static void sub_layer(const oracle_cfg *cfg, const layer_coef *c, double w0,
                      double g0, double mu, double dtau, double B_top,
                      double B_bot, int isothermal, double B_iso, double Fb_top,
                      double Fb_bot, int *etau_hit, sub_rel *o)
{
    double chi, xi, psi;
    if (c->k > 0.0) {
        /* Eqs. B1-B2 */
        double T = exp(-2.0 * sqrt(c->E * (c->E - w0) * (1.0 - w0 * g0)) * dtau);
        double zp = c->zeta_p, zm = c->zeta_m;
        chi = zm * zm * T * T - zp * zp;
        xi = zp * zm * (1.0 - T * T);
        psi = (zm * zm - zp * zp) * T;
    } else if (c->k == 0.0) {
        /* E = w0 = 1.  chi, xi, psi all vanish like k; the relations
         * are homogeneous in them, so use their k -> 0 limits divided by k. */
        chi = -(1.0 + c->q * dtau);
        xi = c->q * dtau;
        psi = -1.0;
    } else {
        /* E < w0 (the raw Eq. 19 fit, clamp off): k of Eq. B2 is not real,
         * the layer has no two-stream solution; NaN marks its fluxes. */
        chi = xi = psi = NAN;
    }
    double Pi = c->Pi;
    double S_up, S_dn;
    *etau_hit = 0;
    if (isothermal) {
        /* Eqs. 2-3 */
        S_up = Pi * B_iso * (chi + xi - psi);
        S_dn = S_up;
    } else {
        double Bt = B_top, Bb = B_bot, Bp;
        if (dtau < (double)1e-4f) {
            /* Sec. 2.2.1: e_tau = 1e-4, gradient off, both B by their mean */
            Bt = Bb = 0.5 * (B_top + B_bot);
            Bp = 0.0;
            *etau_hit = 1;
        } else {
            Bp = (B_bot - B_top) / dtau;   /* dB/dtau, tau increasing downward */
        }
        double Theta = (chi - psi - xi) / (2.0 * c->E * (1.0 - w0 * g0));  /* Eqs. 5, 8 */
        /* Eq. B4 (times chi) */
        S_up = Pi * (Bt * (chi + xi) - psi * Bb + Bp * Theta);
        S_dn = Pi * (Bb * (chi + xi) - psi * Bt - Bp * Theta);
    }
    if (mu > 0.0) {
        double bu, bd;
        if (c->limit_avg) {
            /* Limit mode at |D| < 1e-7: the beam source per unit incident
             * beam is continuous in mu*, so take the mean of its values at
             * mu (1 -+ 5e-6), where |D| ~ 1e-5, with G+- and the sub-layer
             * beam attenuation both evaluated at the moved mu. */
            bu = bd = 0.0;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double mu2 = mu * (1.0 + sgn * 5e-6), Gp, Gm, b1, b2;
                double D2 = resonance_D(w0, g0, c->E, -mu2);
                g_factors(w0, g0, c->E, -mu2, cfg->eps2, D2, &Gp, &Gm);
                beam_terms(chi, xi, psi, Gp, Gm, 1.0, exp(-dtau / mu2), &b1, &b2);
                bu += 0.5 * b1 * Fb_top;
                bd += 0.5 * b2 * Fb_top;
            }
        } else {
            beam_terms(chi, xi, psi, c->Gp, c->Gm, Fb_top, Fb_bot, &bu, &bd);
        }
        S_up += bu;
        S_dn += bd;
    }
    o->chi = chi;
    o->xi = xi;
    o->psi = psi;
    o->S_up = S_up;
    o->S_dn = S_dn;
}

/* ------------------------------------------------------------------ */
/* Per-system setup: sub-layer properties, B at levels, beam at levels. */
/* ------------------------------------------------------------------ */

typedef struct {
    int L, n;            /* layers, sub-layers (= levels - 1) */
    double *dtau_s, *w0_s, *g0_s;   /* [n], sub-layer s joins level s and s+1 */
    double *B_lev;       /* [n+1] B at levels (non-isothermal) */
    double *B_iso;       /* [n] B of each isothermal layer */
    double *tau;         /* [n+1] optical depth from the TOA at each level */
    double *Fb;          /* [n+1] direct beam flux at each level */
    sub_rel *rel;        /* [n] */
} sys_work;

/* Build the per-sub-layer arrays of one system.
 * dtau/w0/g0 are strided views of the cube for this (column, bin, g):
 * element l (API layer, 0 = TOA) is at p[l * stride].
 * Bc[l] = B at the centre of API layer l; Bi[i] = B at API interface i. */
static void setup_system(const oracle_cfg *cfg, int L, const float *dtau,
                         const float *w0, const float *g0, int64_t stride,
                         const double *Bc, const double *Bi, double mu,
                         double Fstar, sys_work *w)
{
    int iso = cfg->isothermal;
    int n = iso ? L : 2 * L;
    w->L = L;
    w->n = n;
    for (int j = 0; j < L; ++j) {          /* internal layer j from the BOA */
        int l = L - 1 - j;                 /* API layer */
        double d = (double)dtau[l * stride];
        double a = (double)w0[l * stride];
        double g = (double)g0[l * stride];
        if (iso) {
            w->dtau_s[j] = d;
            w->w0_s[j] = a;
            w->g0_s[j] = g;
            w->B_iso[j] = Bc[l];
        } else {
            /* two sub-layers with half the optical depth each */
            for (int h = 0; h < 2; ++h) {
                w->dtau_s[2 * j + h] = 0.5 * d;
                w->w0_s[2 * j + h] = a;
                w->g0_s[2 * j + h] = g;
            }
            w->B_lev[2 * j] = Bi[L - j];       /* interface below layer */
            w->B_lev[2 * j + 1] = Bc[l];       /* centre */
        }
    }
    if (!iso) w->B_lev[n] = Bi[0];
    /* optical depth from the TOA and Beer's law, Eq. B6 (mu* = -mu) */
    w->tau[n] = 0.0;
    for (int i = n - 1; i >= 0; --i) w->tau[i] = w->tau[i + 1] + w->dtau_s[i];
    for (int i = 0; i <= n; ++i) {
        if (mu > 0.0) {
            double mus = -mu;
            w->Fb[i] = -mus * Fstar * exp(w->tau[i] / mus);
        } else {
            w->Fb[i] = 0.0;   /* night side, no beam */
        }
    }
}

static void relations(const oracle_cfg *cfg, double mu, sys_work *w,
                      oracle_stats *st)
{
    int iso = cfg->isothermal;
    for (int s = 0; s < w->n; ++s) {
        layer_coef c;
        layer_coeffs(cfg, w->w0_s[s], w->g0_s[s], mu, &c);
        /* count once per layer (both sub-layers share the coefficients) */
        if (st && (iso || (s % 2) == 0)) {
            st->resonance_hits += c.resonance_hit;
            st->eclamp_hits += c.eclamp_hit;
        }
        int et;
        sub_layer(cfg, &c, w->w0_s[s], w->g0_s[s], mu, w->dtau_s[s],
                  iso ? 0.0 : w->B_lev[s + 1], iso ? 0.0 : w->B_lev[s], iso,
                  iso ? w->B_iso[s] : 0.0, w->Fb[s + 1], w->Fb[s], &et,
                  &w->rel[s]);
        if (st) st->etau_hits += et;
    }
}

/* ------------------------------------------------------------------ */
/* Block-tridiagonal assembly (Eq. 12) and block Thomas                 */
/* (Eqs. 13-15).  X_i = (F_up,i, F_dn,i) at level i = 0 (BOA) .. n.     */
/*   row 0:  F_up,0 - F_dn,0 = F_BOA + F_beam,0 (Eq. 10);               */
/*           downward relation of sub-layer 0.                          */
/*   row i:  upward relation of sub-layer i-1; downward of sub-layer i. */
/*   row n:  upward relation of sub-layer n-1; F_dn,n = F_TOA.          */
/* Blocks are stored row-major: M[i*4 + 2*r + c].                       */
/* ------------------------------------------------------------------ */

static void assemble(const oracle_cfg *cfg, const sys_work *w, double F_BOA,
                     double *A, double *B, double *C, double *D)
{
    int n = w->n;
    memset(A, 0, sizeof(double) * 4 * (n + 1));
    memset(B, 0, sizeof(double) * 4 * (n + 1));
    memset(C, 0, sizeof(double) * 4 * (n + 1));
    memset(D, 0, sizeof(double) * 2 * (n + 1));
    for (int i = 0; i <= n; ++i) {
        double *a = A + 4 * i, *b = B + 4 * i, *c = C + 4 * i, *d = D + 2 * i;
        /* first equation of the row */
        if (i == 0) {
            b[0] = 1.0;
            b[1] = -1.0;
            d[0] = F_BOA + w->Fb[0];
        } else {
            const sub_rel *r = &w->rel[i - 1];
            a[0] = -r->psi;
            b[0] = r->chi;
            b[1] = r->xi;
            d[0] = r->S_up;
        }
        /* second equation of the row */
        if (i == n) {
            b[3] = 1.0;
            d[1] = cfg->F_toa;
        } else {
            const sub_rel *r = &w->rel[i];
            b[2] = r->xi;
            b[3] = r->chi;
            c[3] = -r->psi;
            d[1] = r->S_dn;
        }
    }
}

static void mat2_inv(const double *m, double *inv)
{
    double det = m[0] * m[3] - m[1] * m[2];
    inv[0] = m[3] / det;
    inv[1] = -m[1] / det;
    inv[2] = -m[2] / det;
    inv[3] = m[0] / det;
}

static void mat2_mul(const double *x, const double *y, double *o)
{
    double t0 = x[0] * y[0] + x[1] * y[2];
    double t1 = x[0] * y[1] + x[1] * y[3];
    double t2 = x[2] * y[0] + x[3] * y[2];
    double t3 = x[2] * y[1] + x[3] * y[3];
    o[0] = t0; o[1] = t1; o[2] = t2; o[3] = t3;
}

static void mat2_vec(const double *x, const double *v, double *o)
{
    double t0 = x[0] * v[0] + x[1] * v[1];
    double t1 = x[2] * v[0] + x[3] * v[1];
    o[0] = t0; o[1] = t1;
}

/* Eqs. 13-15.  Cp: [4(n+1)], Dp: [2(n+1)], X: [2(n+1)]. */
static void block_thomas(int n, const double *A, const double *B,
                         const double *C, const double *D, double *Cp,
                         double *Dp, double *X)
{
    double M[4], Minv[4], t[4], v[2];
    for (int i = 0; i <= n; ++i) {
        memcpy(M, B + 4 * i, sizeof M);
        v[0] = D[2 * i];
        v[1] = D[2 * i + 1];
        if (i > 0) {
            mat2_mul(A + 4 * i, Cp + 4 * (i - 1), t);   /* A_i C'_{i-1} */
            for (int e = 0; e < 4; ++e) M[e] -= t[e];
            double av[2];
            mat2_vec(A + 4 * i, Dp + 2 * (i - 1), av);  /* A_i D'_{i-1} */
            v[0] -= av[0];
            v[1] -= av[1];
        }
        mat2_inv(M, Minv);
        mat2_mul(Minv, C + 4 * i, Cp + 4 * i);
        mat2_vec(Minv, v, Dp + 2 * i);
    }
    X[2 * n] = Dp[2 * n];
    X[2 * n + 1] = Dp[2 * n + 1];
    for (int i = n - 1; i >= 0; --i) {
        double cx[2];
        mat2_vec(Cp + 4 * i, X + 2 * (i + 1), cx);
        X[2 * i] = Dp[2 * i] - cx[0];
        X[2 * i + 1] = Dp[2 * i + 1] - cx[1];
    }
}

/* ------------------------------------------------------------------ */
/* Iterative multiple scattering (Sec. 2.2.2, "Multiple scattering      */
/* using Thomas's algorithm"): the older approach that the block solve  */
/* replaces.  The pairwise two-stream relation of every sub-layer is     */
/* applied in turn through the whole column, and the passes are         */
/* repeated N times, so radiation is scattered N times in each          */
/* direction.  One sweep here is:                                       */
/*   - a downward pass from the TOA condition F_dn,n = F_TOA: each       */
/*     sub-layer's downward relation gives F_dn at its bottom from F_dn  */
/*     at its top (this pass) and F_up at its bottom (previous sweep);  */
/*   - the BOA condition (Eq. 10): F_up,0 = F_dn,0 + F_BOA + F_beam,0;   */
/*   - an upward pass: each sub-layer's upward relation gives F_up at    */
/*     its top from F_up at its bottom (this pass) and F_dn at its top. */
/* The paper fixes neither the order of the two passes nor the starting */
/* state; we start from zero diffuse flux and go down first, so that    */
/* without scattering (xi = 0: the up and down streams decouple) one    */
/* sweep already gives the exact solution.                              */
/* up, dn: [n+1] at levels (BOA first), the starting state on entry.    */
/* ------------------------------------------------------------------ */
static void sweeps(const oracle_cfg *cfg, const sys_work *w, double F_BOA,
                   int n_sweeps, double *up, double *dn)
{
    int n = w->n;
    for (int it = 0; it < n_sweeps; ++it) {
        dn[n] = cfg->F_toa;
        for (int s = n - 1; s >= 0; --s) {
            /* chi F_dn,bot - psi F_dn,top + xi F_up,bot = S_dn */
            const sub_rel *r = &w->rel[s];
            dn[s] = (r->S_dn + r->psi * dn[s + 1] - r->xi * up[s]) / r->chi;
        }
        up[0] = dn[0] + F_BOA + w->Fb[0];
        for (int s = 0; s < n; ++s) {
            /* chi F_up,top - psi F_up,bot + xi F_dn,top = S_up */
            const sub_rel *r = &w->rel[s];
            up[s + 1] = (r->S_up + r->psi * up[s] - r->xi * dn[s + 1]) / r->chi;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Single-system entry points (used by the pins in the test suite).     */
/* ------------------------------------------------------------------ */

static int alloc_work(sys_work *w, int L)
{
    int n = 2 * L;   /* upper bound for either mode */
    w->dtau_s = malloc(sizeof(double) * n);
    w->w0_s = malloc(sizeof(double) * n);
    w->g0_s = malloc(sizeof(double) * n);
    w->B_lev = malloc(sizeof(double) * (n + 1));
    w->B_iso = malloc(sizeof(double) * n);
    w->tau = malloc(sizeof(double) * (n + 1));
    w->Fb = malloc(sizeof(double) * (n + 1));
    w->rel = malloc(sizeof(sub_rel) * n);
    return w->dtau_s && w->w0_s && w->g0_s && w->B_lev && w->B_iso && w->tau
           && w->Fb && w->rel;
}

static void free_work(sys_work *w)
{
    free(w->dtau_s); free(w->w0_s); free(w->g0_s); free(w->B_lev);
    free(w->B_iso); free(w->tau); free(w->Fb); free(w->rel);
}

/* Assemble the block system of one (column, bin, g) system.
 * dtau/w0/g0: [L] per API layer (0 = TOA).  Bc: [L] centre B, Bi: [L+1]
 * interface B (API order).  F_BOA: pi B(T_int) for this bin.
 * Outputs (levels BOA first, n = L or 2L): A, B, C: [4(n+1)]; D: [2(n+1)];
 * Fb: [n+1] beam at levels.  Returns n. */
int oracle_assemble(const oracle_cfg *cfg, int L, const float *dtau,
                    const float *w0, const float *g0, const double *Bc,
                    const double *Bi, double mu, double Fstar, double F_BOA,
                    double *A, double *B, double *C, double *D, double *Fb)
{
    sys_work w;
    if (!alloc_work(&w, L)) { free_work(&w); return -1; }
    setup_system(cfg, L, dtau, w0, g0, 1, Bc, Bi, mu, Fstar, &w);
    relations(cfg, mu, &w, NULL);
    assemble(cfg, &w, F_BOA, A, B, C, D);
    memcpy(Fb, w.Fb, sizeof(double) * (w.n + 1));
    int n = w.n;
    free_work(&w);
    return n;
}

/* Block Thomas on an assembled system; X: [2(n+1)] = (F_up, F_dn) per level. */
int oracle_block_thomas(int n, const double *A, const double *B,
                        const double *C, const double *D, double *X)
{
    double *Cp = malloc(sizeof(double) * 4 * (n + 1));
    double *Dp = malloc(sizeof(double) * 2 * (n + 1));
    if (!Cp || !Dp) { free(Cp); free(Dp); return -1; }
    block_thomas(n, A, B, C, D, Cp, Dp, X);
    free(Cp);
    free(Dp);
    return 0;
}

/* Solve one system.  Outputs at levels (BOA first, n+1 values each):
 * F_up, F_dn (diffuse) and F_beam.  Returns n, or -1 on allocation failure. */
int oracle_solve_system(const oracle_cfg *cfg, int L, const float *dtau,
                        const float *w0, const float *g0, const double *Bc,
                        const double *Bi, double mu, double Fstar, double F_BOA,
                        double *F_up, double *F_dn, double *F_beam)
{
    int n = cfg->isothermal ? L : 2 * L;
    double *A = malloc(sizeof(double) * 4 * (n + 1));
    double *B = malloc(sizeof(double) * 4 * (n + 1));
    double *C = malloc(sizeof(double) * 4 * (n + 1));
    double *D = malloc(sizeof(double) * 2 * (n + 1));
    double *X = malloc(sizeof(double) * 2 * (n + 1));
    int rc = -1;
    if (A && B && C && D && X) {
        oracle_assemble(cfg, L, dtau, w0, g0, Bc, Bi, mu, Fstar, F_BOA, A, B,
                        C, D, F_beam);
        oracle_block_thomas(n, A, B, C, D, X);
        for (int i = 0; i <= n; ++i) {
            F_up[i] = X[2 * i];
            F_dn[i] = X[2 * i + 1];
        }
        rc = n;
    }
    free(A); free(B); free(C); free(D); free(X);
    return rc;
}

/* n_sweeps sweeps of the iterative method on one system.  F_up, F_dn
 * [n+1] (levels BOA first) hold the starting state on entry and the result
 * on return; F_beam [n+1] receives the direct beam.  Returns n, or -1. */
int oracle_sweep_system(const oracle_cfg *cfg, int L, const float *dtau,
                        const float *w0, const float *g0, const double *Bc,
                        const double *Bi, double mu, double Fstar, double F_BOA,
                        int n_sweeps, double *F_up, double *F_dn, double *F_beam)
{
    sys_work w;
    if (!alloc_work(&w, L)) { free_work(&w); return -1; }
    setup_system(cfg, L, dtau, w0, g0, 1, Bc, Bi, mu, Fstar, &w);
    relations(cfg, mu, &w, NULL);
    sweeps(cfg, &w, F_BOA, n_sweeps, F_up, F_dn);
    memcpy(F_beam, w.Fb, sizeof(double) * (w.n + 1));
    int n = w.n;
    free_work(&w);
    return n;
}

/* ------------------------------------------------------------------ */
/* Whole batch of columns: Planck, every system, spectral sum, heating. */
/* ------------------------------------------------------------------ */

/* Columns are packed in order.  Column c has L_c = n_layers[c] layers and
 * NB_c = n_bins[c] bins; its cube block holds L_c*NB_c*n_g floats laid out
 * [layer][bin][g] (layer 0 = TOA), and blocks follow each other.
 * T_center: [sum L_c]; T_iface, p_iface: [sum (L_c+1)] (interface 0 = TOA,
 * pressures in Pa); mu_star: [n_cols] (cos theta*, <= 0 means no beam);
 * F_star: [sum NB_c] W m^-2 normal to the beam; g_w: [n_g].
 * Outputs: F_up, F_dn (diffuse + beam), F_net: [sum (L_c+1)];
 * Q: [sum L_c] in K s^-1.  Optional per-system outputs (may be NULL):
 * sys_up, sys_dn: [sum (L_c+1)*NB_c*n_g] diffuse fluxes at interfaces,
 * layout [column block][interface][bin][g]. */
int oracle_solve_columns(const oracle_cfg *cfg, int n_cols,
                         const int32_t *n_layers, const int32_t *n_bins,
                         int n_g, const double *g_w, const float *dtau,
                         const float *w0, const float *g0,
                         const double *T_center, const double *T_iface,
                         const double *p_iface, const double *mu_star,
                         const double *F_star, double *F_up, double *F_dn,
                         double *F_net, double *Q, double *sys_up,
                         double *sys_dn, double *toa_up, oracle_stats *stats_out)
{
    gl_init();
    int64_t *cube_off = malloc(sizeof(int64_t) * (n_cols + 1));
    int64_t *lay_off = malloc(sizeof(int64_t) * (n_cols + 1));
    int64_t *bin_off = malloc(sizeof(int64_t) * (n_cols + 1));
    int64_t *sys_off = malloc(sizeof(int64_t) * (n_cols + 1));
    if (!cube_off || !lay_off || !bin_off || !sys_off) {
        free(cube_off); free(lay_off); free(bin_off); free(sys_off);
        return -1;
    }
    cube_off[0] = lay_off[0] = bin_off[0] = sys_off[0] = 0;
    for (int c = 0; c < n_cols; ++c) {
        cube_off[c + 1] = cube_off[c] + (int64_t)n_layers[c] * n_bins[c] * n_g;
        lay_off[c + 1] = lay_off[c] + n_layers[c];
        bin_off[c + 1] = bin_off[c] + n_bins[c];
        sys_off[c + 1] = sys_off[c] + (int64_t)(n_layers[c] + 1) * n_bins[c] * n_g;
    }
    oracle_stats total = {0, 0, 0, 0};
    int failed = 0;

#pragma omp parallel
    {
        oracle_stats st = {0, 0, 0, 0};
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < n_cols; ++c) {
            int L = n_layers[c], NB = n_bins[c];
            int n = cfg->isothermal ? L : 2 * L;
            double mu = mu_star[c];
            const double *Tc = T_center + lay_off[c];
            const double *Ti = T_iface + lay_off[c] + c;
            const double *p = p_iface + lay_off[c] + c;
            double *up = F_up + lay_off[c] + c, *dn = F_dn + lay_off[c] + c;
            double *net = F_net + lay_off[c] + c, *q = Q + lay_off[c];
            double *Bc = malloc(sizeof(double) * L);
            double *Bi = malloc(sizeof(double) * (L + 1));
            double *fu = malloc(sizeof(double) * (n + 1));
            double *fd = malloc(sizeof(double) * (n + 1));
            double *fb = malloc(sizeof(double) * (n + 1));
            double *sum_up = calloc(L + 1, sizeof(double));
            double *sum_dn = calloc(L + 1, sizeof(double));
            if (!Bc || !Bi || !fu || !fd || !fb || !sum_up || !sum_dn) {
#pragma omp atomic write
                failed = 1;
            } else {
                double dwn = (cfg->wn_max - cfg->wn_min) / NB;
                for (int b = 0; b < NB; ++b) {
                    double lo = cfg->wn_min + b * dwn, hi = lo + dwn;
                    if (cfg->wn_edges) {
                        lo = cfg->wn_edges[b];
                        hi = cfg->wn_edges[b + 1];
                    }
                    /* emergent spectrum: the g-weighted upward flux at the TOA
                     * of this bin (the quantity post-processing samples) */
                    double toa_b = 0.0;
                    for (int l = 0; l < L; ++l) Bc[l] = oracle_planck_bin(Tc[l], lo, hi);
                    for (int i = 0; i <= L; ++i) Bi[i] = oracle_planck_bin(Ti[i], lo, hi);
                    double F_BOA = OR_PI * oracle_planck_bin(cfg->T_int, lo, hi);  /* Eq. 10 */
                    double Fs = F_star[bin_off[c] + b];
                    for (int g = 0; g < n_g; ++g) {
                        const float *cb = dtau + cube_off[c] + (int64_t)b * n_g + g;
                        const float *cw = w0 + cube_off[c] + (int64_t)b * n_g + g;
                        const float *cg = g0 + cube_off[c] + (int64_t)b * n_g + g;
                        int64_t stride = (int64_t)NB * n_g;
                        sys_work w;
                        if (!alloc_work(&w, L)) {
                            free_work(&w);
#pragma omp atomic write
                            failed = 1;
                            continue;
                        }
                        setup_system(cfg, L, cb, cw, cg, stride, Bc, Bi, mu, Fs, &w);
                        relations(cfg, mu, &w, &st);
                        double *A = malloc(sizeof(double) * 4 * (n + 1));
                        double *Bm = malloc(sizeof(double) * 4 * (n + 1));
                        double *C = malloc(sizeof(double) * 4 * (n + 1));
                        double *D = malloc(sizeof(double) * 2 * (n + 1));
                        double *Cp = malloc(sizeof(double) * 4 * (n + 1));
                        double *Dp = malloc(sizeof(double) * 2 * (n + 1));
                        double *X = malloc(sizeof(double) * 2 * (n + 1));
                        if (A && Bm && C && D && Cp && Dp && X) {
                            if (cfg->n_sweeps > 0) {
                                /* the iterative method, from zero diffuse flux */
                                for (int i = 0; i <= n; ++i) fu[i] = fd[i] = 0.0;
                                sweeps(cfg, &w, F_BOA, cfg->n_sweeps, fu, fd);
                            } else {
                                assemble(cfg, &w, F_BOA, A, Bm, C, D);
                                block_thomas(n, A, Bm, C, D, Cp, Dp, X);
                                for (int i = 0; i <= n; ++i) {
                                    fu[i] = X[2 * i];
                                    fd[i] = X[2 * i + 1];
                                }
                            }
                            int bad = 0;
                            for (int i = 0; i <= n; ++i) {
                                fb[i] = w.Fb[i];
                                if (!isfinite(fu[i]) || !isfinite(fd[i])) bad = 1;
                            }
                            st.nonfinite += bad;
                            /* interfaces: API interface i sits at level
                             * (L - i) (isothermal) or 2 (L - i). */
                            double wg = g_w[g];
                            toa_b += wg * fu[cfg->isothermal ? L : 2 * L];
                            for (int i = 0; i <= L; ++i) {
                                int lev = cfg->isothermal ? (L - i) : 2 * (L - i);
                                sum_up[i] += wg * fu[lev];
                                sum_dn[i] += wg * (fd[lev] + fb[lev]);  /* beam added */
                                if (sys_up) {
                                    int64_t o = sys_off[c] + ((int64_t)i * NB + b) * n_g + g;
                                    sys_up[o] = fu[lev];
                                    sys_dn[o] = fd[lev];
                                }
                            }
                        } else {
#pragma omp atomic write
                            failed = 1;
                        }
                        free(A); free(Bm); free(C); free(D); free(Cp); free(Dp); free(X);
                        free_work(&w);
                    }
                    if (toa_up) toa_up[bin_off[c] + b] = toa_b;
                }
                for (int i = 0; i <= L; ++i) {
                    up[i] = sum_up[i];
                    dn[i] = sum_dn[i];
                    net[i] = sum_up[i] - sum_dn[i];
                }
                /* Q_l = (g/cp) (F_net,bot - F_net,top) / (p_bot - p_top) */
                for (int l = 0; l < L; ++l)
                    q[l] = cfg->grav / cfg->cp * (net[l + 1] - net[l]) / (p[l + 1] - p[l]);
            }
            free(Bc); free(Bi); free(fu); free(fd); free(fb); free(sum_up); free(sum_dn);
        }
#pragma omp critical
        {
            total.resonance_hits += st.resonance_hits;
            total.etau_hits += st.etau_hits;
            total.eclamp_hits += st.eclamp_hits;
            total.nonfinite += st.nonfinite;
        }
    }
    if (stats_out) *stats_out = total;
    free(cube_off); free(lay_off); free(bin_off); free(sys_off);
    return failed ? -1 : 0;
}
