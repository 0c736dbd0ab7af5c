// rt_kernels.cu -- fused column kernels for sm_103a.
//
// One persistent CTA handles one column at a time (columns are taken from a
// largest-first list through an atomic counter).  Inside a column the CTA
// walks the column's (bin, g) systems in chunks of blockDim, one thread per
// system, g fastest, so that a warp reads 32 consecutive floats of each
// optical-property cube per layer.  For each chunk the CTA:
//   1. evaluates the Planck function per bin at every interface and layer
//      centre of the column into shared memory (bin-integrated B, Sec. 2.2.1);
//   2. per thread: walks the layers from the TOA down, forming the layer
//      coefficients (App. B), the stellar beam (Eq. B6) and its source terms
//      (Eq. B7-B8), the thermal source terms (Eqs. 2-9), and eliminates
//      towards the BOA (Thomas forward sweep, Sec. 2.2.2), keeping per
//      interface what the back-substitution needs in a global scratch laid
//      out [level][thread slot];
//   3. closes the system at the BOA (Eq. 10) and substitutes back to the TOA,
//      reducing the Gauss-weighted fluxes of the 32 systems of each warp with
//      a fixed butterfly, then across warps in a fixed order.
// After the last chunk it writes the column's interface fluxes, net flux and
// heating rate.  Every reduction runs in a fixed order, so a column gives the
// same bits whatever else is in the batch (for a fixed block size).
//
// Two arithmetic variants:
//   fp32_units    -- the FP32 "chosen form": cancellation-free transmission,
//                    reflection and absorption forms, a beam source with the
//                    removable singularity at mu* alpha = 1 divided out, and
//                    departure variables u = F - pi B at every level.  FP64 is
//                    used only to decide the paper's resonance switch when the
//                    FP32 estimate of D lies within 2e-5 of zero.
//   fp64_columns  -- FP64 with the paper's literal formulas, scalar Thomas on
//                    every level (sub-layers not merged).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rt_internal.h"

namespace rt {

// ---------------------------------------------------------------------
// Physical constants (SI defining constants, exact) and Planck series.
// ---------------------------------------------------------------------
constexpr double kH = 6.62607015e-34;
constexpr double kC = 299792458.0;
constexpr double kKB = 1.380649e-23;
constexpr double kC2 = kH * kC / kKB;                       // m K
constexpr double kPlanckK = 2.0 * kKB * kKB * kKB * kKB / (kH * kH * kH * kC * kC);
constexpr double kPi = 3.14159265358979323846;
constexpr double kPi4Over15 = 6.4939394022668291491;      // integral_0^inf x^3/(e^x-1)
constexpr float kPiF = 3.14159265358979323846f;

// Bernoulli numbers B_k give t/(e^t - 1) = sum_k B_k t^k / k!, hence
//   S(x) = integral_0^x t^3/(e^t-1) dt = sum_k B_k x^(k+3) / (k! (k+3)),
// convergent for |x| < 2 pi.  Coefficients c_k = B_k / (k! (k+3)).
#define BC(num, den, kfact, k) ((double)(num) / (double)(den) / ((double)(kfact) * ((k) + 3.0)))
__device__ constexpr double kS0 = 1.0 / 3.0;
__device__ constexpr double kS1 = -1.0 / 8.0;
__device__ constexpr double kS2 = BC(1, 6, 2.0, 2);
__device__ constexpr double kS4 = BC(-1, 30, 24.0, 4);
__device__ constexpr double kS6 = BC(1, 42, 720.0, 6);
__device__ constexpr double kS8 = BC(-1, 30, 40320.0, 8);
__device__ constexpr double kS10 = BC(5, 66, 3628800.0, 10);
__device__ constexpr double kS12 = BC(-691, 2730, 479001600.0, 12);
__device__ constexpr double kS14 = BC(7, 6, 87178291200.0, 14);
__device__ constexpr double kS16 = BC(-3617, 510, 20922789888000.0, 16);
__device__ constexpr double kS18 = BC(43867, 798, 6402373705728000.0, 18);
__device__ constexpr double kS20 = BC(-174611, 330, 2432902008176640000.0, 20);
__device__ constexpr double kS22 = BC(854513, 138, 1.1240007277776077e21, 22);
__device__ constexpr double kS24 = BC(-236364091, 2730, 6.2044840173323941e23, 24);
__device__ constexpr double kS26 = BC(8553103, 6, 4.0329146112660565e26, 26);
__device__ constexpr double kS28 = BC(-23749461029.0, 870, 3.0488834461171386e29, 28);
__device__ constexpr double kS30 = BC(8615841276005.0, 14322, 2.6525285981219105e32, 30);
#undef BC

// FP32: S(x) for x <= 2 (terms to k = 14, relative error < 1e-7).
__device__ __forceinline__ float planck_lower_f(float x) {
    const float x2 = x * x;
    float s = (float)kS14;
    s = fmaf(s, x2, (float)kS12);
    s = fmaf(s, x2, (float)kS10);
    s = fmaf(s, x2, (float)kS8);
    s = fmaf(s, x2, (float)kS6);
    s = fmaf(s, x2, (float)kS4);
    const float head = fmaf(x, fmaf(x, (float)kS2, (float)kS1), (float)kS0);
    return fmaf(x2 * x2, s, head) * x2 * x;
}

// Fast FP32 primitives: MUFU reciprocal, reciprocal square root and
// exponential (ex2 with the argument scaled by log2 e).  Each is accurate to a
// few ulp, far inside the 1e-4 target.
__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fexp(float x) { return __expf(x); }

// (1 - exp(-x)) / x from its Taylor series sum_n (-x)^n / (n+1)! for |x| < 0.25
// (7 terms, truncation below 2e-9), else from the exponential e = exp(-x)
// (relative error of 1 - e below 5e-7 there).
__device__ __forceinline__ float u_series(float x) {
    float p = -1.f / 40320.f;
    p = fmaf(p, x, 1.f / 5040.f);
    p = fmaf(p, x, -1.f / 720.f);
    p = fmaf(p, x, 1.f / 120.f);
    p = fmaf(p, x, -1.f / 24.f);
    p = fmaf(p, x, 1.f / 6.f);
    p = fmaf(p, x, -0.5f);
    return fmaf(p, x, 1.f);
}
__device__ __forceinline__ float one_minus_exp_over_x(float x, float e) {
    const float s = u_series(x);
    const float d = (1.f - e) * frcp(x);
    return (fabsf(x) < 0.25f) ? s : d;
}

// FP32: P(x) = integral_x^inf t^3/(e^t-1) dt for x >= 2 as
//   sum_n e^(-n x) (x^3/n + 3 x^2/n^2 + 6 x/n^3 + 6/n^4), 8 terms.
__device__ __forceinline__ float planck_upper_f(float x) {
    const float e = fexp(-x);
    const float x2 = x * x, x3 = x2 * x;
    float en = e, s = 0.f;
#pragma unroll
    for (int n = 1; n <= 8; ++n) {
        const float y = 1.0f / (float)n;
        const float poly = y * fmaf(y, fmaf(y, fmaf(6.f, y, 6.f * x), 3.f * x2), x3);
        s = fmaf(en, poly, s);
        en *= e;
    }
    return s;
}

// Bin-integrated Planck function (W m^-2 sr^-1) between two wavenumbers
// (cm^-1), FP32.  The difference is taken in the form without cancellation.
__device__ float planck_bin_f(float T, float wlo, float whi) {
    if (!(T > 0.f)) return 0.f;
    const float a = (float)(kC2 * 100.0) * frcp(T);
    const float xlo = a * wlo, xhi = a * whi;
    float d;
    if (xlo >= 2.f) {
        d = planck_upper_f(xlo) - planck_upper_f(xhi);
    } else if (xhi <= 2.f) {
        d = planck_lower_f(xhi) - planck_lower_f(xlo);
    } else {
        d = ((float)kPi4Over15 - planck_lower_f(xlo)) - planck_upper_f(xhi);
    }
    const float T2 = T * T;
    return (float)kPlanckK * (T2 * T2) * d;
}

// FP64 versions (terms to k = 30 below x = 2, 20 exponential terms above).
__device__ __forceinline__ double planck_lower_d(double x) {
    const double x2 = x * x;
    double s = kS30;
    s = fma(s, x2, kS28); s = fma(s, x2, kS26); s = fma(s, x2, kS24);
    s = fma(s, x2, kS22); s = fma(s, x2, kS20); s = fma(s, x2, kS18);
    s = fma(s, x2, kS16); s = fma(s, x2, kS14); s = fma(s, x2, kS12);
    s = fma(s, x2, kS10); s = fma(s, x2, kS8); s = fma(s, x2, kS6);
    s = fma(s, x2, kS4);
    const double head = fma(x, fma(x, kS2, kS1), kS0);
    return fma(x2 * x2, s, head) * x2 * x;
}

__device__ __forceinline__ double planck_upper_d(double x) {
    const double e = exp(-x);
    const double x2 = x * x, x3 = x2 * x;
    double en = e, s = 0.0;
#pragma unroll
    for (int n = 1; n <= 20; ++n) {
        const double y = 1.0 / (double)n;
        const double poly = y * fma(y, fma(y, fma(6.0, y, 6.0 * x), 3.0 * x2), x3);
        s = fma(en, poly, s);
        en *= e;
    }
    return s;
}

__device__ double planck_bin_d(double T, double wlo, double whi) {
    if (!(T > 0.0)) return 0.0;
    const double a = kC2 * 100.0 / T;
    const double xlo = a * wlo, xhi = a * whi;
    double d;
    if (xlo >= 2.0) {
        d = planck_upper_d(xlo) - planck_upper_d(xhi);
    } else if (xhi <= 2.0) {
        d = planck_lower_d(xhi) - planck_lower_d(xlo);
    } else {
        d = (kPi4Over15 - planck_lower_d(xlo)) - planck_upper_d(xhi);
    }
    const double T2 = T * T;
    return kPlanckK * (T2 * T2) * d;
}

// ---------------------------------------------------------------------
// Counters kept in registers and flushed once per CTA.
// ---------------------------------------------------------------------
struct Counters {
    unsigned res, etau, eclamp, inv, nonfinite, fp64;
    unsigned on;   // 1 while the thread works on a real system, 0 on padding lanes
    // FP32 form: raw per-system counts, added (masked by `on`) once per system
    unsigned s_inv, s_ecl, s_etau;
};

__device__ __forceinline__ void flush_counters(const Counters &cn, unsigned long long *stats) {
    unsigned v[6] = {cn.res, cn.etau, cn.eclamp, cn.inv, cn.nonfinite, cn.fp64};
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(stats + i, (unsigned long long)x);
    }
}

// The paper's resonance test (Eq. 11 and the text after it) evaluated in
// FP64 with the same operation order as a plain C evaluation, so the branch
// matches an FP64 reference bit for bit.
__device__ __noinline__ double resonance_D_fp64(float w0f, float g0f, double mu, int improved, int e_clamp) {
    const double w0 = (double)w0f, g0 = (double)g0f;
    double E = 1.0;
    if (improved && w0 > (double)0.1f) {
        double t = __dsub_rn(1.225, __dmul_rn(0.1582, g0));
        t = __dsub_rn(t, __dmul_rn(0.1777, w0));
        t = __dsub_rn(t, __dmul_rn(__dmul_rn(0.07465, g0), g0));
        t = __dadd_rn(t, __dmul_rn(__dmul_rn(0.2351, w0), g0));
        t = __dsub_rn(t, __dmul_rn(__dmul_rn(0.05582, w0), w0));
        E = (e_clamp && t < 1.0) ? 1.0 : t;
    }
    const double mus = -mu;
    double v = __dmul_rn(4.0, E);
    v = __dmul_rn(v, mus);
    v = __dmul_rn(v, mus);
    v = __dmul_rn(v, __dsub_rn(E, w0));
    v = __dmul_rn(v, __dsub_rn(1.0, __dmul_rn(w0, g0)));
    return __dsub_rn(v, 1.0);
}

// ---------------------------------------------------------------------
// FP32 chosen form: one layer.
//
// Notation: q = E (1 - w0 g0), k = sqrt((E - w0)/q) so that the transmission
// exponent of Eq. B2 is 2 q k dtau and zeta_-/zeta_+ = eps = (1-k)/(1+k).
// With x = 2 q k dtau, T = exp(-x), u = (1 - T)/x, h = 2 q dtau u + 2T/(1+k),
// p = 1 + eps T, the relations of Eqs. B1-B3 divided by chi give
//   t = psi/chi = 4T / ((1+k)^2 h p),  r = -xi/chi = eps 2 q dtau u (1+T)/(h p),
//   1-t-r = 4 q k^2 dtau u / ((1+k) p),  1-t+r = 4 q dtau u / ((1+k) h),
// free of cancellation as k -> 0 (w0 -> 1) and dtau -> 0.
// Thermal sources are written for departures u = F - pi B at both ends of
// the sub-layer; with Pi - pi = -pi (E-1)/(E-w0) they carry no difference of
// large terms, and the Planck-gradient term c B' (1-t+r) becomes
// Pi (B_bot - B_top) 2u/((1+k) h) with no division by dtau.
// The beam source (Eqs. B7-B8) per unit beam at the sub-layer top is
// rewritten with rho = mu 2 q k, delta = dtau/mu, m = exp(-delta) and
// Lambda = (T - m)/(1 - rho) (evaluated as m delta expm1(z)/z, z =
// (1-rho) delta, near rho = 1): the factor 1/D of G+- cancels analytically,
// so the source is finite and accurate through mu* alpha = 1.
// Two identical sub-layers (half the optical depth each) are merged into one
// layer with T_L = t^2/(1-r^2), R_L = r (1 + T_L) and combined sources.
// ---------------------------------------------------------------------
struct Layer32 {
    float T, R, Su, Sd, omtr, opr, mlay;
};

// Products are grouped by hand: float multiplication is not reassociated by
// the compiler, and shared factors (1/h and 1/p from one reciprocal of h p,
// 2q, w0 g0, ...) are formed once per layer.
template <bool ISO>
__device__ __forceinline__ Layer32 layer32(float dt, float w0, float g0, float Bt, float Bc, float Bb,
                                           float mu, float imu, double mu_d, bool beam, float Fb,
                                           const KParams &kp, Counters &cn) {
    const bool valid = (dt >= 0.f) && (w0 >= 0.f) && (w0 <= 1.f) && (fabsf(g0) < 1.f);
    cn.s_inv += valid ? 0u : 1u;
    // E of Eq. 19, switched off for w0 <= 0.1, clamped at 1
    const float wg = w0 * g0;
    float em1 = fmaf(g0, fmaf(-0.07465f, g0, -0.1582f), fmaf(w0, fmaf(-0.05582f, w0, -0.1777f), 0.225f));
    em1 = fmaf(0.2351f, wg, em1);
    em1 = (kp.improved && w0 > 0.1f) ? em1 : 0.f;
    const bool clamp = kp.e_clamp && em1 < 0.f;
    cn.s_ecl += clamp ? 1u : 0u;
    em1 = clamp ? 0.f : em1;
    const float omw = 1.f - w0;
    const float ewm = em1 + omw;                 // E - w0
    const float q = (1.f + em1) * (1.f - wg);    // E (1 - w0 g0)
    const float iq = frcp(q);
    const bool cons = ewm == 0.f;                // E = w0 = 1: k = 0, Pi := pi
    const float k = cons ? 0.f : ewm * rsqrtf(ewm * q);
    const float piw = kPiF * frcp(ewm);
    const float Pi = cons ? kPiF : omw * piw;
    const float dPi = cons ? 0.f : -em1 * piw;  // Pi - pi
    const float ip = frcp(1.f + k);
    const float eps = (1.f - k) * ip;
    const float dts = ISO ? dt : 0.5f * dt;

    const float q2 = q + q;
    const float q2d = q2 * dts;
    const float x = q2d * k;
    const float Tm = fexp(-x);
    const float u = one_minus_exp_over_x(x, Tm);
    const float qd = q2d * u;                    // (1 - T)/k
    const float h = fmaf(Tm + Tm, ip, qd);
    const float p = fmaf(eps, Tm, 1.f);
    const float ihp = frcp(h * p);
    const float ih = p * ihp, ipp = h * ihp;     // 1/h, 1/p
    const float ipihp = ip * ihp;
    const float t = (4.f * Tm) * (ip * ipihp);
    const float Y = fmaf(qd, Tm, qd);            // (1 - T^2)/k = qd (1 + T)
    const float r = (eps * ihp) * Y;
    const float k2 = k * k;
    const float omtr = (k2 + k2) * (qd * ip) * ipp;      // 1 - t - r
    const float omr = omtr + t;                          // 1 - r

    float suU, sdU, suL = 0.f, sdL = 0.f;
    if (!ISO) {
        const bool fb = dts < 1e-4f;
        cn.s_etau += fb ? 1u : 0u;
        // Gradient form  su = dPi ((1-r) B1 - t B2) + G (B2 - B1),
        //                sd = dPi ((1-r) B2 - t B1) - G (B2 - B1),
        // with G = Pi 2u/((1+k) h).  The e_tau fallback (isothermal at the mean
        // B, Sec. 2.2.1) is the same expression with B1 = B2 = mean B and
        // G = pi (1 - r + t)/2, so only the inputs are selected.
        const float pig = Pi * (2.f * u) * (ip * ih);
        const float side = (0.5f * kPiF) * (omtr + 2.f * t);
        const float G = fb ? side : pig;
        const float mU = 0.5f * (Bt + Bc), mL = 0.5f * (Bc + Bb);
        const float tU = fb ? mU : Bt, cU = fb ? mU : Bc;    // upper sub-layer ends
        const float cL = fb ? mL : Bc, bL = fb ? mL : Bb;    // lower sub-layer ends
        const float gU = G * (Bc - Bt), gL = G * (Bb - Bc);
        suU = fmaf(dPi, fmaf(omr, tU, -t * cU), gU);
        sdU = fmaf(dPi, fmaf(omr, cU, -t * tU), -gU);
        suL = fmaf(dPi, fmaf(omr, cL, -t * bL), gL);
        sdL = fmaf(dPi, fmaf(omr, bL, -t * cL), -gL);
    } else {
        const float base = dPi * Bc * omtr;
        suU = base + kPiF * (omr * (Bc - Bt) - t * (Bc - Bb));
        sdU = base + kPiF * (omr * (Bc - Bb) - t * (Bc - Bt));
    }

    float m = 1.f;
    if (beam) {
        const float dl = dts * imu;
        m = fexp(-dl);
        const float omm = (dl < 0.25f) ? dl * u_series(dl) : 1.f - m;   // 1 - m
        const float q2k = q2 * k;
        const float rho = mu * q2k;
        const float ie2 = kp.inv_eps2;
        const float A = w0 * fmaf(g0, ie2, q2);
        const float G0h = wg * (0.25f * ie2) * iq;            // G0/2 of Eq. B8
        const float r2 = r + r;
        const float tm1r = -fmaf(t, omm, omtr + r2);           // (t m - 1) - r
        const float rmtm = fmaf(r, m, (omtr + r) - omm);      // r m - (t - m)
        // stable form: the 1/D of G+- divided out (see the block comment)
        const float omrho = 1.f - rho;
        const float z = omrho * dl;
        const float lam_s = (m * dl) * u_series(-z);
        const float lam_d = (Tm - m) * frcp(omrho);
        const float Lam = (fabsf(z) < 0.25f) ? lam_s : lam_d;
        const float SA2 = (0.5f * A) * (ip * ipihp) * (iq * frcp(1.f + rho));   // 2 SA
        const float tq = mu * q2;
        const float TL = Tm * Lam;
        float bu = fmaf(SA2, fmaf((1.f + k) * Y, 1.f, (TL + TL) * (1.f - tq)), G0h * tm1r);
        const float cl = fmaf(Y, fmaf(tq, k2, 1.f), (1.f + tq) * fmaf(Tm, Tm, 1.f));
        float bd = fmaf(SA2, fmaf(Lam, cl, -(Tm * (1.f - k)) * Y), G0h * rmtm);
        // resonance test of Eq. 11 (rare): the FP64 decision, and the paper's
        // switch to D := 2 mu* when |D| < 1e-5, run only if a lane needs them
        const float D32 = fmaf(rho, rho, -1.f);
        const bool near = fabsf(D32) < 2e-5f;
        if (__any_sync(0xffffffffu, near)) {
            bool sw = false;
            if (near) {
                cn.fp64 += cn.on;
                const double D = resonance_D_fp64(w0, g0, mu_d, kp.improved, kp.e_clamp);
                if (fabs(D) < 1e-5) {
                    cn.res += cn.on;
                    sw = kp.resonance_paper != 0;
                }
            }
            if (sw) {
                // paper: D := 2 mu* = -2 mu, literal G+- (no singularity left)
                const float c1 = 0.5f * iq;
                const float lead = -0.5f * A * imu;
                const float Gp = 0.5f * lead * (c1 - mu) + G0h;
                const float Gm = -0.5f * lead * (c1 + mu) - G0h;
                bu = -Gp * (omtr + r + t * omm) + r * Gm;     // Gp (t m - 1) + r Gm
                bd = Gm * (omm - omtr - r) + r * Gp * m;      // Gm (t - m) + r Gp m
            }
        }
        suU = fmaf(Fb, bu, suU);
        sdU = fmaf(Fb, bd, sdU);
        if (!ISO) {
            const float Fc = Fb * m;
            suL = fmaf(Fc, bu, suL);
            sdL = fmaf(Fc, bd, sdL);
        }
    }

    Layer32 o;
    if (ISO) {
        o.T = t;
        o.R = r;
        o.Su = suU;
        o.Sd = sdU;
        o.omtr = omtr;
        o.opr = omtr + 2.f * t;
        o.mlay = m;
    } else {
        // merge upper (top -> centre) and lower (centre -> bottom) sub-layers
        const float opr1 = 1.f + r;
        const float Dr = frcp(omr * opr1);      // 1 / (1 - r^2)
        const float tD = t * Dr;
        o.T = t * tD;
        o.R = fmaf(r, o.T, r);
        o.Su = fmaf(tD, fmaf(r, sdU, suL), suU);
        o.Sd = fmaf(tD, fmaf(r, suL, sdU), sdL);
        o.omtr = (omtr * (omtr + 2.f * t)) * (opr1 * Dr);   // (1-r-t)(1-r+t)/(1-r)
        o.opr = fmaf(omr, o.T, omr);
        o.mlay = m * m;
    }
    return o;
}

// ---------------------------------------------------------------------
// Shared-memory layout (both kernels):
//   acc   double [2 (Lmax+1)]                  column sums (F_up, F_net)
//   wpart R      [2 (Lmax+1) nwarps]            warp partial sums
//   sB    R      [(2 Lmax + 1) nb_chunk]        Planck at levels (2i iface, 2i+1 centre)
//   sFs   R      [nb_chunk]                     stellar flux per bin
//   sFB   R      [nb_chunk]                     F_BOA per bin
//   stoa  R      [block]                        weighted TOA F_up per system
// ---------------------------------------------------------------------
template <typename R>
__host__ __device__ inline size_t smem_bytes_t(int block, int Lmax, int nb_chunk) {
    const int nw = block / 32;
    size_t b = sizeof(double) * 2 * (size_t)(Lmax + 1);
    b += sizeof(R) * 2 * (size_t)(Lmax + 1) * nw;
    b += sizeof(R) * (size_t)(2 * Lmax + 1) * nb_chunk;
    b += sizeof(R) * 2 * (size_t)nb_chunk;
    b += sizeof(R) * (size_t)block;
    return b;
}

int fp32_warp_floats(int Lmax, int nbw, int direct) {
    // Planck [(2 Lmax + 1) nbw] (staged mode only) + F* [nbw] + F_BOA [nbw]
    // + transpose [16][2][33]
    int n = (direct ? 0 : (2 * Lmax + 1) * nbw) + 2 * nbw + 16 * 2 * 33;
    return (n + 3) & ~3;
}
size_t fp32_smem_bytes(int block, int Lmax, int nbw, int direct) {
    return sizeof(float) * (size_t)(block / 32) * fp32_warp_floats(Lmax, nbw, direct);
}
size_t fp64_smem_bytes(int block, int Lmax, int nb_chunk) { return smem_bytes_t<double>(block, Lmax, nb_chunk); }
size_t fp32_scratch_per_slot(int Lmax) { return sizeof(float4) * (size_t)Lmax; }
size_t fp64_scratch_per_slot(int Lmax, int isothermal) {
    const int nlev = isothermal ? Lmax : 2 * Lmax;
    return 2 * sizeof(double2) * (size_t)nlev;
}
int bins_per_chunk(int block, int n_g, int max_bins) {
    int nb = (block - 1) / n_g + 2;
    return nb < max_bins ? nb : max_bins;
}

template <typename R>
struct Smem {
    double *acc;
    R *wpart, *sB, *sFs, *sFB, *stoa;
    __device__ Smem(unsigned char *raw, int Lmax, int nb_chunk, int nwarps) {
        acc = reinterpret_cast<double *>(raw);
        wpart = reinterpret_cast<R *>(acc + 2 * (Lmax + 1));
        sB = wpart + 2 * (Lmax + 1) * nwarps;
        sFs = sB + (2 * Lmax + 1) * nb_chunk;
        sFB = sFs + nb_chunk;
        stoa = sFB + nb_chunk;
    }
};

// Column bookkeeping common to both kernels.
struct ColInfo {
    int c, L, NB, S;
    long long cube0, lay0, if0, bin0, tc_in, if_in, fs_in;
    double mu;
};

__device__ __forceinline__ bool next_column(const KParams &kp, int *s_unit, ColInfo &ci) {
    if (threadIdx.x == 0) *s_unit = atomicAdd(kp.counter, 1);
    __syncthreads();
    const int unit = *s_unit;
    __syncthreads();
    if (unit >= kp.n_cols) return false;
    ci.c = kp.order[unit];
    ci.L = kp.n_layers[ci.c];
    ci.NB = kp.n_bins[ci.c];
    ci.S = ci.NB * kp.n_g;
    ci.cube0 = kp.cube_off[ci.c];
    ci.lay0 = kp.lay_off[ci.c];
    ci.if0 = ci.lay0 + ci.c;
    ci.bin0 = kp.bin_off[ci.c];
    ci.tc_in = kp.tc_off[ci.c];
    ci.if_in = kp.if_off[ci.c];
    ci.fs_in = kp.fs_off[ci.c];
    ci.mu = kp.mu_star[kp.mu_idx[ci.c]];
    return true;
}

// Planck at the 2L+1 levels of the column for bins [b_lo, b_lo + nbc).
template <typename R>
__device__ __forceinline__ void stage_planck(const KParams &kp, const ColInfo &ci, int b_lo, int nbc,
                                             Smem<R> &sm) {
    const int nlev = 2 * ci.L + 1;
    const double dwn = (kp.wn_max - kp.wn_min) / ci.NB;
    auto edge = [&](int e) { return kp.edges ? kp.edges[e] : kp.wn_min + e * dwn; };
    for (int i = threadIdx.x; i < nlev * nbc; i += blockDim.x) {
        const int lev = i / nbc, bb = i - lev * nbc, b = b_lo + bb;
        const double T = (lev & 1) ? kp.T_center[ci.tc_in + (lev >> 1)] : kp.T_iface[ci.if_in + (lev >> 1)];
        const double wlo = edge(b), whi = edge(b + 1);
        if constexpr (sizeof(R) == 4)
            sm.sB[i] = planck_bin_f((float)T, (float)wlo, (float)whi);
        else
            sm.sB[i] = planck_bin_d(T, wlo, whi);
    }
    for (int bb = threadIdx.x; bb < nbc; bb += blockDim.x) {
        const int b = b_lo + bb;
        const double wlo = edge(b), whi = edge(b + 1);
        sm.sFs[bb] = (R)kp.F_star[ci.fs_in + b];
        if constexpr (sizeof(R) == 4)
            sm.sFB[bb] = kPiF * planck_bin_f((float)kp.T_int, (float)wlo, (float)whi);
        else
            sm.sFB[bb] = kPi * planck_bin_d(kp.T_int, wlo, whi);
    }
}

// Butterfly sum of two values over the warp; lane 0 stores the warp partial.
template <typename R>
__device__ __forceinline__ void warp_store(R a, R n, int level, int nwarps, R *wpart) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        wpart[2 * (level * nwarps + w)] = a;
        wpart[2 * (level * nwarps + w) + 1] = n;
    }
}

template <typename R>
__device__ __forceinline__ void fold_warps(int L, int nwarps, Smem<R> &sm) {
    for (int i = threadIdx.x; i <= L; i += blockDim.x) {
        double sa = 0.0, sn = 0.0;
        for (int w = 0; w < nwarps; ++w) {
            sa += (double)sm.wpart[2 * (i * nwarps + w)];
            sn += (double)sm.wpart[2 * (i * nwarps + w) + 1];
        }
        sm.acc[2 * i] += sa;
        sm.acc[2 * i + 1] += sn;
    }
}

__device__ __forceinline__ void write_column(const KParams &kp, const ColInfo &ci, const double *acc) {
    for (int i = threadIdx.x; i <= ci.L; i += blockDim.x) {
        const double up = acc[2 * i], net = acc[2 * i + 1];
        kp.F_up[ci.if0 + i] = up;
        kp.F_net[ci.if0 + i] = net;
        kp.F_dn[ci.if0 + i] = up - net;
    }
    const double gc = kp.grav / kp.cp;
    for (int l = threadIdx.x; l < ci.L; l += blockDim.x) {
        const double dF = acc[2 * (l + 1) + 1] - acc[2 * l + 1];
        const double dp = kp.p_iface[ci.if_in + l + 1] - kp.p_iface[ci.if_in + l];
        kp.Q[ci.lay0 + l] = gc * dF / dp;
    }
}

// ---------------------------------------------------------------------
// FP32 chosen form.
//
// fp32_prep: per column, the Planck function of every bin at the 2L+1
// levels (bin-integrated B, Sec. 2.2.1), F* and F_BOA = pi B(T_int) per bin
// (Eq. 10), and mu, 1/mu, all in FP32 -- the only place the FP32 path reads
// the FP64 per-column inputs.
//
// fp32_units: each warp takes work units of 32 consecutive systems of one
// column (an atomic counter over a largest-column-first list), so no CTA
// barrier is needed and no warp idles on a short column tail.  Per unit the
// warp stages the B values of the bins its systems touch into its own slice
// of shared memory, each lane solves one system, and the weighted interface
// fluxes of the 32 lanes are summed through a padded shared-memory
// transpose (16 interfaces at a time).  The warp that finishes the last unit
// of a column sums the column's unit partials in unit order (FP64) and
// writes fluxes, net flux and heating.
// ---------------------------------------------------------------------
// One (column, level) per warp: lane e evaluates the Planck integral at bin
// edge e (whichever of S(x) or P(x) that edge needs), and bin b takes edges b
// and b+1 from its lane and the next (shuffle).  31 bins per pass.
// x^3 / (e^x - 1), the Planck integrand in x = h c nu / (k T).  Below x = 1/2
// e^x - 1 is formed from its Taylor series (expm1(x) / x to x^6 / 7!,
// truncation < 2e-7 relative) so that small x keeps its digits.
__device__ __forceinline__ float planck_integrand_f(float x) {
    if (x < 0.5f) {
        const float q = fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 5040.f, 1.f / 720.f),
                                                          1.f / 120.f), 1.f / 24.f), 1.f / 6.f), 0.5f), 1.f);
        return x * x * frcp(q);
    }
    return x * x * x * frcp(__expf(x) - 1.f);
}

// Bins narrower than this in x = h c nu / (k T) are integrated by quadrature.
constexpr float kNarrowBin = 0.5f;
// Narrow bins below this width, and below 2% of their centre x, take
// 2-point Gauss-Legendre (nodes -+1/sqrt(3), weights 1); wider ones 4 points.
constexpr float kTwoPointBin = 0.1f;
constexpr float kGL2x = 0.57735026918962576f;
// 4-point Gauss-Legendre on [-1, 1]: outer and inner nodes with their weights.
__constant__ float kGL4x[2] = {0.86113631159405258f, 0.33998104358485626f};
__constant__ float kGL4w[2] = {0.34785484513745386f, 0.65214515486254614f};

__device__ __forceinline__ void planck_level_warp(float T, int NB, float dwn, float wmin,
                                                  const float *edges, const float *dnu, float scale,
                                                  float *dst, int lane) {
    const float a = (T > 0.f) ? (float)(kC2 * 100.0) * frcp(T) : 0.f;
    const float T2 = T * T;
    const float pref = (float)kPlanckK * (T2 * T2) * scale;
    for (int b0 = 0; b0 < NB; b0 += 31) {
        const int e = b0 + lane;
        const float wn = edges ? __ldg(edges + min(e, NB)) : fmaf((float)e, dwn, wmin);
        const float x = a * wn;
        const float x1 = __shfl_down_sync(0xffffffffu, x, 1);
        const int bin = e;
        const bool narrow = !(lane < 31 && bin < NB) || (x1 - x < kNarrowBin);
        // the edge series are needed only when some bin of this pass is wide
        float v = 0.f;
        if (!__all_sync(0xffffffffu, narrow)) v = (x < 2.f) ? planck_lower_f(x) : planck_upper_f(x);
        const float v1 = __shfl_down_sync(0xffffffffu, v, 1);
        if (lane < 31 && bin < NB) {
            float d;
            if (narrow) {
                // narrow bin (e.g. R = 500): the edge difference would lose
                // the digits that the edges' own FP32 rounding carries, so
                // integrate x^3/(e^x - 1) over the bin by Gauss-Legendre (2
                // or 4 points), the width formed from the FP64 edges before
                // rounding (no FP64 arithmetic here: it is slow on this part)
                const float dnu_b = edges ? __ldg(dnu + bin) : dwn;
                const float hh = 0.5f * a * dnu_b;        // half width in x
                const float xm = x + hh;
                float acc;
                if (hh < 0.5f * kTwoPointBin && hh < 0.01f * xm) {
                    // 2 points: below 2e-8 relative for these widths
                    acc = planck_integrand_f(fmaf(-hh, kGL2x, xm)) + planck_integrand_f(fmaf(hh, kGL2x, xm));
                } else {
                    acc = 0.f;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float t = (k < 2) ? -kGL4x[k] : kGL4x[3 - k];
                        const float xk = fmaf(hh, t, xm);
                        acc = fmaf(kGL4w[k < 2 ? k : 3 - k], planck_integrand_f(xk), acc);
                    }
                }
                d = hh * acc;
            } else if (x >= 2.f) {
                d = v - v1;
            } else if (x1 <= 2.f) {
                d = v1 - v;
            } else {
                d = ((float)kPi4Over15 - v) - v1;
            }
            dst[bin] = (T > 0.f) ? pref * d : 0.f;
        }
    }
}

// ---------------------------------------------------------------------
// Input front end (Sec. 2.1.3): optics from the column state and a premixed
// k-table.  Per layer (kt_layer): the bracketing grid cell of (T_center,
// log10 sqrt(p_top p_bot)), clamped, its bilinear weights and the column
// mass dp / g.  Per system (kt_mix): log10 kappa interpolated bilinearly,
// kappa = 10^x, extinction per unit mass E = kappa + s_b + a_b (s_b, a_b:
// the bin's scattering and cloud absorption per unit mass), dtau = E dp / g,
// w0 = s_b / E and the bin's g0.  Every operation is an explicitly rounded
// intrinsic, so that the fused solve and the standalone optics kernel
// produce the same bits.
// ---------------------------------------------------------------------
__device__ __forceinline__ void kt_bracket(const double *grid, int n, double v, int &i, float &w) {
    v = fmin(fmax(v, grid[0]), grid[n - 1]);
    int lo = 0, hi = n - 1;                       // grid[lo] <= v <= grid[hi]
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (grid[m] <= v) lo = m;
        else hi = m;
    }
    i = lo;
    w = (float)__ddiv_rn(__dsub_rn(v, grid[lo]), __dsub_rn(grid[lo + 1], grid[lo]));
}

__device__ __forceinline__ float4 kt_layer(const KParams &kp, double T, double p_top, double p_bot, int S) {
    int iT, iP;
    float wT, wP;
    kt_bracket(kp.kt_T, kp.kt_nT, T, iT, wT);
    kt_bracket(kp.kt_lp, kp.kt_nP, log10(sqrt(__dmul_rn(p_top, p_bot))), iP, wP);
    const int off = (iT * kp.kt_nP + iP) * S;
    return make_float4(__int_as_float(off), wT, wP, (float)__ddiv_rn(__dsub_rn(p_bot, p_top), kp.grav));
}

struct Optics {
    float dt, w0, g0;
};

constexpr float kLog2Of10 = 3.32192809488736234787f;

__device__ __forceinline__ Optics kt_mix(float k00, float k01, float k10, float k11, float4 l4, float4 bq) {
    const float a0 = __fmaf_rn(l4.z, __fsub_rn(k01, k00), k00);     // along log p at T_i
    const float a1 = __fmaf_rn(l4.z, __fsub_rn(k11, k10), k10);     // along log p at T_i+1
    const float x = __fmaf_rn(l4.y, __fsub_rn(a1, a0), a0);         // log10 kappa
    const float kappa = exp2f(__fmul_rn(x, kLog2Of10));
    const float ext = __fadd_rn(__fadd_rn(kappa, bq.x), bq.y);
    Optics o;
    o.dt = __fmul_rn(ext, l4.w);
    o.w0 = ext > 0.f ? __fdiv_rn(bq.x, ext) : 0.f;
    o.g0 = bq.z;
    return o;
}

// The four table corners of system s for a layer whose cell starts at l4.x.
struct Corners {
    float k00, k01, k10, k11;
};

__device__ __forceinline__ Corners kt_corners(const KParams &kp, float4 l4, int S, int s) {
    const float *t = kp.kt_lk + __float_as_int(l4.x) + s;
    const int sP = S, sT = kp.kt_nP * S;
    Corners c;
    c.k00 = __ldg(t);
    c.k01 = __ldg(t + sP);
    c.k10 = __ldg(t + sT);
    c.k11 = __ldg(t + sT + sP);
    return c;
}

__global__ void __launch_bounds__(256) fp32_prep(KParams kp) {
    extern __shared__ float sT[];                 // [2 Lmax + 1] temperatures of one column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = blockIdx.x; c < kp.n_cols; c += gridDim.x) {
        const int L = kp.n_layers[c], NB = kp.n_bins[c];
        const long long tc0 = kp.tc_off[c], ifi = kp.if_off[c], b0 = kp.bin_off[c], fsi = kp.fs_off[c];
        float *B = kp.planck32 + kp.planck_off[c];
        const float dwn = (float)((kp.wn_max - kp.wn_min) / NB);
        const float wmin = (float)kp.wn_min;
        const int nlev = 2 * L + 1;
        __syncthreads();                          // previous column done with sT
        for (int lev = threadIdx.x; lev < nlev; lev += blockDim.x)
            sT[lev] = (float)((lev & 1) ? kp.T_center[tc0 + (lev >> 1)] : kp.T_iface[ifi + (lev >> 1)]);
        if (kp.kt_lk)
            for (int l = threadIdx.x; l < L; l += blockDim.x)
                kp.kt_lay[kp.lay_off[c] + l] =
                    kt_layer(kp, kp.T_center[tc0 + l], kp.p_iface[ifi + l], kp.p_iface[ifi + l + 1], NB * kp.n_g);
        __syncthreads();
        // levels 0..2L, then one extra task for the per-bin and per-column data
        for (int lev = warp; lev <= nlev; lev += nw) {
            if (lev < nlev) {
                planck_level_warp(sT[lev], NB, dwn, wmin, kp.edges32, kp.dnu32, 1.f, B + (long long)lev * NB,
                                  lane);
            } else {
                planck_level_warp((float)kp.T_int, NB, dwn, wmin, kp.edges32, kp.dnu32, kPiF, kp.fboa32 + b0,
                                  lane);
                for (int b = lane; b < NB; b += 32) kp.fs32[b0 + b] = (float)kp.F_star[fsi + b];
                if (lane == 0) {
                    const double mu = kp.mu_star[kp.mu_idx[c]];
                    kp.colf[c] = make_float4((float)mu, mu > 0.0 ? (float)(1.0 / mu) : 0.f,
                                             mu > 0.0 ? 1.f : 0.f, 0.f);
                }
            }
        }
    }
}

__device__ void finalize_column(const KParams &kp, int c, int lane) {
    const int L = kp.n_layers[c];
    const int nu = kp.col_units[c];
    const long long if0 = kp.lay_off[c] + c;
    const float *part = kp.partial + kp.part_off[c];
    const int stride = 2 * (L + 1);
    // unit partials are read through L2 (other SMs wrote them)
    auto sum = [&](int i, int qq) {
        double a = 0.0;
        for (int uidx = 0; uidx < nu; ++uidx) a += (double)__ldcg(part + (long long)uidx * stride + 2 * i + qq);
        return a;
    };
    for (int i = lane; i <= L; i += 32) {
        const double up = sum(i, 0), net = sum(i, 1);
        kp.F_up[if0 + i] = up;
        kp.F_net[if0 + i] = net;
        kp.F_dn[if0 + i] = up - net;
    }
    const float gc = (float)(kp.grav / kp.cp);
    for (int l = lane; l < L; l += 32) {
        const double dF = sum(l + 1, 1) - sum(l, 1);
        const float dp = (float)(kp.p_iface[kp.if_off[c] + l + 1] - kp.p_iface[kp.if_off[c] + l]);
        kp.Q[kp.lay_off[c] + l] = (double)(gc * (float)dF * frcp(dp));
    }
}

// Planck values of a lane's bin: staged in the warp's shared memory (level
// stride nbc) or, when few g-points share a bin (DIRECT), read straight from
// the pre-kernel's table (level stride NB) through the read-only path.
template <bool DIRECT>
__device__ __forceinline__ float ldB(const float *p) {
    if constexpr (DIRECT) return __ldg(p);
    else return *p;
}

template <bool ISO, bool DIRECT, bool KT>
__global__ void __launch_bounds__(kMaxBlock32, 3) fp32_units(KParams kp) {
    extern __shared__ __align__(16) float smem32[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *wsm = smem32 + (size_t)warp * kp.warp_floats;
    const int NG = kp.n_g;
    const int nbw = kp.nbw;
    float *sB = wsm;                               // [(2 L + 1) nbc], staged mode
    float *sFs = wsm + (DIRECT ? 0 : (2 * kp.Lmax + 1) * nbw);    // [nbc]
    float *sFB = sFs + nbw;                        // [nbc]
    float *tb = sFB + nbw;                         // [16][2][33]
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long sstride = kp.n_slots;
    Counters cn = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};

    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(kp.counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= kp.n_units) break;
        const int c = kp.unit_col[unit];
        const int ku = kp.unit_k[unit];
        const int L = kp.n_layers[c], NB = kp.n_bins[c];
        const int S = NB * NG;
        const long long cube0 = kp.cube_off[c];
        const float4 cf = kp.colf[c];
        const float mu = cf.x, imu = cf.y;
        const double mu_d = kp.mu_star[kp.mu_idx[c]];   // only for the rare FP64 resonance test
        const bool beam = cf.z != 0.f;
        const int s0 = ku * 32;
        const int b_lo = s0 / NG;
        const int nbc = min(NB - 1, (s0 + 31) / NG) - b_lo + 1;

        // stage B of the unit's bins at the 2L+1 levels, F* and F_BOA
        {
            const float *Bg = kp.planck32 + kp.planck_off[c] + b_lo;
            const int nlev = 2 * L + 1;
            if constexpr (!DIRECT) {
                for (int i = lane; i < nlev * nbc; i += 32) {
                    const int lev = i / nbc, bb = i - lev * nbc;
                    sB[i] = __ldcg(Bg + (long long)lev * NB + bb);
                }
            }
            if (lane < nbc) {
                sFs[lane] = __ldcg(kp.fs32 + kp.bin_off[c] + b_lo + lane);
                sFB[lane] = __ldcg(kp.fboa32 + kp.bin_off[c] + b_lo + lane);
            }
        }
        __syncwarp();

        // padding lanes of a column's last unit repeat system s0 with zero
        // weight, so the loops below need no per-lane predicates
        const bool active = s0 + lane < S;
        const int s = active ? s0 + lane : s0;
        cn.on = active ? 1u : 0u;
        cn.s_inv = cn.s_ecl = cn.s_etau = 0u;
        const int b = s / NG;
        const int bb = b - b_lo;
        const float wg = active ? kp.g_w32[s - b * NG] : 0.f;
        const int bst = DIRECT ? NB : nbc;         // level stride of Bp
        const float *Bp = DIRECT ? kp.planck32 + kp.planck_off[c] + b : sB + bb;

        // forward elimination, TOA -> BOA, departure variables; the B of a
        // layer's bottom interface is carried as the next layer's top
        float Bt = ldB<DIRECT>(Bp), Bc = ldB<DIRECT>(Bp + bst), Bb = ldB<DIRECT>(Bp + 2 * bst);
        float al = 1.f;                                      // alpha' = 1 - a'
        float bl = (float)kp.F_toa - kPiF * Bt;              // b' at the TOA
        float Fb = beam ? mu * sFs[bb] : 0.f;
        // optics: read from the cubes, or (KT) from the k-table corners of
        // the layer's grid cell, fetched one layer ahead
        const float *pd = nullptr, *pw = nullptr, *pg = nullptr;
        float nd = 0.f, nw = 0.f, ng = 0.f;
        const float4 *klay = nullptr;
        float4 kl_next = make_float4(0.f, 0.f, 0.f, 0.f), kl_after = kl_next, kb = kl_next;
        Corners kc = {0.f, 0.f, 0.f, 0.f};
        if constexpr (KT) {
            klay = kp.kt_lay + kp.lay_off[c];
            kb = __ldg(kp.kt_bin + b);
            kl_next = klay[0];
            kl_after = L > 1 ? klay[1] : kl_next;
            kc = kt_corners(kp, kl_next, S, s);
        } else {
            pd = kp.dtau + cube0 + s;
            pw = kp.w0 + cube0 + s;
            pg = kp.g0 + cube0 + s;
            nd = __ldcs(pd);
            nw = __ldcs(pw);
            ng = __ldcs(pg);
        }
        float4 *sp = kp.scr32 + slot;
        for (int l = 0; l < L; ++l) {
            float dt, w0, g0;
            float nBc = 0.f, nBb = 0.f;
            if constexpr (KT) {
                const Corners cur = kc;
                const float4 kl = kl_next;
                if (l + 1 < L) {                     // prefetch the next layer's corners
                    kl_next = kl_after;
                    kc = kt_corners(kp, kl_next, S, s);
                    if (l + 2 < L) kl_after = klay[l + 2];
                    nBc = ldB<DIRECT>(Bp + 3 * bst);
                    nBb = ldB<DIRECT>(Bp + 4 * bst);
                }
                const Optics o = kt_mix(cur.k00, cur.k01, cur.k10, cur.k11, kl, kb);
                dt = o.dt;
                w0 = o.w0;
                g0 = o.g0;
            } else {
                dt = nd;
                w0 = nw;
                g0 = ng;
                if (l + 1 < L) {                     // prefetch the next layer
                    pd += S; pw += S; pg += S;
                    nd = __ldcs(pd);
                    nw = __ldcs(pw);
                    ng = __ldcs(pg);
                    nBc = ldB<DIRECT>(Bp + 3 * bst);
                    nBb = ldB<DIRECT>(Bp + 4 * bst);
                }
            }
            const Layer32 ly = layer32<ISO>(dt, w0, g0, Bt, Bc, Bb, mu, imu, mu_d, beam, Fb, kp, cn);
            Bp += 2 * bst;
            Bt = Bb;
            Bc = nBc;
            Bb = nBb;
            const float omr = ly.omtr + ly.T;                // 1 - R
            const float ipv = frcp(fmaf(ly.R, al, omr));     // 1 / (1 - R a')
            float4 st;
            st.x = ly.T * ipv;                               // P
            st.y = fmaf(ly.R, bl, ly.Su) * ipv;              // Q
            st.z = al;                                       // alpha' at interface l
            st.w = bl + Fb;                                  // e = b' + F_beam
            __stcg(sp, st);
            sp += sstride;
            const float al_n = fmaf(al, fmaf(ly.R, omr, ly.T * ly.T), ly.omtr * ly.opr) * ipv;
            const float bl_n = ly.Sd + ly.T * fmaf(1.f - al, ly.Su, bl) * ipv;
            al = al_n;
            bl = bl_n;
            Fb *= ly.mlay;
        }

        if (active) {
            cn.inv += cn.s_inv;
            cn.eclamp += cn.s_ecl;
            cn.etau += (ISO ? 1u : 2u) * cn.s_etau;
        }
        // BOA (Eq. 10): u - d = F_BOA + F_beam with d = (1 - alpha') u + b';
        // back-substitution to the TOA; interface sums through the transpose
        const float FBOA = sFB[bb];
        float uu = (FBOA + Fb + bl) * frcp(al);
        bool bad = !isfinite(uu);   // NaN and Inf propagate up the substitution
        float *part = kp.partial + kp.part_off[c] + (long long)ku * 2 * (L + 1);
        // Bp points at level 2L (the BOA interface), whose B is Bt
        tb[lane] = wg * fmaf(kPiF, Bt, uu);
        float nBi = ldB<DIRECT>(Bp - 2 * bst);     // B one interface up
        tb[33 + lane] = wg * FBOA;
        int gi = 1;              // slots used in the current group of 16 interfaces
        int gtop = L;            // interface held in slot 0 of the group
        sp -= sstride;           // interface L-1
        float4 nst = __ldcg(sp);
        for (int i = L - 1; i >= -1; --i) {
            if (i >= 0) {
                const float4 st = nst;
                if (i > 0) {
                    sp -= sstride;
                    nst = __ldcg(sp);
                }
                Bp -= 2 * bst;
                const float Bi = nBi;
                if (i > 0) nBi = ldB<DIRECT>(Bp - 2 * bst);
                uu = fmaf(st.x, uu, st.y);
                const float fup = fmaf(kPiF, Bi, uu);
                Bt = Bi;
                const float fnet = fmaf(st.z, uu, -st.w);
                tb[(gi * 2) * 33 + lane] = wg * fup;
                tb[(gi * 2 + 1) * 33 + lane] = wg * fnet;
                ++gi;
            }
            if (gi == 16 || (i < 0 && gi > 0)) {
                __syncwarp();
                // lane j sums row (slot j & 15, quantity j >> 4) over the 32 lanes
                const int sl = lane & 15, qq = lane >> 4;
                if (sl < gi) {
                    const float *row = tb + (sl * 2 + qq) * 33;
                    float acc = 0.f;
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) acc += row[j];
                    part[2 * (gtop - sl) + qq] = acc;
                }
                __syncwarp();
                gtop -= gi;
                gi = 0;
            }
        }
        bad |= !isfinite(uu);
        if (active && bad) cn.nonfinite++;

        // TOA spectrum: uu and Bp are now at interface 0; each bin's lanes
        // are summed in lane order and added once per unit (a bin of n_g <= 32
        // systems meets at most two units, so the FP64 sum is order-free)
        if (kp.toa) {
            tb[lane] = wg * fmaf(kPiF, Bt, uu);
            __syncwarp();
            if (lane < nbc) {
                const int bt = b_lo + lane;
                const int j0 = max(0, bt * NG - s0);
                const int j1 = min(min(32, S - s0), (bt + 1) * NG - s0);
                float acc = 0.f;
                for (int j = j0; j < j1; ++j) acc += tb[j];
                atomicAdd(kp.toa + kp.bin_off[c] + bt, (double)acc);
            }
            __syncwarp();
        }

        // the warp that completes a column's last unit writes the column
        __threadfence();
        int done = 0;
        if (lane == 0) done = atomicAdd(kp.col_done + c, 1);
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done == kp.col_units[c] - 1) {
            __threadfence();
            finalize_column(kp, c, lane);
        }
        __syncwarp();
    }
    flush_counters(cn, kp.stats);
}

// ---------------------------------------------------------------------
// FP64 plain path: the paper's formulas as written (App. B), scalar
// elimination over every level.
// ---------------------------------------------------------------------
struct Sub64 {
    double t, r, su, sd;
};

__device__ __forceinline__ void g_factors64(double w0, double g0, double E, double mus, double eps2,
                                            double D, double &Gp, double &Gm) {
    const double omwg = 1.0 - w0 * g0;
    const double lead = w0 * (2.0 * E * omwg + g0 / eps2) / D;
    const double tail = w0 * g0 / (2.0 * eps2 * E * omwg);
    Gp = 0.5 * (lead * (mus + 1.0 / (2.0 * E * omwg)) + tail);
    Gm = 0.5 * (lead * (mus - 1.0 / (2.0 * E * omwg)) - tail);
}

__device__ __forceinline__ Sub64 sub64(double dts, double w0, double g0, double E, double B1,
                                       double Biso, double B2, double mu, double Fb1, double Fb2,
                                       const KParams &kp, Counters &cn, bool count_layer) {
    const double omwg = 1.0 - w0 * g0;
    const double k = sqrt((E - w0) / (E * omwg));
    const double zp = 0.5 * (1.0 + k), zm = 0.5 * (1.0 - k);
    const double Pi = (E == w0) ? kPi : kPi * (1.0 - w0) / (E - w0);
    double chi, xi, psi;
    if (k > 0.0) {
        const double T = exp(-2.0 * sqrt(E * (E - w0) * omwg) * dts);
        chi = zm * zm * T * T - zp * zp;
        xi = zp * zm * (1.0 - T * T);
        psi = (zm * zm - zp * zp) * T;
    } else {
        const double q = E * omwg;
        chi = -(1.0 + q * dts);
        xi = q * dts;
        psi = -1.0;
    }
    double Su, Sd;
    if (kp.isothermal) {
        Su = Pi * Biso * (chi + xi - psi);
        Sd = Su;
    } else {
        double Bt = B1, Bb = B2, Bp;
        if (dts < (double)1e-4f) {
            Bt = Bb = 0.5 * (B1 + B2);
            Bp = 0.0;
            cn.etau += cn.on;
        } else {
            Bp = (B2 - B1) / dts;
        }
        const double Theta = (chi - psi - xi) / (2.0 * E * omwg);
        Su = Pi * (Bt * (chi + xi) - psi * Bb + Bp * Theta);
        Sd = Pi * (Bb * (chi + xi) - psi * Bt - Bp * Theta);
    }
    if (mu > 0.0) {
        const double mus = -mu;
        const double D = 4.0 * E * mus * mus * (E - w0) * omwg - 1.0;
        double bu, bd;
        bool avg = false;
        double Dx = D;
        if (fabs(D) < 1e-5) {
            if (count_layer) cn.res += cn.on;
            if (kp.resonance_paper) Dx = 2.0 * mus;
            else if (fabs(D) < 1e-7) avg = true;
        }
        if (!avg) {
            double Gp, Gm;
            g_factors64(w0, g0, E, mus, kp.eps2, Dx, Gp, Gm);
            bu = psi * Gp * Fb2 - (xi * Gm + chi * Gp) * Fb1;
            bd = psi * Gm * Fb1 - (xi * Gp + chi * Gm) * Fb2;
        } else {
            // exact limit: mean of the per-unit-beam source at mu (1 -+ 5e-6)
            bu = bd = 0.0;
            for (int sg = -1; sg <= 1; sg += 2) {
                const double mu2 = mu * (1.0 + sg * 5e-6);
                const double D2 = 4.0 * E * mu2 * mu2 * (E - w0) * omwg - 1.0;
                double Gp, Gm;
                g_factors64(w0, g0, E, -mu2, kp.eps2, D2, Gp, Gm);
                const double m2 = exp(-dts / mu2);
                bu += 0.5 * Fb1 * (psi * Gp * m2 - (xi * Gm + chi * Gp));
                bd += 0.5 * Fb1 * (psi * Gm - (xi * Gp + chi * Gm) * m2);
            }
        }
        Su += bu;
        Sd += bd;
    }
    Sub64 o;
    o.t = psi / chi;
    o.r = -xi / chi;
    o.su = Su / chi;
    o.sd = Sd / chi;
    return o;
}

__global__ void __launch_bounds__(kMaxBlock) fp64_columns(KParams kp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    const int tid = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    Smem<double> sm(smem_raw, kp.Lmax, kp.nb_chunk, nwarps);
    const int NG = kp.n_g;
    const long long slot = (long long)blockIdx.x * blockDim.x + tid;
    double2 *scr = kp.scr64 + slot;           // element (2 lev + j) n_slots + slot
    Counters cn = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    ColInfo ci;
    const bool iso = kp.isothermal;

    while (next_column(kp, &s_unit, ci)) {
        for (int i = tid; i < 2 * (ci.L + 1); i += blockDim.x) sm.acc[i] = 0.0;
        const double mu = ci.mu;
        const bool beam = mu > 0.0;
        const int nsub = iso ? ci.L : 2 * ci.L;
        for (int s0 = 0; s0 < ci.S; s0 += blockDim.x) {
            const int b_lo = s0 / NG;
            const int b_hi = min(ci.NB - 1, (s0 + (int)blockDim.x - 1) / NG);
            const int nbc = b_hi - b_lo + 1;
            stage_planck<double>(kp, ci, b_lo, nbc, sm);
            __syncthreads();

            const int s = s0 + tid;
            const bool active = s < ci.S;
            cn.on = active ? 1u : 0u;
            const int b = active ? s / NG : b_lo;
            const int bb = b - b_lo;
            const double wg = active ? kp.g_w[s - b * NG] : 0.0;
            const double *Bcol = sm.sB + bb;
            const double Fs = sm.sFs[bb];

            double a = 0.0, bv = kp.F_toa;       // F_dn = a F_up + b at the TOA
            double tau = 0.0;
            double Fb = beam ? mu * Fs : 0.0;
            const long long base = ci.cube0 + s;
            for (int l = 0; l < ci.L; ++l) {
                double dt = 0.0, w0 = 0.0, g0 = 0.0;
                float w0f = 0.f, g0f = 0.f;
                if (active) {
                    const long long idx = base + (long long)l * ci.S;
                    dt = (double)__ldg(kp.dtau + idx);
                    w0f = __ldg(kp.w0 + idx);
                    g0f = __ldg(kp.g0 + idx);
                    w0 = (double)w0f;
                    g0 = (double)g0f;
                }
                if (!(dt >= 0.0) || !(w0 >= 0.0 && w0 <= 1.0) || !(g0 > -1.0 && g0 < 1.0)) cn.inv += cn.on;
                double E = 1.0;
                if (kp.improved && w0 > (double)0.1f) {
                    E = 1.225 - 0.1582 * g0 - 0.1777 * w0 - 0.07465 * g0 * g0 + 0.2351 * w0 * g0
                        - 0.05582 * w0 * w0;
                    if (kp.e_clamp && E < 1.0) {
                        E = 1.0;
                        cn.eclamp += cn.on;
                    }
                }
                const int nh = iso ? 1 : 2;
                for (int hsub = 0; hsub < nh; ++hsub) {
                    const double dts = iso ? dt : 0.5 * dt;
                    const int lev = iso ? l : 2 * l + hsub;        // top level of the sub-layer
                    const double B1 = iso ? 0.0 : Bcol[lev * nbc];
                    const double B2 = iso ? 0.0 : Bcol[(lev + 1) * nbc];
                    const double Biso = iso ? Bcol[(2 * l + 1) * nbc] : 0.0;
                    const double tau2 = tau + dts;
                    const double Fb2 = beam ? mu * Fs * exp(-tau2 / mu) : 0.0;
                    const Sub64 sb = sub64(dts, w0, g0, E, B1, Biso, B2, mu, Fb, Fb2, kp, cn, hsub == 0);
                    const double piv = 1.0 - sb.r * a;
                    double2 st0, st1;
                    st0.x = sb.t / piv;                            // P
                    st0.y = (sb.r * bv + sb.su) / piv;             // Q
                    st1.x = a;
                    st1.y = bv + Fb;                               // b + F_beam at the top level
                    scr[(long long)(2 * lev) * kp.n_slots] = st0;
                    scr[(long long)(2 * lev + 1) * kp.n_slots] = st1;
                    const double a_n = sb.r + sb.t * sb.t * a / piv;
                    const double b_n = sb.sd + sb.t * (bv + a * sb.su) / piv;
                    a = a_n;
                    bv = b_n;
                    tau = tau2;
                    Fb = Fb2;
                }
            }
            // BOA (Eq. 10): F_up - F_dn = F_BOA + F_beam, F_dn = a F_up + b
            const double FBOA = sm.sFB[bb];
            double fu = active ? (FBOA + Fb + bv) / (1.0 - a) : 0.0;
            double fnet = active ? (1.0 - a) * fu - (bv + Fb) : 0.0;
            warp_store<double>(wg * fu, wg * fnet, ci.L, nwarps, sm.wpart);
            bool bad = !isfinite(fu);
            for (int lev = nsub - 1; lev >= 0; --lev) {
                if (active) {
                    const double2 st0 = scr[(long long)(2 * lev) * kp.n_slots];
                    const double2 st1 = scr[(long long)(2 * lev + 1) * kp.n_slots];
                    fu = st0.x * fu + st0.y;
                    fnet = (1.0 - st1.x) * fu - st1.y;
                    bad |= !isfinite(fu);
                }
                const bool is_iface = iso || ((lev & 1) == 0);
                if (is_iface) {
                    const int i = iso ? lev : (lev >> 1);
                    warp_store<double>(active ? wg * fu : 0.0, active ? wg * fnet : 0.0, i, nwarps,
                                       sm.wpart);
                }
            }
            if (active && bad) cn.nonfinite++;
            sm.stoa[tid] = active ? wg * fu : 0.0;       // fu is now at interface 0 (TOA)
            __syncthreads();
            fold_warps<double>(ci.L, nwarps, sm);
            if (kp.toa && tid < nbc) {
                // one thread per bin sums its systems in order; a bin split
                // across chunks is continued by the same CTA after a barrier
                const int bt = b_lo + tid;
                const int j0 = max(0, bt * NG - s0);
                const int j1 = min(min((int)blockDim.x, ci.S - s0), (bt + 1) * NG - s0);
                double acc = 0.0;
                for (int j = j0; j < j1; ++j) acc += sm.stoa[j];
                kp.toa[ci.bin0 + bt] += acc;
            }
            __syncthreads();
        }
        write_column(kp, ci, sm.acc);
        __syncthreads();
    }
    flush_counters(cn, kp.stats);
}

// Front end alone: one CTA per column (grid-stride), the column's per-layer
// set-up in shared memory, then every (layer, bin, g) element.
__global__ void __launch_bounds__(256) kt_optics_kernel(KParams kp, const int64_t *pcube_off, float *dtau,
                                                         float *w0, float *g0) {
    extern __shared__ float4 sl[];                // [Lmax]
    const int NG = kp.n_g;
    for (int c = blockIdx.x; c < kp.n_cols; c += gridDim.x) {
        const int L = kp.n_layers[c], NB = kp.n_bins[c], S = NB * NG;
        const long long tc0 = kp.tc_off[c], ifi = kp.if_off[c], base = pcube_off[c];
        __syncthreads();
        for (int l = threadIdx.x; l < L; l += blockDim.x)
            sl[l] = kt_layer(kp, kp.T_center[tc0 + l], kp.p_iface[ifi + l], kp.p_iface[ifi + l + 1], S);
        __syncthreads();
        const long long n = (long long)L * S;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int l = (int)(i / S), s = (int)(i - (long long)l * S);
            const float4 l4 = sl[l];
            const Corners k = kt_corners(kp, l4, S, s);
            const Optics o = kt_mix(k.k00, k.k01, k.k10, k.k11, l4, __ldg(kp.kt_bin + s / NG));
            dtau[base + i] = o.dt;
            w0[base + i] = o.w0;
            g0[base + i] = o.g0;
        }
    }
}

constexpr int kMaxDynSmem = 200 * 1024;

cudaError_t init_kernels() {
    cudaError_t e = cudaSuccess;
    for (auto f : {fp32_units<false, false, false>, fp32_units<true, false, false>,
                   fp32_units<false, true, false>, fp32_units<true, true, false>,
                   fp32_units<false, false, true>, fp32_units<true, false, true>,
                   fp32_units<false, true, true>, fp32_units<true, true, true>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fp64_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

int occupancy(int precision_fp64, int block, size_t smem) {
    if (smem > (size_t)kMaxDynSmem) return 0;
    int n = 0;
    cudaError_t e = precision_fp64
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp64_columns, block, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp32_units<false, false, false>, block, smem);
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_fp32(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s) {
    const int pgrid = kp.n_cols < 4 * 148 ? kp.n_cols : 4 * 148;
    fp32_prep<<<pgrid, 256, sizeof(float) * (2 * kp.Lmax + 1), s>>>(kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int sel = (kp.isothermal ? 1 : 0) | (kp.direct ? 2 : 0) | (kp.kt_lk ? 4 : 0);
    switch (sel) {
        case 0: fp32_units<false, false, false><<<grid, block, smem, s>>>(kp); break;
        case 1: fp32_units<true, false, false><<<grid, block, smem, s>>>(kp); break;
        case 2: fp32_units<false, true, false><<<grid, block, smem, s>>>(kp); break;
        case 3: fp32_units<true, true, false><<<grid, block, smem, s>>>(kp); break;
        case 4: fp32_units<false, false, true><<<grid, block, smem, s>>>(kp); break;
        case 5: fp32_units<true, false, true><<<grid, block, smem, s>>>(kp); break;
        case 6: fp32_units<false, true, true><<<grid, block, smem, s>>>(kp); break;
        default: fp32_units<true, true, true><<<grid, block, smem, s>>>(kp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_kt_optics(const KParams &kp, const int64_t *pcube_off, float *dtau, float *w0,
                             float *g0, cudaStream_t s) {
    const int grid = kp.n_cols < 8 * 148 ? kp.n_cols : 8 * 148;
    kt_optics_kernel<<<grid, 256, sizeof(float4) * kp.Lmax, s>>>(kp, pcube_off, dtau, w0, g0);
    return cudaGetLastError();
}

cudaError_t launch_fp64(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s) {
    fp64_columns<<<grid, block, smem, s>>>(kp);
    return cudaGetLastError();
}

}  // namespace rt
