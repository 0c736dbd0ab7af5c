// rt_kernels.cu -- fused column kernels for sm_103a.
//
// The path for one batch (Sec. 2.2, App. B): per (column, bin, g) system the
// layer coefficients (App. B, Eq. 19), the stellar beam (Eq. B6) and its
// source terms (Eqs. B7-B8), the thermal sources (Eqs. 2-9), the Thomas
// elimination towards the BOA, the BOA closure (Eq. 10) and the substitution
// back to the TOA (Eqs. 12-15); then the Gauss-weighted sum over g and bins,
// net flux and heating.  Every reduction runs in a fixed order, so a column
// gives the same bits whatever else is in the batch.
//
// Kernels:
//   fp32_prep        Planck per bin at every level of every column (and at
//                    T_int), F*, mu, and the k-table cells when the front end
//                    is on; one CTA per column.
//   fp32_units       the FP32 "chosen form": a persistent grid of warps takes
//                    work units of 32 or 64 consecutive systems of a column
//                    (one or two per lane; two use the paired FP32
//                    instructions) from a largest-column-first list;
//                    cancellation-free transmission, reflection and absorption
//                    forms, a beam source with the removable singularity at
//                    mu* alpha = 1 divided out, departure variables u = F - pi
//                    B, merged sub-layers; FP64 only to decide the paper's
//                    resonance switch near |D| = 1e-5.  Each unit leaves its
//                    weighted interface sums as partials.
//   fp32_finalize    one warp per column: the units' partials summed in unit
//                    order (FP64) into fluxes, net flux and heating.
//   kt_optics_kernel the input front end alone (k-table interpolation and
//                    mixing), writing optics cubes.
//   fp64_columns     FP64 with the paper's literal formulas, one CTA per
//                    column, one thread per system, scalar Thomas on every
//                    level (sub-layers not merged).
#include <cuda_runtime.h>
#include <algorithm>
#include <array>
#include <type_traits>
#include <utility>

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

// Fast FP32 primitives: MUFU reciprocal, reciprocal square root and
// exponential (exp(x) = 2^(x log2 e), the PTX ex2 after one multiply).  Each
// is accurate to a few ulp, far inside the 1e-4 target.  The flush-to-zero
// forms are safe here: the solve never feeds them subnormal arguments (E - w0
// and the optical depths are either 0, handled by selects, or far above
// 1e-38), and subnormal exponentials are below every flux floor.
__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float frsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
constexpr float kLog2E = 1.44269504088896340736f;

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
// Bounds-check build (RT_BOUNDS_CHECK): a pointer outside [base, base + n)
// of its array is counted in stats[ST_BOUNDS] and the access is skipped (a
// load gives 0).  Nothing traps.  In the normal build the check is the
// constant true and adds no code.
// ---------------------------------------------------------------------
#ifdef RT_BOUNDS_CHECK
template <class T, class U>
__device__ __forceinline__ bool rt_in_range(const T *p, const U *base, long long n, unsigned long long *stats) {
    const char *c = reinterpret_cast<const char *>(p), *b = reinterpret_cast<const char *>(base);
    const bool ok = base != nullptr && c >= b && c + sizeof(T) <= b + n * (long long)sizeof(U);
    if (!ok) atomicAdd(stats + ST_BOUNDS, 1ull);
    return ok;
}
#define RT_IN(p, base, n) rt_in_range((p), (base), (long long)(n), kp.stats)
#else
#define RT_IN(p, base, n) true
#endif
// base[i] of an array of n elements; a store to it (both checked in bounds builds)
template <class T>
__device__ __forceinline__ T ck_ld(const KParams &kp, const T *base, long long n, long long i) {
    return RT_IN(base + i, base, n) ? base[i] : T{};
}
template <class T>
__device__ __forceinline__ void ck_st(const KParams &kp, T *base, long long n, long long i, T v) {
    if (RT_IN(base + i, base, n)) base[i] = v;
}

// ---------------------------------------------------------------------
// Counters kept in registers and flushed once per CTA.
// ---------------------------------------------------------------------
struct Counters {
    unsigned res, etau, eclamp, inv, nonfinite, fp64;
    unsigned on;   // FP64 path: 1 while the thread works on a real system, 0 on padding lanes
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
// ---------------------------------------------------------------------
// Values of one system (float) or of two systems carried by one lane (V2).
// V2 arithmetic maps onto sm_100+'s paired FP32 instructions (FFMA2, FMUL2,
// FADD2: two IEEE-rounded operations per instruction), so a lane that
// carries two systems issues about half as many FP32 instructions per
// system.  MUFU operations, compares and selects stay per component.
// ---------------------------------------------------------------------
// Stored as a float2 so that the pair stays in an aligned register pair,
// which the paired instructions read and write.
struct V2 {
    float2 v;
    __device__ __forceinline__ V2() {}
    __device__ __forceinline__ V2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit V2(float2 a) : v(a) {}
};
struct M2 {
    bool x, y;
};
struct U2 {
    unsigned x, y;
};

__device__ __forceinline__ float2 f2(V2 a) { return a.v; }
__device__ __forceinline__ V2 v2(float2 a) { return V2(a); }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return v2(__fadd2_rn(f2(a), f2(b))); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return v2(__fmul2_rn(f2(a), f2(b))); }
// a - b as a + (-1) b: one rounding, like the scalar subtraction
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return v2(__ffma2_rn(f2(b), make_float2(-1.f, -1.f), f2(a))); }
__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ M2 operator<(V2 a, V2 b) { return M2{a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ M2 operator<=(V2 a, V2 b) { return M2{a.v.x <= b.v.x, a.v.y <= b.v.y}; }
__device__ __forceinline__ M2 operator>(V2 a, V2 b) { return M2{a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ M2 operator>=(V2 a, V2 b) { return M2{a.v.x >= b.v.x, a.v.y >= b.v.y}; }
__device__ __forceinline__ M2 operator==(V2 a, V2 b) { return M2{a.v.x == b.v.x, a.v.y == b.v.y}; }
__device__ __forceinline__ M2 operator&(M2 a, M2 b) { return M2{a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ M2 operator&(M2 a, bool b) { return M2{a.x && b, a.y && b}; }
__device__ __forceinline__ M2 operator!(M2 a) { return M2{!a.x, !a.y}; }

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ V2 vfma(V2 a, V2 b, V2 c) { return v2(__ffma2_rn(f2(a), f2(b), f2(c))); }
__device__ __forceinline__ float vrcp(float a) { return frcp(a); }
__device__ __forceinline__ V2 vrcp(V2 a) { return V2(frcp(a.v.x), frcp(a.v.y)); }
__device__ __forceinline__ float vrsqrt(float a) { return frsqrt(a); }
__device__ __forceinline__ V2 vrsqrt(V2 a) { return V2(frsqrt(a.v.x), frsqrt(a.v.y)); }
// exp(-a) = 2^(-a log2 e): one (paired) multiply, then ex2 per component
__device__ __forceinline__ float vexpn(float a) { return fex2(a * -kLog2E); }
__device__ __forceinline__ V2 vexpn(V2 a) {
    const float2 y = __fmul2_rn(a.v, make_float2(-kLog2E, -kLog2E));
    return V2(fex2(y.x), fex2(y.y));
}
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ V2 vabs(V2 a) { return V2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ V2 vsel(M2 m, V2 a, V2 b) { return V2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }
__device__ __forceinline__ bool vany(bool m) { return m; }
__device__ __forceinline__ bool vany(M2 m) { return m.x || m.y; }
__device__ __forceinline__ void vcount(unsigned &c, bool m) { c += m ? 1u : 0u; }
__device__ __forceinline__ void vcount(U2 &c, M2 m) {
    c.x += m.x ? 1u : 0u;
    c.y += m.y ? 1u : 0u;
}
// per-component counts added only for systems that are real (`on`)
__device__ __forceinline__ unsigned vmasked(unsigned c, bool on) { return on ? c : 0u; }
__device__ __forceinline__ unsigned vmasked(U2 c, M2 on) { return (on.x ? c.x : 0u) + (on.y ? c.y : 0u); }
__device__ __forceinline__ unsigned vmasked(bool m, bool on) { return (m && on) ? 1u : 0u; }
__device__ __forceinline__ unsigned vmasked(M2 m, M2 on) { return (m.x && on.x ? 1u : 0u) + (m.y && on.y ? 1u : 0u); }

// FP32 series for the bin-integrated Planck function, written over V (one
// value, or two on the paired instructions: every component rounds as the
// scalar form does, so a pair of levels gives the scalar bits).
// S(x) for x <= 2 (terms to k = 14, relative error < 1e-7).
template <class V>
__device__ __forceinline__ V planck_lower_v(V x) {
    const V x2 = x * x;
    V s = V((float)kS14);
    s = vfma(s, x2, V((float)kS12));
    s = vfma(s, x2, V((float)kS10));
    s = vfma(s, x2, V((float)kS8));
    s = vfma(s, x2, V((float)kS6));
    s = vfma(s, x2, V((float)kS4));
    const V head = vfma(x, vfma(x, V((float)kS2), V((float)kS1)), V((float)kS0));
    return (vfma(x2 * x2, s, head) * x2) * x;
}

// P(x) = integral_x^inf t^3/(e^t-1) dt for x >= 2 as
//   sum_n e^(-n x) (x^3/n + 3 x^2/n^2 + 6 x/n^3 + 6/n^4), 8 terms,
// regrouped as e (x^3 A1 + 3 x^2 A2 + 6 x A3 + 6 A4) with
// A_k = sum_n e^(n-1) / n^k evaluated by Horner in e = e^-x <= e^-2.
template <class V>
__device__ __forceinline__ V planck_upper_v(V x) {
    const V e = vexpn(x);
    V a1 = V(1.f / 8.f), a2 = V(1.f / 64.f), a3 = V(1.f / 512.f), a4 = V(1.f / 4096.f);
#pragma unroll
    for (int n = 7; n >= 1; --n) {
        const float y = 1.0f / (float)n;
        a1 = vfma(a1, e, V(y));
        a2 = vfma(a2, e, V(y * y));
        a3 = vfma(a3, e, V(y * y * y));
        a4 = vfma(a4, e, V(y * y * y * y));
    }
    const V poly = vfma(x * x, vfma(x, a1, V(3.f) * a2), vfma(V(6.f) * x, a3, V(6.f) * a4));
    return e * poly;
}
__device__ __forceinline__ float planck_lower_f(float x) { return planck_lower_v(x); }
__device__ __forceinline__ float planck_upper_f(float x) { return planck_upper_v(x); }

template <class V> struct VTraits;
template <> struct VTraits<float> {
    using M = bool;
    using C = unsigned;
};
template <> struct VTraits<V2> {
    using M = M2;
    using C = U2;
};

// (1 - exp(-x)) / x for |x| < 0.25 as a degree-5 polynomial fitted for the least
// maximum relative error on [-0.25, 0.25], constant term fixed at 1 (csrc/fit_series.py):
// 2.9e-9 relative with the FP32 coefficients, 6.1e-8 evaluated in FP32 -- as
// close as the 7-term Taylor sum sum_n (-x)^n / (n+1)! with one multiply-add fewer.
// Above 0.25 the callers use the exponential e = exp(-x) directly (relative error
// of 1 - e below 5e-7 there).
template <class V>
__device__ __forceinline__ V u_series_v(V x) {
    V p = V(-0.0013885563239455223f);
    p = vfma(p, x, V(0.008350598625838757f));
    p = vfma(p, x, V(-0.04166680946946144f));
    p = vfma(p, x, V(0.16666632890701294f));
    p = vfma(p, x, V(-0.5f));
    return vfma(p, x, V(1.f));
}

// Per-system branch counts of one unit (added to the CTA counters for the
// real systems once the unit is done).
template <class V>
struct SysCounts {
    typename VTraits<V>::C inv, ecl, etau;
};

// The paper's resonance switch for the systems whose FP32 |D| is near 1e-5:
// decide |D| < 1e-5 in FP64, and (paper mode) replace the beam source terms
// by the literal G+- of Eq. B8 with D := 2 mu* = -2 mu.
__device__ __forceinline__ void resonance_fix(bool near, bool on, float w0, float g0, float mu, float imu,
                                              double mu_d, float A, float iq, float G0h, float omtr, float r,
                                              float t, float omm, float m, const KParams &kp, Counters &cn,
                                              float &bu, float &bd) {
    bool sw = false;
    if (near) {
        cn.fp64 += on ? 1u : 0u;
        const double D = resonance_D_fp64(w0, g0, mu_d, kp.improved, kp.e_clamp);
        if (fabs(D) < 1e-5) {
            cn.res += on ? 1u : 0u;
            sw = kp.resonance_paper != 0;
        }
    }
    if (sw) {
        const float c1 = 0.5f * iq;
        const float lead = -0.5f * A * imu;
        const float Gp = 0.5f * lead * (c1 - mu) + G0h;
        const float Gm = -0.5f * lead * (c1 + mu) - G0h;
        bu = -Gp * (omtr + r + t * omm) + r * Gm;     // Gp (t m - 1) + r Gm
        bd = Gm * (omm - omtr - r) + r * Gp * m;      // Gm (t - m) + r Gp m
    }
}
__device__ __forceinline__ void resonance_fix(M2 near, M2 on, V2 w0, V2 g0, float mu, float imu, double mu_d,
                                              V2 A, V2 iq, V2 G0h, V2 omtr, V2 r, V2 t, V2 omm, V2 m,
                                              const KParams &kp, Counters &cn, V2 &bu, V2 &bd) {
    resonance_fix(near.x, on.x, w0.v.x, g0.v.x, mu, imu, mu_d, A.v.x, iq.v.x, G0h.v.x, omtr.v.x, r.v.x, t.v.x,
                  omm.v.x, m.v.x, kp, cn, bu.v.x, bd.v.x);
    resonance_fix(near.y, on.y, w0.v.y, g0.v.y, mu, imu, mu_d, A.v.y, iq.v.y, G0h.v.y, omtr.v.y, r.v.y, t.v.y,
                  omm.v.y, m.v.y, kp, cn, bu.v.y, bd.v.y);
}

template <class V>
struct Layer32 {
    V T, R, Su, Sd, omtr, opr, mlay;
};

// One sub-layer's transmission t and reflection r (both sub-layers of a
// non-isothermal layer have the same), 1 - t - r, the sources of the upper
// (top -> centre) and lower (centre -> bottom) sub-layers in departure
// variables, beam included, and the beam's attenuation m across one
// sub-layer.  Isothermal layers use the upper fields only.
template <class V>
struct Sub32 {
    V t, r, omtr, suU, sdU, suL, sdL, m;
    V bu, bd;        // SPLIT: beam source coefficients per unit F_beam at the sub-layer top
};

// Products are grouped by hand: float multiplication is not reassociated by
// the compiler, and shared factors (1/h and 1/p from one reciprocal of h p,
// 2q, w0 g0, ...) are formed once per layer.  Multiply-adds are written as
// vfma so that the scalar and the paired forms round alike.
// SPLIT: the beam terms are left out of the sources and returned as bu, bd
// (the caller applies F_beam; Fb is not read).
template <bool ISO, class V, bool SPLIT = false>
__device__ __forceinline__ Sub32<V> sub32(V dt, V w0, V g0, V Bt, V Bc, V Bb, float mu, float imu,
                                          double mu_d, bool beam, V Fb, const KParams &kp, Counters &cn,
                                          SysCounts<V> &sc, typename VTraits<V>::M on) {
    using M = typename VTraits<V>::M;
    const M valid = (dt >= V(0.f)) & (w0 >= V(0.f)) & (w0 <= V(1.f)) & (vabs(g0) < V(1.f));
    vcount(sc.inv, !valid);
    // E of Eq. 19, switched off for w0 <= 0.1, clamped at 1
    const V wg = w0 * g0;
    // E - 1 in FP32 as nested fused multiply-adds; the clamp's hits are
    // decided on this value (the FP64 path and the reference count on the
    // same FP32 expression)
    V em1 = vfma(g0, vfma(V(-0.07465f), g0, V(-0.1582f)), vfma(w0, vfma(V(-0.05582f), w0, V(-0.1777f)), V(0.225f)));
    em1 = vfma(V(0.2351f), wg, em1);
    em1 = vsel((w0 > V(0.1f)) & (kp.improved != 0), em1, V(0.f));
    const M clamp = (em1 < V(0.f)) & (kp.e_clamp != 0);
    vcount(sc.ecl, clamp);
    em1 = vsel(clamp, V(0.f), em1);
    const V omw = V(1.f) - w0;
    const V ewm = em1 + omw;                      // E - w0
    const V q = (V(1.f) + em1) * (V(1.f) - wg);   // E (1 - w0 g0)
    const V iq = vrcp(q);
    const M cons = ewm == V(0.f);                 // E = w0 = 1: k = 0, Pi := pi
    const V k = vsel(cons, V(0.f), ewm * vrsqrt(ewm * q));
    // Pi and Pi - pi of Eq. B5, both times hs = 1 (isothermal) or 1/2
    // (non-isothermal, where they meet mean values (B1 + B2)/2)
    constexpr float hs = ISO ? 1.f : 0.5f;
    const V piw = V(hs * kPiF) * vrcp(ewm);
    const V Pi = vsel(cons, V(hs * kPiF), omw * piw);
    const V dPi = vsel(cons, V(0.f), -em1 * piw);  // hs (Pi - pi)
    const V opk = V(1.f) + k, omk = V(1.f) - k;
    const V dts = ISO ? dt : V(0.5f) * dt;

    const V q2 = q + q;
    const V q2d = q2 * dts;
    const V x = q2d * k;
    const V Tm = vexpn(x);
    const V u = vsel(vabs(x) < V(0.25f), u_series_v(x), (V(1.f) - Tm) * vrcp(x));
    const V qd = q2d * u;                         // (1 - T)/k
    // with h = (1 + k) qd + 2T and p = (1 + k) + (1 - k) T (the usual
    // denominators times 1 + k), one reciprocal of h p gives t, r, 1/h and 1/p
    const V h = vfma(opk, qd, Tm + Tm);
    const V p = vfma(omk, Tm, opk);
    const V ihp = vrcp(h * p);
    const V t = (V(4.f) * Tm) * ihp;
    const V Y = vfma(qd, Tm, qd);                 // (1 - T^2)/k = qd (1 + T)
    const V r = ((omk * opk) * Y) * ihp;          // (1 - k^2) Y / (h p)
    const V k2 = k * k;
    const V omtr = ((k2 + k2) * qd) * (h * ihp);  // 1 - t - r = 2 k^2 qd / p
    const V omr = omtr + t;                       // 1 - r

    V suU, sdU, suL = V(0.f), sdL = V(0.f);
    if (!ISO) {
        const M fb = dts < V(1e-4f);
        vcount(sc.etau, fb);
        // Gradient form  su = dPi ((1-r) B1 - t B2) + G (B2 - B1),
        //                sd = dPi ((1-r) B2 - t B1) - G (B2 - B1),
        // with G = Pi 2u/((1+k) h), rewritten about the mean B = (B1 + B2)/2 as
        //   su = dPi (1-r-t) B + G' (B2 - B1),  sd = dPi (1-r-t) B - G' (B2 - B1),
        //   G' = G - dPi (1-r+t)/2.
        // The e_tau fallback (isothermal at the mean B, Sec. 2.2.1, written in
        // departures from pi B1 and pi B2) is the same expression with
        // G' = pi (1-r+t)/2, so only G' is selected.
        // (Pi and dPi carry the factor 1/2 here)
        const V pig = (Pi * (V(4.f) * u)) * (p * ihp);           // Pi 2u / h
        const V opt = vfma(V(2.f), t, omtr);                    // 1 - r + t
        const V G = vsel(fb, V(0.5f * kPiF) * opt, vfma(-dPi, opt, pig));
        const V dom = dPi * omtr;
        const V aU = dom * (Bt + Bc), aL = dom * (Bc + Bb);
        const V gU = G * (Bc - Bt), gL = G * (Bb - Bc);
        suU = aU + gU;
        sdU = aU - gU;
        suL = aL + gL;
        sdL = aL - gL;
    } else {
        const V base = (dPi * Bc) * omtr;
        suU = vfma(V(kPiF), vfma(omr, Bc - Bt, -(t * (Bc - Bb))), base);
        sdU = vfma(V(kPiF), vfma(omr, Bc - Bb, -(t * (Bc - Bt))), base);
    }

    V m = V(1.f), bu_o = V(0.f), bd_o = V(0.f);
    if (beam) {
        const V dl = dts * V(imu);
        m = vexpn(dl);
        const V omm = vsel(dl < V(0.25f), dl * u_series_v(dl), V(1.f) - m);   // 1 - m
        const V q2k = q2 * k;
        const V rho = V(mu) * q2k;
        const V Ah = w0 * vfma(g0, V(0.5f * kp.inv_eps2), q);   // A/2
        const V G0h = (wg * V(0.25f * kp.inv_eps2)) * iq;       // G0/2 of Eq. B8
        const V omt = omtr + r;                                  // 1 - t
        const V tm1r = -vfma(t, omm, omt + r);                  // (t m - 1) - r
        const V rmtm = vfma(r, m, omt - omm);                   // r m - (t - m)
        // stable form: the 1/D of G+- divided out (see the block comment)
        const V omrho = V(1.f) - rho;
        const V z = omrho * dl;
        const V lam_s = (m * dl) * u_series_v(-z);
        const V lam_d = (Tm - m) * vrcp(omrho);
        const V Lam = vsel(vabs(z) < V(0.25f), lam_s, lam_d);
        const V SA2 = (Ah * ihp) * (iq * vrcp(V(1.f) + rho));   // 2 SA
        const V tq = V(mu) * q2;
        const V TL = Tm * Lam;
        V bu = vfma(SA2, vfma(opk, Y, TL * vfma(tq, V(-2.f), V(2.f))), G0h * tm1r);
        const V cl = vfma(Y, vfma(tq, k2, V(1.f)), (V(1.f) + tq) * vfma(Tm, Tm, V(1.f)));
        V bd = vfma(SA2, vfma(Lam, cl, -((Tm * omk) * Y)), G0h * rmtm);
        // resonance test of Eq. 11 (rare): the FP64 decision, and the paper's
        // switch to D := 2 mu* when |D| < 1e-5, run only if a lane needs them
        const V D32 = vfma(rho, rho, V(-1.f));
        const M near = vabs(D32) < V(2e-5f);
        if (__any_sync(0xffffffffu, vany(near))) {
            resonance_fix(near, on, w0, g0, mu, imu, mu_d, Ah + Ah, iq, G0h, omtr, r, t, omm, m, kp, cn, bu, bd);
        }
        if (SPLIT) {
            bu_o = bu;
            bd_o = bd;
        } else {
            suU = vfma(Fb, bu, suU);
            sdU = vfma(Fb, bd, sdU);
            if (!ISO) {
                const V Fc = Fb * m;
                suL = vfma(Fc, bu, suL);
                sdL = vfma(Fc, bd, sdL);
            }
        }
    }

    Sub32<V> o;
    o.t = t;
    o.r = r;
    o.omtr = omtr;
    o.suU = suU;
    o.sdU = sdU;
    o.suL = suL;
    o.sdL = sdL;
    o.m = m;
    o.bu = bu_o;
    o.bd = bd_o;
    return o;
}

// The layer as one unit for the Thomas elimination: a non-isothermal
// layer's two sub-layers merged (adding their transmissions, reflections
// and sources).
template <bool ISO, class V>
__device__ __forceinline__ Layer32<V> layer32(V dt, V w0, V g0, V Bt, V Bc, V Bb, float mu, float imu,
                                              double mu_d, bool beam, V Fb, const KParams &kp, Counters &cn,
                                              SysCounts<V> &sc, typename VTraits<V>::M on) {
    const Sub32<V> s = sub32<ISO, V>(dt, w0, g0, Bt, Bc, Bb, mu, imu, mu_d, beam, Fb, kp, cn, sc, on);
    const V t = s.t, r = s.r, omtr = s.omtr;
    const V omr = omtr + t;                       // 1 - r
    Layer32<V> o;
    if (ISO) {
        o.T = t;
        o.R = r;
        o.Su = s.suU;
        o.Sd = s.sdU;
        o.omtr = omtr;
        o.opr = vfma(V(2.f), t, omtr);
        o.mlay = s.m;
    } else {
        // merge upper (top -> centre) and lower (centre -> bottom) sub-layers
        const V opr1 = V(1.f) + r;
        const V Dr = vrcp(omr * opr1);            // 1 / (1 - r^2)
        const V tD = t * Dr;
        o.T = t * tD;
        o.R = vfma(r, o.T, r);
        o.Su = vfma(tD, vfma(r, s.sdU, s.suL), s.suU);
        o.Sd = vfma(tD, vfma(r, s.suL, s.sdU), s.sdL);
        o.omtr = (omtr * vfma(V(2.f), t, omtr)) * (opr1 * Dr);   // (1-r-t)(1-r+t)/(1-r)
        o.opr = vfma(omr, o.T, omr);
        o.mlay = s.m * s.m;
    }
    return o;
}

// ---------------------------------------------------------------------
// Shared-memory layout (both kernels):
//   acc   double [2 (Lmax+1)]                  column sums (F_up, F_net)
//   wpart R      [2 (Lmax+1) nwarps]            warp partial sums
//   sB    R      [staged]                       Planck at levels (2i iface, 2i+1 centre),
//                                               [(2 L + 1) nbc] of the current chunk
//   sFs   R      [nb_chunk]                     stellar flux per bin
//   sFB   R      [nb_chunk]                     F_BOA per bin
//   stoa  R      [block]                        weighted TOA F_up per system
// ---------------------------------------------------------------------
template <typename R>
__host__ __device__ inline size_t smem_bytes_t(int block, int Lmax, int nb_chunk, int staged) {
    const int nw = block / 32;
    size_t b = sizeof(double) * 2 * (size_t)(Lmax + 1);
    b += sizeof(R) * 2 * (size_t)(Lmax + 1) * nw;
    b += sizeof(R) * (size_t)staged;
    b += sizeof(R) * 2 * (size_t)nb_chunk;
    b += sizeof(R) * (size_t)block;
    return b;
}

// The shared-memory ring of the back-substitution: with `depth` levels of
// elimination scratch in flight, depth + 1 slots of one float4 per system,
// the spare slot being the one read a level earlier.
__host__ __device__ constexpr int back_ring_floats(int ns, int depth) { return (depth + 1) * ns * 32 * 4; }
// Inline B: B at the interfaces rides along in a second ring ([slot][32] of
// the lane's ns values).
__host__ __device__ constexpr int back_ringB_floats(int ns, int inline_b, int depth) {
    return inline_b ? (depth + 1) * ns * 32 : 0;
}

int fp32_warp_floats(int Lmax, int nbw, int direct, int ns, int group_shift, int inline_b, int depth, int staged) {
    // back-substitution ring + Planck [staged] (staged mode: the largest
    // (2 L + 1) x bins-per-unit of the batch's columns), or
    // the column's 2 Lmax + 1 level temperatures in FP64 (inline B), or
    // nothing (direct) + F* [nbw] + F_BOA [nbw] + transpose [G][2][33],
    // G = 2^group_shift interfaces per transposed sum (at least 2 NS 32
    // floats for the TOA sum)
    const int tr = std::max((1 << group_shift) * 2 * 33, 64 * ns);
    const int st = !direct ? staged : inline_b ? 2 * (2 * Lmax + 1) : 0;
    int n = back_ring_floats(ns, depth) + back_ringB_floats(ns, inline_b, depth) + st + 2 * nbw + tr;
    return (n + 3) & ~3;
}
size_t fp32_smem_bytes(int block, int Lmax, int nbw, int direct, int ns, int group_shift, int inline_b, int depth,
                       int staged) {
    return sizeof(float) * (size_t)(block / 32) *
           fp32_warp_floats(Lmax, nbw, direct, ns, group_shift, inline_b, depth, staged);
}
size_t fp64_smem_bytes(int block, int Lmax, int nb_chunk, int staged) {
    return smem_bytes_t<double>(block, Lmax, nb_chunk, staged);
}
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
    __device__ Smem(unsigned char *raw, int Lmax, int nb_chunk, int staged, int nwarps) {
        acc = reinterpret_cast<double *>(raw);
        wpart = reinterpret_cast<R *>(acc + 2 * (Lmax + 1));
        sB = wpart + 2 * (Lmax + 1) * nwarps;
        sFs = sB + staged;
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
    ci.mu = ck_ld(kp, kp.mu_star, kp.ext.mu, kp.mu_idx[ci.c]);
    return true;
}

// Planck at the 2L+1 levels of the column for bins [b_lo, b_lo + nbc).
template <typename R>
__device__ __forceinline__ void stage_planck(const KParams &kp, const ColInfo &ci, int b_lo, int nbc,
                                             Smem<R> &sm) {
    const int nlev = 2 * ci.L + 1;
    const double dwn = (kp.wn_max - kp.wn_min) / ci.NB;
    auto edge = [&](int e) { return kp.edges ? kp.edges[e] : kp.wn_min + e * dwn; };
    static_assert(sizeof(R) == 8, "the FP32 form stages B in fp32_units");
    for (int i = threadIdx.x; i < nlev * nbc; i += blockDim.x) {
        const int lev = i / nbc, bb = i - lev * nbc, b = b_lo + bb;
        const double T = (lev & 1) ? ck_ld(kp, kp.T_center, kp.ext.center, ci.tc_in + (lev >> 1))
                                   : ck_ld(kp, kp.T_iface, kp.ext.iface, ci.if_in + (lev >> 1));
        sm.sB[i] = planck_bin_d(T, edge(b), edge(b + 1));
    }
    for (int bb = threadIdx.x; bb < nbc; bb += blockDim.x) {
        const int b = b_lo + bb;
        sm.sFs[bb] = (R)ck_ld(kp, kp.F_star, kp.ext.fstar, ci.fs_in + b);
        sm.sFB[bb] = kPi * planck_bin_d(kp.T_int, edge(b), edge(b + 1));
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

// The warp partials are added to the column sums one at a time in warp
// (system) order, so the order of the additions does not depend on the CTA
// size: a column gives the same bits in any batch and launch shape.
template <typename R>
__device__ __forceinline__ void fold_warps(int L, int nwarps, Smem<R> &sm) {
    for (int i = threadIdx.x; i <= L; i += blockDim.x) {
        double sa = sm.acc[2 * i], sn = sm.acc[2 * i + 1];
        for (int w = 0; w < nwarps; ++w) {
            sa += (double)sm.wpart[2 * (i * nwarps + w)];
            sn += (double)sm.wpart[2 * (i * nwarps + w) + 1];
        }
        sm.acc[2 * i] = sa;
        sm.acc[2 * i + 1] = sn;
    }
}

__device__ __forceinline__ void write_column(const KParams &kp, const ColInfo &ci, const double *acc) {
    for (int i = threadIdx.x; i <= ci.L; i += blockDim.x) {
        const double up = acc[2 * i], net = acc[2 * i + 1];
        ck_st(kp, kp.F_up, kp.ext.out_if, ci.if0 + i, up);
        ck_st(kp, kp.F_net, kp.ext.out_if, ci.if0 + i, net);
        ck_st(kp, kp.F_dn, kp.ext.out_if, ci.if0 + i, up - net);
    }
    const double gc = kp.grav / kp.cp;
    for (int l = threadIdx.x; l < ci.L; l += blockDim.x) {
        const double dF = acc[2 * (l + 1) + 1] - acc[2 * l + 1];
        const double dp = ck_ld(kp, kp.p_iface, kp.ext.iface, ci.if_in + l + 1) -
                          ck_ld(kp, kp.p_iface, kp.ext.iface, ci.if_in + l);
        ck_st(kp, kp.Q, kp.ext.out_lay, ci.lay0 + l, gc * dF / dp);
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
// transpose (16 interfaces at a time), stored as the unit's partials;
// fp32_finalize then sums each column's unit partials in unit order (FP64)
// and writes fluxes, net flux and heating.
// ---------------------------------------------------------------------
// One (column, level) per warp: lane e evaluates the Planck integral at bin
// edge e (whichever of S(x) or P(x) that edge needs), and bin b takes edges b
// and b+1 from its lane and the next (shuffle).  31 bins per pass.
// x^3 / (e^x - 1), the Planck integrand in x = h c nu / (k T), as num/den so
// that two quadrature nodes share one reciprocal:
//   x < 1/2:  x^2 / q,  q = (e^x - 1)/x as a degree-4 polynomial fitted for
//             the least maximum relative error on [0, 1/2], constant term 1
//             (csrc/fit_series.py; 1.0e-7 relative, 1.6e-7 evaluated in FP32,
//             against 2.1e-7 for the Taylor sum to x^6 / 7! with two more
//             multiply-adds), so that small x keeps its digits;
//   x >= 1/2: x^3 m / (1 - m),  m = e^-x  (1 - m >= 0.39: no cancellation,
//             and no overflow however large x is).
// Written over V (one value, or two on the paired instructions) with every
// operation rounded on its own, so that the pre-kernel's table, the solve
// kernel's own evaluation (RT_STAGE_INLINE) and one or two systems per lane
// all give the same bits.
template <class V>
struct PlanckND {
    V num, den;
};
template <class V>
__device__ __forceinline__ PlanckND<V> planck_nd(V x) {
    V q = V(0.010216917842626572f);
    q = vfma(q, x, V(0.040856339037418365f));
    q = vfma(q, x, V(0.1668008267879486f));
    q = vfma(q, x, V(0.4999932050704956f));
    q = vfma(q, x, V(1.f));
    const V xx = x * x;
    const V m = vexpn(x);
    const auto small = x < V(0.5f);
    PlanckND<V> r;
    r.num = vsel(small, xx, (xx * x) * m);
    r.den = vsel(small, q, V(1.f) - m);
    return r;
}
// f(xa) + f(xb) with one reciprocal
template <class V>
__device__ __forceinline__ V planck_pair(V xa, V xb) {
    const PlanckND<V> a = planck_nd(xa), b = planck_nd(xb);
    return vfma(a.num, b.den, b.num * a.den) * vrcp(a.den * b.den);
}

// Bins narrower than this in x = h c nu / (k T) are integrated by quadrature.
constexpr float kNarrowBin = 0.5f;
// Narrow bins below this width, and below 2% of their centre x, take
// 2-point Gauss-Legendre (nodes -+1/sqrt(3), weights 1); wider ones 4 points.
constexpr float kTwoPointBin = 0.1f;
constexpr float kGL2x = 0.57735026918962576f;
// 4-point Gauss-Legendre on [-1, 1]: outer and inner nodes with their weights.
constexpr float kGL4xo = 0.86113631159405258f, kGL4xi = 0.33998104358485626f;
constexpr float kGL4wo = 0.34785484513745386f, kGL4wi = 0.65214515486254614f;

// Integral of x^3/(e^x - 1) over a narrow bin [x, x + 2 hh] (e.g. R = 500)
// by Gauss-Legendre: the edge difference would lose the digits that the
// edges' own FP32 rounding carries, so the half width hh comes from the
// bin width formed in FP64 before rounding.  2 points are below 2e-8
// relative for the widths that take them.
template <class V>
__device__ __forceinline__ V planck_two_point(V x, V hh) {
    const V xm = x + hh;
    return hh * planck_pair(vfma(hh, V(-kGL2x), xm), vfma(hh, V(kGL2x), xm));
}
__device__ __forceinline__ bool planck_takes_two_points(float x, float hh) {
    return hh < 0.5f * kTwoPointBin && hh < __fmul_rn(0.01f, __fadd_rn(x, hh));
}
__device__ __forceinline__ float planck_narrow_f(float x, float hh) {
    if (planck_takes_two_points(x, hh)) return planck_two_point(x, hh);
    const float xm = __fadd_rn(x, hh);
    const float outer = planck_pair(fmaf(hh, -kGL4xo, xm), fmaf(hh, kGL4xo, xm));
    const float inner = planck_pair(fmaf(hh, -kGL4xi, xm), fmaf(hh, kGL4xi, xm));
    return __fmul_rn(hh, fmaf(kGL4wo, outer, __fmul_rn(kGL4wi, inner)));
}

// One edge's series value: S(x) below x = 2, P(x) above.
__device__ __forceinline__ float planck_edge_f(float x) { return (x < 2.f) ? planck_lower_f(x) : planck_upper_f(x); }

// Integral of x^3/(e^x - 1) over a wide bin [x0, x1] from the edge series
// v0, v1 (planck_edge_f), in the difference without cancellation.
__device__ __forceinline__ float planck_wide_f(float x0, float x1, float v0, float v1) {
    if (x0 >= 2.f) return __fsub_rn(v0, v1);
    if (x1 < 2.f) return __fsub_rn(v1, v0);
    return __fsub_rn(__fsub_rn((float)kPi4Over15, v0), v1);
}

// Per-level factors of the bin-integrated Planck function B = K T^4 d(x):
// a = c2 / T (x = a nu) and K T^4 (times `scale`).
struct PlanckLevel {
    float a, pref;
};
__device__ __forceinline__ PlanckLevel planck_level(float T, float scale) {
    PlanckLevel lv;
    lv.a = (T > 0.f) ? __fmul_rn((float)(kC2 * 100.0), frcp(T)) : 0.f;
    const float T2 = __fmul_rn(T, T);
    lv.pref = (T > 0.f) ? __fmul_rn(__fmul_rn((float)kPlanckK, __fmul_rn(T2, T2)), scale) : 0.f;
    return lv;
}

// B of one bin [wn0, wn1] (cm^-1, FP32 edges; dnu its width formed in FP64).
__device__ __forceinline__ float planck_bin32(PlanckLevel lv, float wn0, float wn1, float dnu) {
    const float x0 = __fmul_rn(lv.a, wn0), x1 = __fmul_rn(lv.a, wn1);
    float d;
    if (__fsub_rn(x1, x0) < kNarrowBin)
        d = planck_narrow_f(x0, __fmul_rn(0.5f, __fmul_rn(lv.a, dnu)));
    else
        d = planck_wide_f(x0, x1, planck_edge_f(x0), planck_edge_f(x1));
    return __fmul_rn(lv.pref, d);
}

// B at NQ levels for the warp's chunk of 31 bins [b0, b0 + 31) (the
// pre-kernel's inner loop): lane e holds edge b0 + e at x = a wn (x1: the
// next edge, from lane e + 1); a wide bin takes the difference of its
// edges' series values, the lower edge's from its own lane, the upper's
// from the next lane; a narrow bin its own quadrature.  One vote serves the
// group and the series and the wide-bin difference are formed by selects,
// so that the NQ evaluation chains are independent and can overlap.  The
// values equal planck_bin32's for the same bin and level.
template <int NQ>
__device__ __forceinline__ void planck_chunk_levels(const float (&T)[NQ], const float (&scale)[NQ],
                                                    const float (&wn)[NQ], const float (&dnu_b)[NQ],
                                                    const bool (&inb)[NQ], float (&out)[NQ]) {
    PlanckLevel lv[NQ];
    float x[NQ], x1[NQ], v[NQ], v1[NQ], d[NQ];
    bool nar[NQ];
    bool alln = true, anyn = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        lv[q] = planck_level(T[q], scale[q]);
        x[q] = __fmul_rn(lv[q].a, wn[q]);
        x1[q] = __shfl_down_sync(0xffffffffu, x[q], 1);
        nar[q] = !inb[q] || (__fsub_rn(x1[q], x[q]) < kNarrowBin);
        alln = alln && nar[q];
        anyn = anyn || (inb[q] && nar[q]);
    }
    // the edge series only when some bin of this chunk is wide
    if (!__all_sync(0xffffffffu, alln)) {
        // two levels per paired evaluation (the same bits as one at a time)
#pragma unroll
        for (int q = 0; q + 1 < NQ; q += 2) {
            const V2 xq(x[q], x[q + 1]);
            const V2 lo = planck_lower_v(xq), up = planck_upper_v(xq);
            v[q] = (x[q] < 2.f) ? lo.v.x : up.v.x;
            v[q + 1] = (x[q + 1] < 2.f) ? lo.v.y : up.v.y;
        }
        if constexpr (NQ & 1) {
            const float lo = planck_lower_f(x[NQ - 1]), up = planck_upper_f(x[NQ - 1]);
            v[NQ - 1] = (x[NQ - 1] < 2.f) ? lo : up;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v1[q] = __shfl_down_sync(0xffffffffu, v[q], 1);
        const float dh = __fsub_rn(v[q], v1[q]), dl = __fsub_rn(v1[q], v[q]);
        const float dm = __fsub_rn(__fsub_rn((float)kPi4Over15, v[q]), v1[q]);
        d[q] = (x[q] >= 2.f) ? dh : ((x1[q] < 2.f) ? dl : dm);     // planck_wide_f
    }
    if (__any_sync(0xffffffffu, anyn)) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (nar[q]) d[q] = planck_narrow_f(x[q], __fmul_rn(0.5f, __fmul_rn(lv[q].a, dnu_b[q])));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = __fmul_rn(lv[q].pref, d[q]);
}

// ---------------------------------------------------------------------
// Input front end (Sec. 2.1.3): optics from the column state and a premixed
// k-table.  Per layer (kt_layer): the bracketing grid cell of (T_center,
// log10 sqrt(p_top p_bot)), clamped, its bilinear weights and the column
// mass dp / g.  Per system (kt_mix): log10 kappa interpolated bilinearly,
// kappa = 10^x, extinction per unit mass E = kappa + s_b + a_b (s_b, a_b:
// the bin's scattering and cloud absorption per unit mass), dtau = E dp / g,
// w0 = s_b / E (capped at 1) and the bin's g0.  Every operation is an explicitly rounded
// intrinsic, so that the fused solve and the standalone optics kernel
// produce the same bits.  The cell search compares in FP64 against the
// FP64 grids; the weights, log10 p and dp / g are formed in FP32 (each a few
// ulp: below 1e-5 relative in kappa), which keeps the FP64 pipe, 1/64 of the
// FP32 rate on this part, out of the pre-kernel's critical path.
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
    w = __fdiv_rn(__double2float_rn(__dsub_rn(v, grid[lo])), __double2float_rn(__dsub_rn(grid[lo + 1], grid[lo])));
}

// gT, gP: the table's T and log10 p grids (in shared memory where staged)
__device__ __forceinline__ float4 kt_layer(const KParams &kp, const double *gT, const double *gP, double T,
                                           double p_top, double p_bot, int S) {
    int iT, iP;
    float wT, wP;
    kt_bracket(gT, kp.kt_nT, T, iT, wT);
    // log10 sqrt(p_top p_bot), from the FP64 product
    const float lp = __fmul_rn(0.5f, log10f(__double2float_rn(__dmul_rn(p_top, p_bot))));
    kt_bracket(gP, kp.kt_nP, (double)lp, iP, wP);
    const int off = (iT * kp.kt_nP + iP) * S * 2;   // float offset of the (iT, iT + 1) pairs
    return make_float4(__int_as_float(off), wT, wP,
                       __fdiv_rn(__double2float_rn(__dsub_rn(p_bot, p_top)), __double2float_rn(kp.grav)));
}

struct Optics {
    float dt, w0, g0;
};

constexpr float kLog2Of10 = 3.32192809488736234787f;

// lo = (k00, k10) and hi = (k01, k11): the corners at p_i and p_i+1 for T_i and
// T_i+1, so the two interpolations along log p run as one paired operation
// (each component rounded as the scalar form would round it).
__device__ __forceinline__ Optics kt_mix(float2 lo, float2 hi, float4 l4, float4 bq) {
    const float2 d = __ffma2_rn(lo, make_float2(-1.f, -1.f), hi);                 // k01 - k00, k11 - k10
    const float2 a = __ffma2_rn(make_float2(l4.z, l4.z), d, lo);                  // along log p at T_i, T_i+1
    const float x = __fmaf_rn(l4.y, __fsub_rn(a.y, a.x), a.x);                    // log10 kappa
    const float kappa = fex2(__fmul_rn(x, kLog2Of10));
    const float ext = __fadd_rn(__fadd_rn(kappa, bq.x), bq.y);
    Optics o;
    o.dt = __fmul_rn(ext, l4.w);
    // w0 = s / E by the approximate reciprocal (a few ulp), capped at 1 so
    // that s = E (nothing absorbs) stays a valid albedo
    o.w0 = ext > 0.f ? fminf(__fmul_rn(bq.x, frcp(ext)), 1.f) : 0.f;
    o.g0 = bq.z;
    return o;
}

// The four table corners of system s for a layer whose cell starts at l4.x:
// the table keeps the two T-neighbours of a (T, p) node side by side, so the
// corners are one 8-byte load at p_i and one at p_i+1 (8-byte aligned: the
// offsets are even and the table is a fresh allocation).
struct Corners {
    float2 lo, hi;                                // (k00, k10), (k01, k11)
};

__device__ __forceinline__ Corners kt_corners(const KParams &kp, float4 l4, int S, int s) {
    const float2 *t = reinterpret_cast<const float2 *>(kp.kt_lk + __float_as_int(l4.x)) + s;
    Corners c;
    c.lo = __ldg(t);
    c.hi = __ldg(t + S);
    return c;
}

// One CTA per column (grid-stride).  Warp tasks are (chunk of 31 bins, run
// of levels): the chunk's edges are loaded once and the levels' B computed
// from the shared temperatures; the runs are short enough that every warp
// has work when a column has few bins.  Level 2L+1 stands for T_int (F_BOA =
// pi B(T_int), Eq. 10).
__global__ void __launch_bounds__(256, 4) fp32_prep(KParams kp) {
    extern __shared__ float sT[];                 // [2 Lmax + 2] temperatures of one column, then T_int
    double *sG = (double *)(sT + 2 * kp.Lmax + 2);  // k-table T and log10 p grids (binary searches)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (kp.kt_lk)
        for (int i = threadIdx.x; i < kp.kt_nT + kp.kt_nP; i += blockDim.x)
            sG[i] = i < kp.kt_nT ? kp.kt_T[i] : kp.kt_lp[i - kp.kt_nT];   // read after the loop's first barrier
    for (int c = blockIdx.x; c < kp.n_cols; c += gridDim.x) {
        const int L = kp.n_layers[c], NB = kp.n_bins[c];
        const long long tc0 = kp.tc_off[c], ifi = kp.if_off[c], b0 = kp.bin_off[c], fsi = kp.fs_off[c];
        float *B = kp.planck32 + kp.planck_off[c];
        const float dwn = (float)((kp.wn_max - kp.wn_min) / NB);
        const float wmin = (float)kp.wn_min;
        const int nlev = 2 * L + 1;
        __syncthreads();                          // previous column done with sT
        for (int lev = threadIdx.x; lev <= nlev; lev += blockDim.x)
            sT[lev] = lev == nlev ? (float)kp.T_int
                                  : (float)((lev & 1) ? ck_ld(kp, kp.T_center, kp.ext.center, tc0 + (lev >> 1))
                                                      : ck_ld(kp, kp.T_iface, kp.ext.iface, ifi + (lev >> 1)));
        for (int b = threadIdx.x; b < NB; b += blockDim.x)
            ck_st(kp, kp.fs32, kp.ext.bins, b0 + b, (float)ck_ld(kp, kp.F_star, kp.ext.fstar, fsi + b));
        __syncthreads();
        if (warp == 0) {
            // the coldest level (largest h c / k T) bounds every level's bin
            // widths in x, which lets the solve kernel's inline B skip the
            // per-level narrow-bin tests; 0 when some level is not in (0, 1e20)
            float tmin = 3.0e38f;
            bool ok = true;
            for (int lev = lane; lev < nlev; lev += 32) {
                const float T = sT[lev];
                ok = ok && T > 0.f && T < 1e20f;
                tmin = fminf(tmin, T);
            }
            ok = __all_sync(0xffffffffu, ok);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
            if (lane == 0) {
                const double mu = ck_ld(kp, kp.mu_star, kp.ext.mu, kp.mu_idx[c]);
                if (RT_IN(kp.colf + c, kp.colf, kp.ext.cols)) kp.colf[c] = make_float4((float)mu, mu > 0.0 ? (float)(1.0 / mu) : 0.f, mu > 0.0 ? 1.f : 0.f,
                                         ok ? tmin : 0.f);
            }
        }
        // the layers' k-table cells first: their loads and FP64 compares
        // then overlap the Planck tasks of the other warps
        if (kp.kt_lk)
            for (int l = threadIdx.x; l < L; l += blockDim.x)
                ck_st(kp, kp.kt_lay, kp.ext.out_lay, kp.lay_off[c] + l,
                      kt_layer(kp, sG, sG + kp.kt_nT, ck_ld(kp, kp.T_center, kp.ext.center, tc0 + l),
                               ck_ld(kp, kp.p_iface, kp.ext.iface, ifi + l),
                               ck_ld(kp, kp.p_iface, kp.ext.iface, ifi + l + 1), NB * kp.n_g));
        const int nchunk = (NB + 30) / 31;
        // levels [lev0, nlev]: the 2L+1 levels, then T_int (T_int alone when
        // the solve kernel evaluates B itself)
        const int lev0 = kp.inline_b ? nlev : 0;
        const int nl = nlev + 1 - lev0;
        int run = (int)(((long long)nl * nchunk + nw - 1) / nw);
        run = run < nl ? run : nl;
        const int nrun = (nl + run - 1) / run;
        if (nl == 1) {
            // T_int alone (inline B): four chunks per pass as independent chains
            for (int t0 = 4 * warp; t0 < nchunk; t0 += 4 * nw) {
                float Tq[4], sq[4], wq[4], dq[4], vq[4];
                bool iq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = (t0 + q) * 31 + lane;
                    iq[q] = t0 + q < nchunk && lane < 31 && e < NB;
                    wq[q] = kp.edges32 ? __ldg(kp.edges32 + min(e, NB)) : fmaf((float)e, dwn, wmin);
                    dq[q] = kp.edges32 ? __ldg(kp.dnu32 + min(e, NB - 1)) : dwn;
                    Tq[q] = sT[nlev];
                    sq[q] = kPiF;
                }
                planck_chunk_levels<4>(Tq, sq, wq, dq, iq, vq);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (iq[q]) ck_st(kp, kp.fboa32, kp.ext.bins, b0 + (t0 + q) * 31 + lane, vq[q]);
            }
        } else
        for (int task = warp; task < nchunk * nrun; task += nw) {
            const int ch = task % nchunk, r0 = lev0 + (task / nchunk) * run;
            const int e = ch * 31 + lane, bin = e;
            const bool inb = lane < 31 && bin < NB;
            const float wn = kp.edges32 ? __ldg(kp.edges32 + min(e, NB)) : fmaf((float)e, dwn, wmin);
            const float dnu_b = kp.edges32 ? __ldg(kp.dnu32 + min(bin, NB - 1)) : dwn;
            const int r1 = min(r0 + run, nlev + 1);
            // four levels per pass (independent evaluation chains), then one at a time
            auto store = [&](int lq, float v) {
                if (inb) {
                    if (lq == nlev) ck_st(kp, kp.fboa32, kp.ext.bins, b0 + bin, v);
                    else if (RT_IN(B + (long long)lq * NB + bin, kp.planck32, kp.ext.planck)) B[(long long)lq * NB + bin] = v;
                }
            };
            int lev = r0;
            for (; lev + 4 <= r1; lev += 4) {
                float Tq[4], sq[4], vq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    Tq[q] = sT[lev + q];
                    sq[q] = lev + q == nlev ? kPiF : 1.f;
                }
                const float wq[4] = {wn, wn, wn, wn}, dq[4] = {dnu_b, dnu_b, dnu_b, dnu_b};
                const bool iq[4] = {inb, inb, inb, inb};
                planck_chunk_levels<4>(Tq, sq, wq, dq, iq, vq);
#pragma unroll
                for (int q = 0; q < 4; ++q) store(lev + q, vq[q]);
            }
            for (; lev < r1; ++lev) {
                float Tq[1] = {sT[lev]}, sq[1] = {lev == nlev ? kPiF : 1.f}, vq[1];
                const float wq[1] = {wn}, dq[1] = {dnu_b};
                const bool iq[1] = {inb};
                planck_chunk_levels<1>(Tq, sq, wq, dq, iq, vq);
                store(lev, vq[0]);
            }
        }
    }
}

// A kernel launched with programmatic stream serialization may start while
// the previous kernel on its stream finishes; this waits until that kernel
// has completed and its memory writes are visible (a no-op for a kernel
// launched without the attribute).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ void finalize_column(const KParams &kp, int c, int lane) {
    const int L = kp.n_layers[c];
    const int nu = kp.col_units[c];
    const long long if0 = kp.lay_off[c] + c;
    const float *part = kp.partial + kp.part_off[c];
    const int stride = 2 * (L + 1);
    // Unit partials, read through L2 (other SMs wrote them), are summed in
    // unit order as unevaluated FP32 pairs hi + lo: Knuth's TwoSum gives each
    // addition's rounding error exactly, so hi + lo, formed once in FP64,
    // carries the sum to about eps_f^2 of the summands' magnitudes (an FP64
    // accumulation would run on B300's FP64 units, a small fraction of the
    // FP32 rate, once per unit and interface).
    auto acc = [](float &hi, float &lo, float x) {
        const float s = __fadd_rn(hi, x);
        const float bx = __fadd_rn(s, -hi);
        const float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bx)), __fadd_rn(x, -bx));
        hi = s;
        lo = __fadd_rn(lo, e);
    };
    for (int i = lane; i <= L; i += 32) {
        float uh = 0.f, ul = 0.f, nh = 0.f, nl = 0.f;
        // eight units' loads in flight, then their sums in unit order (a
        // zero past the last unit leaves hi and lo as they are)
        for (int u0 = 0; u0 < nu; u0 += 8) {
            float2 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float *pp = part + (long long)(u0 + k) * stride + 2 * i;   // (w F_up, w F_net), 8-byte aligned
                v[k] = (u0 + k < nu && RT_IN(pp + 1, kp.partial, kp.ext.part))
                           ? __ldcg(reinterpret_cast<const float2 *>(pp)) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc(uh, ul, v[k].x);
                acc(nh, nl, v[k].y);
            }
        }
        const double up = (double)uh + (double)ul, net = (double)nh + (double)nl;
        ck_st(kp, kp.F_up, kp.ext.out_if, if0 + i, up);
        ck_st(kp, kp.F_net, kp.ext.out_if, if0 + i, net);
        ck_st(kp, kp.F_dn, kp.ext.out_if, if0 + i, up - net);
    }
    __syncwarp();        // (orders the warp's F_net stores before the loads below)
    const float gc = (float)(kp.grav / kp.cp);
    for (int l = lane; l < L; l += 32) {
        const double dF = ck_ld(kp, (const double *)kp.F_net, kp.ext.out_if, if0 + l + 1) -
                          ck_ld(kp, (const double *)kp.F_net, kp.ext.out_if, if0 + l);
        const float dp = (float)(ck_ld(kp, kp.p_iface, kp.ext.iface, kp.if_off[c] + l + 1) -
                                 ck_ld(kp, kp.p_iface, kp.ext.iface, kp.if_off[c] + l));
        ck_st(kp, kp.Q, kp.ext.out_lay, kp.lay_off[c] + l, (double)(gc * (float)dF * frcp(dp)));
    }
}

// The columns' outputs, launched after the unit kernel on the same stream (so
// every unit's partials are written): each warp takes columns in turn and sums
// their unit partials in unit order.  Forming them here rather than in the
// warp that finishes a column's last unit spares every unit a device-wide
// memory fence and a returning atomic.
__global__ void __launch_bounds__(128) fp32_finalize(KParams kp) {
    grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int c = w; c < kp.n_cols; c += nw) finalize_column(kp, c, lane);
}

// Where the solve kernel gets a system's B at the levels: staged per unit in
// the warp's shared memory from the pre-kernel's table, read straight from
// that table, or evaluated per system in the kernel (no table; the per-bin
// work is not shared when few g-points share a bin).
constexpr int kStageShared = 0, kStageDirect = 1, kStageInline = 2;

// Planck values of a lane's bin: staged in the warp's shared memory (level
// stride nbc) or, when few g-points share a bin (DIRECT), read straight from
// the pre-kernel's table (level stride NB) through the read-only path.
template <bool DIRECT>
__device__ __forceinline__ float ldB(const float *p) {
    if constexpr (DIRECT) return __ldg(p);
    else return *p;
}
// the same, with DIRECT reads checked against the table in bounds-check builds
template <bool DIRECT>
__device__ __forceinline__ float ldBk(const KParams &kp, const float *p) {
    if constexpr (DIRECT) return RT_IN(p, kp.planck32, kp.ext.planck) ? __ldg(p) : 0.f;
    else return *p;
}

// Invalidate the 128-byte L2 line at p (128-byte aligned) without writing it
// back.  `after` is a value loaded from that line: the compare that reads it
// makes the discard issue only once the load has returned.
__device__ __forceinline__ void discard_l2_after(const void *p, float after) {
    asm volatile(
        "{\n\t.reg .pred d;\n\tsetp.ne.f32 d, %1, %1;\n\tdiscard.global.L2 [%0], 128;\n\t}" ::"l"(p),
        "f"(after)
        : "memory");
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only): the
// copy needs no register while in flight.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}


// Elimination scratch of one interface: (P, Q, alpha', e) of one system in a
// float4; for a lane with two systems, (P, Q) of both and (alpha', e) of
// both in two float4 (component pairs stay in their register pairs).
__device__ __forceinline__ void scr_store(const KParams &kp, float4 *sp, long long, float P, float Q, float a,
                                          float e) {
    if (RT_IN(sp, kp.scr32, kp.ext.scr32)) __stcg(sp, make_float4(P, Q, a, e));
}
__device__ __forceinline__ void scr_store(const KParams &kp, float4 *sp, long long other, V2 P, V2 Q, V2 a, V2 e) {
    if (RT_IN(sp, kp.scr32, kp.ext.scr32)) __stcg(sp, make_float4(P.v.x, P.v.y, Q.v.x, Q.v.y));
    if (RT_IN(sp + other, kp.scr32, kp.ext.scr32)) __stcg(sp + other, make_float4(a.v.x, a.v.y, e.v.x, e.v.y));
}
__device__ __forceinline__ void scr_unpack(const float4 *n, float &P, float &Q, float &a, float &e) {
    P = n[0].x;
    Q = n[0].y;
    a = n[0].z;
    e = n[0].w;
}
__device__ __forceinline__ void scr_unpack(const float4 *n, V2 &P, V2 &Q, V2 &a, V2 &e) {
    P = V2(n[0].x, n[0].y);
    Q = V2(n[0].z, n[0].w);
    a = V2(n[1].x, n[1].y);
    e = V2(n[1].z, n[1].w);
}

// B at the interfaces kept for the back-substitution (RT_STAGE_INLINE):
// [interface][thread slot], the lane's systems side by side.
__device__ __forceinline__ void stB(float *p, float v) { __stcg(p, v); }
__device__ __forceinline__ void stB(V2 *p, V2 v) { __stcg((float2 *)p, v.v); }
__device__ __forceinline__ float ldB_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ V2 ldB_cg(const V2 *p) { return V2(__ldcg((const float2 *)p)); }

// Component access for per-system values (one system per lane: float; two:
// V2) and per-system loads.
__device__ __forceinline__ float &cmp(float &v, int) { return v; }
__device__ __forceinline__ float &cmp(V2 &v, int i) { return i ? v.v.y : v.v.x; }
__device__ __forceinline__ float cmp(const float &v, int) { return v; }
__device__ __forceinline__ float cmp(const V2 &v, int i) { return i ? v.v.y : v.v.x; }
__device__ __forceinline__ float hsum(float v) { return v; }
__device__ __forceinline__ float hsum(V2 v) { return v.v.x + v.v.y; }
__device__ __forceinline__ bool &cmpm(bool &m, int) { return m; }
__device__ __forceinline__ bool &cmpm(M2 &m, int i) { return i ? m.y : m.x; }

// One work unit: SPU = 32 NS consecutive systems of one column, starting at
// system s0 = ku SPG of the column (SPG: the kernel's unit stride).
template <bool ISO, int ST, bool KT, int NS, int SPG, int DEP>
__device__ __forceinline__ void fp32_unit(const KParams &kp, int unit, int lane, float4 *ring, float *ringB, float *sB,
                                          float *sFs, float *sFB,
                                          float *tb, long long slot, long long gthreads, long long sstride,
                                          Counters &cn) {
    using V = typename std::conditional<NS == 2, V2, float>::type;
    using M = typename VTraits<V>::M;
    constexpr bool DIRECT = ST != kStageShared;    // B not staged in shared memory
    constexpr bool INL = ST == kStageInline;       // B evaluated here, per system
    constexpr int SPU = 32 * NS;                   // systems in this unit
    const int NG = kp.n_g;
    const int c = kp.unit_col[unit];
    const int ku = kp.unit_k[unit];
    const int L = kp.n_layers[c], NB = kp.n_bins[c];
    const int S = NB * NG;
    const long long cube0 = kp.cube_off[c];
    const float4 cf = kp.colf[c];
    const float mu = cf.x, imu = cf.y;
    const double mu_d = kp.mu_star[kp.mu_idx[c]];   // only for the rare FP64 resonance test
    const bool beam = cf.z != 0.f;
    const int s0 = ku * SPG;
    const int b_lo = s0 / NG;
    const int nbc = min(NB - 1, (s0 + SPU - 1) / NG) - b_lo + 1;

    // stage B of the unit's bins at the 2L+1 levels, F* and F_BOA: every
    // copy issued at once (cp.async), landing while the lanes set up their
    // systems and the first layer's optics load
    {
        const float *Bg = kp.planck32 + kp.planck_off[c] + b_lo;
        const int nlev = 2 * L + 1;
        if constexpr (!DIRECT) {
            // [bin][level]: unit level stride.  With at most 32 bins, lane
            // (lev0, bb) takes bin bb at levels lev0, lev0 + per, ... (one
            // division per unit instead of one per element)
            if (nbc <= 32) {
                const int per = 32 / nbc, lev0 = lane / nbc, bb = lane - lev0 * nbc;
                if (lev0 < per) {
                    const float *pb = Bg + (long long)lev0 * NB + bb;
                    const long long step = (long long)per * NB;
                    float *dst = sB + bb * nlev;
                    for (int lev = lev0; lev < nlev; lev += per, pb += step) {
                        if (RT_IN(pb, kp.planck32, kp.ext.planck)) cp_async4(dst + lev, pb);
                        else dst[lev] = 0.f;
                    }
                }
            } else {
                for (int i = lane; i < nlev * nbc; i += 32) {
                    const int lev = i / nbc, bb = i - lev * nbc;
                    const float *pb = Bg + (long long)lev * NB + bb;
                    float *dst = sB + bb * nlev + lev;
                    if (RT_IN(pb, kp.planck32, kp.ext.planck)) cp_async4(dst, pb);
                    else *dst = 0.f;
                }
            }
        }
        if constexpr (INL) {
            // the column's temperatures at its 2L+1 levels (2i: interface i,
            // 2i + 1: centre of layer i), in FP64 as given
            double *sT = reinterpret_cast<double *>(sB);
            for (int lev = lane; lev < nlev; lev += 32) {
                const double *pT = (lev & 1) ? kp.T_center + kp.tc_off[c] + (lev >> 1) : kp.T_iface + kp.if_off[c] + (lev >> 1);
                if (RT_IN(pT, (lev & 1) ? kp.T_center : kp.T_iface, (lev & 1) ? kp.ext.center : kp.ext.iface))
                    cp_async8(sT + lev, pT);
                else sT[lev] = 0.0;
            }
        }
        for (int j = lane; j < nbc; j += 32) {
            const long long jb = kp.bin_off[c] + b_lo + j;
            if (RT_IN(kp.fs32 + jb, kp.fs32, kp.ext.bins)) cp_async4(sFs + j, kp.fs32 + jb);
            else sFs[j] = 0.f;
            if (RT_IN(kp.fboa32 + jb, kp.fboa32, kp.ext.bins)) cp_async4(sFB + j, kp.fboa32 + jb);
            else sFB[j] = 0.f;
        }
        cp_async_commit();
    }

    // component i of this lane is system s0 + 32 i + lane; padding
    // systems of a column's last unit repeat system s0 with zero weight,
    // so the loops below need no per-lane predicates
    M on;
    int sI[NS], bI[NS];
    V wg, Fb, Bt, Bc, Bb;
    const float *Bp[NS];
    const int bst = DIRECT ? NB : 1;           // level stride of Bp (a literal 1 when staged)
    // INL: the bins' edges and FP64-formed widths, and the level temperatures
    float wn0[NS], wn1[NS], dnu[NS];
    V wn0v, wn1v, dnuv;
    bool unit_narrow = false;                  // INL: the unit's bins take two points at every level
    const double *sTd = reinterpret_cast<const double *>(sB);   // INL: the level temperatures, staged
    auto B_at = [&](int lev, V &B) {           // B of the lane's systems at level lev
        const PlanckLevel lv = planck_level((float)sTd[lev], 1.f);
        // narrow bins that take two quadrature points (the R = 500 shape):
        // the lane's systems together on the paired instructions; any other
        // bin through the per-system rule (the same bits either way)
        const V a = V(lv.a);
        const V x0 = a * wn0v, hh = V(0.5f) * (a * dnuv), w = a * wn1v - x0;
        bool fast = unit_narrow;
        if (!fast) {
            fast = true;
#pragma unroll
            for (int i = 0; i < NS; ++i)
                fast = fast && cmp(w, i) < kNarrowBin && planck_takes_two_points(cmp(x0, i), cmp(hh, i));
            fast = __all_sync(0xffffffffu, fast);
        }
        if (fast) {
            B = V(lv.pref) * planck_two_point(x0, hh);
        } else {
#pragma unroll
            for (int i = 0; i < NS; ++i) cmp(B, i) = planck_bin32(lv, wn0[i], wn1[i], dnu[i]);
        }
    };
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const bool act = s0 + 32 * i + lane < S;
        cmpm(on, i) = act;
        sI[i] = act ? s0 + 32 * i + lane : s0;
        bI[i] = sI[i] / NG;
        cmp(wg, i) = act ? kp.g_w32[sI[i] - bI[i] * NG] : 0.f;
        Bp[i] = DIRECT ? kp.planck32 + kp.planck_off[c] + bI[i] : sB + (bI[i] - b_lo) * (2 * L + 1);
        if constexpr (INL) {
            if (kp.edges32) {
                wn0[i] = __ldg(kp.edges32 + bI[i]);
                wn1[i] = __ldg(kp.edges32 + bI[i] + 1);
                dnu[i] = __ldg(kp.dnu32 + bI[i]);
            } else {
                const float dwn = (float)((kp.wn_max - kp.wn_min) / NB), wmin = (float)kp.wn_min;
                wn0[i] = fmaf((float)bI[i], dwn, wmin);
                wn1[i] = fmaf((float)(bI[i] + 1), dwn, wmin);
                dnu[i] = dwn;
            }
        }
    }
    // optics: read from the cubes, or (KT) from the k-table corners of
    // the layer's grid cell, fetched one layer ahead
    V nd = V(0.f), nw = V(0.f), ng = V(0.f);
    const float *pd[NS], *pw[NS], *pg[NS];
    const float4 *klay = nullptr;
    float4 kl_next = make_float4(0.f, 0.f, 0.f, 0.f), kl_after = kl_next;
    float4 kb[NS];
    Corners kc[NS];
    if constexpr (KT) {
        klay = kp.kt_lay + kp.lay_off[c];
        kl_next = klay[0];
        kl_after = L > 1 ? klay[1] : kl_next;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            kb[i] = __ldg(kp.kt_bin + bI[i]);
            kc[i] = kt_corners(kp, kl_next, S, sI[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const long long e = cube0 + sI[i];
            pd[i] = kp.dtau + e;
            pw[i] = kp.w0 + e;
            pg[i] = kp.g0 + e;
            cmp(nd, i) = RT_IN(pd[i], kp.dtau, kp.ext.cube) ? __ldcs(pd[i]) : 0.f;
            cmp(nw, i) = RT_IN(pw[i], kp.w0, kp.ext.cube) ? __ldcs(pw[i]) : 0.f;
            cmp(ng, i) = RT_IN(pg[i], kp.g0, kp.ext.cube) ? __ldcs(pg[i]) : 0.f;
        }
    }
    cp_async_wait<0>();
    __syncwarp();                              // the staged values of every lane
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        cmp(Fb, i) = beam ? mu * sFs[bI[i] - b_lo] : 0.f;
        if constexpr (!INL) {
            // the B of a layer's bottom interface is carried as the next layer's top
            cmp(Bt, i) = ldBk<DIRECT>(kp, Bp[i]);
            cmp(Bc, i) = ldBk<DIRECT>(kp, Bp[i] + bst);
            cmp(Bb, i) = ldBk<DIRECT>(kp, Bp[i] + 2 * bst);
        }
    }
    if constexpr (INL) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            cmp(wn0v, i) = wn0[i];
            cmp(wn1v, i) = wn1[i];
            cmp(dnuv, i) = dnu[i];
        }
        // every level of the column is at least as warm as cf.w, so its
        // h c / k T is at most that level's: if the unit's bins pass the
        // two-point tests there (with margins for the FP32 roundings of the
        // per-level tests), they pass at every level and the tests are skipped
        if (cf.w > 0.f) {
            const float am = __fmul_rn(planck_level(cf.w, 1.f).a, 1.0001f);
            bool ok = true;
#pragma unroll
            for (int i = 0; i < NS; ++i)
                ok = ok && fmaf(am, wn1[i] - wn0[i], 1e-6f * am * wn1[i]) < 0.999f * kNarrowBin &&
                     am * dnu[i] < 0.999f * kTwoPointBin &&
                     0.5f * dnu[i] < 0.0099f * (wn0[i] + 0.5f * dnu[i]);
            unit_narrow = __all_sync(0xffffffffu, ok);
        }
        B_at(0, Bt);
        B_at(1, Bc);
        B_at(2, Bb);
    }
    SysCounts<V> sc;
    sc.inv = sc.ecl = sc.etau = typename VTraits<V>::C{};

    // forward elimination, TOA -> BOA, departure variables
    V al = V(1.f);                                       // alpha' = 1 - a'
    V bl = vfma(V(-kPiF), Bt, V((float)kp.F_toa));       // b' at the TOA
    float4 *sp = kp.scr32 + slot;
    V *spB = INL ? (V *)kp.scrB + slot : nullptr;
    // two layers per trip: the carried values (B at the levels, the
    // prefetched optics, alpha' and b') alternate between two register
    // sets instead of being copied at the end of every layer (not with
    // inline B, whose extra live values would spill; the k-table front end
    // spills a few bytes and still gains)
#pragma unroll(INL ? 1 : 2)
    for (int l = 0; l < L; ++l) {
        V dt, w0, g0;
        V nBc = V(0.f), nBb = V(0.f);
        if constexpr (KT) {
            const float4 kl = kl_next;
            Corners cur[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) cur[i] = kc[i];
            if (l + 1 < L) {                     // prefetch the next layer's corners
                kl_next = kl_after;
#pragma unroll
                for (int i = 0; i < NS; ++i) kc[i] = kt_corners(kp, kl_next, S, sI[i]);
                if (l + 2 < L) kl_after = klay[l + 2];
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const Optics o = kt_mix(cur[i].lo, cur[i].hi, kl, kb[i]);
                cmp(dt, i) = o.dt;
                cmp(w0, i) = o.w0;
                cmp(g0, i) = o.g0;
            }
        } else {
            dt = nd;
            w0 = nw;
            g0 = ng;
            if (l + 1 < L) {                     // prefetch the next layer
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    pd[i] += S;
                    pw[i] += S;
                    pg[i] += S;
                    cmp(nd, i) = RT_IN(pd[i], kp.dtau, kp.ext.cube) ? __ldcs(pd[i]) : 0.f;
                    cmp(nw, i) = RT_IN(pw[i], kp.w0, kp.ext.cube) ? __ldcs(pw[i]) : 0.f;
                    cmp(ng, i) = RT_IN(pg[i], kp.g0, kp.ext.cube) ? __ldcs(pg[i]) : 0.f;
                }
            }

        }
        if (l + 1 < L) {
            if constexpr (INL) {
                B_at(2 * l + 3, nBc);
                B_at(2 * l + 4, nBb);
            } else {
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    cmp(nBc, i) = ldBk<DIRECT>(kp, Bp[i] + 3 * bst);
                    cmp(nBb, i) = ldBk<DIRECT>(kp, Bp[i] + 4 * bst);
                }
            }
        }
        if constexpr (INL) {
            if (RT_IN(spB, (V *)kp.scrB, kp.ext.scrB / NS)) stB(spB, Bt);   // B at interface l, for the back-substitution
            spB += gthreads;
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) Bp[i] += 2 * bst;   // level 2 (l + 1)
        const Layer32<V> ly = layer32<ISO, V>(dt, w0, g0, Bt, Bc, Bb, mu, imu, mu_d, beam, Fb, kp, cn, sc, on);
        Bt = Bb;
        Bc = nBc;
        Bb = nBb;
        const V omr = ly.omtr + ly.T;                      // 1 - R
        const V ipv = vrcp(vfma(ly.R, al, omr));           // 1 / (1 - R a')
        const V P = ly.T * ipv;
        const V Qv = vfma(ly.R, bl, ly.Su) * ipv;
        scr_store(kp, sp, gthreads, P, Qv, al, bl + Fb);  // e = b' + F_beam
        sp += sstride;
        const V al_n = vfma(al, vfma(ly.R, omr, ly.T * ly.T), ly.omtr * ly.opr) * ipv;
        const V bl_n = vfma(ly.T * vfma(V(1.f) - al, ly.Su, bl), ipv, ly.Sd);
        al = al_n;
        bl = bl_n;
        Fb = Fb * ly.mlay;
    }

    cn.inv += vmasked(sc.inv, on);
    cn.eclamp += vmasked(sc.ecl, on);
    cn.etau += (ISO ? 1u : 2u) * vmasked(sc.etau, on);
    // BOA (Eq. 10): u - d = F_BOA + F_beam with d = (1 - alpha') u + b';
    // back-substitution to the TOA; interface sums through the transpose
    V FBOA;
#pragma unroll
    for (int i = 0; i < NS; ++i) cmp(FBOA, i) = sFB[bI[i] - b_lo];
    V uu = ((FBOA + Fb) + bl) * vrcp(al);
    bool bad[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) bad[i] = !isfinite(cmp(uu, i));   // NaN and Inf propagate upwards
    float *part = kp.partial + kp.part_off[c] + (long long)ku * 2 * (L + 1);
    // Bt holds B at level 2L (the BOA interface)
    tb[lane] = hsum(wg * vfma(V(kPiF), Bt, uu));
    tb[33 + lane] = hsum(wg * FBOA);
    V nBi = V(0.f);          // Bp is at level 2L; prefetch one interface up (inline B: through the ring)
    if constexpr (!INL) {
#pragma unroll
        for (int i = 0; i < NS; ++i) cmp(nBi, i) = ldBk<DIRECT>(kp, Bp[i] - 2 * bst);
    }
    // The back-substitution does a few operations per level, so each
    // level's scratch is copied into the shared-memory ring DEP levels ahead
    // (cp.async, one commit group per level; level i sits in slot
    // (L - 1 - i) mod (DEP + 1), and the copy of level i - DEP goes to the
    // slot read one level earlier).
    constexpr int D = DEP, NSL = DEP + 1;
    const float4 *sbase = kp.scr32 + slot;
    const V *Bbase = INL ? (const V *)kp.scrB + slot : nullptr;      // inline B at interface i: + i gthreads
    V *rB = reinterpret_cast<V *>(ringB);
    auto issue = [&](int i, int k) {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const float4 *p = sbase + (long long)i * sstride + (long long)j * gthreads;
            if (RT_IN(p, kp.scr32, kp.ext.scr32)) cp_async16(ring + (k * NS + j) * 32 + lane, p);
        }
        if constexpr (INL) {
            const V *pb = Bbase + (long long)i * gthreads;
            if (RT_IN(pb, (const V *)kp.scrB, kp.ext.scrB / NS)) {
                if constexpr (NS == 2) cp_async8(rB + k * 32 + lane, pb);
                else cp_async4(rB + k * 32 + lane, pb);
            }
        }
    };
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (L - 1 - k >= 0) issue(L - 1 - k, k);
        cp_async_commit();
    }
    const int gsh = kp.group_shift, G = 1 << gsh;  // interfaces per transposed sum
    int gi = 1;              // slots used in the current group of G interfaces
    int gtop = L;            // interface held in slot 0 of the group
    for (int i0 = L - 1; i0 >= -1; i0 -= NSL) {
#pragma unroll
        for (int k = 0; k < NSL; ++k) {
            const int i = i0 - k;
            if (i >= 0) {
                cp_async_wait<D - 1>();              // level i has landed
                float4 nst[NS];
#pragma unroll
                for (int j = 0; j < NS; ++j) nst[j] = ring[(k * NS + j) * 32 + lane];
                if (i - D >= 0) issue(i - D, (k + D) % NSL);
                cp_async_commit();
                V Pv, Qq, av, ev;
                scr_unpack(nst, Pv, Qq, av, ev);
#pragma unroll
                for (int j = 0; j < NS; ++j) {
                    // this level's scratch is dead once read: drop its L2
                    // lines (one per 8 lanes) so they are not written back
                    const float4 *p = sbase + (long long)i * sstride + (long long)j * gthreads;
                    if ((lane & 7) == 0 && RT_IN(p, kp.scr32, kp.ext.scr32)) discard_l2_after(p, nst[j].x);
                }
                V Bi = nBi;
                if constexpr (INL) {
                    Bi = rB[k * 32 + lane];
                    const V *pb = Bbase + (long long)i * gthreads;
                    if ((lane & (32 / NS - 1)) == 0 && RT_IN(pb, (const V *)kp.scrB, kp.ext.scrB / NS))
                        discard_l2_after(pb, cmp(Bi, 0));
                }
#pragma unroll
                for (int j = 0; j < NS; ++j) Bp[j] -= 2 * bst;     // level 2i
                if constexpr (!INL) {
                    if (i > 0) {
#pragma unroll
                        for (int j = 0; j < NS; ++j) cmp(nBi, j) = ldBk<DIRECT>(kp, Bp[j] - 2 * bst);
                    }
                }
                uu = vfma(Pv, uu, Qq);
                const V fup = vfma(V(kPiF), Bi, uu);
                Bt = Bi;
                const V fnet = vfma(av, uu, -ev);
                tb[(gi * 2) * 33 + lane] = hsum(wg * fup);
                tb[(gi * 2 + 1) * 33 + lane] = hsum(wg * fnet);
                ++gi;
            }
            if (gi == G || (i < 0 && gi > 0)) {
                __syncwarp();
                // lane j < 2 G sums row (slot j mod G, quantity j / G) over the 32 lanes
                const int sl = lane & (G - 1), qq = lane >> gsh;
                if (qq < 2 && sl < gi) {
                    const float *row = tb + (sl * 2 + qq) * 33;
                    float acc = 0.f;
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) acc += row[j];
                    if (RT_IN(part + 2 * (gtop - sl) + qq, kp.partial, kp.ext.part)) part[2 * (gtop - sl) + qq] = acc;
                }
                __syncwarp();
                gtop -= gi;
                gi = 0;
            }
        }
    }
    cp_async_wait<0>();      // (only empty groups remain)
#pragma unroll
    for (int i = 0; i < NS; ++i)
        if (cmpm(on, i) && (bad[i] || !isfinite(cmp(uu, i)))) cn.nonfinite++;

    // TOA spectrum: uu and Bt are now at interface 0; each bin's systems
    // are summed in system order and added once per unit (a bin of
    // n_g <= 32 NS systems meets at most two units, so the FP64 sum is
    // order-free)
    if (kp.toa) {
        V ft = wg * vfma(V(kPiF), Bt, uu);
#pragma unroll
        for (int i = 0; i < NS; ++i) tb[32 * i + lane] = cmp(ft, i);
        __syncwarp();
        for (int jb = lane; jb < nbc; jb += 32) {
            const int bt = b_lo + jb;
            const int j0 = max(0, bt * NG - s0);
            const int j1 = min(min(SPU, S - s0), (bt + 1) * NG - s0);
            float acc = 0.f;
            for (int j = j0; j < j1; ++j) acc += tb[j];
            if (RT_IN(kp.toa + kp.bin_off[c] + bt, kp.toa, kp.ext.bins)) atomicAdd(kp.toa + kp.bin_off[c] + bt, (double)acc);
        }
        __syncwarp();
    }

    // (the column's outputs are formed from the units' partials by
    // fp32_finalize, after every unit of the launch)
    __syncwarp();
}

// DEP: levels of elimination scratch in flight in the back-substitution
// (kp.back_depth; one instance per offered depth).
template <bool ISO, int ST, bool KT, int NS, int DEP>
__global__ void __launch_bounds__(kMaxBlock32, NS == 2 ? 2 : 3) fp32_units(KParams kp) {
    grid_dependency_wait();                        // the pre-kernel's tables
    constexpr int SPG = 32 * NS;                   // unit stride within a column
    extern __shared__ __align__(16) float smem32[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *wsm = smem32 + (size_t)warp * kp.warp_floats;
    const int nbw = kp.nbw;
    float4 *ring = reinterpret_cast<float4 *>(wsm);   // [DEP + 1][NS][32], back-substitution
    float *ringB = wsm + back_ring_floats(NS, DEP);   // inline B: [DEP + 1][32] x NS
    float *sB = ringB + back_ringB_floats(NS, ST == kStageInline, DEP);   // [nbc][2 L + 1] (bin, level), staged mode
    float *sFs = sB + (ST == kStageShared ? kp.staged : ST == kStageInline ? 2 * (2 * kp.Lmax + 1) : 0);   // [nbc]
    float *sFB = sFs + nbw;                        // [nbc]
    float *tb = sFB + nbw;                         // [G][2][33]
    // scratch slots: component i of this thread at slot + i * (threads in the grid)
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long sstride = kp.n_slots;
    Counters cn = {0, 0, 0, 0, 0, 0, 0};

    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(kp.counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= kp.n_units) break;
        fp32_unit<ISO, ST, KT, NS, SPG, DEP>(kp, unit, lane, ring, ringB, sB, sFs, sFB, tb, slot, gthreads, sstride, cn);
    }
    flush_counters(cn, kp.stats);
}

// ---------------------------------------------------------------------
// The iterative method (Sec. 2.2.2) in the FP32 form: the pairwise two-stream
// relations of every sub-layer applied through the column, repeated N times,
// instead of the elimination.  One sweep is a downward pass from the TOA
// condition (each sub-layer gives d at its bottom from d at its top and the
// previous sweep's u at its bottom), the BOA condition (Eq. 10) and an upward
// pass (each sub-layer gives u at its top from u at its bottom and d at its
// top); the sweeps start from zero diffuse flux.  In departure variables
// (u = F_up - pi B, d = F_dn - pi B at each level, as in the elimination)
// the relations of a sub-layer with transmission t, reflection r and sources
// su, sd read
//   u_top = t u_bot + r d_top + su,   d_bot = t d_top + r u_bot + sd.
//
// Layout.  A warp takes work units of 32 systems of a column (one per lane).
// The coefficient pass streams the cubes once and leaves, per layer, the
// sub-layer sources in the warp's shared memory, the warp sums of w F_beam at
// the interfaces there too, and each lane's (t, r) in a global scratch
// ([layer][thread slot], read back at once, so it stays in L2); the lane
// then loads its t, r into registers next to its level state (u or d at each
// of the 2L+1 levels), so that a sweep reads only the sources from shared
// memory: 8 bytes per layer and pass for four FMAs.  Register arrays need
// compile-time indices, so the passes are unrolled to kSweepMaxLayers layers.
// The last upward pass writes the interface fluxes into the downward
// sources' area (the last downward pass is done by then), swizzled for a
// conflict-free transposed sum.  Keeping (t, r) out of shared memory is what
// lets 8 warps (the register limit) rather than 7 reside on an SM.
// ---------------------------------------------------------------------
// The output rows [2 (Lmax + 1)][32] (XOR-swizzled)
__host__ __device__ inline int sweep_region_floats() { return 64 * (kSweepMaxLayers + 1); }

// Output row element (row, j) of the swizzled rows: lane j's writes to one
// row and the lanes' reads of one column each of their own row hit 32
// different banks.
__device__ __forceinline__ int out_idx(int row, int j) { return row * 32 + (j ^ (row & 31)); }

int sweep_warp_floats(int Lmax, int nbw, int direct, int isothermal) {
    const int per = isothermal ? 32 : 64;          // sources per layer and pass (one or two sub-layers)
    int n = ((direct ? 0 : (2 * Lmax + 1) * nbw) + 3) & ~3;
    n += (2 * nbw + 3) & ~3;                        // F*, F_BOA
    n += (Lmax + 1 + 3) & ~3;                       // warp sums of w F_beam per interface
    n += per * kSweepMaxLayers;                     // SU (every system padded to the register limit)
    n += std::max(per * kSweepMaxLayers, sweep_region_floats());   // SD, then the output rows
    return n;
}
size_t sweep_smem_bytes(int block, int Lmax, int nbw, int direct, int isothermal) {
    return sizeof(float) * (size_t)(block / 32) * sweep_warp_floats(Lmax, nbw, direct, isothermal);
}

// Layers per chunk of the sweep passes: each chunk's source rows are loaded
// while the previous chunk computes.
constexpr int kSweepChunk = 8;
static_assert(kSweepMaxLayers % kSweepChunk == 0, "whole chunks");

// The passes run over all kSweepMaxLayers layers of every system: a column
// with fewer layers is padded below its BOA with exact identity layers (t =
// 1, r = 0, no source, B of the BOA), through which u and d pass unchanged.
// The BOA condition then sits at a compile-time level and the passes need
// no per-layer predicate, clamp or select.

// One upward pass.  X holds d at the levels and u at the padded BOA; on
// return it holds u.  EMIT (last sweep): u and u - d at interface i <= L of
// the column (level 2i, or i for isothermal layers) go to rows 2i and 2i + 1
// of OUT (element of lane j: out_idx); interface kSweepMaxLayers is left to
// the caller.  X is indexed only by the unrolled loop counters, so it stays
// in registers.
template <bool ISO, bool EMIT, int LR, int NLV>
__device__ __forceinline__ void sweep_up(float (&X)[NLV], const float (&t)[LR], const float (&r)[LR], int L, int lane,
                                         float d0, const float *SU, float *OUT) {
    constexpr int CH = kSweepChunk, NC = LR / kSweepChunk;
    using S2 = typename std::conditional<ISO, float, float2>::type;    // sources of one layer
    const S2 *src = reinterpret_cast<const S2 *>(SU) + lane;
    S2 buf[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) buf[k] = src[((NC - 1) * CH + k) * 32];
#pragma unroll
    for (int c = NC - 1; c >= 0; --c) {
        S2 cur[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) cur[k] = buf[k];
        if (c > 0) {
#pragma unroll
            for (int k = 0; k < CH; ++k) buf[k] = src[((c - 1) * CH + k) * 32];
        }
#pragma unroll
        for (int k = CH - 1; k >= 0; --k) {
            const int l = c * CH + k;
            float u, dl;
            if constexpr (ISO) {
                dl = l == 0 ? d0 : X[l];
                u = fmaf(t[l], X[l + 1], fmaf(r[l], dl, cur[k]));
                X[l] = u;
            } else {
                X[2 * l + 1] = fmaf(t[l], X[2 * l + 2], fmaf(r[l], X[2 * l + 1], cur[k].y));   // lower
                dl = l == 0 ? d0 : X[2 * l];
                u = fmaf(t[l], X[2 * l + 1], fmaf(r[l], dl, cur[k].x));                       // upper
                X[2 * l] = u;
            }
            if (EMIT && l <= L) {
                OUT[out_idx(2 * l, lane)] = u;
                OUT[out_idx(2 * l + 1, lane)] = u - dl;
            }
        }
    }
}

// One downward pass: X takes d at every level below the TOA, then u = d +
// (F_BOA + F_beam) at the padded BOA; returns d there.
template <bool ISO, int LR, int NLV>
__device__ __forceinline__ float sweep_down(float (&X)[NLV], const float (&t)[LR], const float (&r)[LR], int lane,
                                            float d0, float ubc, const float *SD) {
    constexpr int CH = kSweepChunk, NC = LR / kSweepChunk;
    using S2 = typename std::conditional<ISO, float, float2>::type;
    const S2 *src = reinterpret_cast<const S2 *>(SD) + lane;
    S2 buf[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) buf[k] = src[k * 32];
    float d = d0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        S2 cur[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) cur[k] = buf[k];
        if (c + 1 < NC) {
#pragma unroll
            for (int k = 0; k < CH; ++k) buf[k] = src[((c + 1) * CH + k) * 32];
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int l = c * CH + k;
            if constexpr (ISO) {
                d = fmaf(t[l], d, fmaf(r[l], X[l + 1], cur[k]));
                X[l + 1] = d;
            } else {
                d = fmaf(t[l], d, fmaf(r[l], X[2 * l + 1], cur[k].x));          // upper sub-layer
                X[2 * l + 1] = d;
                d = fmaf(t[l], d, fmaf(r[l], X[2 * l + 2], cur[k].y));          // lower
                X[2 * l + 2] = d;
            }
        }
    }
    X[NLV - 1] = d + ubc;
    return d;
}

// Column and lane bookkeeping of a sweep unit (re-derived after the sweeps,
// so that none of it is held in registers across them).
struct SweepLane {
    int c, ku, L, NB, S, s0, b_lo, nbc, bI, bst;
    bool on;
    float wg;
    const float *Bp;
};

template <bool DIRECT>
__device__ __forceinline__ SweepLane sweep_lane(const KParams &kp, int unit, int lane, float *sB) {
    SweepLane q;
    const int NG = kp.n_g;
    q.c = kp.unit_col[unit];
    q.ku = kp.unit_k[unit];
    q.L = kp.n_layers[q.c];
    q.NB = kp.n_bins[q.c];
    q.S = q.NB * NG;
    q.s0 = q.ku * 32;
    q.b_lo = q.s0 / NG;
    q.nbc = min(q.NB - 1, (q.s0 + 31) / NG) - q.b_lo + 1;
    // padding lanes of a column's last unit repeat system s0 with zero weight
    q.on = q.s0 + lane < q.S;
    const int sI = q.on ? q.s0 + lane : q.s0;
    q.bI = sI / NG;
    q.wg = q.on ? kp.g_w32[sI - q.bI * NG] : 0.f;
    q.bst = DIRECT ? q.NB : q.nbc;
    q.Bp = DIRECT ? kp.planck32 + kp.planck_off[q.c] + q.bI : sB + (q.bI - q.b_lo);
    return q;
}

// What the sweeps start from: the column's L, d at the TOA level and u - d
// at the BOA (Eq. 10).
struct SweepStart {
    int L;
    float d0, ubc;
};

// The coefficient pass of a sweep unit: stage B, F*, F_BOA; per layer (t, r)
// and the sub-layer sources into shared memory, and the warp sums of w F_beam
// at the interfaces.  (Inlined: as a call, or with the staging issued as
// asynchronous copies, the sweeps' register arrays spill.)
template <bool ISO, bool DIRECT>
__device__ __forceinline__ SweepStart sweep_coefficients(const KParams &kp, int unit, int lane, float *sB, float *sFs,
                                                      float *sFB, float *fbs, float *SU, float *SD, float2 *gtr,
                                                      long long gst) {
    {
        const SweepLane q = sweep_lane<DIRECT>(kp, unit, lane, sB);
        const int L = q.L;
        constexpr int LR = kSweepMaxLayers;
        float d0, ubc;
        {
            const float *Bg = kp.planck32 + kp.planck_off[q.c] + q.b_lo;
            const int nlev = 2 * L + 1;
            if constexpr (!DIRECT) {
                for (int i = lane; i < nlev * q.nbc; i += 32) {
                    const int lev = i / q.nbc, bb = i - lev * q.nbc;
                    const float *pb = Bg + (long long)lev * q.NB + bb;
                    sB[i] = RT_IN(pb, kp.planck32, kp.ext.planck) ? __ldcg(pb) : 0.f;
                }
            }
            for (int j = lane; j < q.nbc; j += 32) {
                const long long jb = kp.bin_off[q.c] + q.b_lo + j;
                sFs[j] = RT_IN(kp.fs32 + jb, kp.fs32, kp.ext.bins) ? __ldcg(kp.fs32 + jb) : 0.f;
                sFB[j] = RT_IN(kp.fboa32 + jb, kp.fboa32, kp.ext.bins) ? __ldcg(kp.fboa32 + jb) : 0.f;
            }
        }
        const long long e0 = kp.cube_off[q.c] + (q.on ? q.s0 + lane : q.s0);
        const float *pd = kp.dtau + e0, *pw = kp.w0 + e0, *pg = kp.g0 + e0;
        auto ld_opt = [&](int l, float &d, float &w, float &g) {    // the optics of layer l
            const long long o = (long long)l * q.S;
            d = RT_IN(pd + o, kp.dtau, kp.ext.cube) ? __ldcs(pd + o) : 0.f;
            w = RT_IN(pw + o, kp.w0, kp.ext.cube) ? __ldcs(pw + o) : 0.f;
            g = RT_IN(pg + o, kp.g0, kp.ext.cube) ? __ldcs(pg + o) : 0.f;
        };
        float nd0, nw0, ng0, nd1 = 0.f, nw1 = 0.f, ng1 = 0.f;
        ld_opt(0, nd0, nw0, ng0);
        if (L > 1) ld_opt(1, nd1, nw1, ng1);
        const float4 cf = kp.colf[q.c];
        const float mu = cf.x, imu = cf.y;
        const double mu_d = ck_ld(kp, kp.mu_star, kp.ext.mu, kp.mu_idx[q.c]);
        const bool beam = cf.z != 0.f;
        __syncwarp();                                              // the staged values of every lane
        float Fb = beam ? mu * sFs[q.bI - q.b_lo] : 0.f;
        const float FBOA = sFB[q.bI - q.b_lo];
        Counters cu = {0, 0, 0, 0, 0, 0, 0};
        SysCounts<float> sc;
        sc.inv = sc.ecl = sc.etau = 0u;
        SysCounts<V2> sc2;
        sc2.inv = sc2.ecl = sc2.etau = U2{0u, 0u};
        const M2 on2 = M2{q.on, q.on};
        auto wsum = [](float v) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            return v;
        };
        auto put = [&](int l, float tl, float rl, float uU, float uL, float dU, float dL) {
            float2 *pt = gtr + l * gst;
            if (RT_IN(pt, reinterpret_cast<float2 *>(kp.scr32), 2 * kp.ext.scr32)) __stcg(pt, make_float2(tl, rl));
            if constexpr (ISO) {
                SU[l * 32 + lane] = uU;
                SD[l * 32 + lane] = dU;
            } else {
                reinterpret_cast<float2 *>(SU)[l * 32 + lane] = make_float2(uU, uL);
                reinterpret_cast<float2 *>(SD)[l * 32 + lane] = make_float2(dU, dL);
            }
        };
        // layers l and l + 1 side by side on the paired instructions (they
        // are independent but for F_beam, applied here from the running
        // product); the next pair's optics prefetched; an odd last layer alone
        float Bt = ldBk<DIRECT>(kp, q.Bp);
        d0 = fmaf(-kPiF, Bt, (float)kp.F_toa);                     // d at the TOA level
        int l = 0;
        for (; l + 1 < L; l += 2) {
            const V2 dt(nd0, nd1), w0(nw0, nw1), g0(ng0, ng1);
            if (l + 2 < L) ld_opt(l + 2, nd0, nw0, ng0);
            if (l + 3 < L) ld_opt(l + 3, nd1, nw1, ng1);
            const float B1 = ldBk<DIRECT>(kp, q.Bp + (2 * l + 1) * q.bst);
            const float B2 = ldBk<DIRECT>(kp, q.Bp + (2 * l + 2) * q.bst);
            const float B3 = ldBk<DIRECT>(kp, q.Bp + (2 * l + 3) * q.bst);
            const float B4 = ldBk<DIRECT>(kp, q.Bp + (2 * l + 4) * q.bst);
            const Sub32<V2> sb = sub32<ISO, V2, true>(dt, w0, g0, V2(Bt, B2), V2(B1, B3), V2(B2, B4), mu, imu, mu_d,
                                                      beam, V2(0.f), kp, cu, sc2, on2);
            const float m0 = sb.m.v.x, m1 = sb.m.v.y;
            const float Fb0 = Fb, Fb1 = ISO ? Fb0 * m0 : Fb0 * (m0 * m0);
            const float fw0 = wsum(q.wg * Fb0), fw1 = wsum(q.wg * Fb1);    // interfaces l, l + 1
            if (lane == 0) {
                fbs[l] = fw0;
                fbs[l + 1] = fw1;
            }
            V2 uU = sb.suU, dU = sb.sdU, uL = sb.suL, dL = sb.sdL;
            if (beam) {
                const V2 F(Fb0, Fb1);
                uU = vfma(F, sb.bu, uU);
                dU = vfma(F, sb.bd, dU);
                if constexpr (!ISO) {
                    const V2 Fc = F * sb.m;
                    uL = vfma(Fc, sb.bu, uL);
                    dL = vfma(Fc, sb.bd, dL);
                }
            }
            put(l, sb.t.v.x, sb.r.v.x, uU.v.x, uL.v.x, dU.v.x, dL.v.x);
            put(l + 1, sb.t.v.y, sb.r.v.y, uU.v.y, uL.v.y, dU.v.y, dL.v.y);
            Fb = ISO ? Fb1 * m1 : Fb1 * (m1 * m1);
            Bt = B4;
        }
        if (l < L) {
            const float Bc = ldBk<DIRECT>(kp, q.Bp + (2 * l + 1) * q.bst);
            const float Bb = ldBk<DIRECT>(kp, q.Bp + (2 * l + 2) * q.bst);
            const float fw = wsum(q.wg * Fb);                          // interface l
            if (lane == 0) fbs[l] = fw;
            const Sub32<float> sb =
                sub32<ISO, float>(nd0, nw0, ng0, Bt, Bc, Bb, mu, imu, mu_d, beam, Fb, kp, cu, sc, q.on);
            put(l, sb.t, sb.r, sb.suU, sb.suL, sb.sdU, sb.sdL);
            Fb *= ISO ? sb.m : sb.m * sb.m;
        }
        // identity layers below the BOA up to the register limit (t = 1, r = 0, no source)
        for (int k = L; k < LR; ++k) put(k, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        {
            const float fw = wsum(q.wg * Fb);                          // the BOA interface
            if (lane == 0) fbs[L] = fw;
        }
        ubc = FBOA + Fb;                                           // u - d at the BOA (Eq. 10)
        cu.inv = vmasked(sc.inv, q.on) + vmasked(sc2.inv, on2);
        cu.eclamp = vmasked(sc.ecl, q.on) + vmasked(sc2.ecl, on2);
        cu.etau = (ISO ? 1u : 2u) * (vmasked(sc.etau, q.on) + vmasked(sc2.etau, on2));
        flush_counters(cu, kp.stats);                              // per unit: nothing kept live
        __syncwarp();
        return SweepStart{L, d0, ubc};
    }
}

template <bool ISO, bool DIRECT>
__device__ __forceinline__ void sweep_unit(const KParams &kp, int unit, int lane, float *sB, float *sFs, float *sFB,
                                           float *fbs, float *SU, float *SD, float *TR, float2 *gtr, long long gst) {
    constexpr int LR = kSweepMaxLayers;
    constexpr int NLV = ISO ? LR + 1 : 2 * LR + 1;    // levels held per lane
    float t[LR], r[LR], X[NLV];
    int L;
    float d0, ubc;

    // ---- coefficient pass into shared memory; then t, r and the starting
    // state into registers
    {
        const SweepStart st = sweep_coefficients<ISO, DIRECT>(kp, unit, lane, sB, sFs, sFB, fbs, SU, SD, gtr, gst);
        L = st.L;
        d0 = st.d0;
        ubc = st.ubc;
        const SweepLane q = sweep_lane<DIRECT>(kp, unit, lane, sB);
#pragma unroll
        for (int l = 0; l < LR; ++l) {
            const float2 *pt = gtr + l * gst;
            const float2 v = RT_IN(pt, reinterpret_cast<const float2 *>(kp.scr32), 2 * kp.ext.scr32)
                                 ? __ldcg(pt) : make_float2(1.f, 0.f);
            t[l] = v.x;
            r[l] = v.y;
        }

        // zero diffuse flux: u = -pi B at every level (the BOA's B below it)
#pragma unroll
        for (int j = 0; j < NLV; ++j) {
            const int lev = ISO ? 2 * j : j;                       // level in the B table
            X[j] = -kPiF * ldBk<DIRECT>(kp, q.Bp + min(lev, 2 * L) * q.bst);
        }
        __syncwarp();
    }

    // ---- the sweeps: registers t, r, X; sources from shared memory
    float dB = 0.f;
    for (int it = 0; it < kp.n_sweeps; ++it) {
        dB = sweep_down<ISO>(X, t, r, lane, d0, ubc, SD);
        if (it + 1 < kp.n_sweeps) {
            sweep_up<ISO, false>(X, t, r, L, lane, d0, SU, TR);
        } else {
            __syncwarp();              // every lane's downward pass has read SD: its area takes the output rows
            sweep_up<ISO, true>(X, t, r, L, lane, d0, SU, TR);
        }
    }
    const bool finite = isfinite(X[0]) && isfinite(dB);

    // ---- interface sums, TOA spectrum, column finalisation
    const SweepLane q = sweep_lane<DIRECT>(kp, unit, lane, sB);
    if (L == LR) {
        // the BOA interface of a column with no padding (the last upward
        // pass emitted it for any other): u = d + (F_BOA + F_beam)
        const float uB = X[NLV - 1];
        TR[out_idx(2 * L, lane)] = uB;
        TR[out_idx(2 * L + 1, lane)] = uB - dB;
    }
    const unsigned bad = __ballot_sync(0xffffffffu, q.on && !finite);
    if (lane == 0 && bad) atomicAdd(kp.stats + ST_NONFINITE, (unsigned long long)__popc(bad));
    // weighted fluxes: F_up = pi B + u; F_net + F_beam = u - d
    for (int i = 0; i <= L; ++i) {
        const float Bi = ldBk<DIRECT>(kp, q.Bp + 2 * i * q.bst);
        TR[out_idx(2 * i, lane)] = q.wg * fmaf(kPiF, Bi, TR[out_idx(2 * i, lane)]);
        TR[out_idx(2 * i + 1, lane)] *= q.wg;
    }
    __syncwarp();
    // row 2i = sum w F_up, row 2i + 1 = sum w (u - d) - sum w F_beam
    float *part = kp.partial + kp.part_off[q.c] + (long long)q.ku * 2 * (L + 1);
    for (int row = lane; row < 2 * (L + 1); row += 32) {
        float acc = 0.f;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) acc += TR[out_idx(row, j)];
        if (row & 1) acc -= fbs[row >> 1];
        if (RT_IN(part + row, kp.partial, kp.ext.part)) part[row] = acc;
    }
    // TOA spectrum: row 0 holds w F_up at the TOA per system
    if (kp.toa) {
        const int NG = kp.n_g;
        for (int jb = lane; jb < q.nbc; jb += 32) {
            const int bt = q.b_lo + jb;
            const int j0 = max(0, bt * NG - q.s0);
            const int j1 = min(min(32, q.S - q.s0), (bt + 1) * NG - q.s0);
            float acc = 0.f;
            for (int j = j0; j < j1; ++j) acc += TR[out_idx(0, j)];
            if (RT_IN(kp.toa + kp.bin_off[q.c] + bt, kp.toa, kp.ext.bins))
                atomicAdd(kp.toa + kp.bin_off[q.c] + bt, (double)acc);
        }
    }
    __syncwarp();

    // (the column's outputs: fp32_finalize, after every unit of the launch)
    __syncwarp();
}

template <bool ISO, bool DIRECT>
__global__ void __launch_bounds__(kMaxBlock32, 1) fp32_sweeps(KParams kp) {
    extern __shared__ __align__(16) float smem32[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *wsm = smem32 + (size_t)warp * kp.warp_floats;
    const int Lm = kp.Lmax, nbw = kp.nbw;
    float *sB = wsm;
    float *sFs = sB + (((DIRECT ? 0 : (2 * Lm + 1) * nbw) + 3) & ~3);
    float *sFB = sFs + nbw;
    float *fbs = sFs + ((2 * nbw + 3) & ~3);
    float *SU = fbs + ((Lm + 1 + 3) & ~3);
    float *SD = SU + (ISO ? 32 : 64) * kSweepMaxLayers;
    float *TR = SD;                                // the output rows, once the last downward pass is done
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gst = (long long)gridDim.x * blockDim.x;
    float2 *gtr = reinterpret_cast<float2 *>(kp.scr32) + slot;   // (t, r) of layer l at gtr[l gst]
    for (;;) {
        int unit = 0;
        if (lane == 0) unit = atomicAdd(kp.counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= kp.n_units) break;
        sweep_unit<ISO, DIRECT>(kp, unit, lane, sB, sFs, sFB, fbs, SU, SD, TR, gtr, gst);
    }
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
    } else if (k == 0.0) {                         // E = w0 = 1: the k -> 0 limit
        const double q = E * omwg;
        chi = -(1.0 + q * dts);
        xi = q * dts;
        psi = -1.0;
    } else {                                       // E < w0 (raw fit): k is not real
        chi = xi = psi = k;                        // NaN
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
    Smem<double> sm(smem_raw, kp.Lmax, kp.nb_chunk, kp.staged, nwarps);
    const int NG = kp.n_g;
    const long long slot = (long long)blockIdx.x * blockDim.x + tid;
    double2 *scr = kp.scr64 + slot;           // element (2 lev + j) n_slots + slot
    Counters cn = {0, 0, 0, 0, 0, 0, 0};
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
                    dt = RT_IN(kp.dtau + idx, kp.dtau, kp.ext.cube) ? (double)__ldg(kp.dtau + idx) : 0.0;
                    w0f = RT_IN(kp.w0 + idx, kp.w0, kp.ext.cube) ? __ldg(kp.w0 + idx) : 0.f;
                    g0f = RT_IN(kp.g0 + idx, kp.g0, kp.ext.cube) ? __ldg(kp.g0 + idx) : 0.f;
                    w0 = (double)w0f;
                    g0 = (double)g0f;
                }
                if (!(dt >= 0.0) || !(w0 >= 0.0 && w0 <= 1.0) || !(g0 > -1.0 && g0 < 1.0)) cn.inv += cn.on;
                double E = 1.0;
                if (kp.improved && w0 > (double)0.1f) {
                    E = 1.225 - 0.1582 * g0 - 0.1777 * w0 - 0.07465 * g0 * g0 + 0.2351 * w0 * g0
                        - 0.05582 * w0 * w0;
                    // hits counted on E - 1 in FP32 as the FP32 form forms it
                    const float w0f = (float)w0, g0f = (float)g0;
                    const float em1f = fmaf(0.2351f, __fmul_rn(w0f, g0f),
                                            fmaf(g0f, fmaf(-0.07465f, g0f, -0.1582f),
                                                 fmaf(w0f, fmaf(-0.05582f, w0f, -0.1777f), 0.225f)));
                    if (kp.e_clamp && em1f < 0.f) cn.eclamp += cn.on;
                    if (kp.e_clamp && E < 1.0) {
                        E = 1.0;
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
                    ck_st(kp, scr, kp.ext.scr64 - slot, (long long)(2 * lev) * kp.n_slots, st0);
                    ck_st(kp, scr, kp.ext.scr64 - slot, (long long)(2 * lev + 1) * kp.n_slots, st1);
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
                    const double2 st0 = ck_ld(kp, (const double2 *)scr, kp.ext.scr64 - slot, (long long)(2 * lev) * kp.n_slots);
                    const double2 st1 = ck_ld(kp, (const double2 *)scr, kp.ext.scr64 - slot,
                                              (long long)(2 * lev + 1) * kp.n_slots);
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
                // one thread per bin adds its systems in system order; a bin
                // split across chunks is continued by the same CTA after a
                // barrier, with the same sequence of additions
                const int bt = b_lo + tid;
                const int j0 = max(0, bt * NG - s0);
                const int j1 = min(min((int)blockDim.x, ci.S - s0), (bt + 1) * NG - s0);
                double acc = ck_ld(kp, kp.toa, kp.ext.bins, ci.bin0 + bt);
                for (int j = j0; j < j1; ++j) acc += sm.stoa[j];
                ck_st(kp, kp.toa, kp.ext.bins, ci.bin0 + bt, acc);
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
            sl[l] = kt_layer(kp, kp.kt_T, kp.kt_lp, ck_ld(kp, kp.T_center, kp.ext.center, tc0 + l),
                             ck_ld(kp, kp.p_iface, kp.ext.iface, ifi + l), ck_ld(kp, kp.p_iface, kp.ext.iface, ifi + l + 1),
                             S);
        __syncthreads();
        const long long n = (long long)L * S;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int l = (int)(i / S), s = (int)(i - (long long)l * S);
            const float4 l4 = sl[l];
            const Corners k = kt_corners(kp, l4, S, s);
            const Optics o = kt_mix(k.lo, k.hi, l4, __ldg(kp.kt_bin + s / NG));
            ck_st(kp, dtau, kp.ext.cube, base + i, o.dt);
            ck_st(kp, w0, kp.ext.cube, base + i, o.w0);
            ck_st(kp, g0, kp.ext.cube, base + i, o.g0);
        }
    }
}

constexpr int kMaxDynSmem = 200 * 1024;

// Instance SEL: ISO = SEL & 1, staging mode (SEL / 2) % 3, KT = (SEL / 6) & 1,
// NS = (SEL / 12) % 2 + 1, DEP = kBackDepthMin + SEL / 24.
template <int SEL>
constexpr auto units_kernel() {
    return &fp32_units<(SEL & 1) != 0, (SEL / 2) % 3, (SEL / 6) % 2 != 0, (SEL / 12) % 2 + 1, kBackDepthMin + SEL / 24>;
}
constexpr int kUnitsInstances = 24 * (kBackDepthMax - kBackDepthMin + 1);
template <int... I>
std::array<const void *, sizeof...(I)> units_kernels(std::integer_sequence<int, I...>) {
    return {(const void *)units_kernel<I>()...};
}

cudaError_t init_kernels() {
    cudaError_t e = cudaSuccess;
    // every instance of the solve kernel: ISO x staging mode (shared,
    // direct, inline) x KT x systems per lane x back-substitution depth
    for (const void *f : units_kernels(std::make_integer_sequence<int, kUnitsInstances>{})) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    if (e != cudaSuccess) return e;
    for (auto f : {fp32_sweeps<false, false>, fp32_sweeps<true, false>, fp32_sweeps<false, true>,
                   fp32_sweeps<true, true>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(fp64_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

int occupancy(int precision_fp64, int block, size_t smem, int ns, int sweeps) {
    if (smem > (size_t)kMaxDynSmem) return 0;
    int n = 0;
    cudaError_t e = sweeps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp32_sweeps<false, false>, block, smem)
                    : precision_fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp64_columns, block, smem)
                    : ns == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp32_units<false, 0, false, 2, 2>,
                                                                            block, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fp32_units<false, 0, false, 1, 2>,
                                                                            block, smem);
    return e == cudaSuccess ? n : 0;
}

// fp32_units instantiations, indexed by isothermal + 2 stage + 6 k-table + 12 (two systems per lane)
// Launch with programmatic stream serialization: the kernel's CTAs may be
// scheduled while the previous kernel on the stream drains; the kernel
// waits (grid_dependency_wait) before it reads that kernel's output.
template <class... A>
static cudaError_t launch_after_previous(void (*f)(A...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                         const KParams &kp) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, kp);
}

template <int SEL>
void units_launch(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s) {
    launch_after_previous(units_kernel<SEL>(), dim3(grid), dim3(block), smem, s, kp);
}
using UnitsLaunch = void (*)(const KParams &, int, int, size_t, cudaStream_t);
template <int... I>
constexpr std::array<UnitsLaunch, sizeof...(I)> units_table(std::integer_sequence<int, I...>) {
    return {&units_launch<I>...};
}
constexpr auto kUnitsLaunch = units_table(std::make_integer_sequence<int, kUnitsInstances>{});

// the columns' outputs after the unit (or sweep) kernel: one warp per column,
// up to 16 four-warp CTAs per SM
static cudaError_t launch_finalize(const KParams &kp, cudaStream_t s) {
    const int g = (kp.n_cols + 3) / 4, cap = 16 * 148;
    const cudaError_t e = launch_after_previous(fp32_finalize, dim3(g < cap ? g : cap), dim3(128), 0, s, kp);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_fp32(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s,
                        cudaEvent_t const *ev) {
    // pre-kernel: 4-warp CTAs when it tabulates B at every level (more columns in flight),
    // 8-warp CTAs when it forms the T_int row alone (the bins are the parallel work)
    const int pblock = kp.inline_b ? 256 : 128;
    const int pcap = (kp.inline_b ? 4 : 8) * 148;
    const int pgrid = kp.n_cols < pcap ? kp.n_cols : pcap;
    if (ev) cudaEventRecord(ev[0], s);
    const size_t psmem = sizeof(float) * (2 * kp.Lmax + 2) + (kp.kt_lk ? sizeof(double) * (kp.kt_nT + kp.kt_nP) : 0);
    fp32_prep<<<pgrid, pblock, psmem, s>>>(kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    const int st = kp.inline_b ? kStageInline : (kp.direct ? kStageDirect : kStageShared);
    const int dep = kp.back_depth < kBackDepthMin ? kBackDepthMin : kp.back_depth > kBackDepthMax ? kBackDepthMax : kp.back_depth;
    const int sel = (kp.isothermal ? 1 : 0) + 2 * st + (kp.kt_lk ? 6 : 0) + (kp.ns == 2 ? 12 : 0) + 24 * (dep - kBackDepthMin);
    kUnitsLaunch[sel](kp, grid, block, smem, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_finalize(kp, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    return e;
}

cudaError_t launch_sweeps(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s,
                          cudaEvent_t const *ev) {
    const int pgrid = kp.n_cols < 8 * 148 ? kp.n_cols : 8 * 148;
    if (ev) cudaEventRecord(ev[0], s);
    fp32_prep<<<pgrid, 128, sizeof(float) * (2 * kp.Lmax + 2), s>>>(kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    if (kp.isothermal) {
        if (kp.direct) fp32_sweeps<true, true><<<grid, block, smem, s>>>(kp);
        else fp32_sweeps<true, false><<<grid, block, smem, s>>>(kp);
    } else {
        if (kp.direct) fp32_sweeps<false, true><<<grid, block, smem, s>>>(kp);
        else fp32_sweeps<false, false><<<grid, block, smem, s>>>(kp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_finalize(kp, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    return e;
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
