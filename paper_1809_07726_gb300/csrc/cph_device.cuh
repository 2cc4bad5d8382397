// Device-side building blocks of the engine: constants, Philox4x32-10,
// fixed-point helpers and the per-pair arithmetic of the OBC generalized-Born
// model ("igb=2", named in the paper's Implicit Solvent Calculations
// section) with Hawkins-Cramer-Truhlar pairwise descreening.
//
// Pair quantities for atom i and a partner j at distance r:
//   H(r, rt, s)  descreening integral of sphere s (partner's scaled radius)
//                outside the ball rt (this atom's offset radius):
//                0 if rt >= r + s; else with L = max(rt, |r - s|), U = r + s
//                H = 1/L - 1/U + (r/4)(1/U^2 - 1/L^2) + ln(L/U)/(2r)
//                    + (s^2/(4r))(1/L^2 - 1/U^2)  [+ 2(1/rt - 1/L) if rt < s - r]
//   When the spheres are disjoint (L = r - s) H depends on r and x = s/r only:
//   H = (1/r) (x/(1 - x^2) - atanh x) = (1/r) sum_{k>=1} 2k/(2k+1) x^(2k+1).
//   The FP32 path evaluates that series (a degree-5 polynomial in x^2, fitted
//   on the interval) whenever x <= 0.35: it needs no transcendental, and it
//   avoids the cancellation of the closed form (whose terms are O(x) while H
//   is O(x^3)).  The fits stay within 2e-8 relative error.
//   Derivatives: in every branch the L- and U-dependence of H cancels (the
//   integrand vanishes on the moving boundary), so
//     dH/dr  = -(1/4)(1/L^2 - 1/U^2)(1 + s^2/r^2) - ln(L/U)/(2 r^2)
//            = -(1/r^2) sum 2k(2k+2)/(2k+1) x^(2k+1)      (disjoint)
//     dH/ds  = (s/(2r))(1/L^2 - 1/U^2) = (1/r^2) sum 2k x^(2k)
//     dH/drt = ((L - r)^2 - s^2)/(2 r L^3) when L = rt, -2/rt^2 when the ball
//              lies inside sphere s, else 0.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace cph {

// Physical constants (kcal/mol, A, e, amu, ps, K, V).
constexpr double kCoulomb = 332.0522173;   // kcal A / (mol e^2)
constexpr double kBoltzmann = 0.0019872041; // kcal / (mol K)
constexpr double kFaraday = 23.0605;       // kcal / (mol V)
constexpr double kAccel = 418.4;           // (kcal/mol/A)/amu -> A/ps^2
constexpr double kLn10 = 2.302585092994046;

// Fixed-point scales of the int64 accumulators.
constexpr double kScaleE = 4294967296.0;   // energies and forces: 2^32
constexpr double kScaleH = 1099511627776.0; // descreening sums: 2^40

// Random-number purposes (last counter word).
constexpr uint32_t kRngLangevin = 1, kRngMcPh = 2, kRngMcRedox = 3, kRngExchange = 4;

// ------------------------------------------------------------------ Philox
// Philox4x32 with ten rounds (Salmon, Moraes, Dror and Shaw, SC'11).  A round
// multiplies counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57, XORs the
// high product words with counter words 1 and 3 and the key, and permutes;
// between rounds the key advances by the Weyl increments 0x9E3779B9 and
// 0xBB67AE85.
struct U4 {
    uint32_t a, b, c, d;
};

__host__ __device__ inline U4 philox4x32_10(U4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * ctr.a;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * ctr.c;
        U4 n;
        n.a = (uint32_t)(p1 >> 32) ^ ctr.b ^ k0;
        n.b = (uint32_t)p1;
        n.c = (uint32_t)(p0 >> 32) ^ ctr.d ^ k1;
        n.d = (uint32_t)p0;
        ctr = n;
    }
    return ctr;
}

// Counter (index, stream, step low word, purpose | step high bits << 8),
// key (seed low word, seed high word).
__host__ __device__ inline U4 draw(uint64_t seed, uint32_t index, uint32_t stream,
                                   uint64_t step, uint32_t purpose) {
    U4 c{index, stream, (uint32_t)step, (purpose & 0xffu) | ((uint32_t)(step >> 32) << 8)};
    return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// u in (0, 1): u32 * 2^-32 + 2^-33, exact in FP64.
__host__ __device__ inline double unit_open(uint32_t u) {
    return (double)u * 2.3283064365386963e-10 + 1.1641532182693481e-10;
}

// ------------------------------------------------------- salt screening
// A GB term of effective distance f (f = R for a self term) carries
// tau(f) = 1/eps_in - exp(-kappa f)/eps_out; d(tau(f)/f)/df = -taud(f)/f^2 with
// taud(f) = tau(f) - kappa f exp(-kappa f)/eps_out.  kappa = 0: both are the
// constant 1/eps_in - 1/eps_out.
// Without salt both are iei - ieo exactly (exp(-0) = 1): the FP64 exponential,
// slow on GB300's narrow FP64 pipe, is skipped.
__host__ __device__ inline double salt_tau(double f, double iei, double ieo, double kappa) {
    if (!(kappa > 0)) return iei - ieo;
    return iei - exp(-kappa * f) * ieo;
}
__host__ __device__ inline double salt_taud(double f, double iei, double ieo, double kappa) {
    if (!(kappa > 0)) return iei - ieo;
    const double es = exp(-kappa * f) * ieo;
    return iei - es - kappa * f * es;
}

// ------------------------------------------------- nonpolar surface term
// ACE approximation (Schaefer & Karplus 1996): E_SA = 4 pi gamma (rho + probe)^2
// (rho / R)^6 per atom; dE_SA/dR = -6 E_SA / R.  gamma = 0: off.
__host__ __device__ inline double sa_ace(double gamma, double probe, double rho, double R) {
    if (gamma == 0.0) return 0.0;
    const double a = rho + probe, t = rho / R, t3 = t * t * t;
    return 4.0 * 3.14159265358979323846 * gamma * a * a * t3 * t3;
}

// --------------------------------------------------------- fixed point
__device__ inline long long to_fixed(float v, float scale) { return __float2ll_rn(v * scale); }
__device__ inline long long to_fixed(double v, double scale) { return __double2ll_rn(v * scale); }

// ---------------------------------------------- MUFU approximations (FP32)
// The PTX ISA's approximate reciprocal square root and base-2 exponential in
// their flush-to-zero forms (rsqrt.approx.ftz.f32, ex2.approx.ftz.f32), written
// as inline PTX.  No operand of the pair loops comes near the denormal range
// (distances >= ~1 A; exp(-D) underflowing to 0 is harmless), so flushing
// changes no result; accuracy is covered by the parity tests against the
// FP64 oracle.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The PTX ISA's approximate reciprocal (rcp.approx.ftz.f32): 1/r^2 in one MUFU
// operation where the tile needs no 1/r.
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float exp2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ------------------------------------------------------------- HCT, FP32
constexpr float kHctXmax = 0.35f;

// Far-pair polynomials in y = (s/r)^2 on [0, 0.35^2]: degree-5 near-minimax
// fits (Chebyshev, relative error) of the series
//   P(y) = sum 2k/(2k+1) y^(k-1),  Q(y) = sum 2k(2k+2)/(2k+1) y^(k-1),
//   S(y) = sum 2k y^(k-1) = 2/(1-y)^2,
// with max relative errors 3.5e-9, 1.4e-8 and 1.8e-8 (gen_hct_poly.py derives
// the coefficients).
// Packed FP32: one float2 carries the same quantity for two pairs, and
// fma.rn.f32x2 / add / mul (sm_100 and later) work on both halves in one
// instruction.  The helpers below take float or float2 alike.
__device__ __forceinline__ float fma_p(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_p(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class T> __device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ float splat<float>(float v) { return v; }
template <> __device__ __forceinline__ float2 splat<float2>(float v) { return make_float2(v, v); }

template <class T> __device__ __forceinline__ T hct_series_h(T y) { // P
    T p = splat<T>(1.361160215f);
    p = fma_p(p, y, splat<T>(0.8443080909f));
    p = fma_p(p, y, splat<T>(0.8931260308f));
    p = fma_p(p, y, splat<T>(0.8570198603f));
    p = fma_p(p, y, splat<T>(0.8000012903f));
    p = fma_p(p, y, splat<T>(0.6666666645f));
    return p;
}

template <class T> __device__ __forceinline__ T hct_series_dr(T y) { // Q
    T p = splat<T>(20.1395503f);
    p = fma_p(p, y, splat<T>(9.836372412f));
    p = fma_p(p, y, splat<T>(8.959016539f));
    p = fma_p(p, y, splat<T>(6.855114687f));
    p = fma_p(p, y, splat<T>(4.800021136f));
    p = fma_p(p, y, splat<T>(2.666666631f));
    return p;
}

template <class T> __device__ __forceinline__ T hct_series_ds(T y) { // S
    T p = splat<T>(18.77114444f);
    p = fma_p(p, y, splat<T>(8.994253274f));
    p = fma_p(p, y, splat<T>(8.065659941f));
    p = fma_p(p, y, splat<T>(5.998104684f));
    p = fma_p(p, y, splat<T>(4.0000197f));
    p = fma_p(p, y, splat<T>(1.999999967f));
    return p;
}

// Born-radius cutoff rc (AMBER's rgbmax; infinity = none): only shells
// t <= rc descreen, so U = min(r + s, rc), the covered shells of a ball inside
// sphere s end at min(s - r, rc), and H = 0 once L >= U.  The derivative forms
// below hold for a moving or a fixed U alike (the integrand vanishes on the
// moving boundaries), except that the covered-shell term stops moving with r
// and s once capped.  With the ball inside sphere s (L = s - r) the closed
// part's dependence on L cancels that of the covered shells, so dH/dr and
// dH/ds are the closed part's explicit partials alone; once the covered
// shells are capped at rc the closed part is empty and both vanish.
__device__ __forceinline__ bool hct_far(float r, float rt, float s, float rc = INFINITY) {
    return (r - s >= rt) && (s <= kHctXmax * r) && (r + s <= rc);
}

struct HctClosed {
    float iL, iU, lg;
};

__device__ __forceinline__ HctClosed hct_closed(float r, float rt, float s, float rc) {
    float U = fminf(r + s, rc);
    float L = fmaxf(rt, fabsf(r - s));
    float iLU = __fdividef(1.f, L * U);
    HctClosed h;
    h.iL = U * iLU;
    h.iU = L * iLU;
    h.lg = logf(L * h.iU); // accurate log: near pairs dominate psi, keep them to ~1 ulp
    return h;
}

// whether the closed-form part is empty (L >= U)
__device__ __forceinline__ bool hct_empty(float r, float rt, float s, float rc) {
    return fmaxf(rt, fabsf(r - s)) >= fminf(r + s, rc);
}

__device__ __forceinline__ float hct(float r, float rinv, float rt, float irt, float s, float rc = INFINITY) {
    if (hct_far(r, rt, s, rc)) {
        float x = s * rinv, y = x * x;
        return x * y * hct_series_h(y) * rinv;
    }
    float h = 0.f;
    if (!hct_empty(r, rt, s, rc)) {
        HctClosed c = hct_closed(r, rt, s, rc);
        h = (c.iL - c.iU) * fmaf((c.iL + c.iU) * 0.25f * rinv, (s - r) * (s + r), 1.f) + 0.5f * rinv * c.lg;
    }
    if (rt < s - r) {
        const float top = fminf(s - r, rc);
        if (rt < top) h += 2.f * (irt - __fdividef(1.f, top));
    }
    return h;
}

__device__ __forceinline__ float hct_dr(float r, float rinv, float rt, float s, float rc = INFINITY) {
    float rinv2 = rinv * rinv;
    if (hct_far(r, rt, s, rc)) {
        float x = s * rinv, y = x * x;
        return -x * y * hct_series_dr(y) * rinv2;
    }
    float d = 0.f;
    if (!hct_empty(r, rt, s, rc)) {
        HctClosed c = hct_closed(r, rt, s, rc);
        d = -0.25f * (c.iL - c.iU) * (c.iL + c.iU) * fmaf(s * s, rinv2, 1.f) - 0.5f * c.lg * rinv2;
    }
    return d;
}

// dH/dr with the fast logarithm (__logf) in the closed form: the chain-rule
// force of a near pair, where the log term is O(1) and its ~1e-7 absolute
// error stays far below the force bar.
__device__ __forceinline__ float hct_dr_fastlog(float r, float rinv, float rt, float s, float rc = INFINITY) {
    float rinv2 = rinv * rinv;
    if (hct_far(r, rt, s, rc)) {
        float x = s * rinv, y = x * x;
        return -x * y * hct_series_dr(y) * rinv2;
    }
    float d = 0.f;
    if (!hct_empty(r, rt, s, rc)) {
        const float U = fminf(r + s, rc), L = fmaxf(rt, fabsf(r - s));
        const float iLU = __fdividef(1.f, L * U), iL = U * iLU, iU = L * iLU;
        d = -0.25f * (iL - iU) * (iL + iU) * fmaf(s * s, rinv2, 1.f) - 0.5f * __logf(L * iU) * rinv2;
    }
    return d;
}

__device__ __forceinline__ float hct_ds(float r, float rinv, float rt, float s, float rc = INFINITY) {
    if (hct_far(r, rt, s, rc)) {
        float x = s * rinv, y = x * x;
        return y * hct_series_ds(y) * rinv * rinv;
    }
    float d = 0.f;
    if (!hct_empty(r, rt, s, rc)) {
        HctClosed c = hct_closed(r, rt, s, rc);
        d = 0.5f * s * rinv * (c.iL - c.iU) * (c.iL + c.iU);
    }
    return d;
}

__device__ __forceinline__ float hct_drt(float r, float rt, float irt, float s, float rc = INFINITY) {
    if (hct_far(r, rt, s, rc)) return 0.f;
    float d = 0.f;
    if (rt < s - r) {
        if (rt < fminf(s - r, rc)) d = -2.f * irt * irt;
    } else if (rt > fabsf(r - s) && !hct_empty(r, rt, s, rc)) {
        float a = rt - r;
        d = (a * a - s * s) * 0.5f * __fdividef(1.f, r) * irt * irt * irt;
    }
    return d;
}

// ------------------------------------------------------------- HCT, FP64
// Closed forms throughout (FP64 has no cancellation problem at these sizes);
// rc as above (infinity = no cutoff).
__device__ __forceinline__ double hct(double r, double rinv, double rt, double irt, double s, double rc = INFINITY) {
    const double U = fmin(r + s, rc), L = fmax(rt, fabs(r - s));
    double h = 0.0;
    if (L < U) {
        double iL = 1.0 / L, iU = 1.0 / U;
        h = (iL - iU) * (1.0 + (iL + iU) * 0.25 * rinv * (s - r) * (s + r)) + 0.5 * rinv * log(L * iU);
    }
    if (rt < s - r) {
        const double top = fmin(s - r, rc);
        if (rt < top) h += 2.0 * (irt - 1.0 / top);
    }
    return h;
}

__device__ __forceinline__ double hct_dr(double r, double rinv, double rt, double s, double rc = INFINITY) {
    const double U = fmin(r + s, rc), L = fmax(rt, fabs(r - s));
    double d = 0.0;
    if (L < U) {
        double iL = 1.0 / L, iU = 1.0 / U;
        double rinv2 = rinv * rinv;
        d = -0.25 * (iL - iU) * (iL + iU) * (1.0 + s * s * rinv2) - 0.5 * log(L * iU) * rinv2;
    }
    return d;
}

__device__ __forceinline__ double hct_ds(double r, double rinv, double rt, double s, double rc = INFINITY) {
    const double U = fmin(r + s, rc), L = fmax(rt, fabs(r - s));
    double d = 0.0;
    if (L < U) {
        double iL = 1.0 / L, iU = 1.0 / U;
        d = 0.5 * s * rinv * (iL - iU) * (iL + iU);
    }
    return d;
}

__device__ __forceinline__ double hct_drt(double r, double rt, double irt, double s, double rc = INFINITY) {
    const double U = fmin(r + s, rc), L = fmax(rt, fabs(r - s));
    if (rt < s - r) return rt < fmin(s - r, rc) ? -2.0 * irt * irt : 0.0;
    if (rt > fabs(r - s) && L < U) {
        double a = rt - r;
        return (a * a - s * s) * 0.5 / r * irt * irt * irt;
    }
    return 0.0;
}

// ------------------------------------------------- compensated summation
// Kahan summation of a tile's partial energies: the energy sums cancel
// strongly (sum |terms| >> |E|), so plain FP32 partials over a 128-atom tile
// would lose ~1e-6 of |E|.  FP64 needs no compensation.
template <class Real>
struct KSum {
    Real s = 0, c = 0;
    __device__ __forceinline__ void add(Real v) {
        const Real y = v - c;
        const Real t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ Real value() const { return s; }
};

template <>
struct KSum<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

// ------------------------------------------------------ precision traits
template <class Real>
struct Prec;

template <>
struct Prec<float> {
    using Acc = long long; // int64 fixed point
    __device__ static float rsqrt(float x) { return rsqrtf(x); }
    __device__ static float expm(float x) { return __expf(-x); } // e^-x
    __device__ static float recip(float x) { return __fdividef(1.f, x); }
    __device__ static void add(Acc& a, float part, float scale) { a += to_fixed(part, scale); }
    __device__ static double value(Acc a, double scale) { return (double)a / scale; }
};

template <>
struct Prec<double> {
    using Acc = double;
    __device__ static double rsqrt(double x) { return 1.0 / sqrt(x); }
    __device__ static double expm(double x) { return exp(-x); }
    __device__ static double recip(double x) { return 1.0 / x; }
    __device__ static void add(Acc& a, double part, double) { a += part; }
    __device__ static double value(Acc a, double) { return a; }
};

} // namespace cph
