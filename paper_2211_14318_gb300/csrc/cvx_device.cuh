// cvx_device.cuh -- device building blocks of the per-point convexification:
// the material law in FP64 (node and leaf evaluation) and in FP32 line form
// (sampling), shared by the kernels of this library only.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "convexify.h"

namespace cvx {

constexpr float kU32 = 5.9604644775390625e-8f;  // unit roundoff of FP32, 2^-24
constexpr float kLn2 = 0.693147180559945309f;
constexpr double kLn2d = 0.693147180559945309417232;
constexpr double kLog2e = 1.442695040888963407359924;

// Material constants in FP64 (one per call).
struct Material {
    double mu, lam, Dinf, D0;
    int energy;
};

// -------------------------------------------------------------------------
// FP64 energy at a point, plane strain (Eqs. 2.1-2.9) and stress (Eq. 2.12).
// W is written through the closed form of Eq. (2.9) in s = psi0(F):
//   s <= beta_k : W = (1 - D(beta_k)) (s - beta_k)
//   s >  beta_k : W = (1 - D_inf)(s - beta_k) + D_inf D_0 (e^{-beta_k/D_0} - e^{-s/D_0})
// and dW/ds = 1 - D(max(s, beta_k)).
// -------------------------------------------------------------------------
__host__ __device__ inline double psi0_nh64(const double F[4], const Material &m, double *lnJ,
                                            double *J) {
    double j = F[0] * F[3] - F[1] * F[2];
    double i1 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3] + 1.0;
    double lj = log(j);
    *lnJ = lj;
    *J = j;
    return 0.5 * m.mu * (i1 - 3.0) - m.mu * lj + 0.5 * m.lam * lj * lj;
}

__host__ __device__ inline double energy64(const double F[4], double beta_k, const Material &m) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        double a = F[0] * F[0] - 1.0, d = F[3] - 1.0;
        return a * a + F[1] * F[1] + F[2] * F[2] + d * d;
    }
    double lj, J;
    double s = psi0_nh64(F, m, &lj, &J);
    if (!(J > 0.0)) return nan("");
    if (s <= beta_k) return (1.0 - m.Dinf * (1.0 - exp(-beta_k / m.D0))) * (s - beta_k);
    return (1.0 - m.Dinf) * (s - beta_k) + m.Dinf * m.D0 * (exp(-beta_k / m.D0) - exp(-s / m.D0));
}

__host__ __device__ inline void stress64(const double F[4], double beta_k, const Material &m,
                                         double P[4]) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        P[0] = 4.0 * F[0] * (F[0] * F[0] - 1.0);
        P[1] = 2.0 * F[1];
        P[2] = 2.0 * F[2];
        P[3] = 2.0 * (F[3] - 1.0);
        return;
    }
    double lj, J;
    double s = psi0_nh64(F, m, &lj, &J);
    if (!(J > 0.0)) {
        P[0] = P[1] = P[2] = P[3] = nan("");
        return;
    }
    double beta = s > beta_k ? s : beta_k;
    double g = 1.0 - m.Dinf * (1.0 - exp(-beta / m.D0));
    double iJ = 1.0 / J;
    double FiT[4] = {F[3] * iJ, -F[2] * iJ, -F[1] * iJ, F[0] * iJ};  // F^{-T}
    for (int k = 0; k < 4; ++k) P[k] = g * (m.mu * (F[k] - FiT[k]) + m.lam * lj * FiT[k]);
}

// Tangent d^2 W / dF dF in FP64 (Eq. 2.12 differentiated once more), as a
// 4 x 4 matrix over the row-major entries of F: A[4 a + b] = dP_a / dF_b.
// With s = psi0(F), g = dW/ds = 1 - D(max(s, beta_k)), and on loading
// (s > beta_k) dg/ds = -D'(s) = -(D_inf / D_0) e^{-s/D_0}:
//   A = g d^2psi0/dF^2 + dg/ds (dpsi0/dF) (x) (dpsi0/dF),
//   dpsi0/dF = mu F + (lam ln J - mu) F^{-T},
//   d^2psi0 / dF_aA dF_bB = mu d_ab d_AB + lam G_aA G_bB + (mu - lam ln J) G_aB G_bA,
// G = F^{-T} (d G_aA / dF_bB = -G_aB G_bA, d ln J / dF = G).
__device__ inline void tangent64(const double F[4], double beta_k, const Material &m,
                                 double A[16]) {
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        for (int k = 0; k < 16; ++k) A[k] = 0.0;
        A[0] = 12.0 * F[0] * F[0] - 4.0;
        A[5] = A[10] = A[15] = 2.0;
        return;
    }
    double lj, J;
    const double s = psi0_nh64(F, m, &lj, &J);
    if (!(J > 0.0)) {
        for (int k = 0; k < 16; ++k) A[k] = nan("");
        return;
    }
    const double beta = s > beta_k ? s : beta_k;
    const double g = 1.0 - m.Dinf * (1.0 - exp(-beta / m.D0));
    const double dg = s > beta_k ? -(m.Dinf / m.D0) * exp(-s / m.D0) : 0.0;
    const double iJ = 1.0 / J;
    // G = F^{-T} in row-major entries: G_11 = F22/J, G_12 = -F21/J, G_21 = -F12/J, G_22 = F11/J
    const double G[4] = {F[3] * iJ, -F[2] * iJ, -F[1] * iJ, F[0] * iJ};
    const double c = m.mu - m.lam * lj;
    double dp[4];
    for (int k = 0; k < 4; ++k) dp[k] = m.mu * F[k] - c * G[k];
    for (int a = 0; a < 2; ++a)
        for (int aa = 0; aa < 2; ++aa)
            for (int b = 0; b < 2; ++b)
                for (int bb = 0; bb < 2; ++bb) {
                    const int r = 2 * a + aa, q = 2 * b + bb;
                    const double d2 = (a == b && aa == bb ? m.mu : 0.0) + m.lam * G[r] * G[q] +
                                      c * G[2 * a + bb] * G[2 * b + aa];
                    A[4 * r + q] = g * d2 + dg * dp[r] * dp[q];
                }
}

// -------------------------------------------------------------------------
// FP64 line function g(t) = W(F + t R) with g' and g'' in closed form, for the
// common-tangent refinement of a split.  Along the line
//   I1' = 2 G:R, I1'' = 2 |R|^2, J' = cof G : R, J'' = 2 det R,
//   s'  = mu/2 I1' + (lam ln J - mu) J'/J,
//   s'' = mu/2 I1'' + lam (J'/J)^2 + (lam ln J - mu)(J''/J - (J'/J)^2),
// and with dW/ds = 1 - D(max(s, beta_k)), d^2W/ds^2 = -D'(s) [s > beta_k]:
//   g' = W_s s',  g'' = W_ss s'^2 + W_s s''.
// -------------------------------------------------------------------------
__device__ inline void line_derivs64(const double F[4], const double R[4], double beta_k,
                                     const Material &m, double t, double *g, double *g1,
                                     double *g2) {
    double G[4];
    for (int k = 0; k < 4; ++k) G[k] = F[k] + t * R[k];
    if (m.energy == CVX_ENERGY_DOUBLE_WELL) {
        const double a = G[0] * G[0] - 1.0, d = G[3] - 1.0;
        *g = a * a + G[1] * G[1] + G[2] * G[2] + d * d;
        *g1 = 4.0 * G[0] * a * R[0] + 2.0 * (G[1] * R[1] + G[2] * R[2] + d * R[3]);
        *g2 = (12.0 * G[0] * G[0] - 4.0) * R[0] * R[0] +
              2.0 * (R[1] * R[1] + R[2] * R[2] + R[3] * R[3]);
        return;
    }
    const double J = G[0] * G[3] - G[1] * G[2];
    if (!(J > 0.0)) {
        *g = *g1 = *g2 = nan("");
        return;
    }
    const double lj = log(J);
    const double I1 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2] + G[3] * G[3] + 1.0;
    const double s = 0.5 * m.mu * (I1 - 3.0) - m.mu * lj + 0.5 * m.lam * lj * lj;
    const double dI1 = 2.0 * (G[0] * R[0] + G[1] * R[1] + G[2] * R[2] + G[3] * R[3]);
    const double ddI1 = 2.0 * (R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + R[3] * R[3]);
    const double dJ = G[3] * R[0] - G[2] * R[1] - G[1] * R[2] + G[0] * R[3];
    const double ddJ = 2.0 * (R[0] * R[3] - R[1] * R[2]);
    const double q = dJ / J;
    const double c = m.lam * lj - m.mu;
    const double s1 = 0.5 * m.mu * dI1 + c * q;
    const double s2 = 0.5 * m.mu * ddI1 + m.lam * q * q + c * (ddJ / J - q * q);
    const double ek = exp(-beta_k / m.D0);
    double Ws, Wss;
    if (s <= beta_k) {
        Ws = 1.0 - m.Dinf * (1.0 - ek);
        Wss = 0.0;
        *g = Ws * (s - beta_k);
    } else {
        const double es = exp(-s / m.D0);
        Ws = 1.0 - m.Dinf * (1.0 - es);
        Wss = -m.Dinf / m.D0 * es;
        *g = (1.0 - m.Dinf) * (s - beta_k) + m.Dinf * m.D0 * (ek - es);
    }
    *g1 = Ws * s1;
    *g2 = Wss * s1 * s1 + Ws * s2;
}

// Newton on the common-tangent conditions of a split (t-, t+) along R,
//   g'(t-) = g'(t+) = (g(t+) - g(t-)) / (t+ - t-),
// written as f1 = g'(t-) - g'(t+), f2 = g'(t-)(t+ - t-) - (g(t+) - g(t-)),
// seeded by the grid bridge, at most 8 iterations.  Returns true, with the
// refined ends and the chord value at 0, only if it converged inside the
// line window, det > 0 at both ends and the chord value is not above h_grid.
__device__ inline bool newton_tangent64(const double F[4], const double R[4], double beta_k,
                                        const Material &m, double t_half, double h_grid,
                                        double &tm, double &tp, double &h) {
    double a = tm, b = tp;
    bool conv = false;
    for (int it = 0; it < 8 && !conv; ++it) {
        double ga, ga1, ga2, gb, gb1, gb2;
        line_derivs64(F, R, beta_k, m, a, &ga, &ga1, &ga2);
        line_derivs64(F, R, beta_k, m, b, &gb, &gb1, &gb2);
        const double f1 = ga1 - gb1, f2 = ga1 * (b - a) - (gb - ga);
        const double j11 = ga2, j12 = -gb2, j21 = ga2 * (b - a), j22 = ga1 - gb1;
        const double det = j11 * j22 - j12 * j21;
        if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
        const double da = (j12 * f2 - j22 * f1) / det;
        const double db = (j21 * f1 - j11 * f2) / det;
        a += da;
        b += db;
        if (!isfinite(a) || !isfinite(b)) return false;
        conv = fabs(da) <= 1e-13 * (1.0 + fabs(a)) && fabs(db) <= 1e-13 * (1.0 + fabs(b));
    }
    if (!conv || !(a >= -t_half && a < 0.0 && b > 0.0 && b <= t_half)) return false;
    double ga, gb, d1, d2;
    line_derivs64(F, R, beta_k, m, a, &ga, &d1, &d2);
    line_derivs64(F, R, beta_k, m, b, &gb, &d1, &d2);
    if (!isfinite(ga) || !isfinite(gb)) return false;
    const double hc = ga + (gb - ga) * (-a / (b - a));
    if (!(hc <= h_grid)) return false;
    tm = a;
    tp = b;
    h = hc;
    return true;
}

// -------------------------------------------------------------------------
// FP32 line form.  Along G(t) = F + t R with R = a (x) b rank one:
//   I1(t) - 3 = |F|^2 - 2 + 2 t (F:R) + t^2 |R|^2,   J(t) = J0 + t (cof F : R).
// With lg = log2 J(t) and d = psi0(t) - beta_k:
//   d = A0 + A1 t + A2 t^2 + lg (B1 + B2 lg),
//   A0 = mu/2 (|F|^2 - 2) - beta_k, A1 = mu F:R, A2 = mu/2 |R|^2,
//   B1 = -mu ln2, B2 = lam/2 ln2^2,
// and the two branches of Eq. (2.9) become, with e_k = exp(-beta_k/D_0),
//   W = (1 - D_inf) d + K1 (1 - exp(-max(d, 0)/D_0)) + K2 min(d, 0),
//   K1 = D_inf D_0 e_k, K2 = D_inf e_k
// (d <= 0 gives (1 - D_inf + D_inf e_k) d = (1 - D(beta_k)) d; d > 0 gives
// (1 - D_inf)(s - beta_k) + D_inf D_0 (e_k - e^{-s/D_0})).  The kernels sample
//   v = kappa' W - C,  kappa' = kappa / (1 - D_inf),  kappa = log2(e) / D_0,
//   C = kappa D_inf D_0 e_k / (1 - D_inf)          (per point),
// i.e. with d scaled by kappa (so that the exponential is one ex2 of
// -max(d, 0)) and the whole divided by 1 - D_inf:
//   v = d + K2' min(d, 0) - K1' 2^{-max(d, 0)},  K1' = C,  K2' = K2 / (1 - D_inf).
// A positive factor and a per-point constant change no hull or direction
// decision; values are mapped back by W = (v + C) / kappa'.  J <= 0 yields
// +inf or NaN, which the hull search ignores.
// -------------------------------------------------------------------------
struct __align__(16) NodeLine {
    float F[4];  // first, so that F and cof F are two 16-byte loads
    float cof[4];
    float A0, B1, B2, K1, K2, mu;  // kappa-scaled (K2 is a ratio)
    float J0;
};

struct DirLine {
    float A1, A2, cJ, J0;  // NH
    float c[5];            // double well: W(t) = sum c_i t^i
};

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic: two independent FP32 values in a 64-bit register
// pair, one fma.rn.f32x2 computing both (each an IEEE fma with round to
// nearest, so results equal the scalar __fmaf_rn ones).  Used by the
// certification pass of the hull search; the sampler stays scalar (measured
// faster inside the full line scan).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float x, float y) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// min of three FP32 values (a NaN operand is ignored, as by fminf)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Warp-wide minimum of FP32 values (one redux.sync; NaN operands are ignored,
// -0 < +0 as for min.f32).
__device__ __forceinline__ float warp_min_f32(float x) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(x));
    return r;
}

// Sample scale kappa' (v = kappa' W - C): log2(e) / (D_0 (1 - D_inf)) for the
// damage energy, 1 for the test energy.
__host__ __device__ inline double line_kappa(const Material &m) {
    return m.energy == CVX_ENERGY_NH_DAMAGE ? kLog2e / (m.D0 * (1.0 - m.Dinf)) : 1.0;
}

// Sample shift C of a point with history beta_k (0 for the test energy).
__host__ __device__ inline double line_shift(const Material &m, double beta_k) {
    if (m.energy != CVX_ENERGY_NH_DAMAGE) return 0.0;
    return kLog2e * m.Dinf * exp(-beta_k / m.D0) / (1.0 - m.Dinf);
}

// Node constants from F (FP64) and beta_k, rounded to FP32.
__device__ inline NodeLine make_node_line(const double F[4], double beta_k, const Material &m) {
    NodeLine nl;
    const double kap = m.energy == CVX_ENERGY_NH_DAMAGE ? kLog2e / m.D0 : 1.0;
    const double a1 = 1.0 - m.Dinf;
    double fsq = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    double ek = exp(-beta_k / m.D0);
    nl.A0 = (float)(kap * (0.5 * m.mu * (fsq - 2.0) - beta_k));
    nl.B1 = (float)(kap * (-m.mu * kLn2d));
    nl.B2 = (float)(kap * (0.5 * m.lam * kLn2d * kLn2d));
    nl.K1 = (float)line_shift(m, beta_k);
    nl.K2 = (float)(m.Dinf * ek / a1);
    nl.mu = (float)(kap * m.mu);
    nl.J0 = (float)(F[0] * F[3] - F[1] * F[2]);
    for (int k = 0; k < 4; ++k) nl.F[k] = (float)F[k];
    nl.cof[0] = (float)F[3];
    nl.cof[1] = (float)(-F[2]);
    nl.cof[2] = (float)(-F[1]);
    nl.cof[3] = (float)F[0];
    return nl;
}

template <int EK>
__device__ __forceinline__ DirLine make_dir_line(const NodeLine &nl, float4 d) {
    DirLine dl;
    // R = a (x) b, a = (d.x, d.y), b = (d.z, d.w)
    float R0 = d.x * d.z, R1 = d.x * d.w, R2 = d.y * d.z, R3 = d.y * d.w;
    if (EK == CVX_ENERGY_NH_DAMAGE) {
        float c1 = nl.F[0] * R0 + nl.F[1] * R1 + nl.F[2] * R2 + nl.F[3] * R3;
        float cJ = nl.cof[0] * R0 + nl.cof[1] * R1 + nl.cof[2] * R2 + nl.cof[3] * R3;
        float rr = (d.x * d.x + d.y * d.y) * (d.z * d.z + d.w * d.w);
        dl.A1 = nl.mu * c1;
        dl.A2 = 0.5f * nl.mu * rr;
        dl.cJ = cJ;
        dl.J0 = nl.J0;
    } else {
        // (G11^2 - 1)^2 + G12^2 + G21^2 + (G22 - 1)^2 as a quartic in t
        float q0 = nl.F[0] * nl.F[0] - 1.0f, q1 = 2.0f * nl.F[0] * R0, q2 = R0 * R0;
        float g22 = nl.F[3] - 1.0f;
        dl.c[0] = q0 * q0 + nl.F[1] * nl.F[1] + nl.F[2] * nl.F[2] + g22 * g22;
        dl.c[1] = 2.0f * q0 * q1 + 2.0f * (nl.F[1] * R1 + nl.F[2] * R2 + g22 * R3);
        dl.c[2] = q1 * q1 + 2.0f * q0 * q2 + R1 * R1 + R2 * R2 + R3 * R3;
        dl.c[3] = 2.0f * q1 * q2;
        dl.c[4] = q2 * q2;
    }
    return dl;
}

// One FP32 sample of v = kappa' W - C at parameter t: 9 FP32-pipe
// instructions and 2 MUFU for the damage energy.
template <int EK>
__device__ __forceinline__ float sample_w(const NodeLine &nl, const DirLine &dl, float t) {
    if (EK == CVX_ENERGY_NH_DAMAGE) {
        const float p = __fmaf_rn(t, __fmaf_rn(t, dl.A2, dl.A1), nl.A0);
        const float J = __fmaf_rn(t, dl.cJ, dl.J0);
        const float lg = lg2_approx(J);
        const float d = __fmaf_rn(lg, __fmaf_rn(lg, nl.B2, nl.B1), p);
        const float e = ex2_approx(-fmaxf(d, 0.0f));
        const float w = __fmaf_rn(nl.K2, fminf(d, 0.0f), d);
        return __fmaf_rn(-nl.K1, e, w);
    } else {
        float w = __fmaf_rn(dl.c[4], t, dl.c[3]);
        w = __fmaf_rn(w, t, dl.c[2]);
        w = __fmaf_rn(w, t, dl.c[1]);
        return __fmaf_rn(w, t, dl.c[0]);
    }
}

// Slope of v along a line at t = 0, per sample step: sl = sa (A1 + cb cJ)
// with, at the node (d0 = d(0), lg0 = log2 J0),
//   dd/dt(0) = A1 + cJ (B1 + 2 B2 lg0) / (J0 ln 2),
//   dv/dd(d0) = 1 + K2' (d0 < 0),  1 + K1' ln 2 2^{-d0} (d0 >= 0),
//   sa = h dv/dd(d0),  cb = (B1 + 2 B2 lg0) / (J0 ln 2).
// Used only to pick the slope of a rigorous lower bound (any slope gives
// one), so its own rounding does not matter.
__device__ inline void center_slope_consts(const NodeLine &nl, double h, float &sa, float &cb) {
    const double J0 = nl.J0, lg0 = J0 > 0.0 ? log2(J0) : 0.0;
    const double d0 = (double)nl.A0 + lg0 * ((double)nl.B1 + (double)nl.B2 * lg0);
    const double dv = d0 < 0.0 ? 1.0 + (double)nl.K2 : 1.0 + (double)nl.K1 * kLn2d * exp2(-d0);
    sa = (float)(h * dv);
    cb = J0 > 0.0 ? (float)(((double)nl.B1 + 2.0 * (double)nl.B2 * lg0) / (J0 * kLn2d)) : 0.0f;
}

// The constants of sample_w<NH> duplicated into register pairs (the node's
// from nh_pair_node, the direction's from the line scan's shared table), and
// two samples at the parameters in T: every FMA of sample_w is one half of a
// fma.rn.f32x2 (so each component is rounded exactly as sample_w rounds it);
// the MUFU operations and the clamps stay scalar.
struct NHPair {
    f32x2 A0, A1, A2, B1, B2, K2, NK1, CJ, J0;
};
__device__ __forceinline__ NHPair nh_pair_node(const NodeLine &nl) {
    NHPair c;
    c.A0 = pk2(nl.A0, nl.A0);
    c.B1 = pk2(nl.B1, nl.B1);
    c.B2 = pk2(nl.B2, nl.B2);
    c.K2 = pk2(nl.K2, nl.K2);
    c.NK1 = pk2(-nl.K1, -nl.K1);
    c.A1 = c.A2 = c.CJ = c.J0 = c.A0;
    return c;
}
__device__ __forceinline__ f32x2 sample_nh2(const NHPair &c, f32x2 T) {
    const f32x2 P = fma2(T, fma2(T, c.A2, c.A1), c.A0);
    float j0, j1;
    upk2(fma2(T, c.CJ, c.J0), j0, j1);
    const f32x2 LG = pk2(lg2_approx(j0), lg2_approx(j1));
    const f32x2 D = fma2(LG, fma2(LG, c.B2, c.B1), P);
    float d0, d1;
    upk2(D, d0, d1);
    const f32x2 E = pk2(ex2_approx(-fmaxf(d0, 0.0f)), ex2_approx(-fmaxf(d1, 0.0f)));
    const f32x2 W = fma2(c.K2, pk2(fminf(d0, 0.0f), fminf(d1, 0.0f)), D);
    return fma2(c.NK1, E, W);
}

// energy64 of the damage energy with the node's e_k = exp(-beta_k / D_0)
// precomputed (the same operations on the same values: bit-identical).
__device__ inline double energy64_ek(const double F[4], double beta_k, double ek,
                                     const Material &m) {
    double lj, J;
    double s = psi0_nh64(F, m, &lj, &J);
    if (!(J > 0.0)) return nan("");
    if (s <= beta_k) return (1.0 - m.Dinf * (1.0 - ek)) * (s - beta_k);
    return (1.0 - m.Dinf) * (s - beta_k) + m.Dinf * m.D0 * (ek - exp(-s / m.D0));
}

// FP64 sample of W along the line: G = F + t R with t = (m - m0) h and R, G
// rounded exactly as the split points are (no contraction).
__device__ __forceinline__ double sample_w64(const double F[4], const double R[4], int m, int m0,
                                             double h, double beta_k, const Material &mat) {
    const double t = __dmul_rn((double)(m - m0), h);
    double G[4];
    for (int k = 0; k < 4; ++k) G[k] = __dadd_rn(F[k], __dmul_rn(t, R[k]));
    return energy64(G, beta_k, mat);
}

// sample_w64 of the damage energy with e_k precomputed (bit-identical).
__device__ __forceinline__ double sample_w64_ek(const double F[4], const double R[4], int m, int m0,
                                                double h, double beta_k, double ek,
                                                const Material &mat) {
    const double t = __dmul_rn((double)(m - m0), h);
    double G[4];
    for (int k = 0; k < 4; ++k) G[k] = __dadd_rn(F[k], __dmul_rn(t, R[k]));
    return energy64_ek(G, beta_k, ek, mat);
}

}  // namespace cvx
