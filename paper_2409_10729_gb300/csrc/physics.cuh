// physics.cuh -- device-side arithmetic of the five-equation RHS.
//
// Stiffened-gas mixture EOS (arXiv 2409.10729, Sec. II-A), WENO5-JS face
// reconstruction and the HLLC flux (Sec. II-B, last paragraph), written for
// the GB300 FP64 and FP32 pipes.  The formulas are the same as the serial
// oracle's, reorganised to spend fewer divisions, which are the expensive
// operations on this part:
//   * WENO weights in product form: omega_k ~ d_k * prod_{j != k} (eps+beta_j)^2,
//     so each face value costs one division instead of six (FP64), or
//     min-normalised reciprocals that cannot overflow (FP32);
//   * candidate stencils multiplied by 1/6 instead of divided by 6;
//   * the HLLC star energy uses one reciprocal 1/(S_K - S*) for both chi_K
//     and the p_K/(S_K - u_K) term.
// Results agree with the oracle to rounding, not bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mfc5 {

// Stiffened-gas mixture constants of N fluids (N <= kMaxFluids), with
// g_i = 1/(gamma_i - 1) and P_i = gamma_i pi_i / (gamma_i - 1):
//   Gamma = sum_i alpha_i g_i = g_N + sum_{i<N} alpha_i (g_i - g_N),
//   Pi    = sum_i alpha_i P_i = P_N + sum_{i<N} alpha_i (P_i - P_N),
// alpha_N = 1 - sum_{i<N} alpha_i.  dg/dP hold g_i - g_N, P_i - P_N (i < N).
constexpr int kMaxFluids = 4;
struct Eos {
    double g[kMaxFluids], P[kMaxFluids];
    double dg[kMaxFluids - 1], dP[kMaxFluids - 1];
    // the same constants rounded to FP32 (on the host), so that the FP32 forms
    // read them without a conversion on GB300's narrow FP64 pipe
    float g32[kMaxFluids], P32[kMaxFluids];
    float dg32[kMaxFluids - 1], dP32[kMaxFluids - 1];
    int nf;
};

// Field layout of an N-fluid state: alpha_i rho_i (i < N), rho u_k, rho E,
// alpha_1 .. alpha_{N-1}.  For two fluids: alpha1 rho1, alpha2 rho2, rho u_k,
// rho E, alpha1 (NEQ = NDIM + 4).
template <int NDIM, int NF = 2>
struct Fields {
    static constexpr int NEQ = 2 * NF + NDIM;
    static constexpr int IU = NF;             // first momentum / velocity
    static constexpr int IE = NF + NDIM;      // energy / pressure
    static constexpr int IA = NF + NDIM + 1;  // alpha_1 (alpha_2 .. alpha_{N-1} follow)
    static constexpr int NA = NF - 1;         // carried volume fractions
};

// Comparisons of FP64 values on the integer pipes, from the two 32-bit words
// of each operand (GB300's narrow FP64 pipe also executes the FP64 compare
// instruction).  The answers are the IEEE compares': false when an operand
// is a NaN, and -0 equal to +0.
__device__ __forceinline__ bool is_nan_w(unsigned h, unsigned l) {
    const unsigned m = h & 0x7fffffffu;
    return m > 0x7ff00000u || (m == 0x7ff00000u && l != 0u);
}

// x > 0
__device__ __forceinline__ bool gt0(double x) {
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    return (h >> 31) == 0u && (h | l) != 0u && !is_nan_w(h, l);
}

// 0 <= x
__device__ __forceinline__ bool ge0(double x) {
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    return ((h >> 31) == 0u && !is_nan_w(h, l)) || (h == 0x80000000u && l == 0u);
}

// a < b
__device__ __forceinline__ bool less(double a, double b) {
    const unsigned ha = (unsigned)__double2hiint(a), la = (unsigned)__double2loint(a);
    const unsigned hb = (unsigned)__double2hiint(b), lb = (unsigned)__double2loint(b);
    const unsigned ma = ha & 0x7fffffffu, mb = hb & 0x7fffffffu;
    const bool lt_mag = ma < mb || (ma == mb && la < lb);   // |a| < |b|
    const bool gt_mag = mb < ma || (ma == mb && lb < la);   // |a| > |b|
    const bool zeros = (ma | la | mb | lb) == 0u;
    const unsigned sa = ha >> 31, sb = hb >> 31;
    const bool r = sa == 0u ? (sb == 0u && lt_mag) : (sb == 0u ? !zeros : gt_mag);
    return r && !is_nan_w(ha, la) && !is_nan_w(hb, lb);
}

template <typename R>
__device__ __forceinline__ bool pos(R x) {
    if constexpr (sizeof(R) == 8) return gt0(x);
    else return x > R(0);
}
template <typename R>
__device__ __forceinline__ bool nonneg(R x) {
    if constexpr (sizeof(R) == 8) return ge0(x);
    else return R(0) <= x;
}
template <typename R>
__device__ __forceinline__ bool lt(R a, R b) {
    if constexpr (sizeof(R) == 8) return less(a, b);
    else return a < b;
}

// Mixture density of the partial densities w[0..NF-1].
template <int NF, typename R>
__device__ __forceinline__ R mix_rho(const R* w) {
    R rho = w[0] + w[1];
#pragma unroll
    for (int i = 2; i < NF; ++i) rho = rho + w[i];
    return rho;
}

template <typename R>
__device__ __forceinline__ R rdiv(R a, R b) { return a / b; }

template <typename R>
__device__ __forceinline__ R sqrt_pos(R x) { return sqrt(x); }

// EOS constants in the working precision R (converted once per thread, so the
// FP32 path issues no FP64 conversions per face).
template <typename R, int NF = 2>
struct EosR {
    R dg[NF - 1], gN, dP[NF - 1], PN;
    __device__ __forceinline__ explicit EosR(const Eos& e) {
        if constexpr (sizeof(R) == 4) {
            gN = e.g32[NF - 1];
            PN = e.P32[NF - 1];
        } else {
            gN = R(e.g[NF - 1]);
            PN = R(e.P[NF - 1]);
        }
#pragma unroll
        for (int i = 0; i < NF - 1; ++i) {
            if constexpr (sizeof(R) == 4) {
                dg[i] = e.dg32[i];
                dP[i] = e.dP32[i];
            } else {
                dg[i] = R(e.dg[i]);
                dP[i] = R(e.dP[i]);
            }
        }
    }
};

// Mixture Gamma and Pi at the carried volume fractions a[0..NF-2].
template <typename R, int NF>
__device__ __forceinline__ void mixture(const EosR<R, NF>& e, const R* a, R& G, R& Pi) {
    G = a[0] * e.dg[0] + e.gN;
    Pi = a[0] * e.dP[0] + e.PN;
#pragma unroll
    for (int i = 1; i < NF - 1; ++i) {
        G = G + a[i] * e.dg[i];
        Pi = Pi + a[i] * e.dP[i];
    }
}

// ---------------------------------------------------------------- WENO5-JS
// v0..v4 = v_{i-2}..v_{i+2}.  vm: left-biased value at i+1/2 (linear weights
// 0.1, 0.6, 0.3); vp: right-biased value at i-1/2 (0.3, 0.6, 0.1).  The three
// Jiang-Shu smoothness indicators of cell i serve both faces.
//
// Written in first differences d1..d4 (d_k = v_k - v_{k-1}):
//   beta0 = 13/12 (d2-d1)^2 + 1/4 (3 d2 - d1)^2
//   beta1 = 13/12 (d3-d2)^2 + 1/4 (d2 + d3)^2
//   beta2 = 13/12 (d4-d3)^2 + 1/4 (3 d3 - d4)^2
// and each candidate value as v_i plus a correction:
//   left:  (5 d2 - 2 d1)/6, (d2 + 2 d3)/6, (4 d3 - d4)/6
//   right: (d1 - 4 d2)/6, -(2 d2 + d3)/6, (2 d4 - 5 d3)/6
// (the same polynomials as the textbook forms), so uniform data reconstructs
// exactly.  FP64: product-form weights and one reciprocal for both faces.
// FP32: weights relative to the smoothest stencil, the linear weights and
// the 1/6 folded into the corrections, one fast reciprocal per face.
// FP32 WENO5 from the smoothness indicators: weights relative to the smoothest
// stencil, the linear weights and the 1/6 of the candidates folded into the
// corrections, one reciprocal per face.
__device__ __forceinline__ void weno5_tail32(float v2, float d1, float d2, float d3, float d4, float b0, float b1,
                                             float b2, float eps, float& vm, float& vp) {
    float s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
    s0 = s0 * s0;
    s1 = s1 * s1;
    s2 = s2 * s2;
    // weights relative to the smoothest stencil, all in (0, 1]
    const float smin = fminf(s0, fminf(s1, s2));
    const float m0 = __fdividef(smin, s0);
    const float m1 = __fdividef(smin, s1);
    const float m2 = __fdividef(smin, s2);
    // face values v_i + sum_k d_k m_k c_k / sum_k d_k m_k with the linear
    // weights d_k and the 1/6 of the candidates folded into the
    // corrections c_k, and one reciprocal per face
    const float t1 = float(0.6) * m1;
    const float Dm = fmaf(float(0.1), m0, fmaf(float(0.3), m2, t1));
    const float Dp = fmaf(float(0.3), m0, fmaf(float(0.1), m2, t1));
    const float d2x02 = float(0.2) * d2, d3x02 = float(0.2) * d3;
    const float cm0 = fmaf(float(0.5 / 6.0), d2, float(-0.2 / 6.0) * d1);  // 0.1 (5 d2 - 2 d1)/6
    const float cm1 = fmaf(float(0.1), d2, d3x02);  // 0.6 (d2 + 2 d3)/6
    const float cm2 = fmaf(-float(0.05), d4, d3x02);  // 0.3 (4 d3 - d4)/6
    const float cp0 = fmaf(float(0.05), d1, -d2x02);  // 0.3 (d1 - 4 d2)/6
    const float cp1 = fmaf(-float(0.1), d3, -d2x02);  // -0.6 (2 d2 + d3)/6
    const float cp2 = fmaf(float(0.2 / 6.0), d4, float(-0.5 / 6.0) * d3);  // 0.1 (2 d4 - 5 d3)/6
    const float Nm = fmaf(m0, cm0, fmaf(m1, cm1, m2 * cm2));
    const float Np = fmaf(m0, cp0, fmaf(m1, cp1, m2 * cp2));
    vm = fmaf(Nm, __fdividef(1.0f, Dm), v2);
    vp = fmaf(Np, __fdividef(1.0f, Dp), v2);
}

// FP32 WENO5 of cell i from values carried along the pencil: the first
// differences d1..d4 of v_{i-2}..v_{i+2} and the curvature parts
// C_k = 13/12 (d_{k+2} - d_{k+1})^2 of the three indicators.  d1..d3 and C0, C1
// are d2..d4 and C1, C2 of cell i-1, so a sweep forms one difference and one
// curvature part per cell and field.
__device__ __forceinline__ void weno5_dc(float v2, float d1, float d2, float d3, float d4, float C0, float C1,
                                         float C2, float eps, float& vm, float& vp) {
    const float Q0 = 3.0f * d2 - d1, Q1 = d2 + d3, Q2 = 3.0f * d3 - d4;
    const float b0 = fmaf(0.25f * Q0, Q0, C0);
    const float b1 = fmaf(0.25f * Q1, Q1, C1);
    const float b2 = fmaf(0.25f * Q2, Q2, C2);
    weno5_tail32(v2, d1, d2, d3, d4, b0, b1, b2, eps, vm, vp);
}

template <typename R>
__device__ __forceinline__ void weno5(R v0, R v1, R v2, R v3, R v4, R eps, R& vm, R& vp) {
    const R c13 = R(13.0 / 12.0);
    R d1 = v1 - v0, d2 = v2 - v1, d3 = v3 - v2, d4 = v4 - v3;
    R D0 = d2 - d1, D1 = d3 - d2, D2 = d4 - d3;
    R Q0 = R(3) * d2 - d1, Q1 = d2 + d3, Q2 = R(3) * d3 - d4;
    R b0 = c13 * D0 * D0 + R(0.25) * Q0 * Q0;
    R b1 = c13 * D1 * D1 + R(0.25) * Q1 * Q1;
    R b2 = c13 * D2 * D2 + R(0.25) * Q2 * Q2;
    if constexpr (sizeof(R) == 4) {
        weno5_tail32(v2, d1, d2, d3, d4, b0, b1, b2, eps, vm, vp);
        return;
    }
    R s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
    s0 = s0 * s0;
    s1 = s1 * s1;
    s2 = s2 * s2;
    // product form: weight of stencil k is proportional to d_k * s_j * s_l
    R m0 = s1 * s2, m1 = s0 * s2, m2 = s0 * s1;
    R am0 = R(0.1) * m0, am1 = R(0.6) * m1, am2 = R(0.3) * m2;
    R ap0 = R(0.3) * m0, ap1 = R(0.6) * m1, ap2 = R(0.1) * m2;
    R Nm = am0 * (R(5) * d2 - R(2) * d1) + am1 * (d2 + R(2) * d3) + am2 * (R(4) * d3 - d4);
    R Np = ap0 * (d1 - R(4) * d2) - ap1 * (R(2) * d2 + d3) + ap2 * (R(2) * d4 - R(5) * d3);
    R Dm = am0 + am1 + am2, Dp = ap0 + ap1 + ap2;
    R r = rdiv(R(1), R(6) * Dm * Dp);
    vm = v2 + Nm * Dp * r;
    vp = v2 + Np * Dm * r;
}

// WENO3-JS (Sec. II-B's third-order option; Jiang & Shu, stencils {i-1, i}
// and {i, i+1}, beta_k the squared first differences d1 = v_i - v_{i-1},
// d2 = v_{i+1} - v_i).  In difference form the candidates are v_i +- d_k/2:
//   v_{i+1/2}^- = v_i + (w0 d1 + w1 d2)/2,  linear weights (1/3, 2/3)
//   v_{i-1/2}^+ = v_i - (w0 d1 + w1 d2)/2,  linear weights (2/3, 1/3)
// with the same weight scaling as weno5 and one reciprocal for both faces.
template <typename R>
__device__ __forceinline__ void weno3(R v1, R v2, R v3, R eps, R& vm, R& vp) {
    R d1 = v2 - v1, d2 = v3 - v2;
    R s0 = eps + d1 * d1, s1 = eps + d2 * d2;
    s0 = s0 * s0;
    s1 = s1 * s1;
    R m0, m1;
    if constexpr (sizeof(R) == 8) {
        m0 = s1;   // product form: weight of stencil k proportional to d_k * s_other
        m1 = s0;
    } else {
        R smin = fminf(s0, s1);
        m0 = __fdividef(smin, s0);
        m1 = __fdividef(smin, s1);
    }
    R am0 = R(1.0 / 3.0) * m0, am1 = R(2.0 / 3.0) * m1;
    R ap0 = R(2.0 / 3.0) * m0, ap1 = R(1.0 / 3.0) * m1;
    R Dm = am0 + am1, Dp = ap0 + ap1;
    R r = rdiv(R(1), R(2) * Dm * Dp);
    vm = v2 + (am0 * d1 + am1 * d2) * Dp * r;
    vp = v2 - (ap0 * d1 + ap1 * d2) * Dm * r;
}

// WENO5-JS on a non-uniform grid from the cell's table T (kTabDoubles values,
// the same for every lane of a warp): candidates q_k^+- = cp_k.v, cm_k.v,
// smoothness beta_k = (B_k.v)^2 + 13/3 (C_k.v)^2, linear weights dp, dm;
// weights scaled as in weno5 (product form in FP64, relative to the smoothest
// stencil in FP32), one reciprocal for both faces.
template <typename R>
__device__ __forceinline__ void weno5_tab(const R* __restrict__ T, R v0, R v1, R v2, R v3, R v4, R eps, R& vm,
                                          R& vp) {
    const R v[5] = {v0, v1, v2, v3, v4};
    R qp[3], qm[3], s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R a = R(0), b = R(0), c = R(0), d = R(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const R x = v[k + j];
            a += __ldg(T + 3 * k + j) * x;
            b += __ldg(T + 9 + 3 * k + j) * x;
            c += __ldg(T + 18 + 3 * k + j) * x;
            d += __ldg(T + 27 + 3 * k + j) * x;
        }
        qp[k] = a;
        qm[k] = b;
        const R beta = c * c + R(13.0 / 3.0) * (d * d);
        s[k] = (eps + beta) * (eps + beta);
    }
    R m0, m1, m2;
    if constexpr (sizeof(R) == 8) {
        m0 = s[1] * s[2];
        m1 = s[0] * s[2];
        m2 = s[0] * s[1];
    } else {
        R smin = fminf(s[0], fminf(s[1], s[2]));
        m0 = __fdividef(smin, s[0]);
        m1 = __fdividef(smin, s[1]);
        m2 = __fdividef(smin, s[2]);
    }
    const R ap0 = __ldg(T + 36) * m0, ap1 = __ldg(T + 37) * m1, ap2 = __ldg(T + 38) * m2;
    const R am0 = __ldg(T + 39) * m0, am1 = __ldg(T + 40) * m1, am2 = __ldg(T + 41) * m2;
    const R Dp = ap0 + ap1 + ap2, Dm = am0 + am1 + am2;
    const R r = rdiv(R(1), Dp * Dm);
    vm = (ap0 * qp[0] + ap1 * qp[1] + ap2 * qp[2]) * Dm * r;
    vp = (am0 * qm[0] + am1 * qm[1] + am2 * qm[2]) * Dp * r;
}

// ---------------------------------------------------------------- HLLC
// Flux through a face normal to DIR from reconstructed primitive states
// (alpha1 rho1, alpha2 rho2, u_k, p, alpha1).  uf receives the velocity of the
// selected region (u_K outside the fan, S* inside), which also carries the
// alpha1 slot: F_alpha = alpha1_K * uf.  Region choice follows
// 0<=S_L: F_L; S_L<0<=S*: F*_L; S*<0<=S_R: F*_R; else F_R.
// Returns true when a face state is non-physical (rho<=0, c^2<=0, NaN).
template <int NDIM, int DIR, typename R, int NF = 2>
__device__ __forceinline__ bool hllc(const EosR<R, NF>& e, const R* wL, const R* wR, R* F, R& uf) {
    using FL = Fields<NDIM, NF>;
    const int IE = FL::IE, IA = FL::IA, IU = FL::IU;
    R rhoL = mix_rho<NF>(wL);
    R rhoR = mix_rho<NF>(wR);
    R GL, PiL, GR, PiR;
    mixture(e, wL + IA, GL, PiL);
    mixture(e, wR + IA, GR, PiR);
    R pL = wL[IE], pR = wR[IE];
    R c2L = rdiv((GL + R(1)) * pL + PiL, GL * rhoL);
    R c2R = rdiv((GR + R(1)) * pR + PiR, GR * rhoR);
    bool bad = !pos(rhoL) || !pos(rhoR) || !pos(c2L) || !pos(c2R);
    R cL = sqrt_pos(c2L), cR = sqrt_pos(c2R);
    R uL = wL[IU + DIR], uR = wR[IU + DIR];
    const R aL = uL - cL, aR = uR - cR, bL = uL + cL, bR = uR + cR;
    R SL = lt(aL, aR) ? aL : aR;
    R SR = lt(bR, bL) ? bL : bR;
    R mL = rhoL * (SL - uL), mR = rhoR * (SR - uR);
    R Ss = rdiv(pR - pL + uL * mL - uR * mR, mL - mR);
    const bool left = nonneg(SL) || nonneg(Ss);
    const bool star = left ? !nonneg(SL) : nonneg(SR);
    // selected side K (element-wise select keeps both states in registers)
    R w[FL::NEQ];
#pragma unroll
    for (int f = 0; f < FL::NEQ; ++f) w[f] = left ? wL[f] : wR[f];
    R rho = left ? rhoL : rhoR;
    R G = left ? GL : GR;
    R Pi = left ? PiL : PiR;
    R SK = left ? SL : SR;
    R p = w[IE];
    R un = w[IU + DIR];
    R ke = R(0);
#pragma unroll
    for (int k = 0; k < NDIM; ++k) ke += w[IU + k] * w[IU + k];
    ke = R(0.5) * rho * ke;
    R E = G * p + Pi + ke;
#pragma unroll
    for (int i = 0; i < NF; ++i) F[i] = w[i] * un;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) F[IU + k] = rho * w[IU + k] * un;
    F[IU + DIR] += p;
    F[IE] = (E + p) * un;
    uf = un;
    if (star) {
        R inv = rdiv(R(1), SK - Ss);
        R chi = (SK - un) * inv;
        R dchi = chi - R(1);
#pragma unroll
        for (int i = 0; i < NF; ++i) F[i] += SK * (dchi * w[i]);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            R ms = (k == DIR) ? chi * rho * Ss : chi * rho * w[IU + k];
            F[IU + k] += SK * (ms - rho * w[IU + k]);
        }
        R dS = Ss - un;
        R Es = chi * (E + dS * rho * Ss) + dS * p * inv;
        F[IE] += SK * (Es - E);
        uf = Ss;
    }
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) F[IA + i] = w[IA + i] * uf;
    return bad;
}

}  // namespace mfc5
