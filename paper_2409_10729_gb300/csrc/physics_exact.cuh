// physics_exact.cuh -- FP64 RHS arithmetic in the reference operation order.
//
// The same stiffened-gas EOS (arXiv 2409.10729, Sec. II-A), WENO5-JS and
// HLLC (Sec. II-B) as physics.cuh, but every formula is evaluated in the
// textbook order the serial FP64 oracle uses, with one IEEE rounding per
// operation.  Compiled with -fmad=false (no contraction of a*b+c), the
// results are bit-identical to that order.  Where several quotients share a
// denominator, the quotient is formed from a correctly rounded reciprocal
// y = RN(1/b) and one FMA correction (Markstein's theorem, "Computation of
// elementary functions on the IBM RISC System/6000", 1990):
//   q = RN(a y),  r = RN(a - b q) (exact),  a/b rounded = RN(q + r y),
// which is the correctly rounded a/b for operands without overflow or
// underflow -- the same bits as a division, at a third of the cost.
#pragma once
#include "physics.cuh"

namespace mfc5 {
namespace exact {

// Correctly rounded a/b given y = RN(1/b).
__device__ __forceinline__ double div_rcp(double a, double b, double y) {
    double q = __dmul_rn(a, y);
    double r = __fma_rn(-b, q, a);
    return __fma_rn(r, y, q);
}

__device__ __forceinline__ double rcp(double b) { return __drcp_rn(b); }

__device__ __forceinline__ double sq(double x) { return x * x; }

// Gamma = sum_i alpha_i g_i, Pi = sum_i alpha_i P_i over the NF fluids, the
// carried fractions a[0..NF-2] first and alpha_N = 1 - a[0] - ... - a[NF-2]
// last (two fluids: a1 g1 + (1 - a1) g2).
template <int NF>
__device__ __forceinline__ void mixture(const Eos& e, const double* a, double& G, double& Pi) {
    double aN = 1.0 - a[0];
#pragma unroll
    for (int i = 1; i < NF - 1; ++i) aN = aN - a[i];
    double sg = a[0] * e.g[0], sp = a[0] * e.P[0];
#pragma unroll
    for (int i = 1; i < NF - 1; ++i) {
        sg = sg + a[i] * e.g[i];
        sp = sp + a[i] * e.P[i];
    }
    G = sg + aN * e.g[NF - 1];
    Pi = sp + aN * e.P[NF - 1];
}

template <int NF>
__device__ __forceinline__ double mix_rho(const double* q) {
    double rho = q[0] + q[1];
#pragma unroll
    for (int i = 2; i < NF; ++i) rho = rho + q[i];
    return rho;
}

// 0.5 rho |u|^2 in the oracle's order, whose sum starts from 0.0: 0.0 + u_0^2
// is u_0^2 itself (a square is never -0), so the sum starts there.
template <int NDIM>
__device__ __forceinline__ double kinetic(double rho, const double* u) {
    double s = u[0] * u[0];
#pragma unroll
    for (int k = 1; k < NDIM; ++k) s = s + u[k] * u[k];
    return 0.5 * rho * s;
}

// Conservative -> primitive (u_k = rho u_k / rho, p = (rho E - ke - Pi)/Gamma).
template <int NDIM, int NF = 2>
__device__ __forceinline__ void cons_to_prim(const Eos& e, const double* q, double* w) {
    using FL = Fields<NDIM, NF>;
    double rho = mix_rho<NF>(q);
    double y = rcp(rho);
    double u[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) u[k] = div_rcp(q[FL::IU + k], rho, y);
    double ke = kinetic<NDIM>(rho, u);
    double G, Pi;
    mixture<NF>(e, q + FL::IA, G, Pi);
    double p = (q[FL::IE] - ke - Pi) / G;
#pragma unroll
    for (int i = 0; i < NF; ++i) w[i] = q[i];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) w[FL::IU + k] = u[k];
    w[FL::IE] = p;
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) w[FL::IA + i] = q[FL::IA + i];
}

// Primitive -> conservative (rho E = Gamma p + Pi + ke).
template <int NDIM, int NF = 2>
__device__ __forceinline__ void prim_to_cons(const Eos& e, const double* w, double* q) {
    using FL = Fields<NDIM, NF>;
    double rho = mix_rho<NF>(w);
    double u[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) u[k] = w[FL::IU + k];
    double ke = kinetic<NDIM>(rho, u);
    double G, Pi;
    mixture<NF>(e, w + FL::IA, G, Pi);
#pragma unroll
    for (int i = 0; i < NF; ++i) q[i] = w[i];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) q[FL::IU + k] = rho * u[k];
    q[FL::IE] = G * w[FL::IE] + Pi + ke;
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) q[FL::IA + i] = w[FL::IA + i];
}

__device__ __forceinline__ double sound2(double G, double Pi, double rho, double p) {
    return ((G + 1.0) * p + Pi) / (G * rho);
}

// WENO5-JS: left-biased value at i+1/2 and right-biased value at i-1/2 from
// v0..v4 = v_{i-2}..v_{i+2}; weights a_k = d_k/(eps+beta_k)^2, omega_k = a_k/sum(a),
// candidate values (.)/6, face value sum omega_k p_k.
//
// Products by a power of two (2, 4, 1/4) are exact, so RN(RN(2 v) + x) equals
// the single fused RN(2 v + x): those sums are written as FMAs (fma2 below),
// which changes no result bit (barring a product in the subnormal range,
// below 2^-1022, that a scaling by 1/4 would round).
__device__ __forceinline__ double fma2(double k, double v, double x) { return __fma_rn(k, v, x); }

// Two correctly rounded operations of WENO5 computed from the IEEE 754
// binary64 fields on the integer pipes (GB300's FP64 pipe retires two
// operations per SM and clock): the product of v by a small odd integer K and
// the quotient x/6, both on 32-bit words (32-bit multiplies, multiply-highs,
// shifts and adds; no floating-point or 64-bit integer instruction).  Same bits as the FP64 operation for every input: zeros
// are returned directly, and subnormal, infinite or NaN operands and results
// near the exponent limits take the FP64 instruction.
//
// K v: with v = +-M 2^(e-1075), M in [2^52, 2^53), the product M K has 54 to
// 57 bits; it is rounded to 53 bits (ties to even) by adding 2^(s-1) - 1 plus
// the lowest kept bit before the shift by s.  The rounded significand (up to
// 2^53) is added onto the shifted exponent field, so a carry out of the
// significand raises the exponent.
template <unsigned K>
__device__ __forceinline__ double mul_small(double v) {
    static_assert(K % 2 == 1 && K >= 3 && K <= 15, "odd factor 3..15");
    constexpr unsigned S0 = K < 4 ? 1 : (K < 8 ? 2 : 3);   // M K in [2^(52+S0), 2^(54+S0))
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned e = (hi >> 20) & 0x7ffu;
    // subnormals, |v| >= 2^1019, infinities and NaNs
    if (__builtin_expect(e > 2041u || (e == 0u && ((hi << 1) | lo) != 0u), 0)) return (double)K * v;
    // P = M K in two 32-bit words (M = mh:lo): no 64-bit integer instruction
    const unsigned mh = (hi & 0x000fffffu) | 0x00100000u;
    const unsigned pl = lo * K;
    const unsigned ph = mh * K + __umulhi(lo, K);
    const unsigned s = S0 + ((ph >> (21 + S0)) & 1u);   // P >= 2^(53+S0): one more bit to drop
    const unsigned add = ((1u << (s - 1u)) - 1u) + ((pl >> s) & 1u);
    const unsigned nl = pl + add;
    const unsigned nh = ph + (nl < pl ? 1u : 0u);
    const unsigned rl = __funnelshift_r(nl, nh, s), rh = nh >> s;
    const bool zero = e == 0u;   // +-0: K 0 = 0 with the sign kept
    const unsigned oh = zero ? hi : (hi & 0x80000000u) + ((e + s - 1u) << 20) + rh;
    const unsigned ol = zero ? lo : rl;
    return __hiloint2double((int)oh, (int)ol);
}

// x/6: with x = +-M 2^(e-1075), x/6 = +-(M 2^k / 3) 2^(e-1076-k), where k = 2
// for M < 3 2^51 and k = 1 otherwise puts M 2^k / 3 in [2^52, 2^53).  A third
// of an integer is never halfway between two integers, so the round-to-nearest
// significand is floor((M 2^k + 1) / 3) and never reaches 2^53.
__device__ __forceinline__ double div6(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (__builtin_expect(e == 2047u || (e < 4u && ((hi << 1) | lo) != 0u), 0)) return x / 6.0;
    // N = M 2^k + 1 in two 32-bit words (M = mh:lo), then N / 3 word by word:
    // H = 3 q1 + r1, L = 3 qL + rL and 2^32 = 3 * 1431655765 + 1 give
    // N / 3 = q1 2^32 + r1 * 1431655765 + qL + (r1 + rL >= 3), whose low word never carries
    const unsigned mh = (hi & 0x000fffffu) | 0x00100000u;
    const unsigned k = mh < 0x00180000u ? 2u : 1u;
    const unsigned L = (lo << k) | 1u, H = __funnelshift_l(lo, mh, k);
    const unsigned q1 = __umulhi(H, 0xAAAAAAABu) >> 1, r1 = H - 3u * q1;
    const unsigned qL = __umulhi(L, 0xAAAAAAABu) >> 1, rL = L - 3u * qL;
    const unsigned q0 = r1 * 1431655765u + qL + (r1 + rL >= 3u ? 1u : 0u);
    const bool zero = e == 0u;   // +-0 (subnormals took the division)
    const unsigned oh = zero ? hi : (hi & 0x80000000u) + ((e - 2u - k) << 20) + q1;
    const unsigned ol = zero ? lo : q0;
    return __hiloint2double((int)oh, (int)ol);
}

// The curvature term of a Jiang-Shu smoothness indicator on the three cells
// a, b, c: 13/12 (a - 2 b + c)^2.  The stencil {i-1, i, i+1} gives beta_1 of
// cell i, beta_2 of cell i-1 and beta_0 of cell i+1 the same term, formed
// from the same three values in the same order -- the same bits -- so a sweep
// that slides along a pencil can form it once per cell and pass it on.
__device__ __forceinline__ double curv(double a, double b, double c) {
    const double c13 = 13.0 / 12.0;
    return c13 * sq(fma2(-2.0, b, a) + c);
}

// WENO5-JS given the curvature terms t0 = curv(v0, v1, v2), t1 = curv(v1, v2,
// v3) and t2 = curv(v2, v3, v4) of the three smoothness indicators.
__device__ __forceinline__ void weno5_t(double eps, double v0, double v1, double v2, double v3, double v4,
                                        double t0, double t1, double t2, double& vm, double& vp) {
    // b0 = c13 (v0 - 2 v1 + v2)^2 + 1/4 (v0 - 4 v1 + 3 v2)^2, and likewise b1, b2
    const double v2x3 = mul_small<3>(v2);
    double b0 = fma2(0.25, sq(fma2(-4.0, v1, v0) + v2x3), t0);
    double b1 = fma2(0.25, sq(v1 - v3), t1);
    double b2 = fma2(0.25, sq(fma2(-4.0, v3, v2x3) + v4), t2);
    double s0 = sq(eps + b0), s1 = sq(eps + b1), s2 = sq(eps + b2);
    double y0 = rcp(s0), y1 = rcp(s1), y2 = rcp(s2);

    double a0 = div_rcp(0.1, s0, y0);
    double a1 = div_rcp(0.6, s1, y1);
    double a2 = div_rcp(0.3, s2, y2);
    double s = a0 + a1 + a2;
    double ys = rcp(s);
    const double v2x5 = mul_small<5>(v2), v2x11 = mul_small<11>(v2);
    double p0 = div6(fma2(2.0, v0, -mul_small<7>(v1)) + v2x11);     // (2 v0 - 7 v1 + 11 v2)/6
    double p1 = div6(fma2(2.0, v3, -v1 + v2x5));                    // (-v1 + 5 v2 + 2 v3)/6
    double p2 = div6(fma2(2.0, v2, mul_small<5>(v3)) - v4);         // (2 v2 + 5 v3 - v4)/6
    vm = div_rcp(a0, s, ys) * p0 + div_rcp(a1, s, ys) * p1 + div_rcp(a2, s, ys) * p2;

    a0 = div_rcp(0.3, s0, y0);
    a1 = div_rcp(0.6, s1, y1);
    a2 = div_rcp(0.1, s2, y2);
    s = a0 + a1 + a2;
    ys = rcp(s);
    p0 = div6(fma2(2.0, v2, -v0 + mul_small<5>(v1)));               // (-v0 + 5 v1 + 2 v2)/6
    p1 = div6(fma2(2.0, v1, v2x5) - v3);                            // (2 v1 + 5 v2 - v3)/6
    p2 = div6(fma2(2.0, v4, v2x11 - mul_small<7>(v3)));             // (11 v2 - 7 v3 + 2 v4)/6
    vp = div_rcp(a0, s, ys) * p0 + div_rcp(a1, s, ys) * p1 + div_rcp(a2, s, ys) * p2;
}

// The right-face candidates of cell i, (-v_{i-2} + 5 v_{i-1} + 2 v_i)/6 and
// (2 v_{i-1} + 5 v_i - v_{i+1})/6, are the left-face candidates p1 and p2 of
// cell i-1, formed from the same values in the same order (the same bits):
// weno5_tc takes them as r0, r1 and returns this cell's p1, p2 for the next.
__device__ __forceinline__ void weno5_tc(double eps, double v0, double v1, double v2, double v3, double v4,
                                         double t0, double t1, double t2, double& r0, double& r1, double& vm,
                                         double& vp) {
    const double v2x3 = mul_small<3>(v2);
    double b0 = fma2(0.25, sq(fma2(-4.0, v1, v0) + v2x3), t0);
    double b1 = fma2(0.25, sq(v1 - v3), t1);
    double b2 = fma2(0.25, sq(fma2(-4.0, v3, v2x3) + v4), t2);
    double s0 = sq(eps + b0), s1 = sq(eps + b1), s2 = sq(eps + b2);
    double y0 = rcp(s0), y1 = rcp(s1), y2 = rcp(s2);

    double a0 = div_rcp(0.1, s0, y0);
    double a1 = div_rcp(0.6, s1, y1);
    double a2 = div_rcp(0.3, s2, y2);
    double s = a0 + a1 + a2;
    double ys = rcp(s);
    const double v2x5 = mul_small<5>(v2), v2x11 = mul_small<11>(v2);
    double p0 = div6(fma2(2.0, v0, -mul_small<7>(v1)) + v2x11);     // (2 v0 - 7 v1 + 11 v2)/6
    double p1 = div6(fma2(2.0, v3, -v1 + v2x5));                    // (-v1 + 5 v2 + 2 v3)/6
    double p2 = div6(fma2(2.0, v2, mul_small<5>(v3)) - v4);         // (2 v2 + 5 v3 - v4)/6
    vm = div_rcp(a0, s, ys) * p0 + div_rcp(a1, s, ys) * p1 + div_rcp(a2, s, ys) * p2;

    a0 = div_rcp(0.3, s0, y0);
    a1 = div_rcp(0.6, s1, y1);
    a2 = div_rcp(0.1, s2, y2);
    s = a0 + a1 + a2;
    ys = rcp(s);
    p0 = div6(fma2(2.0, v4, v2x11 - mul_small<7>(v3)));             // (11 v2 - 7 v3 + 2 v4)/6
    vp = div_rcp(a0, s, ys) * r0 + div_rcp(a1, s, ys) * r1 + div_rcp(a2, s, ys) * p0;
    r0 = p1;
    r1 = p2;
}

// The right-face candidates r0, r1 of the cell whose window is v0..v3 (as in weno5_t).
__device__ __forceinline__ void weno5_right01(double v0, double v1, double v2, double v3, double& r0, double& r1) {
    r0 = div6(fma2(2.0, v2, -v0 + mul_small<5>(v1)));
    r1 = div6(fma2(2.0, v1, mul_small<5>(v2)) - v3);
}

__device__ __forceinline__ void weno5(double eps, double v0, double v1, double v2, double v3, double v4,
                                      double& vm, double& vp) {
    weno5_t(eps, v0, v1, v2, v3, v4, curv(v0, v1, v2), curv(v1, v2, v3), curv(v2, v3, v4), vm, vp);
}

// WENO3-JS in the reference order: v1..v3 = v_{i-1}..v_{i+1}; weights
// a_k = d_k/(eps+beta_k)^2 with d = (1/3, 2/3) at i+1/2 and (2/3, 1/3) at
// i-1/2, omega_k = a_k/sum(a), candidates (.)/2 (an exact halving).
__device__ __forceinline__ void weno3(double eps, double v1, double v2, double v3, double& vm, double& vp) {
    const double c1 = 1.0 / 3.0, c2 = 2.0 / 3.0;
    double b0 = sq(v2 - v1), b1 = sq(v3 - v2);
    double s0 = sq(eps + b0), s1 = sq(eps + b1);
    double y0 = rcp(s0), y1 = rcp(s1);

    double a0 = div_rcp(c1, s0, y0);
    double a1 = div_rcp(c2, s1, y1);
    double s = a0 + a1;
    double ys = rcp(s);
    double p0 = (-v1 + 3.0 * v2) * 0.5;
    double p1 = (v2 + v3) * 0.5;
    vm = div_rcp(a0, s, ys) * p0 + div_rcp(a1, s, ys) * p1;

    a0 = div_rcp(c2, s0, y0);
    a1 = div_rcp(c1, s1, y1);
    s = a0 + a1;
    ys = rcp(s);
    p0 = (v1 + v2) * 0.5;
    p1 = (3.0 * v2 - v3) * 0.5;
    vp = div_rcp(a0, s, ys) * p0 + div_rcp(a1, s, ys) * p1;
}

struct Face {
    double rho, p, G, Pi, E, c2;
};

template <int NDIM, int NF = 2>
__device__ __forceinline__ void face_from_prim(const Eos& e, const double* w, Face& s) {
    using FL = Fields<NDIM, NF>;
    s.rho = mix_rho<NF>(w);
    s.p = w[FL::IE];
    mixture<NF>(e, w + FL::IA, s.G, s.Pi);
    s.E = s.G * s.p + s.Pi + kinetic<NDIM>(s.rho, w + FL::IU);
    s.c2 = sound2(s.G, s.Pi, s.rho, s.p);
}

// Physical flux of side K (primitives w, face state K) normal to DIR; the
// volume-fraction slots carry alpha_i,K u_n.
template <int NDIM, int DIR, int NF = 2>
__device__ __forceinline__ void phys_flux(const double* w, const Face& K, double* F) {
    using FL = Fields<NDIM, NF>;
    double un = w[FL::IU + DIR];
#pragma unroll
    for (int i = 0; i < NF; ++i) F[i] = w[i] * un;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) F[FL::IU + k] = K.rho * w[FL::IU + k] * un;
    F[FL::IU + DIR] = F[FL::IU + DIR] + K.p;
    F[FL::IE] = (K.E + K.p) * un;
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) F[FL::IA + i] = w[FL::IA + i] * un;
}

// HLLC flux through a face normal to DIR; regions 0<=S_L: F_L, S_L<0<=S*: F*_L,
// S*<0<=S_R: F*_R, else F_R; the alpha1 slot carries alpha1_K times the
// region velocity, returned in uf.  Returns true for a non-physical face state.
template <int NDIM, int DIR, int NF = 2>
__device__ __forceinline__ bool hllc(const Eos& e, const double* wL, const double* wR, double* F, double& uf) {
    using FL = Fields<NDIM, NF>;
    Face L, R;
    face_from_prim<NDIM, NF>(e, wL, L);
    face_from_prim<NDIM, NF>(e, wR, R);
    bool bad = !gt0(L.rho) || !gt0(R.rho) || !gt0(L.c2) || !gt0(R.c2);
    double cL = sqrt(L.c2), cR = sqrt(R.c2);
    double uL = wL[FL::IU + DIR], uR = wR[FL::IU + DIR];
    const double aL = uL - cL, aR = uR - cR, bL = uL + cL, bR = uR + cR;
    double SL = less(aL, aR) ? aL : aR;
    double SR = less(bR, bL) ? bL : bR;
    double num = R.p - L.p + L.rho * uL * (SL - uL) - R.rho * uR * (SR - uR);
    double den = L.rho * (SL - uL) - R.rho * (SR - uR);
    double Ss = num / den;
    const bool left = ge0(SL) || ge0(Ss);
    const bool star = left ? !ge0(SL) : ge0(SR);
    double w[FL::NEQ];
#pragma unroll
    for (int f = 0; f < FL::NEQ; ++f) w[f] = left ? wL[f] : wR[f];
    Face K;
    K.rho = left ? L.rho : R.rho;
    K.p = left ? L.p : R.p;
    K.G = left ? L.G : R.G;
    K.Pi = left ? L.Pi : R.Pi;
    K.E = left ? L.E : R.E;
    double SK = left ? SL : SR;
    double un = w[FL::IU + DIR];
    phys_flux<NDIM, DIR, NF>(w, K, F);
    uf = un;
    if (star) {
        double chi = (SK - un) / (SK - Ss);
#pragma unroll
        for (int i = 0; i < NF; ++i) F[i] = F[i] + SK * (chi * w[i] - w[i]);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            double mstar = (k == DIR) ? chi * K.rho * Ss : chi * K.rho * w[FL::IU + k];
            F[FL::IU + k] = F[FL::IU + k] + SK * (mstar - K.rho * w[FL::IU + k]);
        }
        double Estar = chi * (K.E + (Ss - un) * (K.rho * Ss + K.p / (SK - un)));
        F[FL::IE] = F[FL::IE] + SK * (Estar - K.E);
#pragma unroll
        for (int i = 0; i < FL::NA; ++i) F[FL::IA + i] = w[FL::IA + i] * Ss;
        uf = Ss;
    }
    return bad;
}

// S contribution of one cell: sum_d (|u_d| + c)/dx_d, from the conservative state.
template <int NDIM, int NF = 2>
__device__ __forceinline__ double cell_wavespeed(const Eos& e, const double* q, const double* dx,
                                                 const double* rdx, bool& bad) {
    using FL = Fields<NDIM, NF>;
    double w[FL::NEQ];
    cons_to_prim<NDIM, NF>(e, q, w);
    double rho = mix_rho<NF>(w);
    double G, Pi;
    mixture<NF>(e, w + FL::IA, G, Pi);
    double c2 = sound2(G, Pi, rho, w[FL::IE]);
    bad |= !gt0(mix_rho<NF>(q)) || !gt0(rho) || !gt0(c2);
    double cs = sqrt(c2);
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s = s + div_rcp(fabs(w[FL::IU + d]) + cs, dx[d], rdx[d]);
    bad |= !less(s, INFINITY);
    return s;
}

}  // namespace exact
}  // namespace mfc5
