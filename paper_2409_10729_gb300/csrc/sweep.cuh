// sweep.cuh -- the fused per-direction sweep kernel.
//
// One launch handles one direction d of one RHS evaluation (arXiv
// 2409.10729, Sec. II-B): for every cell it converts conservative to
// primitive variables (Sec. II-A EOS), reconstructs both face values of every
// primitive with WENO5-JS, solves HLLC at every face once, and forms
//   L_d = (F_{i-1/2} - F_{i+1/2}) / dx_d  (+ alpha1_i (u_f,i+1/2 - u_f,i-1/2) / dx_d)
// which it stores into, adds to, or finishes the RHS accumulator with.  The
// last direction's sweep also applies the SSP-RK3 stage update and, on the
// third stage, reduces the CFL wave speed of the new state.
//
// Thread mapping.  A warp owns 32 adjacent pencils along d and a segment of
// `seg` cells of each -- or, in the balanced split, an even share of all the
// sweep's cells, one or more such segments of consecutive pencil groups
// (sweep_balanced).  For d = y, z the 32 lanes run along x, so every load
// is one coalesced row.  For d = x the lanes run along y: each lane loads
// its own row, whose 32-byte sector stays in L1 for the lane's next cells,
// and the RHS goes out through a shared-memory tile as whole sectors.  Each
// thread slides a five-cell window of
// primitives along its pencil in registers: per cell it takes one new cell,
// runs WENO once (both faces) and HLLC once (the face between the previous
// cell and this one), so no face is computed twice except at the two ends of
// a segment.  Boundary ghosts come from index clamping (transmissive) or
// wrapping (periodic) in the loads.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include <string.h>

#include <type_traits>

#include "mfc.h"
#include "mfc_internal.cuh"
#include "physics_exact.cuh"

namespace mfc5 {

__device__ __forceinline__ int bc_index(int j, int n, int periodic) {
    if (j >= 0 && j < n) return j;
    if (periodic) {
        int r = j % n;
        return r < 0 ? r + n : r;
    }
    return j < 0 ? 0 : n - 1;
}

// Fields a sweep reads per cell, in load order.  FP64: the conservative
// state.  Mixed: the FP32 state with the pressure stored as field NEQ (formed
// in FP64 when the state was written) read in place of rho E.
template <int NDIM, typename R, int NF = 2>
struct LoadSet {
    static constexpr int N = Fields<NDIM, NF>::NEQ;
    __device__ static constexpr int field(int k) {
        return (sizeof(R) == 8 || k != Fields<NDIM, NF>::IE) ? k : N;
    }
};

// Primitives from the loaded values v[] (see LoadSet).
template <int NDIM, int NF = 2>
__device__ __forceinline__ void to_prim(const EosR<double, NF>& e, const double* v, double* w) {
    using FL = Fields<NDIM, NF>;
    double r = 1.0 / mix_rho<NF>(v);
    double ke2 = 0.0;
#pragma unroll
    for (int i = 0; i < NF; ++i) w[i] = v[i];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        double u = v[FL::IU + k] * r;
        w[FL::IU + k] = u;
        ke2 += v[FL::IU + k] * u;
    }
    double G, Pi;
    mixture(e, v + FL::IA, G, Pi);
    w[FL::IE] = (v[FL::IE] - 0.5 * ke2 - Pi) / G;
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) w[FL::IA + i] = v[FL::IA + i];
}

template <int NDIM, int NF = 2>
__device__ __forceinline__ void to_prim(const EosR<float, NF>& e, const float* v, float* w) {
    using FL = Fields<NDIM, NF>;
    float r = __fdividef(1.0f, mix_rho<NF>(v));
#pragma unroll
    for (int i = 0; i < NF; ++i) w[i] = v[i];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) w[FL::IU + k] = v[FL::IU + k] * r;
    w[FL::IE] = v[FL::IE];  // stored pressure
#pragma unroll
    for (int i = 0; i < FL::NA; ++i) w[FL::IA + i] = v[FL::IA + i];
}

// Exact float -> double and round-to-nearest-even double -> float conversions
// done on the integer pipes by rearranging the IEEE 754 bit fields (binary32:
// 8-bit exponent bias 127, 23-bit fraction; binary64: 11-bit bias 1023,
// 52-bit fraction).  They return the same bits as the hardware conversions
// (zeros and subnormals of the -ftz build flush to signed zero; the rare
// out-of-range cases take the hardware path) and keep the conversions of the
// mixed form's FP64 stage update off GB300's narrow FP64 pipe.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = e == 0u ? 0u : (u & 0x7fffffu);
    const unsigned ed = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
    const unsigned hi = (u & 0x80000000u) | (ed << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}

__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned s = hi & 0x80000000u;
    if (e == 0u) return __uint_as_float(s);                  // zero (and FP64 subnormals)
    if (e < 897u || e > 1150u) return __double2float_rn(x);  // outside the normal float range
    unsigned mag = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    mag += (rem > 0x10000000u) || (rem == 0x10000000u && (mag & 1u));
    return __uint_as_float(s | mag);
}

// Pressure from an FP64 conservative state, mixed form: the cancelling part
// rho E - Pi is formed in FP64, the rest in FP32.
template <int NDIM, int NF = 2>
__device__ __forceinline__ float mixed_pressure(const Eos& e, const double* q, const float* q32) {
    using FL = Fields<NDIM, NF>;
    float rho = mix_rho<NF>(q32);
    float r = __fdividef(1.0f, rho);
    float ke2 = 0.0f;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) ke2 += q32[FL::IU + k] * (q32[FL::IU + k] * r);
    double Pi = q[FL::IA] * e.dP[0] + e.P[NF - 1];
#pragma unroll
    for (int i = 1; i < FL::NA; ++i) Pi = Pi + q[FL::IA + i] * e.dP[i];
    double num = (q[FL::IE] - Pi) - f2d_bits(0.5f * ke2);
    float G = q32[FL::IA] * e.dg32[0] + e.g32[NF - 1];
#pragma unroll
    for (int i = 1; i < FL::NA; ++i) G = G + q32[FL::IA + i] * e.dg32[i];
    return __fdividef(d2f_bits(num), G);
}

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Per-cell wave speed sum_d (|u_d| + c) / dx_d from primitives.
template <int NDIM, typename R, int NF = 2, typename T = double>
__device__ __forceinline__ R cell_wavespeed(const EosR<R, NF>& e, const R* w, const T* inv_dx, bool& bad) {
    using FL = Fields<NDIM, NF>;
    R rho = mix_rho<NF>(w);
    R G, Pi;
    mixture(e, w + FL::IA, G, Pi);
    R c2 = rdiv((G + R(1)) * w[FL::IE] + Pi, G * rho);
    bad |= !pos(rho) || !pos(c2);
    R c = sqrt_pos(c2);
    R s = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s += (fabs(w[FL::IU + d]) + c) * R(inv_dx[d]);
    bad |= !lt(s, R(INFINITY));
    return s;
}

// Width, RN(1/width) and 1/width of a cell in every direction (uniform, or
// the cell's own on non-uniform directions); the cell is `i` along the sweep
// direction DIR, `ia` along the lanes' direction and `b` along the third.
template <int DIR, bool NU>
__device__ __forceinline__ void cell_geometry(const SweepArgs& a, int i, int ia, int b, double* dx, double* rdx,
                                              double* idx) {
    int c[3];
    c[DIR] = i;
    c[DIR == 0 ? 1 : 0] = ia;
    c[DIR == 2 ? 1 : 2] = b;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        dx[d] = a.dx[d];
        rdx[d] = a.rdx[d];
        idx[d] = a.inv_dx[d];
        if (NU && a.cw[d]) {
            dx[d] = __ldg(a.cw[d] + c[d]);
            rdx[d] = __ldg(a.crw[d] + c[d]);
            idx[d] = rdx[d];
        }
    }
}

// Output tile of the x-direction sweep: per warp, per field, 32 rows x CH
// cells (CH * sizeof(R) = 32 bytes, one DRAM sector), padded by one element
// per row so that the 32 lanes write 32 different banks.
template <typename R>
struct XStage {
    static constexpr int CH = 32 / sizeof(R);   // cells per row and sector along x
    static constexpr int PITCH = CH + 1;        // padded row pitch (conflict-free accesses)
};

template <int FORM>
using FormReal = typename std::conditional<FORM == FORM_MIXED || FORM == FORM_GATED, float, double>::type;

// ---- gate network on the tensor cores, FP32-accurate ----------------------
// A warp evaluates the network for its 32 cells x 2 sensors = 64 samples at
// once, as four 16-row m16n8k16 tiles (rows 0-31: the warp's density
// stencils, 32-63: its pressure stencils), f16 operands, FP32 accumulation.
// To keep FP32 accuracy every FP32 operand v (inputs, weights, hidden
// activations) is split into two f16 halves, v = hi + lo with hi = f16(v)
// and lo = f16(v - hi), and each product is formed as hi*hi + lo*hi + hi*lo:
// products of f16 values are exact in FP32, the neglected lo*lo is below
// 2^-22 of the product, and a lo below the f16 normal range keeps an
// absolute error under 2^-25.  Layer 1 (5 -> 32) packs the three terms into
// one K = 16 contraction -- A row = [x_hi, x_lo, x_hi, 0], B column =
// [w_hi; w_hi; w_lo; 0]; layers 2 (32 -> 32) and 3 (32 -> 1, w3 in every
// column) run the three terms as six K = 16 MMAs per output tile.  Biases
// enter as the accumulator input; one layer's accumulator fragments are the
// next layer's A fragments, so activations never leave registers.
struct GateSmem {
    unsigned w1f[4][32][2];        // layer-1 B fragments (K = 16 packing), per n-tile and lane
    unsigned w2h[2][4][32][2];     // layer-2 B fragments, high halves: per k-tile, n-tile, lane
    unsigned w2l[2][4][32][2];     // layer-2 B fragments, low halves
    unsigned w3h[2][32][2];        // layer-3 B fragments (w3 in every column), high halves
    unsigned w3l[2][32][2];        // layer-3 B fragments, low halves
    float b1[32], b2[32], b3;
};

// f16 halves of an FP32 value: hi = f16(v), lo = f16(v - hi).
__device__ __forceinline__ __half f16_hi(float v) { return __float2half_rn(v); }
__device__ __forceinline__ __half f16_lo(float v) { return __float2half_rn(v - __half2float(__float2half_rn(v))); }

// Two halves packed as one 32-bit operand register (a in the low 16 bits).
__device__ __forceinline__ unsigned pack2(__half a, __half b) {
    return (unsigned)__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16);
}

// max(a, 0) and max(b, 0) split into packed high and low halves.
__device__ __forceinline__ void relu_split(float a, float b, unsigned& hi, unsigned& lo) {
    a = fmaxf(a, 0.f);
    b = fmaxf(b, 0.f);
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    hi = pack2(ha, hb);
    lo = pack2(__float2half_rn(a - __half2float(ha)), __float2half_rn(b - __half2float(hb)));
}

// Fill the block's fragment tables from the 1281 weights (all threads).
// Fragment layouts follow the PTX m16n8k16 f16 B operand: lane (g = lane / 4,
// t = lane % 4) holds column n = g, rows k = 2t, 2t + 1 in its first register
// and k = 2t + 8, 2t + 9 in its second.
__device__ __forceinline__ void gate_fill(GateSmem& g, const float* __restrict__ w) {
    constexpr int OB1 = 160, OW2 = 192, OB2 = 1216, OW3 = 1248, OB3 = 1280;
    // layer-1 operand row k of neuron n: [w_hi (k < 5), w_hi (k < 10), w_lo (k < 15), 0]
    auto b1k = [&](int n, int k) -> __half {
        if (k < 5) return f16_hi(w[n * 5 + k]);
        if (k < 10) return f16_hi(w[n * 5 + k - 5]);
        if (k < 15) return f16_lo(w[n * 5 + k - 10]);
        return __float2half_rn(0.f);
    };
    for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) {
        int nt = i / 32, l = i % 32, gq = l / 4, t = l % 4;
        int n = nt * 8 + gq, k = 2 * t;
        g.w1f[nt][l][0] = pack2(b1k(n, k), b1k(n, k + 1));
        g.w1f[nt][l][1] = pack2(b1k(n, k + 8), b1k(n, k + 9));
    }
    for (int i = threadIdx.x; i < 2 * 4 * 32; i += blockDim.x) {
        int kt = i / 128, nt = (i / 32) % 4, l = i % 32, gq = l / 4, t = l % 4;
        int n = nt * 8 + gq, k = kt * 16 + 2 * t;
        const float* r = w + OW2 + n * 32;
        g.w2h[kt][nt][l][0] = pack2(f16_hi(r[k]), f16_hi(r[k + 1]));
        g.w2h[kt][nt][l][1] = pack2(f16_hi(r[k + 8]), f16_hi(r[k + 9]));
        g.w2l[kt][nt][l][0] = pack2(f16_lo(r[k]), f16_lo(r[k + 1]));
        g.w2l[kt][nt][l][1] = pack2(f16_lo(r[k + 8]), f16_lo(r[k + 9]));
    }
    for (int i = threadIdx.x; i < 2 * 32; i += blockDim.x) {
        int kt = i / 32, l = i % 32, t = l % 4;
        int k = kt * 16 + 2 * t;
        const float* r = w + OW3;
        g.w3h[kt][l][0] = pack2(f16_hi(r[k]), f16_hi(r[k + 1]));
        g.w3h[kt][l][1] = pack2(f16_hi(r[k + 8]), f16_hi(r[k + 9]));
        g.w3l[kt][l][0] = pack2(f16_lo(r[k]), f16_lo(r[k + 1]));
        g.w3l[kt][l][1] = pack2(f16_lo(r[k + 8]), f16_lo(r[k + 9]));
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        g.b1[i] = w[OB1 + i];
        g.b2[i] = w[OB2 + i];
    }
    if (threadIdx.x == 0) g.b3 = w[OB3];
}

// Shared-memory loads the compiler keeps at their place of use: the gate's
// weight fragments are re-read per evaluation instead of being held in
// registers across the whole pencil.
__device__ __forceinline__ unsigned lds_u32(const void* p) {
    unsigned v, a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ uint2 lds_u64(const void* p) {
    uint2 v;
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.b32 {%0,%1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* row) {
    unsigned a = (unsigned)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void mma_k16c(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1, float c0, float c1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%10,%11};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1));
}

// d += a b, f16 operands, f32 accumulate.
__device__ __forceinline__ void mma_k16(float* d, const unsigned* a, uint2 b) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// One sample's layer-1 A row, 16 halves as two 16-byte chunks:
// [x_hi(5), x_lo(5), x_hi(5), 0].
__device__ __forceinline__ void gate_row(const float* x, uint4& r0, uint4& r1) {
    __half h[5], l[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        h[k] = f16_hi(x[k]);
        l[k] = __float2half_rn(x[k] - __half2float(h[k]));
    }
    const __half z = __float2half_rn(0.f);
    r0 = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], l[0]), pack2(l[1], l[2]));
    r1 = make_uint4(pack2(l[3], l[4]), pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], z));
}

// Logits of this lane's cell for both sensors.  xr, xp: the normalised
// density and pressure stencils of the lane's cell; need_r, need_p: whether
// the caller uses that logit -- a 16-sample tile none of whose samples is
// needed is skipped (its logits are left as they were).  With `both`, a
// pressure logit is needed only where the density sensor came out smooth
// (not needed, or logit < 0): the gate wants both smooth.  tile: this warp's
// 2 KB A tile (64 rows x 16 halves).  Must be called by all 32 lanes together.
__device__ __forceinline__ void gate_logits(const GateSmem& g, uint4* tile, const float* xr, const float* xp,
                                            bool need_r, bool need_p, bool both, float& zr, float& zp) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    const unsigned nr = __ballot_sync(0xffffffffu, need_r);
    unsigned np = __ballot_sync(0xffffffffu, need_p);
    // row r's two 16-byte chunks are stored swapped when bit 2 of r is set,
    // so that the eight rows an ldmatrix phase reads fall in distinct banks
    const int sw = (lane >> 2) & 1;
    __syncwarp();
    {
        uint4 r0, r1;
        gate_row(xr, r0, r1);
        tile[2 * lane + sw] = r0;
        tile[2 * lane + (sw ^ 1)] = r1;
        gate_row(xp, r0, r1);
        tile[2 * (32 + lane) + sw] = r0;
        tile[2 * (32 + lane) + (sw ^ 1)] = r1;
    }
    __syncwarp();
    // sample row r of m-tile mt ends in fragment group r % 8, half r / 8 (c[0]
    // or c[2]); the lane's own rows are (mt = lane / 16, r = lane % 16) for
    // the density and (mt = 2 + lane / 16, same r) for the pressure
    const int src = 4 * (lane & 7), half = (lane >> 3) & 1, hi16 = lane >> 4;
#pragma unroll 1
    for (int mt = 0; mt < 4; ++mt) {
        if (both && mt == 2) np = __ballot_sync(0xffffffffu, need_p && (!need_r || zr < 0.f));
        if ((((mt < 2 ? nr : np) >> (16 * (mt & 1))) & 0xffffu) == 0u) continue;   // uniform over the warp
        unsigned a[4];
        ldsm_x4(a[0], a[1], a[2], a[3], tile + 2 * (16 * mt + (lane & 15)) + ((lane >> 4) ^ ((lane >> 2) & 1)));
        // layer 1: its accumulator fragments become layer 2's A fragments
        // (k-tile nt / 2; rows g in registers 0, 2, rows g + 8 in 1, 3)
        unsigned hh[2][4], hl[2][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint2 bb = lds_u64(&g.b1[nt * 8 + 2 * t]);
            const uint2 w = lds_u64(&g.w1f[nt][lane][0]);
            float c[4];
            mma_k16c(c, a[0], a[1], a[2], a[3], w.x, w.y, __uint_as_float(bb.x), __uint_as_float(bb.y));
            relu_split(c[0], c[1], hh[nt >> 1][(nt & 1) * 2], hl[nt >> 1][(nt & 1) * 2]);
            relu_split(c[2], c[3], hh[nt >> 1][(nt & 1) * 2 + 1], hl[nt >> 1][(nt & 1) * 2 + 1]);
        }
        // layers 2 and 3, k-tile by k-tile of layer 3: layer-2 n-tiles 2 kt
        // and 2 kt + 1 form layer 3's A fragments of k-tile kt
        const float b3 = __uint_as_float(lds_u32(&g.b3));
        float z[4] = {b3, b3, b3, b3};
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            unsigned gh[4], gl[4];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int nt = 2 * kt + j;
                const uint2 bb = lds_u64(&g.b2[nt * 8 + 2 * t]);
                float c[4] = {__uint_as_float(bb.x), __uint_as_float(bb.y), __uint_as_float(bb.x),
                              __uint_as_float(bb.y)};
                const uint2 h0 = lds_u64(&g.w2h[0][nt][lane][0]), h1 = lds_u64(&g.w2h[1][nt][lane][0]);
                mma_k16(c, hh[0], h0);
                mma_k16(c, hh[1], h1);
                mma_k16(c, hl[0], h0);
                mma_k16(c, hl[1], h1);
                const uint2 l0 = lds_u64(&g.w2l[0][nt][lane][0]), l1 = lds_u64(&g.w2l[1][nt][lane][0]);
                mma_k16(c, hh[0], l0);
                mma_k16(c, hh[1], l1);
                relu_split(c[0], c[1], gh[j * 2], gl[j * 2]);
                relu_split(c[2], c[3], gh[j * 2 + 1], gl[j * 2 + 1]);
            }
            const uint2 wh = lds_u64(&g.w3h[kt][lane][0]), wl = lds_u64(&g.w3l[kt][lane][0]);
            mma_k16(z, gh, wh);
            mma_k16(z, gl, wh);
            mma_k16(z, gh, wl);
        }
        const float v0 = __shfl_sync(0xffffffffu, z[0], src), v1 = __shfl_sync(0xffffffffu, z[2], src);
        const float v = half ? v1 : v0;
        if (mt == hi16) zr = v;
        if (mt == 2 + hi16) zp = v;
    }
}

// Relative round-off floor of the gate's flat test (MFC_GATE_FLOOR).
constexpr float kGateFloor32 = (float)MFC_GATE_FLOOR;

// Normalised sensor stencil: x_k = (v_k - v_2) / max_j |v_j - v_2|.  Returns
// false, with x = 0, when the stencil is flat -- max_j |v_j - v_2| <= floor
// |v_2| -- and counts as smooth without the network.
__device__ __forceinline__ bool gate_input(const float* v, float* x) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) m = fmaxf(m, fabsf(v[k] - v[2]));
    const bool live = m > kGateFloor32 * fabsf(v[2]);
    const float r = live ? __frcp_rn(m) : 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) x[k] = (v[k] - v[2]) * r;
    return live;
}

// Linear-weight (fifth-order upwind) face values of cell i: the WENO5
// candidates combined with the linear weights, written in differences.
__device__ __forceinline__ void linear5(float v0, float v1, float v2, float v3, float v4, float& vm, float& vp) {
    float d1 = v1 - v0, d2 = v2 - v1, d3 = v3 - v2, d4 = v4 - v3;
    vm = v2 + (0.1f * (5.f * d2 - 2.f * d1) + 0.6f * (d2 + 2.f * d3) + 0.3f * (4.f * d3 - d4)) * (1.f / 6.f);
    vp = v2 + (0.3f * (d1 - 4.f * d2) - 0.6f * (2.f * d2 + d3) + 0.1f * (2.f * d4 - 5.f * d3)) * (1.f / 6.f);
}

// A reconstructed face state is usable when rho > 0, 0 <= alpha1 <= 1 and
// p + pi_inf of the mixture is positive ((Gamma + 1) p + Pi > 0).
template <int NDIM>
__device__ __forceinline__ bool face_ok(const EosR<float, 2>& e, const float* w) {
    using FL = Fields<NDIM>;
    float a1 = w[FL::IA];
    float G, Pi;
    mixture(e, w + FL::IA, G, Pi);
    return (w[0] + w[1] > 0.f) && (a1 >= 0.f) && (a1 <= 1.f) && ((G + 1.f) * w[FL::IE] + Pi > 0.f);
}

// ---- TMA staging (MFC_TMA_YZ builds) ----------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// True once the phase of `bar` with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One 4-D box of the tensor map into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Minimum resident blocks for the register allocator, in blocks of the
// sweep's own size (x sweeps run one-warp blocks, each with its own output
// tile in static shared memory).
template <int FORM, int MODE, int DIR, int NF = 2>
constexpr int sweep_min_blocks() {
    if (NF > 2) return 1;   // more fields per cell: no register cap (the two-fluid caps spill)
    constexpr int per128 = FORM == FORM_MIXED   ? (MODE == SW_LAST_RK ? MFC_MIN_BLOCKS_MIXED_RK
                                                   : DIR == 0         ? MFC_MIN_BLOCKS_MIXED_X
                                                                      : MFC_MIN_BLOCKS_MIXED)
                           : FORM == FORM_GATED ? (MODE == SW_LAST_RK ? MFC_MIN_BLOCKS_GATED_RK : MFC_MIN_BLOCKS_GATED)
                                                : MFC_MIN_BLOCKS_FP64;
    return per128 * 128 / sweep_threads(DIR);
}

// NU: some direction of the grid is non-uniform (tables, per-cell widths);
// the uniform-grid kernels carry none of that code.
template <int NDIM, int DIR, int MODE, int FORM, bool NU, int NF>
__global__ void __launch_bounds__(sweep_threads(DIR), sweep_min_blocks<FORM, MODE, DIR, NF>())
sweep_kernel(const SweepArgs a, const __grid_constant__ CUtensorMap tmap) {
    using R = FormReal<FORM>;
    constexpr bool EXACT = FORM == FORM_FP64_EXACT;
    constexpr bool GATED = FORM == FORM_GATED;
    using FL = Fields<NDIM, NF>;
    using LS = LoadSet<NDIM, R, NF>;
    constexpr int NEQ = FL::NEQ, IE = FL::IE, IA = FL::IA, NA = FL::NA;
    constexpr int NL = LS::N;
    constexpr bool MIXED = FORM == FORM_MIXED || FORM == FORM_GATED;
    constexpr int CH = XStage<R>::CH, PITCH = XStage<R>::PITCH;
    constexpr int WARPS = sweep_threads(DIR) / 32;
    // x sweep writing the accumulator: the warp collects each sector's worth
    // of cells (CH along x) of its 32 rows here and stores whole sectors
    constexpr bool OSTAGE_ON = DIR == 0 && MODE == SW_FIRST;
    constexpr int OSTAGE = NEQ * 32 * PITCH;
    __shared__ R ostage[OSTAGE_ON ? WARPS * OSTAGE : 1];
    __shared__ GateSmem gsm[GATED ? 1 : 0 + 1];
    __shared__ uint4 gtile[GATED ? WARPS * 128 : 1];
    // TMA staging of the FP32 y/z sweeps: per warp two slots of NL fields x
    // kTmaCells cells x 32 lanes, one mbarrier per slot
    constexpr bool TMA = MFC_TMA_YZ && (FORM == FORM_MIXED || FORM == FORM_GATED) && (DIR == 1 || DIR == 2) && !NU;
    constexpr int TC = kTmaCells, TSLOT = NL * TC * 32;
    __shared__ __align__(128) float tbuf[TMA ? WARPS * 2 * TSLOT : 1];
    __shared__ __align__(8) uint64_t tbar[TMA ? WARPS * 2 : 1];
    if constexpr (GATED) {
        gate_fill(gsm[0], a.gate_w);   // every thread, before any warp leaves
        __syncthreads();
    }

    const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
    const int na = DIR == 0 ? n1 : n0;
    const int nb = DIR == 2 ? n1 : n2;
    const int ns = a.n[DIR];
    const long long sa = DIR == 0 ? (long long)n0 : 1LL;
    const long long sb = DIR == 2 ? (long long)n0 : (long long)n0 * n1;
    const long long ss = DIR == 0 ? 1LL : (DIR == 1 ? (long long)n0 : (long long)n0 * n1);
    const long long nchunk = (na + 31) >> 5;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    // This warp's cells in pencil-group order: group g = chunk + nchunk b
    // (32 adjacent pencils), cell j along the pencil at index g ns + j.
    // Balanced mapping: an even share of all of them, which may span the end
    // of one group and the start of the next (one piece each).  Seg mapping:
    // one segment of `seg` cells of one group.
    // (Forms on the seg mapping only, sweep_balanced false, run the piece loop
    // once on gseg, sseg0, sseg1.)
    constexpr bool BAL = sweep_balanced(FORM, NF);
    long long r0, r1, gseg = 0;
    int sseg0 = 0, sseg1 = 0;
    if (BAL && a.nwarps > 0) {
        if (warp >= a.nwarps) return;  // uniform over the warp
        const long long T = nchunk * nb * ns;
        r0 = warp * T / a.nwarps;
        r1 = (warp + 1) * T / a.nwarps;
    } else {
        const int seg = a.seg;
        const long long nseg = (ns + seg - 1) / seg;
        if (warp >= nchunk * nseg * nb) return;  // uniform over the warp
        const long long rest = warp / nchunk;
        gseg = warp % nchunk + nchunk * (rest / nseg);
        sseg0 = (int)(rest % nseg) * seg;
        sseg1 = min(sseg0 + seg, ns);
        r0 = gseg * ns + sseg0;
        r1 = gseg * ns + sseg1;
    }
    const long long nc = a.ncell;
    const R inv_dx = sizeof(R) == 4 ? R(a.inv_dx32[DIR]) : R(a.inv_dx[DIR]);
    const R eps = R(a.eps);
    // FP64 reference-order form: a uniform width along DIR that is a power of two
    // (zero fraction bits) with a normal reciprocal, which a.rdx then holds exactly
    const unsigned dxh = (unsigned)__double2hiint(a.dx[DIR]), dxe = (dxh >> 20) & 0x7ffu;
    const bool pow2_dx = EXACT && (dxh & 0x800fffffu) == 0u && __double2loint(a.dx[DIR]) == 0 && dxe - 2u < 2043u;
    const EosR<R, NF> er(a.eos);
    const R* __restrict__ qin = static_cast<const R*>(a.qin);
    const int wib = threadIdx.x >> 5;

    // the FP64 reference-order kernels are FP64-pipe bound with latency to spare:
    // the registers of a prefetched cell go to the carried candidates instead
    constexpr bool PCARRY = EXACT && !GATED && !NU && NF == 2 && MFC_CAND_CARRY;
    constexpr bool PREFETCH = MFC_PREFETCH != 0 && !PCARRY;
    constexpr bool EPI_PREFETCH = PREFETCH && MIXED;
    bool bad_any = false, tma_fail = false;
    R smax = R(0);
    unsigned n_gated = 0, n_fallback = 0, n_cells = 0, n_flat = 0;
    double dt = 0.0;
    if (MODE == SW_LAST_RK) dt = a.ctrl->dt;
    // FP32 forms: SSP-RK3 in increment form, q^(k) = q^n + D_k with FP32
    // increments D_1 = dt L(q^n), D_2 = (D_1 + dt L(q^(1)))/4,
    // D_3 = 2 (D_2 + dt L(q^(2)))/3 -- the same stages as
    // q^(2) = 3/4 q^n + 1/4 (q^(1) + dt L), q^(3) = 1/3 q^n + 2/3 (q^(2) + dt L) --
    // and one FP64 addition per field forms q^(k) from the FP64 q^n
    const float dt32 = float(dt);
    const float kfac = a.stage == 2 ? 0.25f : (2.0f / 3.0f);

    for (long long r = r0; r < r1;) {
        long long g = gseg;
        int s0 = sseg0, s1 = sseg1;
        if constexpr (BAL) {
            g = r / ns;
            s0 = (int)(r - g * ns);
            s1 = (int)min((long long)ns, r1 - g * ns);
        }
        r = g * ns + s1;
        const int chunk = (int)(g % nchunk);
        const int b = (int)(g / nchunk);
        const int ia = chunk * 32 + lane;
        const bool active = ia < na;
        // inactive lanes follow a valid pencil so that every address is in bounds;
        // their results are discarded
        const long long base = (long long)(active ? ia : na - 1) * sa + (long long)b * sb;
        bool bad = false;
        unsigned p_gated = 0, p_fallback = 0, p_cells = 0, p_flat = 0;

        // Values of loaded cell k (index s0 - 3 + k along the pencil) -> v[].
        // Along y and z the warp's 32 loads form one coalesced row per field;
        // along x each lane reads its own row, and the 32-byte sector it brings
        // into L1 serves the lane's next CH - 1 cells.
        // TMA staging: interior segments (no ghost cell) of launches given a
        // tensor map read their cells from the warp's shared-memory slots; chunk
        // ck (cells s0 - 3 + ck TC ..) lands in slot ck & 1, and starting to read
        // chunk ck refills the other slot with chunk ck + 1.  Waits are bounded:
        // a box that never lands sets status bit 2 instead of hanging.
        const int kcells = s1 - s0 + 6;
        const bool use_tma = TMA && a.tmap && a.nwarps == 0 && s0 >= 3 && s1 + 3 <= ns;
        auto tma_issue = [&](int ck) {   // one lane
            if constexpr (TMA) {
                uint64_t* bar = tbar + wib * 2 + (ck & 1);
                float* dst = tbuf + (wib * 2 + (ck & 1)) * TSLOT;
                mbar_expect_tx(bar, (unsigned)(TSLOT * sizeof(float)));
                const int jc = s0 - 3 + ck * TC;
#pragma unroll
                for (int f = 0; f < NL; ++f) {
                    if constexpr (DIR == 1) tma_load_4d(dst + f * TC * 32, &tmap, chunk * 32, jc, b, LS::field(f), bar);
                    else tma_load_4d(dst + f * TC * 32, &tmap, chunk * 32, b, jc, LS::field(f), bar);
                }
            }
        };
        if constexpr (TMA) {
            if (use_tma) {
                if (lane == 0) {
                    mbar_init(tbar + wib * 2, 1);
                    mbar_init(tbar + wib * 2 + 1, 1);
                    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
                }
                __syncwarp();
                if (lane == 0) tma_issue(0);
            }
        }

        // FP32 x sweep with rows of a multiple of 4 cells: 16-byte aligned rows,
        // loaded four cells at a time (cells are fetched in order along the row)
        constexpr bool XVEC = MIXED && DIR == 0 && MFC_XVEC;
        const bool xvec_ok = XVEC && (n0 & 3) == 0;
        float xq[XVEC ? NL : 1][3];
        int xpend = 0;

        // A ghost cell beyond a side that borders another block (block
        // decomposition) comes from that side's halo buffer; any other from the
        // BC index map.  j is the same for the whole warp.
        auto fetch = [&](int k, R* v) {
            if constexpr (TMA) {
                if (use_tma) {
                    const int ck = k / TC, cc = k - ck * TC;
                    if (cc == 0) {
                        bool ok = false;
                        for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(tbar + wib * 2 + (ck & 1), (ck >> 1) & 1);
                        tma_fail |= !ok;
                        if ((ck + 1) * TC < kcells) {
                            // every lane's reads of the slot being refilled (chunk
                            // ck - 1) are ordered before the copy that overwrites it
                            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                            __syncwarp();
                            if (lane == 0) tma_issue(ck + 1);
                        }
                    }
                    const float* src = tbuf + (wib * 2 + (ck & 1)) * TSLOT + cc * 32 + lane;
#pragma unroll
                    for (int f = 0; f < NL; ++f) v[f] = src[f * TC * 32];
                    return;
                }
            }
            const int j = s0 - 3 + k;
            if constexpr (XVEC) {
                // FP32 x sweep: four cells of the lane's row per 16-byte load, the
                // three not yet used kept in registers for the next steps
                if (xpend > 0) {
#pragma unroll
                    for (int f = 0; f < NL; ++f) {
                        v[f] = xq[f][0];
                        xq[f][0] = xq[f][1];
                        xq[f][1] = xq[f][2];
                    }
                    --xpend;
                    return;
                }
                if (xvec_ok && (j & 3) == 0 && j >= 0 && j + 3 < ns) {
#pragma unroll
                    for (int f = 0; f < NL; ++f) {
                        const float4 t = __ldg(reinterpret_cast<const float4*>(qin + LS::field(f) * nc + base + j));
                        v[f] = t.x;
                        xq[f][0] = t.y;
                        xq[f][1] = t.z;
                        xq[f][2] = t.w;
                    }
                    xpend = 3;
                    return;
                }
            }
            const R* h = j < 0 ? static_cast<const R*>(a.hlo) : (j >= ns ? static_cast<const R*>(a.hhi) : nullptr);
            if (h) {
                // the pencil's position in the plane normal to DIR, from its first
                // cell `base` (x fastest): y + n1 z along x, x + n0 z along y, x + n0 y along z
                long long p;
                if constexpr (DIR == 0) p = base / n0;
                else if constexpr (DIR == 1) p = base % n0 + (long long)n0 * (base / ((long long)n0 * n1));
                else p = base;
                const long long hc = (long long)(j < 0 ? j + 3 : j - ns) * a.hplane + p;
#pragma unroll
                for (int f = 0; f < NL; ++f) v[f] = __ldg(h + (long long)LS::field(f) * 3 * a.hplane + hc);
            } else {
                const long long c = base + (long long)bc_index(j, ns, a.periodic) * ss;
#pragma unroll
                for (int f = 0; f < NL; ++f) v[f] = __ldg(qin + LS::field(f) * nc + c);
            }
        };

        R W[5][NEQ];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            R v[NL];
            fetch(k, v);
            if constexpr (EXACT) exact::cons_to_prim<NDIM, NF>(a.eos, v, W[k]);
            else to_prim<NDIM, NF>(er, v, W[k]);
            bad |= !pos(mix_rho<NF>(W[k]));
        }
        // FP64 reference-order form: the smoothness indicators' curvature terms
        // of the window's stencils {i-2..i}, {i-1..i+1} (cell i = window centre),
        // carried along the pencil so that each is formed once (exact::curv)
        constexpr bool TCARRY = EXACT && !GATED && !NU && NF == 2;
        double Tm[TCARRY ? NEQ : 1], T0[TCARRY ? NEQ : 1];
        if constexpr (TCARRY) {
#pragma unroll
            for (int f = 0; f < NEQ; ++f) {
                Tm[f] = exact::curv(W[0][f], W[1][f], W[2][f]);
                T0[f] = exact::curv(W[1][f], W[2][f], W[3][f]);
            }
        }
        // and the right-face candidates of the window's centre cell, carried as
        // the left-face candidates of the cell before it (exact::weno5_tc)
        double Pr0[PCARRY ? NEQ : 1], Pr1[PCARRY ? NEQ : 1];
        if constexpr (PCARRY) {
#pragma unroll
            for (int f = 0; f < NEQ; ++f) exact::weno5_right01(W[0][f], W[1][f], W[2][f], W[3][f], Pr0[f], Pr1[f]);
        }
        // mixed form, x sweep: the first differences d1..d3 and curvature parts C0, C1
        // of the window's centre cell, carried along the pencil (weno5_dc); the y and
        // z sweeps, register-capped for occupancy, lose more to spills than it saves
        constexpr bool DCARRY = FORM == FORM_MIXED && !NU && DIR == 0 && MFC_DIFF_CARRY;
        float Dd1[DCARRY ? NEQ : 1], Dd2[DCARRY ? NEQ : 1], Dd3[DCARRY ? NEQ : 1];
        float Cc0[DCARRY ? NEQ : 1], Cc1[DCARRY ? NEQ : 1];
        const float c13f = float(13.0 / 12.0);
        if constexpr (DCARRY) {
#pragma unroll
            for (int f = 0; f < NEQ; ++f) {
                Dd1[f] = float(W[1][f] - W[0][f]);
                Dd2[f] = float(W[2][f] - W[1][f]);
                Dd3[f] = float(W[3][f] - W[2][f]);
                const float D0 = Dd2[f] - Dd1[f], D1 = Dd3[f] - Dd2[f];
                Cc0[f] = c13f * D0 * D0;
                Cc1[f] = c13f * D1 * D1;
            }
        }
        R vmPrev[NEQ], Fprev[NEQ];
        R ufPrev = R(0), alphaCell[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) alphaCell[i] = R(0);
#pragma unroll
        for (int f = 0; f < NEQ; ++f) vmPrev[f] = Fprev[f] = R(0);

        for (int j = s0 - 1; j <= s1; ++j) {
            // the cell that enters the window at the end of this iteration: its
            // loads are issued now and complete under this iteration's arithmetic
            R vnext[NL];
            if (PREFETCH && j < s1) fetch(j + 3 - (s0 - 3), vnext);
            // the FP32 forms also issue the stage-update operands of the cell
            // this iteration completes (cell j - 1) here, ahead of the stencil work
            R accp[NEQ], qkp[NEQ];
            double qnp[NEQ];
            if constexpr (EPI_PREFETCH) {
                if (j > s0) {
                    const long long c = base + (long long)(j - 1) * ss;
                    if constexpr (NDIM > 1 && MODE != SW_FIRST) {
                        const R* acc = static_cast<const R*>(a.acc);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) accp[f] = acc[f * nc + c];
                    }
                    if constexpr (MODE == SW_LAST_RK) {
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) qnp[f] = __ldg(a.qn + f * nc + c);
                        if (a.stage != 1) {
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) qkp[f] = a.dinc[f * nc + c];   // D_(k-1)
                        }
                    }
                }
            }
            R vm[NEQ], vp[NEQ];
            bool use_weno = true;
            if constexpr (GATED) {
                // gate: linear weights when the density and the pressure stencil
                // are both smooth -- flat (below the round-off floor), or called
                // smooth by the network (logit < 0) -- and the faces stay physical;
                // all 32 lanes take part in the tensor-core evaluation, which a
                // warp step whose stencils are all flat skips
                float sr[5], sp[5], xr[5], xp[5], zr = -1.f, zp = -1.f;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    sr[k] = W[k][0] + W[k][1];
                    sp[k] = W[k][IE];
                }
                const bool live_r = gate_input(sr, xr), live_p = gate_input(sp, xp);
                const bool warp_flat = !__any_sync(0xffffffffu, live_r || live_p);
                if (!warp_flat)
                    gate_logits(gsm[0], gtile + (threadIdx.x >> 5) * 128, xr, xp, live_r, live_p, true, zr, zp);
                const bool smooth = (!live_r || zr < 0.f) && (!live_p || zp < 0.f);
                if (smooth) {
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) linear5(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
                    use_weno = !(face_ok<NDIM>(er, vm) && face_ok<NDIM>(er, vp));
                }
                if (j >= s0 && j < s1) {   // count each cell once (not the segment halos)
                    p_fallback += smooth && use_weno;
                    p_gated += smooth && !use_weno;
                    p_cells += 1;
                    p_flat += warp_flat;
                    if (a.gate_dec && active) a.gate_dec[base + (long long)j * ss] = smooth ? (use_weno ? 2 : 1) : 0;
                }
            }
            if (use_weno) {
                if (NU && a.tab) {   // non-uniform direction: this cell's table (uniform over the warp)
                    const R* T = static_cast<const R*>(a.tab) + (long long)(j + 1) * kTabDoubles;
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) weno5_tab<R>(T, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], eps, vm[f], vp[f]);
                } else if (GATED || a.order == 5) {
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) {
                        if constexpr (PCARRY) {
                            const double Tp = exact::curv(W[2][f], W[3][f], W[4][f]);
                            exact::weno5_tc(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], Tm[f], T0[f], Tp,
                                            Pr0[f], Pr1[f], vm[f], vp[f]);
                            Tm[f] = T0[f];
                            T0[f] = Tp;
                        } else if constexpr (TCARRY) {
                            const double Tp = exact::curv(W[2][f], W[3][f], W[4][f]);
                            exact::weno5_t(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], Tm[f], T0[f], Tp,
                                           vm[f], vp[f]);
                            Tm[f] = T0[f];
                            T0[f] = Tp;
                        } else if constexpr (EXACT) {
                            exact::weno5(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
                        } else if constexpr (DCARRY) {
                            const float d4 = float(W[4][f] - W[3][f]);
                            const float D2 = d4 - Dd3[f];
                            const float C2 = c13f * D2 * D2;
                            float fm, fp;
                            weno5_dc(float(W[2][f]), Dd1[f], Dd2[f], Dd3[f], d4, Cc0[f], Cc1[f], C2, float(eps), fm, fp);
                            vm[f] = R(fm);
                            vp[f] = R(fp);
                            Dd1[f] = Dd2[f];
                            Dd2[f] = Dd3[f];
                            Dd3[f] = d4;
                            Cc0[f] = Cc1[f];
                            Cc1[f] = C2;
                        } else {
                            weno5(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], eps, vm[f], vp[f]);
                        }
                    }
                } else {   // WENO3 (uniform over the launch): cells i-1 .. i+1 of the window
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) {
                        if constexpr (EXACT) exact::weno3(a.eps, W[1][f], W[2][f], W[3][f], vm[f], vp[f]);
                        else weno3(W[1][f], W[2][f], W[3][f], eps, vm[f], vp[f]);
                    }
                }
            }
            if (j >= s0) {
                R F[NEQ], uf;
                if constexpr (EXACT) bad |= exact::hllc<NDIM, DIR, NF>(a.eos, vmPrev, vp, F, uf);
                else bad |= hllc<NDIM, DIR, R, NF>(er, vmPrev, vp, F, uf);
                if (j > s0 && (active || OSTAGE_ON)) {
                    // cell i = j - 1 is complete: faces i-1/2 (Fprev) and i+1/2 (F)
                    R L[NEQ];
                    if constexpr (EXACT) {
                        // (F_{i-1/2} - F_{i+1/2})/dx, then + alpha1 (u_f+ - u_f-)/dx
                        double dx = a.dx[DIR], rdx = a.rdx[DIR];
                        if (NU && a.cw[DIR]) {   // non-uniform: the cell's own width
                            dx = __ldg(a.cw[DIR] + (j - 1));
                            rdx = __ldg(a.crw[DIR] + (j - 1));
                        }
                        if (pow2_dx && !(NU && a.cw[DIR])) {
                            // a power-of-two width: x / dx and x * (1/dx) are the same real
                            // number, so one multiplication gives the quotient's bits
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) L[f] = (Fprev[f] - F[f]) * rdx;
#pragma unroll
                            for (int i = 0; i < NA; ++i) L[IA + i] = L[IA + i] + alphaCell[i] * (uf - ufPrev) * rdx;
                        } else {
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) L[f] = exact::div_rcp(Fprev[f] - F[f], dx, rdx);
#pragma unroll
                            for (int i = 0; i < NA; ++i)
                                L[IA + i] = L[IA + i] + exact::div_rcp(alphaCell[i] * (uf - ufPrev), dx, rdx);
                        }
                    } else {
                        R idx = inv_dx;
                        if (NU && a.cw[DIR]) {
                            if constexpr (sizeof(R) == 8) idx = __ldg(a.crw[DIR] + (j - 1));
                            else idx = __ldg(a.crw32[DIR] + (j - 1));
                        }
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) L[f] = (Fprev[f] - F[f]) * idx;
#pragma unroll
                        for (int i = 0; i < NA; ++i) L[IA + i] += alphaCell[i] * (uf - ufPrev) * idx;
                    }
                    const long long c = base + (long long)(j - 1) * ss;
                    if constexpr (OSTAGE_ON) {
                        R* o = ostage + (threadIdx.x >> 5) * OSTAGE + lane * PITCH + ((j - 1) & (CH - 1));
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) o[f * 32 * PITCH] = L[f];
                    } else if constexpr (MODE == SW_FIRST) {
                        R* acc = static_cast<R*>(a.acc);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) acc[f * nc + c] = L[f];
                    } else if constexpr (MODE == SW_MID) {
                        R* acc = static_cast<R*>(a.acc);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) acc[f * nc + c] = (EPI_PREFETCH ? accp[f] : acc[f * nc + c]) + L[f];
                    } else if constexpr (MODE == SW_LAST_RHS) {
                        const R* acc = static_cast<const R*>(a.acc);
                        double* out = static_cast<double*>(a.qout);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) {
                            R tot = NDIM > 1 ? (EPI_PREFETCH ? accp[f] : acc[f * nc + c]) + L[f] : L[f];
                            out[f * nc + c] = double(tot);
                        }
                    } else {  // SW_LAST_RK
                        const R* acc = static_cast<const R*>(a.acc);
                        double qnew[NEQ];
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) {
                            R tot = NDIM > 1 ? (EPI_PREFETCH ? accp[f] : acc[f * nc + c]) + L[f] : L[f];
                            double qn = EPI_PREFETCH ? qnp[f] : a.qn[f * nc + c];
                            if constexpr (MIXED) {
                                // D_k in FP32 from D_(k-1) and the FP32 L; q^(k) = q^n + D_k in FP64
                                float Dk;
                                if (a.stage == 1) {
                                    Dk = dt32 * float(tot);
                                } else {
                                    const float Dp = EPI_PREFETCH ? float(qkp[f]) : a.dinc[f * nc + c];
                                    Dk = kfac * fmaf(dt32, float(tot), Dp);
                                }
                                if (a.stage != 3) a.dinc[f * nc + c] = Dk;
                                qnew[f] = qn + f2d_bits(Dk);
                            } else {
                                double dL = dt * double(tot);
                                if (a.stage == 1) {
                                    qnew[f] = qn + dL;
                                } else {
                                    double qkd = double(qin[f * nc + c]);
                                    if (a.stage == 2)
                                        qnew[f] = 0.75 * qn + 0.25 * (qkd + dL);
                                    else
                                        qnew[f] = (1.0 / 3.0) * qn + (2.0 / 3.0) * (qkd + dL);
                                }
                            }
                        }
                        if constexpr (!MIXED) {
                            double* out = static_cast<double*>(a.qout);
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) out[f * nc + c] = qnew[f];
                            if (a.stage == 3) {
                                R s;
                                double dx3[3], rdx3[3], idx3[3];
                                cell_geometry<DIR, NU>(a, j - 1, active ? ia : na - 1, b, dx3, rdx3, idx3);
                                if constexpr (EXACT) {
                                    s = exact::cell_wavespeed<NDIM, NF>(a.eos, qnew, dx3, rdx3, bad);
                                } else {
                                    double wn[NEQ];
                                    to_prim<NDIM, NF>(er, qnew, wn);
                                    s = cell_wavespeed<NDIM, double, NF>(er, wn, idx3, bad);
                                }
                                smax = s > smax ? s : smax;
                            }
                        } else {
                            float q32[NEQ];
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) q32[f] = d2f_bits(qnew[f]);
                            float pnew = mixed_pressure<NDIM, NF>(a.eos, qnew, q32);
                            float* o32 = static_cast<float*>(a.stage == 3 ? a.qout2 : a.qout);
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) o32[f * nc + c] = q32[f];
                            o32[NEQ * nc + c] = pnew;
                            if (a.stage == 3) {
                                double* o64 = static_cast<double*>(a.qout);
#pragma unroll
                                for (int f = 0; f < NEQ; ++f) o64[f * nc + c] = qnew[f];
                                float v[NEQ], wn[NEQ];
#pragma unroll
                                for (int f = 0; f < NEQ; ++f) v[f] = q32[f];
                                v[IE] = pnew;
                                to_prim<NDIM, NF>(er, v, wn);
                                float idx32[3] = {a.inv_dx32[0], a.inv_dx32[1], a.inv_dx32[2]};
                                if constexpr (NU) {
                                    double dx3[3], rdx3[3], idx3[3];
                                    cell_geometry<DIR, NU>(a, j - 1, active ? ia : na - 1, b, dx3, rdx3, idx3);
#pragma unroll
                                    for (int d = 0; d < 3; ++d) idx32[d] = float(idx3[d]);
                                }
                                R s = cell_wavespeed<NDIM, float, NF>(er, wn, idx32, bad);
                                smax = s > smax ? s : smax;
                            }
                        }
                    }
                }
#pragma unroll
                for (int f = 0; f < NEQ; ++f) Fprev[f] = F[f];
                ufPrev = uf;
                if constexpr (OSTAGE_ON) {
                    // cell i = j - 1 closes a sector (or the segment): the warp writes
                    // cells max(x0, s0) .. i of its rows, whole sectors per row
                    const int i = j - 1;
                    if (j > s0 && ((i & (CH - 1)) == CH - 1 || j == s1)) {
                        __syncwarp();
                        const int x0 = i & ~(CH - 1), lo = max(x0, s0);
                        const int t = lane % CH, x = x0 + t;
                        const R* o = ostage + (threadIdx.x >> 5) * OSTAGE;
                        R* acc = static_cast<R*>(a.acc);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            const int r = lane / CH + (32 / CH) * k;
                            const int row = chunk * 32 + r;
                            if (x >= lo && x <= i && row < na) {
                                const long long cc = (long long)row * sa + (long long)b * sb + x;
#pragma unroll
                                for (int f = 0; f < NEQ; ++f) acc[f * nc + cc] = o[(f * 32 + r) * PITCH + t];
                            }
                        }
                        __syncwarp();
                    }
                }
            }
#pragma unroll
            for (int f = 0; f < NEQ; ++f) vmPrev[f] = vm[f];
#pragma unroll
            for (int i = 0; i < NA; ++i) alphaCell[i] = W[2][IA + i];
            if (j < s1) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) W[k][f] = W[k + 1][f];
                if (!PREFETCH) fetch(j + 3 - (s0 - 3), vnext);
                if constexpr (EXACT) exact::cons_to_prim<NDIM, NF>(a.eos, vnext, W[4]);
                else to_prim<NDIM, NF>(er, vnext, W[4]);
                bad |= !pos(mix_rho<NF>(W[4]));
            }
        }
        // only cells this lane owns count (inactive lanes and segment halos excluded)
        bad_any |= bad && active;
        if (active) {
            n_gated += p_gated;
            n_fallback += p_fallback;
            n_cells += p_cells;
            n_flat += p_flat;
        }
        if constexpr (!BAL) break;   // the seg mapping gives one piece
    }

    if constexpr (MODE == SW_LAST_RK) {
        if (a.stage == 3) {
            R m = warp_max(smax);
            if (lane == 0 && m > R(0))
                atomicMax(&a.ctrl->S_bits, (unsigned long long)__double_as_longlong(double(m)));
        }
    }
    if (__any_sync(0xffffffffu, bad_any) && lane == 0) atomicOr(&a.ctrl->status, 1u);
    if constexpr (TMA) {
        if (__any_sync(0xffffffffu, tma_fail) && lane == 0) atomicOr(&a.ctrl->status, 4u);
    }
    if constexpr (GATED) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_gated += __shfl_xor_sync(0xffffffffu, n_gated, o);
            n_fallback += __shfl_xor_sync(0xffffffffu, n_fallback, o);
            n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
            n_flat += __shfl_xor_sync(0xffffffffu, n_flat, o);
        }
        if (lane == 0) {
            atomicAdd(&a.ctrl->gated, (unsigned long long)n_gated);
            atomicAdd(&a.ctrl->fallback, (unsigned long long)n_fallback);
            atomicAdd(&a.ctrl->cells, (unsigned long long)n_cells);
            atomicAdd(&a.ctrl->flat, (unsigned long long)n_flat);
        }
    }
}

// Resident blocks of one sweep kernel on the current device (occupancy x
// SMs), looked up once per kernel and device (devices may differ in SM count).
template <int NDIM, int DIR, int MODE, int FORM, bool NU, int NF>
long long sweep_slots() {
    constexpr int kMaxDev = 64;
    static long long cache[kMaxDev];   // 0: not yet looked up (a benign race: every writer stores the same value)
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (dev >= 0 && dev < kMaxDev && cache[dev] > 0) return cache[dev];
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<NDIM, DIR, MODE, FORM, NU, NF>,
                                                      sweep_threads(DIR), 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long slots = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < kMaxDev) cache[dev] = slots;
    return slots;
}

// Cells per warp along the pencil.  Short segments duplicate halo work (two
// extra reconstructions and one extra Riemann solve per segment), long ones
// leave fewer blocks to spread over the SMs.  Start from the longest power of
// two up to 32 that still gives 152 x 256 threads (4 where none does), then
// double while the grid still fills the resident blocks MFC_MIN_WAVES times
// over, up to MFC_MAX_SEG.
inline int pick_seg(int dir, const int* n, int threads, long long slots) {
    int seg = 32;
    while (seg > 4 && sweep_warps(dir, n, seg) * 32 < 152LL * 256) seg >>= 1;
    while (seg < MFC_MAX_SEG &&
           (sweep_warps(dir, n, 2 * seg) * 32 + threads - 1) / threads >= MFC_MIN_WAVES * slots)
        seg <<= 1;
    return seg;
}

template <int NDIM, int DIR, int MODE, int FORM, bool NU, int NF>
cudaError_t launch_kernel(const SweepArgs& a0, cudaStream_t s) {
    constexpr int T = sweep_threads(DIR);
    constexpr bool TMA = MFC_TMA_YZ && (FORM == FORM_MIXED || FORM == FORM_GATED) && (DIR == 1 || DIR == 2) && !NU;
    SweepArgs a = a0;
    const long long slots = sweep_slots<NDIM, DIR, MODE, FORM, NU, NF>();
    constexpr bool BAL = sweep_balanced(FORM, NF);
    long long blocks;
    if (BAL && !(TMA && a.tmap)) {
        // balanced mapping: MFC_BAL_WAVES x the resident warps, each taking at
        // least MFC_BAL_MIN_CELLS cells
        const long long cells = sweep_group_cells(DIR, a.n);
        long long w = slots * (T / 32) * MFC_BAL_WAVES;
        const long long wmax = (cells + MFC_BAL_MIN_CELLS - 1) / MFC_BAL_MIN_CELLS;
        if (w > wmax) w = wmax;
        a.nwarps = w;
        a.seg = 0;
        blocks = (w * 32 + T - 1) / T;
    } else {
        a.nwarps = 0;
        a.seg = pick_seg(DIR, a.n, T, slots);
        blocks = (sweep_warps(DIR, a.n, a.seg) * 32 + T - 1) / T;
    }
    if (blocks <= 0 || a.dry) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    CUtensorMap tm;
    if (a.tmap) tm = *static_cast<const CUtensorMap*>(a.tmap);
    else memset(&tm, 0, sizeof(tm));
    sweep_kernel<NDIM, DIR, MODE, FORM, NU, NF><<<(unsigned)blocks, T, 0, s>>>(a, tm);
    return cudaGetLastError();
}

template <int NDIM, int DIR, int MODE, int FORM, int NF>
cudaError_t launch_one(const SweepArgs& a, cudaStream_t s) {
    const bool nu = a.cw[0] || a.cw[1] || a.cw[2];
    if constexpr (FORM != FORM_GATED && NF == 2) {
        if (nu) return launch_kernel<NDIM, DIR, MODE, FORM, true, NF>(a, s);
    }
    if (nu) return cudaErrorInvalidValue;   // non-uniform grids: two fluids, non-gated forms
    return launch_kernel<NDIM, DIR, MODE, FORM, false, NF>(a, s);
}

// Launch one sweep: the valid (direction, mode) pairs are x FIRST, y MID
// (3-D), and LAST_RK / LAST_RHS on the last direction.
template <int NDIM, int FORM, int NF>
cudaError_t launch_sweep_t(int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    constexpr int LAST = NDIM - 1;
    if (dir == 0 && mode == SW_FIRST && NDIM > 1) {
        if constexpr (NDIM > 1) return launch_one<NDIM, 0, SW_FIRST, FORM, NF>(a, s);
    } else if (dir == 1 && mode == SW_MID && NDIM == 3) {
        if constexpr (NDIM == 3) return launch_one<NDIM, 1, SW_MID, FORM, NF>(a, s);
    } else if (dir == LAST && mode == SW_LAST_RK) {
        return launch_one<NDIM, LAST, SW_LAST_RK, FORM, NF>(a, s);
    } else if (dir == LAST && mode == SW_LAST_RHS) {
        return launch_one<NDIM, LAST, SW_LAST_RHS, FORM, NF>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <int FORM, int NF>
cudaError_t launch_sweep_nf(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    switch (ndim) {
        case 1: return launch_sweep_t<1, FORM, NF>(dir, mode, a, s);
        case 2: return launch_sweep_t<2, FORM, NF>(dir, mode, a, s);
        case 3: return launch_sweep_t<3, FORM, NF>(dir, mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

// Dispatch on the number of dimensions and of fluids (a.eos.nf): 2 in every
// form, 3 and 4 in the non-gated forms.
template <int FORM>
cudaError_t launch_sweep_any(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    if (a.eos.nf == 2) return launch_sweep_nf<FORM, 2>(ndim, dir, mode, a, s);
    if constexpr (FORM != FORM_GATED) {
        if (a.eos.nf == 3) return launch_sweep_nf<FORM, 3>(ndim, dir, mode, a, s);
        if (a.eos.nf == 4) return launch_sweep_nf<FORM, 4>(ndim, dir, mode, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mfc5
