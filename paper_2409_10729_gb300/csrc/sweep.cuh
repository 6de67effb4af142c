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
// `seg` cells of each.  For d = y, z the 32 lanes run along x, so every load
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
#include <cuda_fp16.h>

#include <type_traits>

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
    float G = q32[FL::IA] * float(e.dg[0]) + float(e.g[NF - 1]);
#pragma unroll
    for (int i = 1; i < FL::NA; ++i) G = G + q32[FL::IA + i] * float(e.dg[i]);
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
template <int NDIM, typename R, int NF = 2>
__device__ __forceinline__ R cell_wavespeed(const EosR<R, NF>& e, const R* w, const double* inv_dx, bool& bad) {
    using FL = Fields<NDIM, NF>;
    R rho = mix_rho<NF>(w);
    R G, Pi;
    mixture(e, w + FL::IA, G, Pi);
    R c2 = rdiv((G + R(1)) * w[FL::IE] + Pi, G * rho);
    bad |= !(rho > R(0)) || !(c2 > R(0));
    R c = sqrt_pos(c2);
    R s = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s += (fabs(w[FL::IU + d]) + c) * R(inv_dx[d]);
    bad |= !(s < R(INFINITY));
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

// ---- gate network on the tensor cores -------------------------------------
// A warp evaluates the network for its 32 cells x 2 sensors = 64 samples at
// once: layer 1 (5 -> 32, K padded to 8) as 4x4 mma.m16n8k8 and layer 2
// (32 -> 32) as 4x4x2 mma.m16n8k16, fp16 operands with FP32 accumulation;
// the fragments of layer 1's result are layer 2's A fragments as they stand.
// The 32 -> 1 output is a dot product of the layer-2 fragments with w3,
// reduced over the four lanes of a fragment group.
struct GateSmem {
    unsigned w1f[4][32];       // layer-1 B fragments, per n-tile and lane
    unsigned w2f[2][4][32][2]; // layer-2 B fragments, per k-tile, n-tile, lane
    unsigned w3f[2][32][2];    // layer-3 B fragments (w3 in every column), per k-tile, lane
    float b1[32], b2[32], b3;
};

__device__ __forceinline__ unsigned pack_half2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&h);
}

// max(lo, 0) and max(hi, 0) rounded to f16 and packed (lo in the low half).
__device__ __forceinline__ unsigned relu_half2(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Fill the block's fragment tables from the 1281 weights (all threads).
// Fragment layouts follow the PTX m16n8k8 / m16n8k16 f16 B operand: lane
// (g = lane / 4, t = lane % 4) holds column n = g, rows k = 2t, 2t + 1 (and
// k = 2t + 8, 2t + 9 in its second register for k16).
__device__ __forceinline__ void gate_fill(GateSmem& g, const float* __restrict__ w) {
    constexpr int OB1 = 160, OW2 = 192, OB2 = 1216, OW3 = 1248, OB3 = 1280;
    for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) {
        int nt = i / 32, l = i % 32, gq = l / 4, t = l % 4;
        int n = nt * 8 + gq, k = 2 * t;
        float lo = k < 5 ? w[n * 5 + k] : 0.f, hi = k + 1 < 5 ? w[n * 5 + k + 1] : 0.f;
        g.w1f[nt][l] = pack_half2(lo, hi);
    }
    for (int i = threadIdx.x; i < 2 * 4 * 32; i += blockDim.x) {
        int kt = i / 128, nt = (i / 32) % 4, l = i % 32, gq = l / 4, t = l % 4;
        int n = nt * 8 + gq, k = kt * 16 + 2 * t;
        g.w2f[kt][nt][l][0] = pack_half2(w[OW2 + n * 32 + k], w[OW2 + n * 32 + k + 1]);
        g.w2f[kt][nt][l][1] = pack_half2(w[OW2 + n * 32 + k + 8], w[OW2 + n * 32 + k + 9]);
    }
    for (int i = threadIdx.x; i < 2 * 32; i += blockDim.x) {
        int kt = i / 32, l = i % 32, t = l % 4;
        int k = kt * 16 + 2 * t;
        g.w3f[kt][l][0] = pack_half2(w[OW3 + k], w[OW3 + k + 1]);
        g.w3f[kt][l][1] = pack_half2(w[OW3 + k + 8], w[OW3 + k + 9]);
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

__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, const void* row) {
    unsigned a = (unsigned)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* row) {
    unsigned a = (unsigned)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// d = a b + c, f16 operands, f32 accumulate (c and d distinct).
__device__ __forceinline__ void mma_k8(float* d, unsigned a0, unsigned a1, unsigned b0, float c0, float c1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%7,%8};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0), "f"(c0), "f"(c1));
}

__device__ __forceinline__ void mma_k16c(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1, float c0, float c1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%10,%11};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1));
}

// d += a b, f16 operands, f32 accumulate.
__device__ __forceinline__ void mma_k16(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                        unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Logits of this lane's cell for both sensors.  xr, xp: the normalised
// density and pressure stencils of the lane's cell; tile: this warp's 1 KB
// A tile (64 rows x 8 halves).  Must be called by all 32 lanes together.
// All three layers run as m16n8 MMAs over four 16-row tiles (rows 0-31: the
// warp's density stencils, 32-63: its pressure stencils).  Biases enter as
// the accumulator input; ReLU and the f16 rounding of the hidden activations
// are one conversion, and the accumulator layout of one layer is the A
// fragment layout of the next, so the activations never leave registers.
__device__ __forceinline__ void gate_logits(const GateSmem& g, uint4* tile, const float* xr, const float* xp,
                                            float& zr, float& zp) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    __syncwarp();
    tile[lane] = make_uint4(pack_half2(xr[0], xr[1]), pack_half2(xr[2], xr[3]), pack_half2(xr[4], 0.f), 0u);
    tile[32 + lane] = make_uint4(pack_half2(xp[0], xp[1]), pack_half2(xp[2], xp[3]), pack_half2(xp[4], 0.f), 0u);
    __syncwarp();
    // sample row r of m-tile mt ends in fragment group r % 8, half r / 8 (c[0]
    // or c[2]); the lane's own rows are (mt = lane / 16, r = lane % 16) for
    // the density and (mt = 2 + lane / 16, same r) for the pressure
    const int src = 4 * (lane & 7), half = (lane >> 3) & 1, hi16 = lane >> 4;
#pragma unroll 1
    for (int mt = 0; mt < 4; ++mt) {
        unsigned a0, a1, h1[2][4], h2[2][4];
        ldsm_x2(a0, a1, tile + 16 * mt + (lane & 15));
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint2 bb = lds_u64(&g.b1[nt * 8 + 2 * t]);
            float c[4];
            mma_k8(c, a0, a1, lds_u32(&g.w1f[nt][lane]), __uint_as_float(bb.x), __uint_as_float(bb.y));
            h1[nt >> 1][(nt & 1) * 2 + 0] = relu_half2(c[0], c[1]);
            h1[nt >> 1][(nt & 1) * 2 + 1] = relu_half2(c[2], c[3]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint2 bb = lds_u64(&g.b2[nt * 8 + 2 * t]);
            const uint2 w0 = lds_u64(&g.w2f[0][nt][lane][0]), w1 = lds_u64(&g.w2f[1][nt][lane][0]);
            float c[4];
            mma_k16c(c, h1[0][0], h1[0][1], h1[0][2], h1[0][3], w0.x, w0.y, __uint_as_float(bb.x),
                     __uint_as_float(bb.y));
            mma_k16(c, h1[1][0], h1[1][1], h1[1][2], h1[1][3], w1.x, w1.y);
            h2[nt >> 1][(nt & 1) * 2 + 0] = relu_half2(c[0], c[1]);
            h2[nt >> 1][(nt & 1) * 2 + 1] = relu_half2(c[2], c[3]);
        }
        const uint2 w0 = lds_u64(&g.w3f[0][lane][0]), w1 = lds_u64(&g.w3f[1][lane][0]);
        const float b3 = __uint_as_float(lds_u32(&g.b3));
        float c[4];
        mma_k16c(c, h2[0][0], h2[0][1], h2[0][2], h2[0][3], w0.x, w0.y, b3, b3);
        mma_k16(c, h2[1][0], h2[1][1], h2[1][2], h2[1][3], w1.x, w1.y);
        const float v0 = __shfl_sync(0xffffffffu, c[0], src), v1 = __shfl_sync(0xffffffffu, c[2], src);
        const float v = half ? v1 : v0;
        if (mt == hi16) zr = v;
        if (mt == 2 + hi16) zp = v;
    }
}

// Normalised sensor stencil (v_k - v_2) / (max_k |v_k - v_2| + 1e-12).
__device__ __forceinline__ void gate_input(const float* v, float* x) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) m = fmaxf(m, fabsf(v[k] - v[2]));
    float r = __fdividef(1.f, m + 1e-12f);
#pragma unroll
    for (int k = 0; k < 5; ++k) x[k] = (v[k] - v[2]) * r;
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
sweep_kernel(const SweepArgs a) {
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
    __shared__ uint4 gtile[GATED ? WARPS * 64 : 1];
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
    const int seg = a.seg;
    const long long nchunk = (na + 31) >> 5;
    const long long nseg = (ns + seg - 1) / seg;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nchunk * nseg * nb) return;  // uniform over the warp
    const int chunk = (int)(warp % nchunk);
    const long long rest = warp / nchunk;
    const int segi = (int)(rest % nseg);
    const int b = (int)(rest / nseg);
    const int ia = chunk * 32 + lane;
    const bool active = ia < na;
    const int s0 = segi * seg;
    const int s1 = min(s0 + seg, ns);
    // inactive lanes follow a valid pencil so that every address is in bounds;
    // their results are discarded
    const long long base = (long long)(active ? ia : na - 1) * sa + (long long)b * sb;
    const long long nc = a.ncell;
    const R inv_dx = R(a.inv_dx[DIR]);
    const R eps = R(a.eps);
    const EosR<R, NF> er(a.eos);
    const R* __restrict__ qin = static_cast<const R*>(a.qin);

    // Values of loaded cell k (index s0 - 3 + k along the pencil) -> v[].
    // Along y and z the warp's 32 loads form one coalesced row per field;
    // along x each lane reads its own row, and the 32-byte sector it brings
    // into L1 serves the lane's next CH - 1 cells.
    // A ghost cell beyond a side that borders another block (block
    // decomposition) comes from that side's halo buffer; any other from the
    // BC index map.  j is the same for the whole warp.
    auto fetch = [&](int k, R* v) {
        const int j = s0 - 3 + k;
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

    constexpr bool PREFETCH = MFC_PREFETCH != 0;
    constexpr bool EPI_PREFETCH = PREFETCH && MIXED;
    bool bad = false;
    R smax = R(0);
    unsigned n_gated = 0, n_fallback = 0, n_cells = 0, n_flat = 0;
    // gated form: the network's logit at zero input (tensor-core path, as for
    // any other input), for warp steps whose stencils are all flat
    float z_flat = 0.f;
    if constexpr (GATED) {
        const float x0[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        float zr0, zp0;
        gate_logits(gsm[0], gtile + (threadIdx.x >> 5) * 64, x0, x0, zr0, zp0);
        z_flat = zr0;
    }
    double dt = 0.0;
    if (MODE == SW_LAST_RK) dt = a.ctrl->dt;
    // SSP-RK3 stage coefficients q^(k+1) = rk_a q^n + rk_b (q^(k) + dt L)
    const double rk_a = a.stage == 2 ? 0.75 : (1.0 / 3.0), rk_b = a.stage == 2 ? 0.25 : (2.0 / 3.0);
    const float bdt32 = float(a.stage == 1 ? dt : rk_b * dt);

    R W[5][NEQ];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        R v[NL];
        fetch(k, v);
        if constexpr (EXACT) exact::cons_to_prim<NDIM, NF>(a.eos, v, W[k]);
        else to_prim<NDIM, NF>(er, v, W[k]);
        bad |= !(mix_rho<NF>(W[k]) > R(0));
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
                        for (int f = 0; f < NEQ; ++f) qkp[f] = __ldg(qin + f * nc + c);
                    }
                }
            }
        }
        R vm[NEQ], vp[NEQ];
        bool use_weno = true;
        if constexpr (GATED) {
            // gate: linear weights when the network calls both the density and
            // the pressure stencil smooth (logit < 0) and the faces stay physical;
            // all 32 lanes take part in the tensor-core evaluation
            float sr[5], sp[5], zr = z_flat, zp = z_flat;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                sr[k] = W[k][0] + W[k][1];
                sp[k] = W[k][IE];
            }
            bool flat = true;
#pragma unroll
            for (int k = 0; k < 5; ++k) flat = flat && sr[k] == sr[2] && sp[k] == sp[2];
            // all 32 stencil pairs flat: every network input is exactly zero and
            // every logit is the output at zero, evaluated once per warp below
            const bool warp_flat = __all_sync(0xffffffffu, flat);
            if (!warp_flat) {
                float xr[5], xp[5];
                gate_input(sr, xr);
                gate_input(sp, xp);
                gate_logits(gsm[0], gtile + (threadIdx.x >> 5) * 64, xr, xp, zr, zp);
            }
            const bool smooth = zr < 0.f && zp < 0.f;
            if (smooth) {
#pragma unroll
                for (int f = 0; f < NEQ; ++f) linear5(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
                use_weno = !(face_ok<NDIM>(er, vm) && face_ok<NDIM>(er, vp));
            }
            if (j >= s0 && j < s1) {   // count each cell once (not the segment halos)
                n_fallback += smooth && use_weno;
                n_gated += smooth && !use_weno;
                n_cells += 1;
                n_flat += warp_flat;
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
                    if constexpr (TCARRY) {
                        const double Tp = exact::curv(W[2][f], W[3][f], W[4][f]);
                        exact::weno5_t(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], Tm[f], T0[f], Tp,
                                       vm[f], vp[f]);
                        Tm[f] = T0[f];
                        T0[f] = Tp;
                    } else if constexpr (EXACT) {
                        exact::weno5(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
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
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) L[f] = exact::div_rcp(Fprev[f] - F[f], dx, rdx);
#pragma unroll
                    for (int i = 0; i < NA; ++i)
                        L[IA + i] = L[IA + i] + exact::div_rcp(alphaCell[i] * (uf - ufPrev), dx, rdx);
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
                            // q^(k+1) = a q^n + b q^(k) + (b dt) L, accumulated in FP64
                            // from the FP32 increment (b dt) L (L itself is FP32)
                            const double inc = f2d_bits(bdt32 * tot);
                            if (a.stage == 1) {
                                qnew[f] = qn + inc;
                            } else {
                                const double qkd = f2d_bits(EPI_PREFETCH ? qkp[f] : qin[f * nc + c]);
                                qnew[f] = __fma_rn(rk_a, qn, __fma_rn(rk_b, qkd, inc));
                            }
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
                            double dx3[3], rdx3[3], idx3[3];
                            cell_geometry<DIR, NU>(a, j - 1, active ? ia : na - 1, b, dx3, rdx3, idx3);
                            R s = cell_wavespeed<NDIM, float, NF>(er, wn, idx3, bad);
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
            bad |= !(mix_rho<NF>(W[4]) > R(0));
        }
    }
    bad = bad && active;

    if constexpr (MODE == SW_LAST_RK) {
        if (a.stage == 3) {
            R m = warp_max(smax);
            if (lane == 0 && m > R(0))
                atomicMax(&a.ctrl->S_bits, (unsigned long long)__double_as_longlong(double(m)));
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&a.ctrl->status, 1u);
    if constexpr (GATED) {
        // only cells this lane owns count (inactive lanes and segment halos excluded)
        if (!active) n_gated = n_fallback = n_cells = n_flat = 0;
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
    SweepArgs a = a0;
    a.seg = pick_seg(DIR, a.n, T, sweep_slots<NDIM, DIR, MODE, FORM, NU, NF>());
    const long long blocks = (sweep_warps(DIR, a.n, a.seg) * 32 + T - 1) / T;
    if (blocks <= 0 || a.dry) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    sweep_kernel<NDIM, DIR, MODE, FORM, NU, NF><<<(unsigned)blocks, T, 0, s>>>(a);
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
