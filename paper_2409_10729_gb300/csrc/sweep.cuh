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
// is one coalesced row.  For d = x the lanes run along y; their cells are
// staged through shared memory in chunks of 32 bytes along x per row (one
// full DRAM sector), loaded cooperatively by the warp so that every global
// load touches whole sectors.  Each thread slides a five-cell window of
// primitives along its pencil in registers: per cell it takes one new cell,
// runs WENO once (both faces) and HLLC once (the face between the previous
// cell and this one), so no face is computed twice except at the two ends of
// a segment.  Boundary ghosts come from index clamping (transmissive) or
// wrapping (periodic) in the loads.
#pragma once
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
template <int NDIM, typename R>
struct LoadSet {
    static constexpr int N = NDIM + 4;
    __device__ static constexpr int field(int k) {
        return (sizeof(R) == 8 || k != 2 + NDIM) ? k : NDIM + 4;
    }
};

// Primitives from the loaded values v[] (see LoadSet).
template <int NDIM>
__device__ __forceinline__ void to_prim(const EosR<double>& e, const double* v, double* w) {
    using FL = Fields<NDIM>;
    double r = 1.0 / (v[0] + v[1]);
    double ke2 = 0.0;
    w[0] = v[0];
    w[1] = v[1];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        double u = v[2 + k] * r;
        w[2 + k] = u;
        ke2 += v[2 + k] * u;
    }
    double G, Pi;
    mixture(e, v[FL::IA], G, Pi);
    w[FL::IE] = (v[FL::IE] - 0.5 * ke2 - Pi) / G;
    w[FL::IA] = v[FL::IA];
}

template <int NDIM>
__device__ __forceinline__ void to_prim(const EosR<float>& e, const float* v, float* w) {
    using FL = Fields<NDIM>;
    float r = __fdividef(1.0f, v[0] + v[1]);
    w[0] = v[0];
    w[1] = v[1];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) w[2 + k] = v[2 + k] * r;
    w[FL::IE] = v[FL::IE];  // stored pressure
    w[FL::IA] = v[FL::IA];
}

// Pressure from an FP64 conservative state, mixed form: the cancelling part
// rho E - Pi is formed in FP64, the rest in FP32.
template <int NDIM>
__device__ __forceinline__ float mixed_pressure(const Eos& e, const double* q) {
    using FL = Fields<NDIM>;
    float rho = float(q[0] + q[1]);
    float r = __fdividef(1.0f, rho);
    float ke2 = 0.0f;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        float m = float(q[2 + k]);
        ke2 += m * (m * r);
    }
    double a1 = q[FL::IA];
    double num = (q[FL::IE] - (a1 * e.dP + e.P2)) - double(0.5f * ke2);
    float G = float(a1) * float(e.dg) + float(e.g2);
    return __fdividef(float(num), G);
}

// FP64 primitives of one cell of an FP64 conservative state (standalone use).
template <int NDIM>
__device__ __forceinline__ void load_prim(const double* __restrict__ q, long long c, long long nc,
                                          const EosR<double>& e, double* w) {
    double v[NDIM + 4];
#pragma unroll
    for (int f = 0; f < NDIM + 4; ++f) v[f] = __ldg(q + f * nc + c);
    to_prim<NDIM>(e, v, w);
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
template <int NDIM, typename R>
__device__ __forceinline__ R cell_wavespeed(const EosR<R>& e, const R* w, const double* inv_dx, bool& bad) {
    using FL = Fields<NDIM>;
    R rho = w[0] + w[1];
    R G, Pi;
    mixture(e, w[FL::IA], G, Pi);
    R c2 = rdiv((G + R(1)) * w[FL::IE] + Pi, G * rho);
    bad |= !(rho > R(0)) || !(c2 > R(0));
    R c = sqrt_pos(c2);
    R s = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s += (fabs(w[2 + d]) + c) * R(inv_dx[d]);
    bad |= !(s < R(INFINITY));
    return s;
}

// Shared-memory staging of the x-direction sweep: per warp, per loaded
// field, 32 rows x CH cells (CH * sizeof(R) = 32 bytes), padded by one
// element per row so that the 32 lanes read 32 different banks.
template <typename R>
struct XStage {
    static constexpr int CH = 32 / sizeof(R);
    static constexpr int PITCH = CH + 1;
};

template <int FORM>
using FormReal = typename std::conditional<FORM == FORM_MIXED || FORM == FORM_GATED, float, double>::type;

// Gate-network argument of a sweep: the 1281 weights for the gated form,
// nothing otherwise.
template <int FORM>
struct GateArg {
    float w[FORM == FORM_GATED ? kGateParams : 1];
};

// Logit of the gate network for a normalised stencil x[5]; th indexes the
// kernel-parameter copy of the weights at compile-time offsets.
__device__ __forceinline__ float gate_logit(const float* th, const float* x) {
    constexpr int H = 32, OB1 = 160, OW2 = 192, OB2 = 1216, OW3 = 1248, OB3 = 1280;
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float a = th[OB1 + j];
#pragma unroll
        for (int i = 0; i < 5; ++i) a = fmaf(th[j * 5 + i], x[i], a);
        h1[j] = fmaxf(a, 0.f);
    }
    float z = th[OB3];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float a = th[OB2 + j];
#pragma unroll
        for (int i = 0; i < H; ++i) a = fmaf(th[OW2 + j * H + i], h1[i], a);
        z = fmaf(th[OW3 + j], fmaxf(a, 0.f), z);
    }
    return z;
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
__device__ __forceinline__ bool face_ok(const EosR<float>& e, const float* w) {
    using FL = Fields<NDIM>;
    float a1 = w[FL::IA];
    float G, Pi;
    mixture(e, a1, G, Pi);
    return (w[0] + w[1] > 0.f) && (a1 >= 0.f) && (a1 <= 1.f) && ((G + 1.f) * w[FL::IE] + Pi > 0.f);
}

template <int NDIM, int DIR, int MODE, int FORM>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(const SweepArgs a, const GateArg<FORM> gate) {
    using R = FormReal<FORM>;
    constexpr bool EXACT = FORM == FORM_FP64_EXACT;
    constexpr bool GATED = FORM == FORM_GATED;
    using FL = Fields<NDIM>;
    using LS = LoadSet<NDIM, R>;
    constexpr int NEQ = FL::NEQ, IE = FL::IE, IA = FL::IA;
    constexpr int NL = LS::N;
    constexpr bool MIXED = FORM == FORM_MIXED || FORM == FORM_GATED;
    constexpr int CH = XStage<R>::CH, PITCH = XStage<R>::PITCH;
    constexpr int WARPS = kSweepThreads / 32;
    __shared__ R stage[DIR == 0 ? WARPS * NL * 32 * PITCH : 1];

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
    const EosR<R> er(a.eos);
    const R* __restrict__ qin = static_cast<const R*>(a.qin);
    R* st = stage + (threadIdx.x >> 5) * (NL * 32 * PITCH);

    // Values of loaded cell k (x-index s0 - 3 + k along the pencil) -> v[].
    auto fetch = [&](int k, R* v) {
        const int j = s0 - 3 + k;
        if constexpr (DIR != 0) {
            const long long c = base + (long long)bc_index(j, ns, a.periodic) * ss;
#pragma unroll
            for (int f = 0; f < NL; ++f) v[f] = __ldg(qin + LS::field(f) * nc + c);
        } else {
            const int slot = k % CH;
            if (slot == 0) {
                // the warp stages cells j .. j+CH-1 of its 32 rows
                __syncwarp();
                const int t = lane % CH;
                const int xg = bc_index(j + t, ns, a.periodic);
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    const int r = lane / CH + (32 / CH) * i;
                    const int row = min(chunk * 32 + r, na - 1);
                    const long long c = (long long)row * sa + (long long)b * sb + xg;
#pragma unroll
                    for (int f = 0; f < NL; ++f) st[(f * 32 + r) * PITCH + t] = __ldg(qin + LS::field(f) * nc + c);
                }
                __syncwarp();
            }
#pragma unroll
            for (int f = 0; f < NL; ++f) v[f] = st[(f * 32 + lane) * PITCH + slot];
        }
    };

    bool bad = false;
    R smax = R(0);
    unsigned n_gated = 0, n_fallback = 0, n_cells = 0;
    double dt = 0.0;
    if (MODE == SW_LAST_RK) dt = a.ctrl->dt;

    R W[5][NEQ];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        R v[NL];
        fetch(k, v);
        if constexpr (EXACT) exact::cons_to_prim<NDIM>(a.eos, v, W[k]);
        else to_prim<NDIM>(er, v, W[k]);
        bad |= !(W[k][0] + W[k][1] > R(0));
    }
    R vmPrev[NEQ], Fprev[NEQ];
    R ufPrev = R(0), alphaCell = R(0);
#pragma unroll
    for (int f = 0; f < NEQ; ++f) vmPrev[f] = Fprev[f] = R(0);

    for (int j = s0 - 1; j <= s1; ++j) {
        R vm[NEQ], vp[NEQ];
        bool use_weno = true;
        if constexpr (GATED) {
            // gate: linear weights when the network calls both the density and
            // the pressure stencil smooth (logit < 0) and the faces stay physical
            float sens[5], x[5];
            bool smooth = true;
#pragma unroll 1
            for (int sensor = 0; sensor < 2 && smooth; ++sensor) {
#pragma unroll
                for (int k = 0; k < 5; ++k) sens[k] = sensor == 0 ? W[k][0] + W[k][1] : W[k][IE];
                gate_input(sens, x);
                smooth = gate_logit(gate.w, x) < 0.f;
            }
            if (smooth) {
#pragma unroll
                for (int f = 0; f < NEQ; ++f) linear5(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
                use_weno = !(face_ok<NDIM>(er, vm) && face_ok<NDIM>(er, vp));
            }
            if (j >= s0 && j < s1) {   // count each cell once (not the segment halos)
                n_fallback += smooth && use_weno;
                n_gated += smooth && !use_weno;
                n_cells += 1;
            }
        }
        if (use_weno) {
#pragma unroll
            for (int f = 0; f < NEQ; ++f) {
                if constexpr (EXACT) exact::weno5(a.eps, W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], vm[f], vp[f]);
                else weno5(W[0][f], W[1][f], W[2][f], W[3][f], W[4][f], eps, vm[f], vp[f]);
            }
        }
        if (j >= s0) {
            R F[NEQ], uf;
            if constexpr (EXACT) bad |= exact::hllc<NDIM, DIR>(a.eos, vmPrev, vp, F, uf);
            else bad |= hllc<NDIM, DIR, R>(er, vmPrev, vp, F, uf);
            if (j > s0 && active) {
                // cell i = j - 1 is complete: faces i-1/2 (Fprev) and i+1/2 (F)
                R L[NEQ];
                if constexpr (EXACT) {
                    // (F_{i-1/2} - F_{i+1/2})/dx, then + alpha1 (u_f+ - u_f-)/dx
                    const double dx = a.dx[DIR], rdx = a.rdx[DIR];
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) L[f] = exact::div_rcp(Fprev[f] - F[f], dx, rdx);
                    L[IA] = L[IA] + exact::div_rcp(alphaCell * (uf - ufPrev), dx, rdx);
                } else {
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) L[f] = (Fprev[f] - F[f]) * inv_dx;
                    L[IA] += alphaCell * (uf - ufPrev) * inv_dx;
                }
                const long long c = base + (long long)(j - 1) * ss;
                if constexpr (MODE == SW_FIRST) {
                    R* acc = static_cast<R*>(a.acc);
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) acc[f * nc + c] = L[f];
                } else if constexpr (MODE == SW_MID) {
                    R* acc = static_cast<R*>(a.acc);
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) acc[f * nc + c] = acc[f * nc + c] + L[f];
                } else if constexpr (MODE == SW_LAST_RHS) {
                    const R* acc = static_cast<const R*>(a.acc);
                    double* out = static_cast<double*>(a.qout);
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) {
                        R tot = NDIM > 1 ? acc[f * nc + c] + L[f] : L[f];
                        out[f * nc + c] = double(tot);
                    }
                } else {  // SW_LAST_RK
                    const R* acc = static_cast<const R*>(a.acc);
                    double qnew[NEQ];
#pragma unroll
                    for (int f = 0; f < NEQ; ++f) {
                        R tot = NDIM > 1 ? acc[f * nc + c] + L[f] : L[f];
                        double qn = a.qn[f * nc + c];
                        double dL = dt * double(tot);
                        if (a.stage == 1) {
                            qnew[f] = qn + dL;
                        } else {
                            double qk = double(qin[f * nc + c]);
                            if (a.stage == 2)
                                qnew[f] = 0.75 * qn + 0.25 * (qk + dL);
                            else
                                qnew[f] = (1.0 / 3.0) * qn + (2.0 / 3.0) * (qk + dL);
                        }
                    }
                    if constexpr (!MIXED) {
                        double* out = static_cast<double*>(a.qout);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) out[f * nc + c] = qnew[f];
                        if (a.stage == 3) {
                            R s;
                            if constexpr (EXACT) {
                                s = exact::cell_wavespeed<NDIM>(a.eos, qnew, a.dx, a.rdx, bad);
                            } else {
                                double wn[NEQ];
                                to_prim<NDIM>(er, qnew, wn);
                                s = cell_wavespeed<NDIM, double>(er, wn, a.inv_dx, bad);
                            }
                            smax = s > smax ? s : smax;
                        }
                    } else {
                        float pnew = mixed_pressure<NDIM>(a.eos, qnew);
                        float* o32 = static_cast<float*>(a.stage == 3 ? a.qout2 : a.qout);
#pragma unroll
                        for (int f = 0; f < NEQ; ++f) o32[f * nc + c] = float(qnew[f]);
                        o32[NEQ * nc + c] = pnew;
                        if (a.stage == 3) {
                            double* o64 = static_cast<double*>(a.qout);
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) o64[f * nc + c] = qnew[f];
                            float v[NEQ], wn[NEQ];
#pragma unroll
                            for (int f = 0; f < NEQ; ++f) v[f] = float(qnew[f]);
                            v[IE] = pnew;
                            to_prim<NDIM>(er, v, wn);
                            R s = cell_wavespeed<NDIM, float>(er, wn, a.inv_dx, bad);
                            smax = s > smax ? s : smax;
                        }
                    }
                }
            }
#pragma unroll
            for (int f = 0; f < NEQ; ++f) Fprev[f] = F[f];
            ufPrev = uf;
        }
#pragma unroll
        for (int f = 0; f < NEQ; ++f) vmPrev[f] = vm[f];
        alphaCell = W[2][IA];
        if (j < s1) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int f = 0; f < NEQ; ++f) W[k][f] = W[k + 1][f];
            R v[NL];
            fetch(j + 3 - (s0 - 3), v);
            if constexpr (EXACT) exact::cons_to_prim<NDIM>(a.eos, v, W[4]);
            else to_prim<NDIM>(er, v, W[4]);
            bad |= !(W[4][0] + W[4][1] > R(0));
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
        if (!active) n_gated = n_fallback = n_cells = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_gated += __shfl_xor_sync(0xffffffffu, n_gated, o);
            n_fallback += __shfl_xor_sync(0xffffffffu, n_fallback, o);
            n_cells += __shfl_xor_sync(0xffffffffu, n_cells, o);
        }
        if (lane == 0) {
            atomicAdd(&a.ctrl->gated, (unsigned long long)n_gated);
            atomicAdd(&a.ctrl->fallback, (unsigned long long)n_fallback);
            atomicAdd(&a.ctrl->cells, (unsigned long long)n_cells);
        }
    }
}

// Launch one sweep: the valid (direction, mode) pairs are x FIRST, y MID
// (3-D), and LAST_RK / LAST_RHS on the last direction.
template <int NDIM, int FORM>
cudaError_t launch_sweep_t(int dir, int mode, const SweepArgs& a, const GateArg<FORM>& g, cudaStream_t s) {
    long long warps = sweep_warps(dir, a.n, a.seg);
    long long blocks = (warps * 32 + kSweepThreads - 1) / kSweepThreads;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks), block(kSweepThreads);
    constexpr int LAST = NDIM - 1;
    if (dir == 0 && mode == SW_FIRST && NDIM > 1) {
        if constexpr (NDIM > 1) sweep_kernel<NDIM, 0, SW_FIRST, FORM><<<grid, block, 0, s>>>(a, g);
    } else if (dir == 1 && mode == SW_MID && NDIM == 3) {
        if constexpr (NDIM == 3) sweep_kernel<NDIM, 1, SW_MID, FORM><<<grid, block, 0, s>>>(a, g);
    } else if (dir == LAST && mode == SW_LAST_RK) {
        sweep_kernel<NDIM, LAST, SW_LAST_RK, FORM><<<grid, block, 0, s>>>(a, g);
    } else if (dir == LAST && mode == SW_LAST_RHS) {
        sweep_kernel<NDIM, LAST, SW_LAST_RHS, FORM><<<grid, block, 0, s>>>(a, g);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_sweep_any(int ndim, int dir, int mode, const SweepArgs& a, const GateArg<FORM>& g,
                             cudaStream_t s) {
    switch (ndim) {
        case 1: return launch_sweep_t<1, FORM>(dir, mode, a, g, s);
        case 2: return launch_sweep_t<2, FORM>(dir, mode, a, g, s);
        case 3: return launch_sweep_t<3, FORM>(dir, mode, a, g, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfc5
