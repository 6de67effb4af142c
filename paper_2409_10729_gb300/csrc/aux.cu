// aux.cu -- small kernels around the sweeps: primitive -> conservative
// conversion, the FP32 working copy of the mixed form, the standalone CFL
// wave-speed reduction, and the per-step control kernel.  Built with
// -fmad=false: the conversion and the wave speed follow the reference
// operation order bit for bit, so every form starts from the same state.
#include <stdint.h>

#include <type_traits>

#include "sweep.cuh"

namespace mfc5 {

constexpr int kAuxThreads = 256;

static unsigned aux_blocks(long long n) {
    long long b = (n + kAuxThreads - 1) / kAuxThreads;
    if (b < 1) b = 1;
    if (b > 152LL * 64) b = 152LL * 64;  // grid-stride beyond this
    return (unsigned)b;
}

// Primitive (alpha1 rho1, alpha2 rho2, u_k, p, alpha1) -> conservative, in
// place (Sec. II-A: rho E = Gamma p + Pi + rho |u|^2 / 2), in the reference
// operation order (this file is built with -fmad=false).
template <int NDIM, int NF>
__global__ void prim_to_cons_kernel(double* q, long long nc, Eos e) {
    using FL = Fields<NDIM, NF>;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        double w[FL::NEQ], v[FL::NEQ];
#pragma unroll
        for (int f = 0; f < FL::NEQ; ++f) w[f] = q[f * nc + c];
        exact::prim_to_cons<NDIM, NF>(e, w, v);
#pragma unroll
        for (int f = 0; f < FL::NEQ; ++f) q[f * nc + c] = v[f];
    }
}

// FP32 working copy (conservatives + pressure) of an FP64 state, mixed form.
template <int NDIM, int NF>
__global__ void make_mixed_state_kernel(const double* __restrict__ qn, float* __restrict__ s0,
                                        long long nc, Eos e) {
    using FL = Fields<NDIM, NF>;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        double q[FL::NEQ];
        float q32[FL::NEQ];
#pragma unroll
        for (int f = 0; f < FL::NEQ; ++f) {
            q[f] = qn[f * nc + c];
            q32[f] = d2f_bits(q[f]);
            s0[f * nc + c] = q32[f];
        }
        s0[FL::NEQ * nc + c] = mixed_pressure<NDIM, NF>(e, q, q32);
    }
}

// S = max over cells of sum_d (|u_d| + c)/dx_d of an FP64 state, in the
// reference operation order.
template <int NDIM, int NF>
__global__ void wavespeed_kernel(const double* __restrict__ q, long long nc, Eos e, double dx0, double dx1,
                                 double dx2, double rdx0, double rdx1, double rdx2, DevCtrl* ctrl, int n0, int n1,
                                 Geom3 g) {
    using FL = Fields<NDIM, NF>;
    double dx[3] = {dx0, dx1, dx2};
    double rdx[3] = {rdx0, rdx1, rdx2};
    double smax = 0.0;
    bool bad = false;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // every thread of a warp runs the same number of iterations so that the
    // warp reduction below sees all 32 lanes
    long long iters = (nc + stride - 1) / stride;
    // uniform over the launch: only a non-uniform grid needs the cell's
    // coordinates (64-bit divisions, kept off the uniform-grid path)
    const bool nu = g.cw[0] || g.cw[1] || g.cw[2];
    for (long long it = 0; it < iters; ++it) {
        long long c = start + it * stride;
        if (c < nc) {
            double v[FL::NEQ];
#pragma unroll
            for (int f = 0; f < FL::NEQ; ++f) v[f] = __ldg(q + f * nc + c);
            if (nu) {   // non-uniform directions: the cell's own width
                const long long ci[3] = {c % n0, (c / n0) % n1, c / ((long long)n0 * n1)};
#pragma unroll
                for (int d = 0; d < NDIM; ++d)
                    if (g.cw[d]) {
                        dx[d] = __ldg(g.cw[d] + ci[d]);
                        rdx[d] = __ldg(g.crw[d] + ci[d]);
                    }
            }
            double s = exact::cell_wavespeed<NDIM, NF>(e, v, dx, rdx, bad);
            smax = s > smax ? s : smax;
        }
    }
    double m = warp_max(smax);
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(&ctrl->S_bits, (unsigned long long)__double_as_longlong(m));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctrl->status, 1u);
}

// Start of a step: take S of the current state, set dt, advance t, and clear
// the accumulator that the step's last sweep fills with S of the new state.
__global__ void step_begin_kernel(DevCtrl* ctrl) {
    double S = __longlong_as_double((long long)ctrl->S_bits);
    double dt = ctrl->dt_fixed > 0.0 ? ctrl->dt_fixed : ctrl->cfl / S;
    if (!(dt > 0.0) || !(dt < INFINITY)) ctrl->status |= 2u;
    ctrl->S = S;
    ctrl->dt = dt;
    ctrl->t += dt;
    ctrl->S_bits = 0ULL;
}

__global__ void f32_to_f64_kernel(const float* __restrict__ src, double* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = double(src[i]);
}

// Calls f.template operator()<NDIM, NF>() for the runtime ndim and fluid count.
template <typename Fn>
cudaError_t dispatch_nd_nf(int ndim, int nf, Fn&& f) {
    auto by_nf = [&](auto nd) -> cudaError_t {
        constexpr int ND = decltype(nd)::value;
        switch (nf) {
            case 2: return f.template operator()<ND, 2>();
            case 3: return f.template operator()<ND, 3>();
            case 4: return f.template operator()<ND, 4>();
            default: return cudaErrorInvalidValue;
        }
    };
    switch (ndim) {
        case 1: return by_nf(std::integral_constant<int, 1>());
        case 2: return by_nf(std::integral_constant<int, 2>());
        case 3: return by_nf(std::integral_constant<int, 3>());
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prim_to_cons(int ndim, double* q, long long nc, const Eos& e, cudaStream_t s) {
    unsigned g = aux_blocks(nc);
    return dispatch_nd_nf(ndim, e.nf, [&]<int ND, int NF>() {
        prim_to_cons_kernel<ND, NF><<<g, kAuxThreads, 0, s>>>(q, nc, e);
        return cudaGetLastError();
    });
}

cudaError_t launch_make_mixed_state(int ndim, const double* qn, float* s0, long long nc, const Eos& e,
                                    cudaStream_t s) {
    unsigned g = aux_blocks(nc);
    return dispatch_nd_nf(ndim, e.nf, [&]<int ND, int NF>() {
        make_mixed_state_kernel<ND, NF><<<g, kAuxThreads, 0, s>>>(qn, s0, nc, e);
        return cudaGetLastError();
    });
}

cudaError_t launch_wavespeed(int ndim, const double* q, const int* n, const double* const* cw,
                             const double* const* crw, long long nc, const double* dx, const double* rdx,
                             const Eos& e, DevCtrl* ctrl, cudaStream_t s) {
    cudaError_t err = cudaMemsetAsync(&ctrl->S_bits, 0, sizeof(unsigned long long), s);
    if (err != cudaSuccess) return err;
    Geom3 g3;
    for (int d = 0; d < 3; ++d) {
        g3.cw[d] = cw ? cw[d] : nullptr;
        g3.crw[d] = crw ? crw[d] : nullptr;
    }
    unsigned g = aux_blocks(nc);
    return dispatch_nd_nf(ndim, e.nf, [&]<int ND, int NF>() {
        wavespeed_kernel<ND, NF><<<g, kAuxThreads, 0, s>>>(q, nc, e, dx[0], dx[1], dx[2], rdx[0], rdx[1], rdx[2],
                                                          ctrl, n[0], n[1], g3);
        return cudaGetLastError();
    });
}

cudaError_t launch_step_begin(DevCtrl* ctrl, cudaStream_t s) {
    step_begin_kernel<<<1, 1, 0, s>>>(ctrl);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* src, double* dst, long long n, cudaStream_t s) {
    f32_to_f64_kernel<<<aux_blocks(n), kAuxThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

// 16-byte grid-stride copy; one side is page-locked host memory read or
// written through its device mapping.
__global__ void copy16_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, long long n16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// True when [p, p + bytes) starts and ends in page-locked host memory that
// the current device reaches at the same address (unified addressing).
static bool host_mapped(const void* p, size_t bytes) {
    const void* ends[2] = {p, static_cast<const char*>(p) + (bytes - 1)};
    for (const void* e : ends) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, e) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer != e) return false;
    }
    return true;
}

cudaError_t host_copy(void* dst, const void* src, size_t bytes, bool to_device, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const void* host = to_device ? src : dst;
    const bool aligned = (((uintptr_t)dst | (uintptr_t)src | bytes) & 15u) == 0;
    if (aligned && host_mapped(host, bytes)) {
        const long long n16 = (long long)(bytes / 16);
        long long blocks = (n16 + 511) / 512;
        if (blocks > kHostCopyBlocks) blocks = kHostCopyBlocks;
        copy16_kernel<<<(unsigned)blocks, 512, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16);
        return cudaGetLastError();
    }
    return cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, s);
}

}  // namespace mfc5

namespace mfc5 {

// ---------------------------------------------------------------------------
// ALU peak probe: independent FMA chains (8 per thread) over a grid of 152 x 8
// blocks; the result is stored so the chains are not removed.  Used only to
// measure the FP64/FP32 roofline denominators.
template <typename R>
__global__ void fma_probe_kernel(R* sink, int iters, R a, R b) {
    R x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == R(12345.678)) sink[0] = s;  // practically never taken; keeps the chains live
}

cudaError_t run_fma_probe(int fp64, double* tflops, cudaStream_t s) {
    const int blocks = 152 * 8, threads = 256;
    const int iters = fp64 ? 256 : 8192;
    void* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 16);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        if (fp64)
            fma_probe_kernel<double><<<blocks, threads, 0, s>>>((double*)sink, iters, 0.999999, 1e-7);
        else
            fma_probe_kernel<float><<<blocks, threads, 0, s>>>((float*)sink, iters, 0.9999f, 1e-5f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaGetLastError();
}

}  // namespace mfc5

namespace mfc5 {

// Self-check of the integer-pipe conversions against the hardware ones on
// pseudo-random bit patterns spanning every exponent (splitmix64 sequence).
__global__ void conversion_check_kernel(long long n, unsigned long long seed, unsigned* mismatches) {
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)i * 0x9e3779b97f4a7c15ULL;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        // doubles around the float range (exponents 880..1170) and arbitrary floats
        unsigned long long db = (z & 0x800fffffffffffffULL) | ((unsigned long long)(880 + (z >> 52) % 291) << 52);
        double x = __longlong_as_double((long long)db);
        float fr = __uint_as_float((unsigned)(z >> 17));
        float a = d2f_bits(x), b = __double2float_rn(x);
        if (__float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b)) ++bad;
        unsigned e = (__float_as_uint(fr) >> 23) & 0xffu;
        if (e != 0u && e != 0xffu) {   // normal floats (flushed subnormals and NaN payloads aside)
            double c = f2d_bits(fr), d = (double)fr;
            if (__double_as_longlong(c) != __double_as_longlong(d)) ++bad;
        }
    }
    if (bad) atomicAdd(mismatches, bad);
}

// Self-check of the FP64 form's integer-pipe products K v and quotients x/6
// against the FP64 instructions, and of its integer-word compares (x > 0,
// 0 <= x, x < y) against the FP64 compares: pseudo-random patterns over every
// exponent, with a share of zeros, subnormals, infinities, NaNs and exponents
// at the ends of the range where the integer path hands over to the FP64 one;
// the second compare operand is another such pattern, x itself or x with its
// lowest bit or its sign flipped.
__global__ void exact_ops_check_kernel(long long n, unsigned long long seed, unsigned* mismatches) {
    unsigned bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)i * 0x9e3779b97f4a7c15ULL;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        unsigned long long bits = z;
        const unsigned sel = (unsigned)(i & 15);
        if (sel == 0) bits &= 0x8000000000000000ULL;                              // +-0
        else if (sel == 1) bits &= 0x800fffffffffffffULL;                         // subnormal
        else if (sel == 2) bits = (bits & 0x800fffffffffffffULL) | ((unsigned long long)((z >> 11) % 10) << 52);
        else if (sel == 3) bits = (bits & 0x800fffffffffffffULL) | ((unsigned long long)(2047 - (z >> 11) % 10) << 52);
        else if (sel == 4) bits = (bits & 0x800fffffffffffffULL) | ((unsigned long long)(1018 + (z >> 11) % 12) << 52);
        const double x = __longlong_as_double((long long)bits);
        const double r[5] = {exact::mul_small<3>(x), exact::mul_small<5>(x), exact::mul_small<7>(x),
                             exact::mul_small<11>(x), exact::div6(x)};
        const double h[5] = {__dmul_rn(3.0, x), __dmul_rn(5.0, x), __dmul_rn(7.0, x), __dmul_rn(11.0, x),
                             __ddiv_rn(x, 6.0)};
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if (__double_as_longlong(r[k]) != __double_as_longlong(h[k]) && !(r[k] != r[k] && h[k] != h[k]))
                ++bad;
        unsigned long long w = z * 0xd6e8feb86659fd93ULL;
        w ^= w >> 32;
        const unsigned pick = (unsigned)(i >> 4) & 3u;
        if (pick == 0u) w = bits;
        else if (pick == 1u) w = bits ^ 1ULL;
        else if (pick == 2u) w = bits ^ 0x8000000000000000ULL;
        else if ((w & 7u) == 0u) w &= 0x8000000000000000ULL;   // +-0 now and then
        const double y = __longlong_as_double((long long)w);
        bad += (gt0(x) != (x > 0.0)) + (ge0(x) != (0.0 <= x)) + (less(x, y) != (x < y)) + (less(y, x) != (y < x));
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace mfc5

extern "C" int mfc_selfcheck_conversions(long long n, unsigned long long seed, long long* mismatches) {
    if (n <= 0 || !mismatches) return -1;
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) return -3;
    cudaMemset(d, 0, sizeof(unsigned));
    mfc5::conversion_check_kernel<<<152 * 8, 256>>>(n, seed, d);
    unsigned h = 0;
    cudaError_t err = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) return -3;
    *mismatches = (long long)h;
    return 0;
}

extern "C" int mfc_selfcheck_exact_ops(long long n, unsigned long long seed, long long* mismatches) {
    if (n <= 0 || !mismatches) return -1;
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) return -3;
    cudaMemset(d, 0, sizeof(unsigned));
    mfc5::exact_ops_check_kernel<<<152 * 8, 256>>>(n, seed, d);
    unsigned h = 0;
    cudaError_t err = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess) return -3;
    *mismatches = (long long)h;
    return 0;
}
