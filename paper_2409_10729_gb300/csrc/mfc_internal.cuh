// mfc_internal.cuh -- shared declarations of the CUDA library (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "physics.cuh"

namespace mfc5 {

// Non-uniform grids: doubles per cell of a WENO5 table -- face-value
// functionals at i+1/2 (3 stencils x 3 values) and i-1/2, the functionals b
// and c of each stencil's quadratic (smoothness b^2 + 13/3 c^2), and the
// linear weights at i+1/2 and i-1/2.
constexpr int kTabDoubles = 42;

// Number of fluids of a params struct (0 means 2).
inline int params_nfluids(int nfluids) { return nfluids == 0 ? 2 : nfluids; }

// Mixture constants of nf fluids from their gamma and pi_inf.
inline Eos make_eos(const double* gamma, const double* pi_inf, int nf) {
    Eos e{};
    e.nf = nf;
    for (int i = 0; i < nf; ++i) {
        e.g[i] = 1.0 / (gamma[i] - 1.0);
        e.P[i] = gamma[i] * pi_inf[i] / (gamma[i] - 1.0);
    }
    for (int i = 0; i < nf - 1; ++i) {
        e.dg[i] = e.g[i] - e.g[nf - 1];
        e.dP[i] = e.P[i] - e.P[nf - 1];
    }
    for (int i = 0; i < nf; ++i) {
        e.g32[i] = (float)e.g[i];
        e.P32[i] = (float)e.P[i];
    }
    for (int i = 0; i < nf - 1; ++i) {
        e.dg32[i] = (float)e.dg[i];
        e.dP32[i] = (float)e.dP[i];
    }
    return e;
}

// Per-direction cell widths and RN(1/width) of a non-uniform grid (null where
// the direction is uniform), by value for kernels.
struct Geom3 {
    const double* cw[3];
    const double* crw[3];
};

// Tables of cells -1 .. n and widths of cells 0 .. n-1 of one direction from
// its n + 1 cell edges (false: edges not strictly increasing, or degenerate).
bool build_grid_tables(const double* edges, int n, int periodic, std::vector<double>& tab,
                       std::vector<double>& width);

// Step control block, resident in device memory so that consecutive steps
// need no host round trip (dt of step n+1 comes from S(q^{n+1}), reduced by
// the last sweep of step n).
struct DevCtrl {
    unsigned long long S_bits;  // max of the per-cell wave speed, as the bits of a positive double
    double S;                   // wave speed the current step's dt was taken from
    double dt;                  // current step size
    double t;                   // time accumulated since the last reset
    double cfl;                 // CFL number (CFL mode)
    double dt_fixed;            // > 0 selects fixed-dt mode
    unsigned int status;        // bit 0: non-physical face state; bit 1: bad wave speed or dt
    unsigned int pad;
    unsigned long long gated;   // gated form: cell reconstructions done with linear weights
    unsigned long long fallback;  // gated form: gated cells recomputed with WENO (non-physical faces)
    unsigned long long cells;   // gated form: cell reconstructions evaluated
    unsigned long long flat;    // gated form: of those, in warp steps whose stencils were all flat
};

enum SweepMode {
    SW_FIRST = 0,     // acc  = L_d
    SW_MID = 1,       // acc += L_d
    SW_LAST_RK = 2,   // L = acc + L_d; RK stage update; stage 3 also reduces S
    SW_LAST_RHS = 3   // out = acc + L_d (FP64 output)
};

struct SweepArgs {
    const void* qin;      // state whose stencils are read (FP64 cons, or FP32 cons+p)
    void* acc;            // RHS accumulator (FP64 or FP32)
    const double* qn;     // RK base state q^n (FP64)
    void* qout;           // stage output (FP64 or FP32), or FP64 RHS output
    void* qout2;          // mixed form, stage 3: FP32 copy of q^{n+1} with p
    float* dinc;          // FP32 forms: the RK increment D_k of the stage (neq fields), read and rewritten
    int n[3];
    long long ncell;
    double inv_dx[3];     // n/(hi - lo) per direction (reformulated forms)
    double dx[3];         // (hi - lo)/n per direction
    double rdx[3];        // RN(1/dx) per direction (reference-order form)
    float inv_dx32[3];    // inv_dx rounded to FP32 (FP32 forms)
    Eos eos;
    double eps;
    int order;            // WENO order, 3 or 5
    int periodic;         // along the sweep direction
    int seg;              // cells per thread along the sweep direction (set at launch)
    long long nwarps;     // > 0: balanced mapping, the launch's warps split the
                          // pencil cells evenly (set at launch); 0: seg mapping
    int dry;              // 1: only pick the launch shape (fills the occupancy caches), launch nothing
    int stage;            // 1, 2, 3
    DevCtrl* ctrl;
    const float* gate_w;  // gated form: the 1281 network weights (device)
    // non-uniform grids (null where the direction is uniform):
    const void* tab;      // sweep direction: WENO5 tables of cells -1 .. n (FP64 or FP32 per form)
    const double* cw[3];  // per direction: cell widths
    const double* crw[3]; // per direction: RN(1/width)
    const float* crw32[3];  // per direction: 1/width in FP32 (FP32 forms)
    // block decomposition (Sec. III-A): the sweep direction's ghost layers
    // beyond a side that borders another block, [field][layer 0..2][plane],
    // in the stage state's element type (null where the side is a domain
    // boundary and the BC applies); hplane = cells of the plane normal to it
    const void* hlo;      // cells -3 .. -1 (layer l = cell l - 3)
    const void* hhi;      // cells n .. n + 2 (layer l = cell n + l)
    long long hplane;
    // gated form: per-cell decisions of this sweep's direction (0 WENO,
    // 1 linear, 2 fallback to WENO), or null
    signed char* gate_dec;
    // FP32 y/z sweeps staged through TMA (MFC_TMA_YZ builds): host address of
    // the CUtensorMap of the stage input for this direction, or null
    const void* tmap;
};

// TMA staging of the FP32 forms' y and z sweeps: 0 = direct loads (default),
// 1 = interior pencil segments staged through shared memory by
// cp.async.bulk.tensor, kTmaCells cells per box, double-buffered per warp.
#ifndef MFC_TMA_YZ
#define MFC_TMA_YZ 0
#endif
// FP32 x sweeps: 1 = 16-byte row loads of four cells per field (rows of a
// multiple of 4 cells), 0 = one cell per load
#ifndef MFC_XVEC
#define MFC_XVEC 1
#endif
constexpr int kTmaCells = 4;

// Arithmetic forms of the sweep kernels:
//   FORM_FP64_FAST   FP64, formulas reorganised for fewer FP64 instructions
//   FORM_MIXED       FP32 stencils/Riemann, FP64 pressure numerator and RK update
//   FORM_FP64_EXACT  FP64 in the reference operation order (bit-identical to it)
//   FORM_GATED       FORM_MIXED with the MLP gate (linear weights in smooth cells)
enum Form { FORM_FP64_FAST = 0, FORM_MIXED = 1, FORM_FP64_EXACT = 2, FORM_GATED = 3 };

// Number of parameters of the gate network (W1[32][5], b1, W2[32][32], b2, w3, b3).
constexpr int kGateParams = 1281;

cudaError_t launch_sweep_fp64(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_mixed(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp64x(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_gated(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_gate_samples(int ndim, const double* q, const int* n, const int* periodic, const Eos& e,
                                double eps, float tau, float* X, float* Y, cudaStream_t s);

// auxiliary kernels (aux.cu)
cudaError_t launch_prim_to_cons(int ndim, double* q, long long ncell, const Eos& e, cudaStream_t s);
cudaError_t launch_make_mixed_state(int ndim, const double* qn, float* s0, long long ncell,
                                    const Eos& e, cudaStream_t s);
cudaError_t launch_wavespeed(int ndim, const double* q, const int* n, const double* const* cw,
                             const double* const* crw, long long ncell, const double* dx,
                             const double* rdx, const Eos& e, DevCtrl* ctrl, cudaStream_t s);
cudaError_t launch_step_begin(DevCtrl* ctrl, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float* src, double* dst, long long count, cudaStream_t s);
// Host <-> device copy of a state-sized array.  When the host side is
// page-locked and mapped into the device's address space (unified
// addressing), and both addresses and the size are multiples of 16 bytes, the
// SMs copy it (copy16_kernel, kHostCopyBlocks blocks of 512 threads); else
// cudaMemcpyAsync.  Measured on GB300 (0.94 GB, host memory over NVLink-C2C):
// the SM copy takes 4.5 ms (H2D) / 4.9 ms (D2H) every time, while the copy
// engine took the same when copies ran back to back but up to 56 ms for the
// first copy after a few hundred ms without host transfers.
constexpr int kHostCopyBlocks = 152 * 4;
cudaError_t host_copy(void* dst, const void* src, size_t bytes, bool to_device, cudaStream_t s);
// block decomposition (blocks.cu): the three boundary layers of side `side`
// (0 low, 1 high) of direction `dir` of a state of nfields fields, element
// size elem (4 or 8 bytes), into out[field][layer][plane]; the start of a
// step with a given dt
cudaError_t launch_pack_side(const void* q, void* out, int elem, int nfields, long long nc, const int* n, int dir,
                             int side, cudaStream_t s);
cudaError_t launch_block_begin(DevCtrl* ctrl, double dt, cudaStream_t s);
cudaError_t run_fma_probe(int fp64, double* tflops, cudaStream_t s);

// thread-block size of every sweep launch
constexpr int kSweepThreads = 128;
// threads per block of the sweep along direction d
__host__ __device__ constexpr int sweep_threads(int dir) { return dir == 0 ? 32 : kSweepThreads; }
// Resident sweep blocks per SM requested from the register allocator,
// counted in 128-thread blocks, per form, and for the FP32 forms separately
// for the x sweep and for the last sweep with its stage update (1: up to 255
// registers a thread; 2: 255; 3: 168; 4: 128).  The FP64 forms are bound by the FP64 pipe and lose nothing at
// two blocks; the FP32 forms need the warps to cover their load latency.
// Pencil segments per warp (cells along the sweep direction) are lengthened
// up to MFC_MAX_SEG cells while the grid still fills the device's resident
// blocks MFC_MIN_WAVES times (measured best at 256^3: FP64 64 cells, mixed
// 32; at 512^3: mixed 128).
#ifndef MFC_MAX_SEG
#define MFC_MAX_SEG 128
#endif
#ifndef MFC_MIN_WAVES
#define MFC_MIN_WAVES 6
#endif
// Balanced work split (default): the launch has exactly MFC_BAL_WAVES times
// the device's resident warps, and warp w takes cells [w T / W, (w + 1) T / W)
// of the T = (pencil groups x cells per pencil) cells in pencil-group order --
// one or more pieces of consecutive pencil groups -- so every warp does the
// same work and no partial last wave is left.  Warps take at least
// MFC_BAL_MIN_CELLS cells (small grids launch fewer warps).  Used by the
// forms where it measured faster: FP64 (256^3: 0.956 -> 0.913 ns), FP64-fast
// (0.552 -> 0.523) and the mixed form with more than two fluids (0.0179 ->
// 0.0171).  The two-fluid mixed form keeps the seg mapping: its sweeps are
// register-capped, and the piece loop cost more than the balance gained
// (512^3: 0.0149 -> 0.0170); so does the gated form, whose cost per warp
// depends on the data (warp steps with all stencils flat skip the network),
// where many short blocks let the block scheduler even it out.  0: the seg
// mapping everywhere (and always for MFC_TMA_YZ sweeps).
#ifndef MFC_BALANCE
#define MFC_BALANCE 1
#endif
#ifndef MFC_BAL_WAVES
#define MFC_BAL_WAVES 1
#endif
#ifndef MFC_BAL_MIN_CELLS
#define MFC_BAL_MIN_CELLS 32
#endif
__host__ __device__ constexpr bool sweep_balanced(int form, int nf) {
    return MFC_BALANCE && (form == FORM_FP64_EXACT || form == FORM_FP64_FAST || (form == FORM_MIXED && nf > 2));
}
#ifndef MFC_MIN_BLOCKS_FP64
#define MFC_MIN_BLOCKS_FP64 1
#endif
#ifndef MFC_MIN_BLOCKS_MIXED
#define MFC_MIN_BLOCKS_MIXED 4
#endif
#ifndef MFC_MIN_BLOCKS_MIXED_X
#define MFC_MIN_BLOCKS_MIXED_X 2
#endif
#ifndef MFC_MIN_BLOCKS_MIXED_RK
#define MFC_MIN_BLOCKS_MIXED_RK 3
#endif
#ifndef MFC_MIN_BLOCKS_GATED
#define MFC_MIN_BLOCKS_GATED 2
#endif
#ifndef MFC_MIN_BLOCKS_GATED_RK
#define MFC_MIN_BLOCKS_GATED_RK 2
#endif
// 1: the sweeps issue the loads of the cell entering the stencil window at the
// top of each step along the pencil (they complete under that step's
// arithmetic); 0: at the bottom, just before they are used.
// FP64 reference-order sweeps: carry two WENO5 candidate values per field
// from cell to cell (1) or form them in every cell (0)
// mixed form, uniform grids, x sweep: carry WENO5 first differences and
// curvature parts from cell to cell (1) or form them in every cell (0)
#ifndef MFC_DIFF_CARRY
#define MFC_DIFF_CARRY 1
#endif
#ifndef MFC_CAND_CARRY
#define MFC_CAND_CARRY 1
#endif
#ifndef MFC_PREFETCH
#define MFC_PREFETCH 1
#endif

// Cells of a sweep counted in warp units: pencil groups (32 adjacent pencils)
// times cells per pencil.
__host__ __device__ inline long long sweep_group_cells(int dir, const int* n) {
    int na = dir == 0 ? n[1] : n[0];
    int nb = dir == 2 ? n[1] : n[2];
    return (long long)((na + 31) / 32) * nb * n[dir];
}

__host__ __device__ inline long long sweep_warps(int dir, const int* n, int seg) {
    int na = dir == 0 ? n[1] : n[0];
    int nb = dir == 2 ? n[1] : n[2];
    int ns = n[dir];
    long long nchunk = (na + 31) / 32;
    long long nseg = (ns + seg - 1) / seg;
    return nchunk * nseg * nb;
}

}  // namespace mfc5
