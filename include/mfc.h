/*
 * mfc.h -- C ABI of the GB300 five-equation solver library (libmfc5.so).
 *
 * The library evaluates and advances the semi-discrete two-fluid
 * five-equation (Allaire) model with the stiffened-gas equation of state
 * (arXiv 2409.10729, Sec. II-A), discretised by finite volumes on a uniform
 * Cartesian grid with WENO5-JS reconstruction of primitive variables and HLLC
 * fluxes (Sec. II-B, Eq. (eqn:discretization) and its cell-integrated form),
 * advanced in time by Shu-Osher SSP-RK3.  All compute runs in the library's
 * own CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - State layout: conservative q[f][z][y][x], x fastest, interior cells
 *     only, FP64.  f = 0: alpha1*rho1, 1: alpha2*rho2, 2..2+d-1: rho*u_k,
 *     2+d: rho*E, 3+d: alpha1, with d = ndim and neq = d + 4 fields.  The
 *     primitive layout w has u_k in place of rho*u_k and p in place of rho*E.
 *   - Pointers flagged on_device = 1 are device pointers on the device the
 *     context was created on; on_device = 0 means host memory.  Copies are
 *     ordered on the context's stream; calls that return host data
 *     synchronise that stream before returning.  A host array in page-locked
 *     memory mapped into the device's address space (cudaHostAlloc, or
 *     memory pinned by PyTorch, under unified addressing), with its address
 *     and size multiples of 16 bytes, is copied by the GPU's SMs through that
 *     mapping; it must lie within one page-locked allocation.  Other host
 *     memory goes through cudaMemcpyAsync.
 *   - The context owns all device memory it allocates; the caller owns every
 *     pointer it passes in and keeps it valid until the call returns.
 *   - Every call returns an mfc_status.  Nothing aborts, traps or prints.
 *   - One context must not be used from two threads at once.
 */
#ifndef MFC5_H
#define MFC5_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfc_ctx mfc_ctx;

typedef enum {
    MFC_OK = 0,
    MFC_EINVAL = -1,        /* bad argument or parameter */
    MFC_ENOMEM = -2,        /* device or pinned-host allocation failed */
    MFC_ECUDA = -3,         /* a CUDA runtime call failed (see mfc_last_cuda_error) */
    MFC_ENONPHYSICAL = -4,  /* a face or cell state had rho<=0, c^2<=0 or NaN */
    MFC_ESTATE = -5,        /* call out of order (e.g. stepping before a state is set) */
    MFC_ETOOBIG = -6        /* problem larger than mfc_rhs_noalloc's fixed scratch */
} mfc_status;

typedef enum {
    MFC_FP64 = 0,      /* every step in FP64, in the textbook operation order of each formula
                          (bit-identical to a serial evaluation in that order) */
    MFC_MIXED = 1,     /* FP32 state/stencils/Riemann; FP64 pressure recovery and RK update */
    MFC_GATED = 2,     /* MFC_MIXED plus an MLP gate choosing linear-weight WENO in smooth cells */
    MFC_FP64_FAST = 3  /* FP64 with the formulas reorganised for fewer FP64 instructions
                          (WENO in differences, product-form weights, FMA); agrees with
                          MFC_FP64 to rounding, amplified by the flow over long runs */
} mfc_precision;

typedef enum { MFC_BC_TRANSMISSIVE = 0, MFC_BC_PERIODIC = 1 } mfc_bc;

#define MFC_MAX_FLUIDS 4

/* Problem statement (Sec. II-A/B): a uniform grid, N stiffened gases, BCs.
 * State layout with N fluids (N = nfluids): alpha_i rho_i (i = 1..N),
 * rho u_k (k < ndim), rho E, alpha_1 .. alpha_{N-1} (alpha_N = 1 - sum):
 * neq = 2 N + ndim fields; two fluids: alpha1 rho1, alpha2 rho2, rho u_k,
 * rho E, alpha1 (neq = ndim + 4). */
typedef struct {
    int ndim;          /* 1, 2 or 3 */
    int n[3];          /* cells per dimension; entries beyond ndim are ignored (treated as 1) */
    double lo[3];      /* lower corner; dx_d = (hi[d] - lo[d]) / n[d] */
    double hi[3];      /* upper corner */
    int bc[3][2];      /* mfc_bc per dimension and side; periodic must be set on both sides */
    double gamma[MFC_MAX_FLUIDS];   /* ratio of specific heats of fluids 1..N (> 1) */
    double pi_inf[MFC_MAX_FLUIDS];  /* stiffness pi_inf of fluids 1..N (>= 0), in pressure units */
    double weno_eps;   /* WENO epsilon, absolute (1e-6 is the usual choice) */
    int precision;     /* mfc_precision */
    int weno_order;    /* reconstruction (Sec. II-B): 5 = WENO5-JS, 3 = WENO3-JS (Jiang-Shu, two
                          two-cell stencils, linear weights 1/3, 2/3); 0 means 5.  WENO3 is
                          available in every precision except MFC_GATED (MFC_EINVAL) */
    int nfluids;       /* N, 2 .. MFC_MAX_FLUIDS; 0 means 2.  N > 2: not with MFC_GATED or
                          mfc_set_grid (MFC_EINVAL) */
} mfc_params;

/* Creates a context: validates params (MFC_EINVAL), allocates the state,
 * stage and accumulator buffers on the current CUDA device (MFC_ENOMEM; also
 * returned, before any device call, for more than 2^36 cells) and
 * binds the CUDA stream `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream).  *out receives the context, or NULL on failure. */
int mfc_create(const mfc_params* params, void* cuda_stream, mfc_ctx** out);

/* Frees every resource of the context after synchronising its stream.
 * NULL is accepted and ignored. */
int mfc_destroy(mfc_ctx* ctx);

/* Sets the current state q^n from conservative FP64 values, layout above,
 * neq * ncells doubles.  Also computes the CFL wave speed of that state. */
int mfc_set_state(mfc_ctx* ctx, const double* q, int on_device);

/* Same as mfc_set_state, from primitive FP64 values w (alpha1 rho1, alpha2
 * rho2, u_k, p, alpha1); the conversion to conservative variables uses the
 * mixture EOS of Sec. II-A and runs on the GPU. */
int mfc_set_state_prim(mfc_ctx* ctx, const double* w, int on_device);

/* Copies the current state q^n (always FP64, conservative) to q. */
int mfc_get_state(mfc_ctx* ctx, double* q, int on_device);

/* Evaluates the semi-discrete right-hand side L(q^n) of the cell-integrated
 * form of Eq. (eqn:discretization) -- flux differences of all directions plus
 * the alpha1 term alpha1 * div(u) -- and writes it to rhs (FP64, state
 * layout).  Returns MFC_ENONPHYSICAL if a reconstructed face state was
 * non-physical; rhs is written either way. */
int mfc_rhs(mfc_ctx* ctx, double* rhs, int on_device);

/* S = max over cells of sum_d (|u_d| + c)/dx_d for the current state
 * [1/time units]; the CFL step is dt = cfl / S. */
int mfc_max_wavespeed(mfc_ctx* ctx, double* s);

/* Advances nsteps SSP-RK3 steps.  Each step uses dt_n = cfl / S(q^n), with S
 * computed on the GPU at the end of the previous step (no host round trip).
 * *t_advanced (may be NULL) receives the sum of the dt_n.  Returns
 * MFC_ENONPHYSICAL after the last step if any state during the run was
 * non-physical; the state is left as computed. */
int mfc_step_rk3(mfc_ctx* ctx, double cfl, int nsteps, double* t_advanced);

/* Advances nsteps SSP-RK3 steps of fixed size dt > 0. */
int mfc_step_rk3_dt(mfc_ctx* ctx, double dt, int nsteps);

/* Number of kernel launches one call of mfc_step_rk3 with nsteps = 1 makes
 * (a step is replayed from a captured CUDA graph of these launches). */
int mfc_launches_per_step(mfc_ctx* ctx, int* launches);

/* Per-kernel timing.  While enabled, mfc_step_rk3/mfc_step_rk3_dt launch
 * kernels directly (no graph) and bracket each launch with CUDA events on the
 * context's stream; the accumulated device time per kernel kind can be read
 * with mfc_kernel_time.  Enabling or disabling resets the accumulators. */
int mfc_set_timing(mfc_ctx* ctx, int enable);

/* Kernel kind `index` (0-based): its name, the summed device time in ms and
 * the number of launches since timing was enabled.  Returns MFC_EINVAL when
 * index is out of range. */
int mfc_kernel_time(mfc_ctx* ctx, int index, const char** name, double* ms, long long* launches);

/* ---- gated form (MFC_GATED): the troubled-cell network ------------------
 * No counterpart in the paper.  Per cell and direction two sensor stencils
 * are read from the five stencil cells' primitives: the mixture density
 * alpha1 rho1 + alpha2 rho2 and the pressure.  A sensor stencil s is flat
 * when max_k |s_k - s_2| <= MFC_GATE_FLOOR |s_2| (a round-off floor) and then
 * counts as smooth; otherwise a 5 -> 32 -> 32 -> 1 perceptron (ReLU hidden
 * layers, logistic output; FP32 arithmetic, evaluated on the tensor cores
 * with every operand split into two f16 halves) reads the normalised stencil
 * x_k = (s_k - s_2) / max_j |s_j - s_2| and calls it smooth when its logit
 * is negative.  A cell whose two sensors are smooth is reconstructed with
 * the linear WENO5 weights in that direction, unless a linear face state has
 * rho <= 0, alpha1 outside [0, 1] or (Gamma + 1) p + Pi <= 0 (then WENO5-JS,
 * the fallback); every other cell with full WENO5-JS.  Parameters
 * (MFC_MLP_NPARAMS floats): W1[32][5], b1[32], W2[32][32], b2[32], w3[32], b3. */
#define MFC_GATE_FLOOR 1e-4
#define MFC_MLP_NPARAMS 1281

/* Makes direction `dir` (0 <= dir < ndim) non-uniform: `edges` is a host
 * array of the n[dir] + 1 cell edges, strictly increasing (e.g. the
 * tanh-refined grids of Sec. III-A); lo/hi of the params no longer apply to
 * that direction.  The reconstruction becomes Shu's WENO5 for non-uniform
 * cells (per-cell candidate coefficients, smoothness indicators and linear
 * weights, computed here from the edges), and the flux divergence and CFL
 * bound use each cell's own width; ghost-cell widths follow the BC (copied
 * at transmissive, wrapped at periodic boundaries).  Only WENO5 in the FP64,
 * FP64-fast and mixed forms: MFC_EINVAL for WENO3 or MFC_GATED contexts, a
 * bad direction, or edges that are not strictly increasing.  Synchronises
 * the context's stream; the wave speed of a state already set is
 * recomputed.  The edges are copied.  On MFC_ENOMEM or MFC_ECUDA while the
 * new tables are allocated or copied, the context keeps its previous grid. */
int mfc_set_grid(mfc_ctx* ctx, int dir, const double* edges);

/* Sets the gate weights of a MFC_GATED context (host array of n =
 * MFC_MLP_NPARAMS finite floats, copied).  Stepping a gated context before
 * this returns MFC_ESTATE. */
int mfc_set_mlp_weights(mfc_ctx* ctx, const float* w, int n);

/* Gate statistics of the last mfc_rhs / mfc_step_rk3 call: cell
 * reconstructions (cells x directions x stages) evaluated, done with linear
 * weights, and gated but recomputed with WENO because a face was non-physical. */
int mfc_gate_stats(mfc_ctx* ctx, long long* gated, long long* fallback, long long* cells);

/* Of the cell reconstructions counted by mfc_gate_stats, those whose warp
 * step had flat density and pressure stencils (below the round-off floor) in
 * all 32 pencils: every one counts as smooth and the network is not
 * evaluated for that step.  MFC_EINVAL on a NULL argument. */
int mfc_gate_flat(mfc_ctx* ctx, long long* flat);

/* L(q^n) of a MFC_GATED context as mfc_rhs, and the gate's decision for
 * every direction and cell: decisions[d * ncells + cell] = 0 (WENO5-JS),
 * 1 (linear weights) or 2 (called smooth, but a linear face was non-physical:
 * WENO5-JS).  decisions is host (on_device = 0) or device memory with room
 * for ndim * ncells bytes.  The first call allocates a device buffer of that
 * size (MFC_ENOMEM).  MFC_EINVAL for other forms; synchronises the stream. */
int mfc_gate_rhs(mfc_ctx* ctx, double* rhs, signed char* decisions, int on_device);

/* Labelled training samples from the current state (FP64 WENO5-JS weights):
 * for every direction d and cell c, two samples (mixture-density stencil,
 * pressure stencil), index (d * ncells + c) * 2 + sensor; X[sample][5] the
 * normalised stencil, Y[sample] = 1 when some primitive's nonlinear weight at
 * either face departs from its linear weight by more than tau (relative) on
 * a stencil of that primitive that is not flat (variation above
 * MFC_GATE_FLOOR of its centre value: below it the two reconstructions differ
 * by round-off), else 0; a flat sensor stencil, which the gate never shows
 * the network, gets X = 0 and Y = -1.
 * X, Y are device pointers with room for capacity >= 2 * ndim * ncells
 * samples; *count receives that number.  Synchronises the context stream. */
int mfc_gate_samples(mfc_ctx* ctx, float* X, float* Y, long long capacity, float tau, long long* count);

/* Training kernels (device pointers; cuda_stream a cudaStream_t, NULL = default).
 * mfc_mlp_loss_grad: mean weighted binary cross-entropy of n samples
 *   (l = wp y softplus(-z) + (1 - y) softplus(z), z the logit) into *loss and
 *   its gradient into grad[MFC_MLP_NPARAMS] (both overwritten).
 * mfc_mlp_adam: one Adam step t (1-based) of theta with moments m, v.
 * mfc_mlp_forward: logits z[n] of X[n][5] (FP32 CUDA cores).
 * mfc_mlp_forward_tc: the same logits as the gated sweep computes them --
 *   every layer on the tensor cores, operands split into two f16 halves
 *   (hi * hi + lo * hi + hi * lo), FP32 accumulation. */
int mfc_mlp_nparams(void);
int mfc_mlp_loss_grad(const float* X, const float* Y, long long n, const float* theta, float pos_weight,
                      float* grad, float* loss, void* cuda_stream);
int mfc_mlp_adam(float* theta, const float* grad, float* m, float* v, int t, float lr, float beta1, float beta2,
                 float eps, void* cuda_stream);
int mfc_mlp_forward(const float* X, long long n, const float* theta, float* z, void* cuda_stream);
int mfc_mlp_forward_tc(const float* X, long long n, const float* theta, float* z, void* cuda_stream);

/* Instrumentation, no counterpart in the paper: measures the sustained FMA
 * throughput of the current device with independent FMA chains, FP64
 * (fp64 != 0) or FP32, in TFLOP/s (2 flops per FMA).  Used as the ALU
 * roofline denominator.  Allocates and frees 16 bytes of device memory and
 * synchronises the legacy default stream. */
int mfc_alu_peak(int fp64, double* tflops);

/* ---- block decomposition (Sec. III-A) --------------------------------------
 * The global grid is split into Cartesian blocks, one context per block (on
 * one GPU or several).  A block needs three ghost layers of the stage state
 * beyond every side that borders another block; they are exchanged once per
 * RK stage, and dt comes from the wave speed reduced over all blocks.  One
 * SSP-RK3 step of a decomposed grid, driven by the caller:
 *   S   = max over blocks of mfc_block_wavespeed     (dt = cfl / S)
 *   mfc_block_begin_step(b, dt) for every block
 *   for stage k = 1, 2, 3:
 *     mfc_block_pack(b, k, send_b) for every block
 *     copy each packed side into the facing side of the neighbour's halo
 *     mfc_block_stage(b, k, halo_b) for every block
 * The result is bit-identical to the undecomposed grid's in every form: a
 * cell's update depends only on the cells of its stencils and on dt.
 *
 * Halo layout of a block (mfc_halo_layout): one segment per side (d, s) that
 * borders another block, in the order (x low, x high, y low, y high, z low,
 * z high); a segment is [field][layer 0..2][plane], the plane index being a
 * cell's position in the plane normal to d, x fastest (y + ny z normal to x,
 * x + nx z normal to y, x + nx y normal to z).  Layer l of the low side is
 * the block's cell l - 3 along d, of the high side its cell n_d + l.  The
 * fields are the stage state's: the neq conservative FP64 fields in the FP64
 * forms; in the FP32 forms, neq FP32 fields and the pressure (neq + 1).
 * mfc_block_pack writes a block's own boundary layers in the same layout (low
 * side: its cells 0, 1, 2; high side: n_d - 3 .. n_d - 1), so the packed low
 * side of block B is the high-side halo segment of B's low neighbour, and the
 * packed high side the low-side segment of its high neighbour. */
typedef struct {
    int lo[3];   /* global index of the block's first cell per dimension (0 beyond ndim) */
    int n[3];    /* cells of the block per dimension (1 beyond ndim); at least 3 along a
                    dimension in which the block has a neighbour */
} mfc_block;

/* Creates the context of one block of the grid `global` (validated as by
 * mfc_create).  Its state, stage and accumulator buffers hold the block's
 * cells only (layout as above, with the block's n); the grid spacing is the
 * global grid's.  A side borders another block unless it is a domain
 * boundary of a non-periodic dimension, or the block spans a periodic
 * dimension (then it wraps onto itself).  MFC_EINVAL for a block outside the
 * grid or thinner than 3 cells in a dimension with a neighbour.  Such a
 * context takes the state calls (mfc_set_state, mfc_get_state, ...) for its
 * own cells; mfc_rhs, mfc_step_rk3 and mfc_step_rk3_dt return MFC_ESTATE when
 * it has a neighbour (use the calls below), and mfc_set_grid MFC_EINVAL. */
int mfc_create_block(const mfc_params* global, const mfc_block* block, void* cuda_stream, mfc_ctx** out);

/* Halo layout: offset[2 d + s] = element offset of side (d, s)'s segment, or
 * -1 where that side has no neighbour (offset has room for 6); *total = the
 * elements of the pack and halo buffers; *elem_bytes = 8 (FP64 forms) or 4
 * (FP32 forms).  Any output may be NULL.  A context that is not a block
 * reports no segments. */
int mfc_halo_layout(mfc_ctx* ctx, long long* offset, long long* total, int* elem_bytes);

/* Packs the boundary layers of the state that stage `stage` (1..3) reads
 * (q^n for stage 1) into the device buffer `out` (halo layout, caller-owned,
 * `total` elements).  Ordered on the context's stream; does not synchronise. */
int mfc_block_pack(mfc_ctx* ctx, int stage, void* out);

/* Starts a step of size dt > 0 (cfl / S with S reduced over all blocks):
 * the counterpart of the first kernel of mfc_step_rk3's step. */
int mfc_block_begin_step(mfc_ctx* ctx, double dt);

/* Stage `stage` (1..3) of SSP-RK3 on the block: the direction sweeps with
 * the stage update folded into the last; ghost cells beyond a side with a
 * neighbour are read from `halo` (device, halo layout, filled with the
 * neighbours' packed layers of the same stage's input; may be NULL for a
 * block without neighbours).  Stage 3 also reduces the block's wave speed.
 * Ordered on the context's stream; does not synchronise. */
int mfc_block_stage(mfc_ctx* ctx, int stage, const void* halo);

/* The block's wave speed S: of the state set last (mfc_set_state*), or, after
 * a stage 3, of the new state.  Synchronises the stream.  Returns
 * MFC_ENONPHYSICAL (and clears the flag) when a state or face since the last
 * such report was non-physical. */
int mfc_block_wavespeed(mfc_ctx* ctx, double* s);

/* L(q^n) of the block (as mfc_rhs) with the ghost cells beyond its sides
 * with neighbours taken from `halo` (the neighbours' packed stage-1 layers). */
int mfc_block_rhs(mfc_ctx* ctx, const void* halo, double* rhs, int on_device);

/* Capacity, in doubles, of the fixed device scratch used by mfc_rhs_noalloc
 * (16 MiB): it must hold neq * ncells doubles plus a 32-double control block. */
#define MFC_NOALLOC_MAX_DOUBLES (2 * 1024 * 1024)

/* The right-hand side L(q) of mfc_rhs, FP64 only, for callers that cannot
 * allocate device memory when they need it -- e.g. code living inside a
 * framework whose pool allocator owns the whole GPU, or a long-running
 * service that must keep a fixed footprint and avoid cudaMalloc's implicit
 * device synchronisation after start-up.  There is no counterpart in the
 * paper; the arithmetic is that of mfc_rhs.
 *   params       problem statement; precision must be MFC_FP64 (else MFC_EINVAL)
 *   q            device pointer, conservative FP64 state, layout above
 *   rhs          device pointer, receives L(q), same layout; the ranges
 *                [q, q + neq*ncells) and [rhs, rhs + neq*ncells) must not
 *                overlap (MFC_EINVAL): the last sweep writes L into cells
 *                that other warps still read as stencil input
 *   cuda_stream  cudaStream_t the kernels run on (NULL = legacy default)
 * No context, no allocation of any kind: the only scratch (accumulator and
 * status word) is a fixed array in device memory that belongs to the loaded
 * library and is held on every device that loads it until process exit.
 * Problems with neq * ncells + 32 > MFC_NOALLOC_MAX_DOUBLES are rejected with
 * MFC_ETOOBIG before anything is launched.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture begins, and do not call again on a device after
 * cudaDeviceReset() on it.  Every call shares the array: calls whose kernels
 * may overlap on the GPU race and must be serialised by the caller.  Every
 * call synchronises `cuda_stream` before returning, to read the status word;
 * returns MFC_ENONPHYSICAL as mfc_rhs does. */
int mfc_rhs_noalloc(const mfc_params* params, const double* q, double* rhs, void* cuda_stream);

/* Instrumentation, no counterpart in the paper: checks the mixed form's
 * integer-pipe float<->double conversions against the hardware conversions on
 * n pseudo-random bit patterns (all exponent ranges); *mismatches receives the
 * number of differing results (0 expected).  Allocates 4 bytes of device
 * memory and synchronises the legacy default stream. */
int mfc_selfcheck_conversions(long long n, unsigned long long seed, long long* mismatches);

/* Instrumentation, no counterpart in the paper: checks the FP64 form's
 * integer-pipe WENO5 operations (products by 3, 5, 7 and 11, quotients by 6)
 * against the FP64 instructions, and its integer-word compares (x > 0, 0 <= x,
 * x < y) against the FP64 compares, on n pseudo-random patterns (all
 * exponents, zeros, subnormals, infinities, NaNs); *mismatches receives the number of
 * differing results (0 expected).  Allocates 4 bytes of device memory and
 * synchronises the legacy default stream. */
int mfc_selfcheck_exact_ops(long long n, unsigned long long seed, long long* mismatches);

/* Message for a status code (static storage). */
const char* mfc_strerror(int status);

/* The last CUDA error code the library saw in this context (0 if none). */
int mfc_last_cuda_error(mfc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MFC5_H */
