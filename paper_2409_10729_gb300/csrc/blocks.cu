// blocks.cu -- kernels of the block decomposition (arXiv 2409.10729,
// Sec. III-A): the global grid is split into Cartesian blocks, each with
// three ghost layers per side that borders another block, exchanged once per
// RK stage, and the CFL wave speed is reduced over all blocks.
//
// pack_side_kernel copies the three boundary layers of one side of a block's
// stage state into a contiguous buffer laid out as [field][layer][plane]: for
// the low side the block's cells 0, 1, 2, for the high side n-3, n-2, n-1, in
// that order.  That is exactly the layout of the neighbour's halo on the
// facing side (its cells n, n+1, n+2 beyond its high side, or -3, -2, -1
// beyond its low side), so a packed side is handed over with one copy.
// The plane index of a cell is its position in the plane normal to the
// direction, x fastest: y + ny z (normal to x), x + nx z (normal to y),
// x + nx y (normal to z).
#include "mfc_internal.cuh"

namespace mfc5 {

template <typename T>
__global__ void pack_side_kernel(const T* __restrict__ q, T* __restrict__ out, long long nc, int nfields, int n0,
                                 int n1, int n2, int dir, int side) {
    const int nd = dir == 0 ? n0 : (dir == 1 ? n1 : n2);
    const long long plane = nc / nd;
    const long long total = (long long)nfields * 3 * plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i % plane;
        const long long fl = i / plane;
        const int l = (int)(fl % 3), f = (int)(fl / 3);
        const int j = side ? nd - 3 + l : l;
        long long c;
        if (dir == 0) {
            c = j + (long long)n0 * p;                               // p = y + n1 z
        } else if (dir == 1) {
            const long long x = p % n0, z = p / n0;                  // p = x + n0 z
            c = x + (long long)n0 * (j + (long long)n1 * z);
        } else {
            c = p + (long long)n0 * n1 * j;                          // p = x + n0 y
        }
        out[i] = q[(long long)f * nc + c];
    }
}

// Start of a step whose dt the caller took from the wave speed reduced over
// all blocks: set dt, advance t, clear the accumulator the step's last sweep
// fills with S of the new state.
__global__ void block_begin_kernel(DevCtrl* ctrl, double dt) {
    ctrl->S = __longlong_as_double((long long)ctrl->S_bits);
    if (!(dt > 0.0) || !(dt < INFINITY)) ctrl->status |= 2u;
    ctrl->dt = dt;
    ctrl->t += dt;
    ctrl->S_bits = 0ULL;
}

cudaError_t launch_pack_side(const void* q, void* out, int elem, int nfields, long long nc, const int* n, int dir,
                             int side, cudaStream_t s) {
    const long long plane = nc / n[dir];
    const long long total = (long long)nfields * 3 * plane;
    long long blocks = (total + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152LL * 32) blocks = 152LL * 32;   // grid-stride beyond this
    if (elem == 8)
        pack_side_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double*>(q),
                                                                   static_cast<double*>(out), nc, nfields, n[0],
                                                                   n[1], n[2], dir, side);
    else
        pack_side_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float*>(q),
                                                                  static_cast<float*>(out), nc, nfields, n[0], n[1],
                                                                  n[2], dir, side);
    return cudaGetLastError();
}

cudaError_t launch_block_begin(DevCtrl* ctrl, double dt, cudaStream_t s) {
    block_begin_kernel<<<1, 1, 0, s>>>(ctrl, dt);
    return cudaGetLastError();
}

}  // namespace mfc5
