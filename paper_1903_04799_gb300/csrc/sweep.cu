// sweep.cu -- fused stream + collide over the whole lattice of a context
// (Sec. III, Eq. "lb"); the per-cell arithmetic is in sweep_body.cuh.
//
// Grid (x-blocks, y-blocks, z-planes).  The update is the in-place AA pattern
// (see lbsq_internal.cuh): even steps read and write a cell's own 19 slots,
// odd steps read and write its 19 neighbour slots.  The kernels are
// geometry-free: solid cells are swept too (their slots are private to them,
// and every slot a fluid cell reads from a solid neighbour is rewritten by the
// link kernel after the sweep), so no flag field is read.
#include "sweep_body.cuh"

namespace lbsq {

template <int S, int P>
__global__ void __launch_bounds__(256) k_sweep(const SweepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = sweep_plane(a);
    if (x >= a.nx || z < 0) return;
    sweep_one<S, P>(a, x, blockIdx.y, z);
}

template <int S, int P>
__global__ void __launch_bounds__(256, 2) k_sweep2(const SweepArgs a) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = sweep_plane(a);
    if (x0 >= a.nx || y >= a.ny || z < 0) return;
    sweep_two<S, P>(a, x0, y, z);
}

template <int S>
static void launch_s(const SweepArgs& a, int parity, int variant, int gz, cudaStream_t st) {
    if constexpr (S != ST_F64) {
        if (variant != 1 && a.nx % 2 == 0) {
            const int pairs = a.nx / 2;
            int bx = ((pairs + 31) / 32) * 32;
            if (bx > 128) bx = 128;
            const int by = 256 / bx;
            dim3 block(bx, by), grid((pairs + bx - 1) / bx, (a.ny + by - 1) / by, gz);
            if (parity == 0) k_sweep2<S, 0><<<grid, block, 0, st>>>(a);
            else k_sweep2<S, 1><<<grid, block, 0, st>>>(a);
            return;
        }
    }
    int bx = ((a.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    dim3 grid((a.nx + bx - 1) / bx, a.ny, gz);
    if (parity == 0) k_sweep<S, 0><<<grid, bx, 0, st>>>(a);
    else k_sweep<S, 1><<<grid, bx, 0, st>>>(a);
}

// variant: 0 = default (two cells per thread where nx is even, FP64 one cell),
// 1 = one cell per thread, 2 = two cells per thread where possible.
// zmode / win / gz: plane selection (see SweepArgs); gz = grid planes (nz for
// modes 0 and 1, an upper bound of the window length for mode 2).  Odd steps
// sweep the planes in descending order.
void launch_sweep(const Lattice& L, double lambda_e, double lambda_o, int parity, int variant, int zmode,
                  const int* win, int gz, cudaStream_t st) {
    SweepArgs a = sweep_args(L, lambda_e, lambda_o);
    a.zmode = zmode;
    a.win = win;
    a.reverse = parity;
    if (gz <= 0) return;
    switch (L.storage) {
        case ST_F64: launch_s<ST_F64>(a, parity, variant, gz, st); break;
        case ST_F32: launch_s<ST_F32>(a, parity, variant, gz, st); break;
        case ST_F16: launch_s<ST_F16>(a, parity, variant, gz, st); break;
        default: launch_s<ST_BF16>(a, parity, variant, gz, st); break;
    }
}

}  // namespace lbsq
