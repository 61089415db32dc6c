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

// 16-bit storages: the packed two-cell form, three blocks per SM.
template <int S, int P>
__global__ void __launch_bounds__(256, 3) k_sweep2p(const SweepArgs a) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = sweep_plane(a);
    if (x0 >= a.nx || y >= a.ny || z < 0) return;
    sweep_two16<S, P>(a, x0, y, z);
}

// 16-bit storages with nx % 128 == 0 and 19 Np < 2^31: a warp per 128 cells
// of a row, eight rows per block (see sweep_four).
template <int S, int P>
__global__ void __launch_bounds__(256, 2) k_sweep4(const SweepArgs a) {
    const int lane = threadIdx.x;
    const int x0 = 128 * blockIdx.x + 4 * lane;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = sweep_plane(a);
    if (y >= a.ny || z < 0) return;  // a whole warp
    sweep_four<S, P>(a, x0, y, z, lane);
}

template <int S>
static void launch_s(const SweepArgs& a, int parity, int variant, int gz, cudaStream_t st) {
    if constexpr (S == ST_F16 || S == ST_BF16) {
        if (variant == 3 && a.nx % 128 == 0 && 19 * a.Np < (int64_t(1) << 31)) {
            dim3 block(32, 8), grid(a.nx / 128, (a.ny + 7) / 8, gz);
            if (parity == 0) k_sweep4<S, 0><<<grid, block, 0, st>>>(a);
            else k_sweep4<S, 1><<<grid, block, 0, st>>>(a);
            return;
        }
    }
    if constexpr (S != ST_F64) {
        if (variant != 1 && a.nx % 2 == 0) {
            const int pairs = a.nx / 2;
            int bx = ((pairs + 31) / 32) * 32;
            if (bx > 128) bx = 128;
            const int by = 256 / bx;
            dim3 block(bx, by), grid((pairs + bx - 1) / bx, (a.ny + by - 1) / by, gz);
            if constexpr (S == ST_F16 || S == ST_BF16) {
                if (variant == 4 && 19 * a.Np < (int64_t(1) << 31)) {  // the packed form
                    if (parity == 0) k_sweep2p<S, 0><<<grid, block, 0, st>>>(a);
                    else k_sweep2p<S, 1><<<grid, block, 0, st>>>(a);
                    return;
                }
            }
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

// variant: 0 = default (reduced storages with even nx: two cells per thread;
// FP64: one), 1 = one cell per thread, 2 = two cells per thread where
// possible, 3 = FP16 / BF16: four cells per thread where possible (else as
// 2), 4 = FP16 / BF16: two cells per thread, packed (else as 2).
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
