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
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y, z);
    if (x >= a.nx || y < 0) return;
    sweep_one<S, P>(a, x, y, z);
}

template <int S, int P, bool O32>
__global__ void __launch_bounds__(256, 2) k_sweep2(const SweepArgs a) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    if (x0 >= a.nx || y < 0) return;
    sweep_two<S, P, O32>(a, x0, y, z);
}

// 16-bit storages: the packed two-cell form, three blocks per SM.
template <int S, int P>
__global__ void __launch_bounds__(256, 3) k_sweep2p(const SweepArgs a) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    if (x0 >= a.nx || y < 0) return;
    sweep_two16<S, P>(a, x0, y, z);
}

// 16-bit storages with nx % 128 == 0 and 19 Np < 2^31: a warp per 128 cells
// of a row, eight rows per block (see sweep_four).
template <int S, int P, int ROWS>
__global__ void __launch_bounds__(32 * ROWS, 2) k_sweep4(const SweepArgs a) {
    const int lane = threadIdx.x;
    const int x0 = 128 * blockIdx.x + 4 * lane;
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    if (y < 0) return;  // a whole warp
    sweep_four<S, P>(a, x0, y, z, lane);
}

// 16-bit storages, two cells per thread on kPlanes consecutive plane slots,
// software-pipelined (see load_pair16).
constexpr int kPlanes = 4;

template <int S, int P>
__global__ void __launch_bounds__(256, 2) k_sweep2z(const SweepArgs a, int slots) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int ly = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= a.nx) return;
    const int p0 = blockIdx.z * kPlanes;
    unsigned int cur[Q], nxt[Q];
    int z = sweep_plane_at(a, p0);
    int y = z < 0 ? -1 : sweep_row(a, ly, z);  // the row depends on the plane in the far sweep
    if (y >= 0) load_pair16<S, P>(a, x0, y, z, cur);
    for (int k = 0; k < kPlanes && p0 + k < slots; ++k) {
        const int zn = (k + 1 < kPlanes && p0 + k + 1 < slots) ? sweep_plane_at(a, p0 + k + 1) : -1;
        const int yn = zn < 0 ? -1 : sweep_row(a, ly, zn);
        if (yn >= 0) load_pair16<S, P>(a, x0, yn, zn, nxt);  // in flight during the collision below
        if (y >= 0) collide_store_pair16<S, P>(a, x0, y, z, cur);
#pragma unroll
        for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
        z = zn;
        y = yn;
    }
}

// 16-bit storages with nx % 4 == 0, nx <= 768: blocks of whole rows, four
// cells per thread (see sweep_four_rows); dynamic shared memory of
// 10 x rows x nx elements on odd steps.
template <int S, int P, bool O32>
__global__ void __launch_bounds__(P == 0 ? 256 : 192, 2) k_sweep4r(const SweepArgs a) {
    extern __shared__ unsigned short rowbuf[];
    const int z = sweep_plane(a);
    if (z < 0) return;  // the whole block
    const int y = sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    sweep_four_rows<S, P, O32>(a, y < 0 ? 0 : y, z, y >= 0, rowbuf);
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Planes ahead for the two-cell form's L2 prefetch (SweepArgs::pf): past the
// planes that the resident blocks (two per SM) cover, plus two.  Measured on
// GB300 (whole-lattice sweeps at 256^3): FP32 0.959 -> 0.990 of the copy
// bandwidth, FP16 0.745 -> 0.684.  Whole-lattice FP32 sweeps only: a prefetch
// installs its lines in L2 at normal priority, and beside the body kernels of
// a split step (far sweeps) that evicted their code again (128^3 step 0.050 ->
// 0.056 ms).
static int prefetch_ahead(const SweepArgs& a, int storage, const dim3& grid) {
    if (a.zmode != 0 || storage != ST_F32) return 0;
    const long long per_plane = (long long)grid.x * grid.y;
    const int ahead = (int)((2LL * sm_count() + per_plane - 1) / per_plane) + 2;
    return ahead < a.nz ? ahead : 0;
}

bool sweep_async_supported(const SweepArgs& a, int storage_bytes);
void launch_sweep_async(const SweepArgs& a, int storage, int parity, int gz, int gy, cudaStream_t st);

template <int S>
static void launch_s(const SweepArgs& a, int parity, int variant, int gz, int gy, cudaStream_t st) {
    if constexpr (S == ST_F16 || S == ST_BF16) {
        if (variant == 7 && sweep_async_supported(a, 2)) {
            launch_sweep_async(a, S, parity, gz, gy, st);
            return;
        }
        if (variant == 5 && a.nx % 2 == 0) {
            const int pairs = a.nx / 2;
            int bx = ((pairs + 31) / 32) * 32;
            if (bx > 128) bx = 128;
            const int by = 256 / bx;
            dim3 block(bx, by), grid((pairs + bx - 1) / bx, (gy + by - 1) / by, (gz + kPlanes - 1) / kPlanes);
            if (parity == 0) k_sweep2z<S, 0><<<grid, block, 0, st>>>(a, gz);
            else k_sweep2z<S, 1><<<grid, block, 0, st>>>(a, gz);
            return;
        }
        // default: even steps in whole-row four-cell blocks (aligned 8-byte
        // chunks: 0.86 of the copy bandwidth at 256^3, against 0.74 for two
        // cells), odd steps in the two-cell form (0.63; the whole-row form's
        // odd steps, with their x-shifts through shared memory, measured 0.62)
        const bool rows4 = a.nx % 4 == 0 && a.nx <= 768;
        if ((variant == 6 || (variant == 0 && parity == 0)) && rows4) {
            // odd steps (more live values) in blocks of at most 192 threads
            const int tx = a.nx / 4, ty = (parity == 0 ? 256 : 192) / tx > 0 ? (parity == 0 ? 256 : 192) / tx : 1;
            dim3 block(tx, ty), grid(1, (gy + ty - 1) / ty, gz);
            const bool o32 = 19 * a.Np < (int64_t(1) << 32);  // element offsets fit 32 bits
            if (parity == 0) {
                if (o32) k_sweep4r<S, 0, true><<<grid, block, 0, st>>>(a);
                else k_sweep4r<S, 0, false><<<grid, block, 0, st>>>(a);
            } else {
                const size_t smem = (size_t)10 * ty * a.nx * sizeof(unsigned short);
                if (o32) k_sweep4r<S, 1, true><<<grid, block, smem, st>>>(a);
                else k_sweep4r<S, 1, false><<<grid, block, smem, st>>>(a);
            }
            return;
        }
        if (variant == 3 && a.nx % 128 == 0 && 19 * a.Np < (int64_t(1) << 31)) {
            // odd steps hold more live values (the x-shifted chunks): 6 rows per
            // block leave them 170 registers a thread at 2 blocks per SM
            if (parity == 0) {
                dim3 block(32, 8), grid(a.nx / 128, (gy + 7) / 8, gz);
                k_sweep4<S, 0, 8><<<grid, block, 0, st>>>(a);
            } else {
                dim3 block(32, 6), grid(a.nx / 128, (gy + 5) / 6, gz);
                k_sweep4<S, 1, 6><<<grid, block, 0, st>>>(a);
            }
            return;
        }
    }
    if constexpr (S != ST_F64) {
        if (variant != 1 && a.nx % 2 == 0) {
            const int pairs = a.nx / 2;
            int bx = ((pairs + 31) / 32) * 32;
            if (bx > 128) bx = 128;
            const int by = 256 / bx;
            dim3 block(bx, by), grid((pairs + bx - 1) / bx, (gy + by - 1) / by, gz);
            if constexpr (S == ST_F16 || S == ST_BF16) {
                if (variant == 4 && 19 * a.Np < (int64_t(1) << 31)) {  // the packed form
                    if (parity == 0) k_sweep2p<S, 0><<<grid, block, 0, st>>>(a);
                    else k_sweep2p<S, 1><<<grid, block, 0, st>>>(a);
                    return;
                }
            }
            SweepArgs b = a;
            b.pf = prefetch_ahead(a, S, grid);
            if (19 * a.Np < (int64_t(1) << 32)) {  // element offsets fit 32 bits
                if (parity == 0) k_sweep2<S, 0, true><<<grid, block, 0, st>>>(b);
                else k_sweep2<S, 1, true><<<grid, block, 0, st>>>(b);
            } else {
                if (parity == 0) k_sweep2<S, 0, false><<<grid, block, 0, st>>>(b);
                else k_sweep2<S, 1, false><<<grid, block, 0, st>>>(b);
            }
            return;
        }
    }
    int bx = ((a.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    dim3 grid((a.nx + bx - 1) / bx, gy, gz);
    if (parity == 0) k_sweep<S, 0><<<grid, bx, 0, st>>>(a);
    else k_sweep<S, 1><<<grid, bx, 0, st>>>(a);
}

// variant: 0 = default (FP16 / BF16: even steps as 6, odd steps as 2; other
// reduced storages with even nx: two cells per thread; FP64: one), 1 = one
// cell per thread, 2 = two cells per thread where
// possible, 3 = FP16 / BF16: four cells per thread where possible (else as
// 2), 4 = FP16 / BF16: two cells per thread, packed (else as 2), 5 = FP16 /
// BF16: two cells per thread on kPlanes planes, software-pipelined (else as 2),
// 6 = FP16 / BF16: four cells per thread in blocks of whole rows, odd-step
// x-shifts through shared memory (nx % 4 == 0, nx <= 768; else as 2), 7 =
// FP16 / BF16: persistent CTAs, loads staged in shared memory by asynchronous
// 16-byte copies (sweep_async.cu; nx % 8 == 0, nx <= 512; else as 2).
// zmode / win / gz / gy: cell selection (see SweepArgs); gz and gy = grid
// planes and rows (nz and ny for modes 0 and 1, upper bounds of the window's
// z and y lengths for mode 2).  Odd steps sweep the planes in descending
// order.
void launch_sweep(const Lattice& L, double lambda_e, double lambda_o, int parity, int variant, int zmode,
                  const int* win, int gz, int gy, cudaStream_t st) {
    SweepArgs a = sweep_args(L, lambda_e, lambda_o);
    a.zmode = zmode;
    a.win = win;
    a.reverse = parity;
    if (gz <= 0 || gy <= 0) return;
    switch (L.storage) {
        case ST_F64: launch_s<ST_F64>(a, parity, variant, gz, gy, st); break;
        case ST_F32: launch_s<ST_F32>(a, parity, variant, gz, gy, st); break;
        case ST_F16: launch_s<ST_F16>(a, parity, variant, gz, gy, st); break;
        default: launch_s<ST_BF16>(a, parity, variant, gz, gy, st); break;
    }
}

}  // namespace lbsq
