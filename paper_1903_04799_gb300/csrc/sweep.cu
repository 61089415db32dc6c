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

template <int S, int P, bool NATIVE>
__global__ void __launch_bounds__(256) k_sweep(const SweepArgs a) {
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // before any exit (see sr_step)
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y, z);
    if (x >= a.nx || y < 0) return;
    sweep_one<S, P, NATIVE>(a, x, y, z, skey);
}

// FP64 storage, double-float collision (sweep_df.cuh), one cell per thread,
// three blocks per SM (80 registers, 40 bytes of spill): 24 warps per SM hide
// the loads better than 16 at 122 registers (256^3: 0.77 -> 0.83 of the copy
// bandwidth).
template <int P, bool O32, bool LE1>
__global__ void __launch_bounds__(256, 3) k_sweep_df(const SweepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y, z);
    if (x >= a.nx || y < 0) return;
    sweep_one_df<P, O32, LE1>(a, x, y, z);
}

template <bool O32, bool LE1>
static void launch_df(const SweepArgs& a, int parity, const dim3& grid, int bx, cudaStream_t st) {
    if (parity == 0) k_sweep_df<0, O32, LE1><<<grid, bx, 0, st>>>(a);
    else k_sweep_df<1, O32, LE1><<<grid, bx, 0, st>>>(a);
}

template <int S, int P, bool O32>
__global__ void __launch_bounds__(256, 2) k_sweep2(const SweepArgs a) {
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // before any exit (see sr_step)
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    if (x0 >= a.nx || y < 0) return;
    sweep_two<S, P, O32>(a, x0, y, z, skey);
}

// 16-bit storages with nx % 4 == 0, nx <= 768: blocks of whole rows, four
// cells per thread (see sweep_four_rows); dynamic shared memory of
// 10 x rows x nx elements on odd steps.
template <int S, int P, bool O32>
__global__ void __launch_bounds__(P == 0 ? 256 : 192, 2) k_sweep4r(const SweepArgs a) {
    extern __shared__ unsigned short rowbuf[];
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // before any exit (see sr_step)
    const int z = sweep_plane(a);
    if (z < 0) return;  // the whole block
    const int y = sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    sweep_four_rows<S, P, O32>(a, y < 0 ? 0 : y, z, y >= 0, rowbuf, skey);
}

// 16-bit storages with nx % 4 == 0, odd steps of split sweeps: four cells per
// thread without shared memory (see sweep_four_odd), blocks of at most 192
// threads (167 registers, no spill; at 256 threads the 128-register cap
// spills 72-80 bytes and measured 3-4 % slower).
template <int S, bool O32>
__global__ void __launch_bounds__(192, 2) k_sweep4o(const SweepArgs a) {
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // before any exit (see sr_step)
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int z = sweep_plane(a);
    const int y = z < 0 ? -1 : sweep_row(a, blockIdx.y * blockDim.y + threadIdx.y, z);
    if (x0 >= a.nx || y < 0) return;
    sweep_four_odd<S, O32>(a, x0, y, z, skey);
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

// Planes ahead for the L2 prefetch of the sources (SweepArgs::pf): just past
// the planes that the resident blocks (two per SM for FP32, three for FP64)
// cover; FP32 adds two more.
// Measured on GB300, whole-lattice sweeps:
//   FP32 (two-cell form, 256^3): 0.959 -> 0.990 of the copy bandwidth;
//   FP64 (double-float form): 256^3 0.65 -> 0.75 at 1 or 2 planes ahead,
//     0.66 at 4, 0.60 at 5; 192^3 0.56 -> 0.72; 128^3 0.64 -> 0.78;
//   16-bit sweeps: see prefetch_ahead16.
// FP32 prefetches in whole-lattice sweeps only: a prefetch installs its lines
// in L2 at normal priority, and beside the body kernels of a split step (far
// sweeps) that evicted their code again (128^3 step 0.050 -> 0.056 ms).  The
// FP64 sweep is long against its body step, and prefetches in split sweeps
// too (256^3 pusher, whole step: 13 970 -> 15 830 MLUPS).
static int prefetch_ahead(const SweepArgs& a, int storage, const dim3& grid) {
    if (storage == ST_F32 ? a.zmode != 0 : storage != ST_F64) return 0;
    const long long per_plane = (long long)grid.x * grid.y;
    const long long resident = (storage == ST_F32 ? 2LL : 3LL) * sm_count();
    const int ahead = (int)((resident + per_plane - 1) / per_plane) + (storage == ST_F32 ? 2 : 0);
    return ahead < a.nz ? ahead : 0;
}

// Planes ahead for the L2 prefetch of the 16-bit sweeps (sweep_four_rows on
// even steps, sweep_two on odd steps): `extra` past the planes the resident
// blocks (two per SM) cover.  Measured on GB300 at 256^3 over both parities,
// against no prefetch: FP16 0.765 -> 0.807 with the even steps' (2 past; 0 or
// 4: the same within 0.3 %), -> 0.840 with the odd steps' too (0 past; 2 or
// 4: within 0.4 %); BF16 0.679 -> 0.703 -> 0.710.  Split sweeps prefetch
// too: the 256^3 pusher's whole step, FP16 0.2516 -> 0.2468 ms, BF16 0.2841 ->
// 0.2850 ms.  (An earlier measurement of the two-cell form prefetching on both
// parities, 0.745 -> 0.684, was taken before the sweeps' traffic was marked
// evict-first.)
static int prefetch_ahead16(const SweepArgs& a, const dim3& grid, int extra) {
    const long long per_plane = (long long)grid.x * grid.y;
    const long long resident = 2LL * sm_count();
    const int ahead = (int)((resident + per_plane - 1) / per_plane) + extra;
    return ahead < a.nz ? ahead : 0;
}

template <int S>
static void launch_s(const SweepArgs& a, int parity, int variant, int gz, int gy, cudaStream_t st) {
    const bool o32 = 19 * a.Np < (int64_t(1) << 32);  // element offsets fit 32 bits
    if constexpr (S == ST_F64) {
        int bx = ((a.nx + 31) / 32) * 32;
        if (bx > 256) bx = 256;
        dim3 grid((a.nx + bx - 1) / bx, gy, gz);
        SweepArgs b = a;
        b.pf = prefetch_ahead(a, S, grid);
        if (variant == 1) {  // FP64 arithmetic
            if (parity == 0) k_sweep<S, 0, true><<<grid, bx, 0, st>>>(a);
            else k_sweep<S, 1, true><<<grid, bx, 0, st>>>(a);
        } else if (o32) {
            if (a.K.df.le1) launch_df<true, true>(b, parity, grid, bx, st);
            else launch_df<true, false>(b, parity, grid, bx, st);
        } else {
            if (a.K.df.le1) launch_df<false, true>(b, parity, grid, bx, st);
            else launch_df<false, false>(b, parity, grid, bx, st);
        }
    } else {
    if constexpr (S == ST_F16 || S == ST_BF16) {
        // default: even steps in whole-row four-cell blocks (aligned 8-byte
        // chunks: 0.86 of the copy bandwidth at 256^3, against 0.74 for two
        // cells), odd steps in the two-cell form (0.63 before the L2
        // prefetch; the whole-row form's odd steps, with their x-shifts
        // through shared memory, measured 0.62), or in split sweeps as below
        const bool rows4 = a.nx % 4 == 0 && a.nx <= 768;
        // odd steps of split sweeps (far and near, mode 1 and 2): four cells per
        // thread.  Measured on GB300, 256^3 pusher, whole step against the
        // two-cell form: FP16 0.242 -> 0.232 ms, BF16 with stochastic rounding
        // 0.260 -> 0.252 ms (BF16 to nearest 0.243 -> 0.245).  In
        // whole-lattice sweeps the two-cell form stays ahead (bare 256^3 step:
        // FP16 0.210 against 0.214 ms, BF16 to nearest 0.211 against 0.223),
        // so they keep it; why the split steps favour four cells is not known.
        if (variant == 0 && parity == 1 && a.nx % 4 == 0 && a.zmode != 0) {
            const int quads = a.nx / 4;
            int bx = ((quads + 31) / 32) * 32;
            if (bx > 64) bx = 64;
            const int by = 192 / bx > 0 ? 192 / bx : 1;
            dim3 block(bx, by), grid((quads + bx - 1) / bx, (gy + by - 1) / by, gz);
            SweepArgs b = a;
            b.pf = prefetch_ahead16(a, grid, 0);
            if (o32) k_sweep4o<S, true><<<grid, block, 0, st>>>(b);
            else k_sweep4o<S, false><<<grid, block, 0, st>>>(b);
            return;
        }
        if ((variant == 3 || (variant == 0 && parity == 0)) && rows4) {
            // odd steps (more live values) in blocks of at most 192 threads
            const int tx = a.nx / 4, ty = (parity == 0 ? 256 : 192) / tx > 0 ? (parity == 0 ? 256 : 192) / tx : 1;
            dim3 block(tx, ty), grid(1, (gy + ty - 1) / ty, gz);
            if (parity == 0) {
                SweepArgs b = a;
                b.pf = prefetch_ahead16(a, grid, 2);
                if (o32) k_sweep4r<S, 0, true><<<grid, block, 0, st>>>(b);
                else k_sweep4r<S, 0, false><<<grid, block, 0, st>>>(b);
            } else {
                const size_t smem = (size_t)10 * ty * a.nx * sizeof(unsigned short);
                if (o32) k_sweep4r<S, 1, true><<<grid, block, smem, st>>>(a);
                else k_sweep4r<S, 1, false><<<grid, block, smem, st>>>(a);
            }
            return;
        }
    }
    if (variant != 1 && a.nx % 2 == 0) {
        const int pairs = a.nx / 2;
        int bx = ((pairs + 31) / 32) * 32;
        if (bx > 128) bx = 128;
        const int by = 256 / bx;
        dim3 block(bx, by), grid((pairs + bx - 1) / bx, (gy + by - 1) / by, gz);
        SweepArgs b = a;
        b.pf = prefetch_ahead(a, S, grid);
        if (S == ST_F16 || S == ST_BF16) b.pf = parity == 1 ? prefetch_ahead16(a, grid, 0) : 0;
        if (o32) {
            if (parity == 0) k_sweep2<S, 0, true><<<grid, block, 0, st>>>(b);
            else k_sweep2<S, 1, true><<<grid, block, 0, st>>>(b);
        } else {
            if (parity == 0) k_sweep2<S, 0, false><<<grid, block, 0, st>>>(b);
            else k_sweep2<S, 1, false><<<grid, block, 0, st>>>(b);
        }
        return;
    }
    int bx = ((a.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    dim3 grid((a.nx + bx - 1) / bx, gy, gz);
    if (parity == 0) k_sweep<S, 0, false><<<grid, bx, 0, st>>>(a);
    else k_sweep<S, 1, false><<<grid, bx, 0, st>>>(a);
    }
}

// variant: 0 = default (FP64: double-float collision, one cell per thread;
// FP32: two cells per thread (even nx); FP16 / BF16: even steps as 3, odd
// steps as 2, or four cells per thread without shared memory in split
// sweeps), 1 = one cell per thread (FP64: FP64 arithmetic), 2 = two
// cells per thread where possible (not FP64), 3 = FP16 / BF16: four cells per
// thread in blocks of whole rows on both parities, odd-step x-shifts through
// shared memory (nx % 4 == 0, nx <= 768; else as 2).
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
    a.sr_writer = zmode != 2;  // of a split step's two sweeps, the far one advances the step counter
    if (gz <= 0 || gy <= 0) return;
    switch (L.storage) {
        case ST_F64: launch_s<ST_F64>(a, parity, variant, gz, gy, st); break;
        case ST_F32: launch_s<ST_F32>(a, parity, variant, gz, gy, st); break;
        case ST_F16: launch_s<ST_F16>(a, parity, variant, gz, gy, st); break;
        default: launch_s<ST_BF16>(a, parity, variant, gz, gy, st); break;
    }
}

}  // namespace lbsq
