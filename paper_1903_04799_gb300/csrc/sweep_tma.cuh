// sweep_tma.cuh -- the 16-bit storages' sweep in tiles of whole rows staged
// through shared memory by bulk asynchronous copies (the tensor memory
// accelerator's cp.async.bulk), in a pipeline of ST stages.
//
// A tile is Y = min(16, C / nx) rows (y, z) of one plane (C = 2048 cells
// with two stages, 1024 with three; 64 <= nx <= 1024), all nx cells of each.
// The slots the tile's cells read and write are, for each direction i, whole
// rows of one plane: even steps (P = 0) plane i at the cell's own row, odd
// steps (P = 1) plane opp(i) at row (y - c_iy, z - c_iz), each cell's
// element shifted by -c_ix within the row.  Every slot belongs to one cell,
// so the rows are the tile's alone: they are copied in whole (16-byte
// aligned, nx % 8 == 0), each cell collides in place in shared memory -- the
// outgoing f_i goes to the slot it read f_ib from -- and the same rows are
// copied back.
// The x-shifts of the odd steps, periodic wrap included, are shared-memory
// indexing; global memory sees only whole aligned rows.
//
// A block is ST stages of one tile each, 256 consumer threads (four cells at
// a time, collide_four) and one producer warp.  The producer loads tile k + ST
// into a stage as soon as the stores of tile k, which used it, have read it
// out; consumers wait for a stage's loads on its `full` barrier and signal
// the producer on its `done` barrier.  Blocks take tiles in sweep order,
// strided by the grid (one persistent block per SM).
//
// Measured on GB300 (FP16, 256^3, both parities): 0.56 of the copy
// bandwidth with two stages (4 KB copies), 0.41 with three (2 KB copies),
// against 0.78 for the default forms; the bitwise results agree with them.
// One block of 288 threads fits an SM (167 registers a thread), and its eight
// consumer warps, issuing some 160 million warp instructions a sweep, cannot
// keep the copies coming; smaller copies cost more per byte.  Kept as
// sweep variants 4 and 5, not the default.
//
// Every wait polls at most kTmaSpin times; a wait that runs out sets the
// lattice's error word to LB_ERR_TIMEOUT (6) and the block's abort flag, the
// other waits then end at their next poll, and the producer waits (again
// bounded) for the copies it issued before the block exits.
#pragma once

#include "sweep_body.cuh"

namespace lbsq {

constexpr int kTmaConsumers = 256;                 // four cells at a time each
constexpr int kTmaThreads = kTmaConsumers + 32;    // and one producer warp
// cells per tile at ST stages: 2048 (two stages), 1024 (three), so that the
// stages fit the 227 KB of shared memory a block may have
constexpr int tma_tile_cells(int ST) { return ST == 2 ? 2048 : 1024; }
constexpr int kTmaCells = 2048;                    // the largest
constexpr long long kTmaSpin = 1ll << 24;          // polls before a wait gives up
constexpr int kTmaHeader = 128;                    // barriers and flags, ahead of the stages
constexpr int kTmaMaxY = 16;                       // rows per tile at most

__device__ __forceinline__ uint32_t tma_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tma_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tma_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tma_smem(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma_smem(bar)) : "memory");
}
__device__ __forceinline__ bool tma_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tma_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared, completing `bytes` on the barrier
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tma_smem(dst)),
                 "l"(src), "r"(bytes), "r"(tma_smem(bar))
                 : "memory");
}
// shared -> global, in the issuing thread's current bulk group
__device__ __forceinline__ void tma_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(tma_smem(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread's bulk groups have read their sources / have completed
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory, ordered before later async-proxy reads
__device__ __forceinline__ void tma_fence_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for phase `parity` of a barrier; false if it ran out or the
// block aborted (*abort set by another waiter).
__device__ __forceinline__ bool tma_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
    for (long long n = 0; n < kTmaSpin; ++n) {
        if (tma_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort) return false;
    }
    atomicCAS(err, 0, 6);  // LB_ERR_TIMEOUT
    *abort = 1;
    return false;
}

// Rows of tile t: plane z, and for each of its Y rows the lattice row or -1
// (outside the selection, see sweep_row), into ys if not null.  Returns the
// number of rows swept; *mine (if not null) receives row r's entry.
__device__ __forceinline__ int tma_tile_rows(const SweepArgs& a, int t, int Y, int nty, int& z, int* ys, int r = -1,
                                             int* mine = nullptr) {
    const int bz = t / nty, ly0 = (t - bz * nty) * Y;
    z = sweep_plane_at(a, bz);
    int n = 0;
    for (int q = 0; q < Y; ++q) {
        const int y = z < 0 ? -1 : sweep_row(a, ly0 + q, z);
        if (ys) ys[q] = y;
        if (q == r) *mine = y;
        n += y >= 0;
    }
    return n;
}

// Element offset in F of row (y, z) of plane `plane` for direction i's
// buffer: P = 0 plane i at (y, z), P = 1 plane opp(i) at (y - c_iy, z - c_iz).
template <int P>
__device__ __forceinline__ int64_t tma_row(const SweepArgs& a, int i, int y, int z) {
    if (P == 0) return (int64_t)i * a.Np + (int64_t)a.nx * (y + (int64_t)a.ny * z);
    int ys = y - cy(i), zs = z - cz(i);
    ys = ys < 0 ? ys + a.ny : (ys >= a.ny ? ys - a.ny : ys);
    zs = zs < 0 ? zs + a.nz : (zs >= a.nz ? zs - a.nz : zs);
    return (int64_t)opp(i) * a.Np + (int64_t)a.nx * (ys + (int64_t)a.ny * zs);
}

// The producer warp's copies of one tile, one lane per direction: load
// (into `buf`, on barrier `bar`) or store (from `buf`).  A direction's rows
// are consecutive in memory unless the selection leaves one out or the
// source rows wrap around y; each run of consecutive rows is one copy.
template <int P, bool LOAD>
__device__ __forceinline__ void tma_tile_copies(const SweepArgs& a, unsigned short* buf, int Y, int z, const int* ys,
                                                uint64_t* bar) {
    unsigned short* F = (unsigned short*)a.F;
    const int i = threadIdx.x & 31;
    if (i >= Q) return;
    const int nx = a.nx;
    int r0 = 0;
    while (r0 < Y) {
        if (ys[r0] < 0) {
            ++r0;
            continue;
        }
        const int64_t first = tma_row<P>(a, i, ys[r0], z);
        int len = 1;
        while (r0 + len < Y && ys[r0 + len] >= 0 && tma_row<P>(a, i, ys[r0 + len], z) == first + (int64_t)len * nx)
            ++len;
        unsigned short* sb = buf + (int64_t)(i * Y + r0) * nx;
        const uint32_t bytes = (uint32_t)len * (uint32_t)nx * 2u;
        if (LOAD) tma_load(sb, F + first, bytes, bar);
        else tma_store(F + first, sb, bytes);
        r0 += len;
    }
}

// The four cells x0 .. x0 + 3 of row r of a tile, in place in the stage's
// buffers (direction i's rows at buf + (i Y + r') nx).
template <int S, int P>
__device__ __forceinline__ void tma_four_cells(const SweepArgs& a, unsigned short* buf, int Y, int r, int x0, int y,
                                               int z, uint32_t skey) {
    const int nx = a.nx;
    auto at = [&](int x) -> int { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    auto rowp = [&](int i) -> unsigned short* { return buf + (int64_t)(i * Y + r) * nx; };
    uint2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short* b = rowp(i);
        const unsigned long long v = *reinterpret_cast<const unsigned long long*>(b + x0);
        unsigned long long w = v;
        if (P == 1 && cx(i) == 1) {  // sources x0 - 1 .. x0 + 2
            w = (v << 16) | (unsigned long long)b[at(x0 - 1)];
        } else if (P == 1 && cx(i) == -1) {  // sources x0 + 1 .. x0 + 4
            w = (v >> 16) | ((unsigned long long)b[at(x0 + 4)] << 48);
        }
        g[i] = make_uint2((unsigned int)w, (unsigned int)(w >> 32));
    }
    collide_four<S>(g, a, skey, x0, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // the outgoing f_i goes where f_ib was read: direction ib's buffer,
        // element x (even steps) or x + c_ix (odd steps)
        unsigned short* b = rowp(opp(i));
        const uint2 o = g[i];
        if (P == 0 || cx(i) == 0) {
            *reinterpret_cast<uint2*>(b + x0) = o;
        } else {
            // targets t0 .. t0 + 3: the outer two alone (their neighbours
            // belong to other threads' cells), the inner two as one aligned word
            const int t0 = cx(i) == 1 ? x0 + 1 : x0 - 1;
            b[at(t0)] = (unsigned short)(o.x & 0xffffu);
            *reinterpret_cast<unsigned int*>(b + t0 + 1) = (o.x >> 16) | (o.y << 16);
            b[at(t0 + 3)] = (unsigned short)(o.y >> 16);
        }
    }
}

template <int S, int P, int ST>
__global__ void __launch_bounds__(kTmaThreads, 1) k_sweep_tma(const SweepArgs a, int Y, int nty, int ntiles) {
    extern __shared__ __align__(128) unsigned char tma_smem_raw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(tma_smem_raw);
    uint64_t* done = full + ST;
    volatile int* abort = reinterpret_cast<volatile int*>(done + ST);
    int* ring = const_cast<int*>(abort) + 1;  // [ST] tile of each stage (producer)
    int* rows = ring + ST;                    // [kTmaMaxY] rows of the tile being copied (producer)
    unsigned short* stage0 = reinterpret_cast<unsigned short*>(tma_smem_raw + kTmaHeader);
    const int64_t stage_elems = (int64_t)Q * Y * a.nx;
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // every thread (see sr_step)
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            tma_bar_init(full + s, 1);
            tma_bar_init(done + s, kTmaConsumers);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int z = 0;
    if (threadIdx.x >= kTmaConsumers) {
        // ---- producer warp
        const int lane = threadIdx.x & 31;
        // copies of tile t (rows into `rows`, by lane 0) from or into stage s
        auto copies = [&](int t, int s, bool load) -> int {
            int zt = 0, n = 0;
            if (lane == 0) n = tma_tile_rows(a, t, Y, nty, zt, rows);
            n = __shfl_sync(0xffffffffu, n, 0);
            zt = __shfl_sync(0xffffffffu, zt, 0);
            __syncwarp();
            if (n == 0) return 0;
            if (load) {
                if (lane == 0) tma_arrive_expect(full + s, (uint32_t)(n * Q) * (uint32_t)a.nx * 2u);
                __syncwarp();
                tma_tile_copies<P, true>(a, stage0 + s * stage_elems, Y, zt, rows, full + s);
            } else {
                tma_tile_copies<P, false>(a, stage0 + s * stage_elems, Y, zt, rows, nullptr);
                tma_commit();
            }
            __syncwarp();
            return n;
        };
        int k = 0;  // tiles loaded
        for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
            if (tma_tile_rows(a, t, Y, nty, z, nullptr) == 0) continue;
            const int s = k % ST;
            if (k >= ST) {  // stage s holds tile k - ST: store it once the consumers are done with it
                if (!tma_wait(done + s, (uint32_t)(((k - ST) / ST) & 1), abort, a.err)) break;
                copies(ring[s], s, false);
                tma_wait_read();
                __syncwarp();
            }
            copies(t, s, true);
            if (lane == 0) ring[s] = t;
            __syncwarp();
            ++k;
        }
        // the last stages' stores (or, after an abort, the loads still in flight)
        for (int j = k > ST ? k - ST : 0; j < k; ++j) {
            const int s = j % ST;
            const uint32_t ph = (uint32_t)((j / ST) & 1);
            if (!*abort && tma_wait(done + s, ph, abort, a.err)) {
                copies(ring[s], s, false);
            } else if (lane == 0) {
                tma_wait(full + s, ph, abort, a.err);
            }
        }
        tma_wait_all();
        return;
    }
    // ---- consumers: groups of four cells, group q = row q / (nx / 4)
    const int per_row = a.nx / 4, groups = Y * per_row;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tma_tile_rows(a, t, Y, nty, z, nullptr) == 0) continue;
        const int s = k % ST;
        if (!tma_wait(full + s, (uint32_t)((k / ST) & 1), abort, a.err)) break;
        const int ly0 = (t % nty) * Y;
        for (int q = threadIdx.x; q < groups; q += kTmaConsumers) {
            const int r = q / per_row, x0 = 4 * (q - r * per_row);
            const int y = sweep_row(a, ly0 + r, z);
            if (y >= 0) tma_four_cells<S, P>(a, stage0 + s * stage_elems, Y, r, x0, y, z, skey);
        }
        tma_fence_shared();
        tma_arrive(done + s);
        ++k;
    }
}

}  // namespace lbsq
