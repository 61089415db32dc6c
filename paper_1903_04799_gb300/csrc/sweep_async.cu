// sweep_async.cu -- the fused stream + collide sweep of the 16-bit storages
// (Sec. III, Eq. "lb") with its loads staged through shared memory by
// asynchronous copies (cp.async, 16 bytes a copy).
//
// Persistent CTAs, two per SM, walk items of R whole rows of one plane (R * nx
// = 512 cells, two per thread).  Every thread issues its share of an item's
// 16-byte copies, global -> shared memory, and commits them as one group; the
// copies of the next kIn - 1 items stay in flight while the threads collide
// the current one out of shared memory.  The bytes in flight then no longer
// depend on registers, which bound every register-fed 16-bit form, and the
// odd step's x-shifts (with the periodic wrap) are done in shared memory:
// even steps store the collided pairs straight to global memory; odd steps
// assemble the x-shifted rows in shared memory and store them in aligned
// 16-byte chunks.  All global accesses are evict-first in L2, as the other
// sweeps' (ld_stream / st_stream).
//
// A bulk-copy (cp.async.bulk) form of this kernel, one 1 KB copy per
// direction and item from a single warp, measured 0.44 of the copy bandwidth:
// the copies queue on the SM's copy engine.  Per-thread 16-byte copies go
// through the load path instead.
//
// In-place AA pattern (see lbsq_internal.cuh): on even steps the cells of row
// (y, z) read and write the 19 rows of their own (y, z); on odd steps they read
// row (y - c_y, z - c_z) of direction opp(i), x-shifted by -c_x, and write row
// (y + c_y, z + c_z) of direction i, x-shifted by +c_x.  Each of those whole
// rows (periodic in x) belongs to the cells of row (y, z) alone, so items never
// share a row, and the near-body window, which spans whole x-rows, splits the
// sweep row by row.  nx % 8 == 0 keeps every 16-byte chunk aligned.
#include "sweep_body.cuh"

namespace lbsq {

namespace {

constexpr int kTT = 256;         // threads per CTA, two CTAs per SM
constexpr int kItemCells = 512;  // R * nx cells per item, two per thread
constexpr int kIn = 4;           // input buffers: copies run kIn - 1 items ahead

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 16 bytes global -> shared memory, asynchronous, cached in L2 only
__device__ __forceinline__ void copy16(void* dst, const void* src, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// this thread's copies of all but the newest kIn - 1 groups have landed
__device__ __forceinline__ void copy_wait_older() { asm volatile("cp.async.wait_group %0;" ::"n"(kIn - 1) : "memory"); }

__device__ __forceinline__ void copy_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrapn(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Item k: grid rows b*R .. b*R + R - 1 of plane slot p.
struct Item {
    int z;  // plane, or -1
    int b;  // row block
};

__device__ __forceinline__ Item item_of(const SweepArgs& a, long long k, int nyb) {
    Item it;
    const int p = (int)(k / nyb);
    it.b = (int)(k - (long long)p * nyb);
    it.z = sweep_plane_at(a, p);
    return it;
}

// Row y of row r of an item, or -1 (outside the lattice, the part of the
// near-body window this sweep leaves out, or no plane).
__device__ __forceinline__ int item_row(const SweepArgs& a, const Item& it, int R, int r) {
    return it.z < 0 ? -1 : sweep_row(a, it.b * R + r, it.z);
}

// Global row of direction array d at plane z, row y.
__device__ __forceinline__ unsigned short* grow(unsigned short* F, const SweepArgs& a, int d, int y, int z) {
    return F + (int64_t)d * a.Np + ((int64_t)z * a.ny + y) * a.nx;
}

// All threads: this thread's 16-byte copies of item `it` into input buffer
// `in` (rows [i][r]), committed as one group (empty if it has none).
template <int P>
__device__ __forceinline__ void issue_item(const SweepArgs& a, const Item& it, int R, unsigned short* in,
                                           uint64_t pol) {
    unsigned short* F = (unsigned short*)a.F;
    const int cpr = a.nx / 8;  // chunks per row
    const int per_dir = R * cpr;
    for (int c = threadIdx.x; c < Q * per_dir; c += kTT) {
        const int i = c / per_dir, rem = c - i * per_dir;
        const int r = rem / cpr, q = rem - r * cpr;
        const int y = item_row(a, it, R, r);
        if (y < 0) continue;
        const unsigned short* src = P == 0 ? grow(F, a, i, y, it.z)
                                           : grow(F, a, opp(i), wrapn(y - cy(i), a.ny), wrapn(it.z - cz(i), a.nz));
        copy16(in + (int64_t)(i * R + r) * a.nx + 8 * q, src + 8 * q, pol);
    }
    copy_commit();
}

// Two cells x0, x0 + 1 of row r (lattice row y, plane z): input rows
// in[i][r].  Even steps store the pairs to global memory; odd steps write the
// x-shifted results to the output rows out[i][r].
template <int S, int P>
__device__ __forceinline__ void collide_two(const SweepArgs& a, int R, int r, int x0, int y, int z,
                                            const unsigned short* in, unsigned short* out) {
    const int nx = a.nx;
    const float rho0 = (float)a.rho0 * a.scale;  // scaled units (see kScaled)
    unsigned int g[Q];  // the pair, packed e0 | e1 << 16
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short* row = in + (i * R + r) * nx;
        if (P == 0 || cx(i) == 0) {
            g[i] = *reinterpret_cast<const unsigned int*>(row + x0);
        } else {
            // sources x0 - 1, x0 (c_x = +1) or x0 + 1, x0 + 2 (c_x = -1)
            const int s0 = x0 - cx(i);
            g[i] = (unsigned int)row[wrapn(s0, nx)] | ((unsigned int)row[wrapn(s0 + 1, nx)] << 16);
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float gc[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) gc[i] = dec16<S>(c ? (g[i] >> 16) : (g[i] & 0xffffu), 1.0f);
        collide_trt<float, true>(gc, a.K, rho0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned int e = enc16<S>(gc[i], 1.0f);
            g[i] = c ? ((g[i] & 0xffffu) | (e << 16)) : ((g[i] & 0xffff0000u) | e);
        }
    }
    unsigned short* F = (unsigned short*)a.F;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (P == 0) {
            st_stream(reinterpret_cast<unsigned int*>(grow(F, a, opp(i), y, z) + x0), g[i]);
        } else if (cx(i) == 0) {
            *reinterpret_cast<unsigned int*>(out + (i * R + r) * nx + x0) = g[i];
        } else {
            // targets x0 + 1, x0 + 2 (c_x = +1) or x0 - 1, x0 (c_x = -1)
            unsigned short* row = out + (i * R + r) * nx;
            const int t0 = x0 + cx(i);
            row[wrapn(t0, nx)] = (unsigned short)(g[i] & 0xffffu);
            row[wrapn(t0 + 1, nx)] = (unsigned short)(g[i] >> 16);
        }
    }
}

// Odd steps, all threads: the output rows of item `it` to global memory in
// aligned 16-byte chunks, row out[d][r] to row (y + c_y, z + c_z) of array d.
__device__ __forceinline__ void store_item(const SweepArgs& a, const Item& it, int R, const unsigned short* out) {
    unsigned short* F = (unsigned short*)a.F;
    const int cpr = a.nx / 8;
    const int per_dir = R * cpr;
    for (int c = threadIdx.x; c < Q * per_dir; c += kTT) {
        const int d = c / per_dir, rem = c - d * per_dir;
        const int r = rem / cpr, q = rem - r * cpr;
        const int y = item_row(a, it, R, r);
        if (y < 0) continue;
        unsigned short* dst = grow(F, a, d, wrapn(y + cy(d), a.ny), wrapn(it.z + cz(d), a.nz)) + 8 * q;
        st_stream(reinterpret_cast<uint4*>(dst), *reinterpret_cast<const uint4*>(out + (int64_t)(d * R + r) * a.nx + 8 * q));
    }
}

// R rows per item, nyb row blocks per plane slot, gz plane slots.
template <int S, int P>
__global__ void __launch_bounds__(kTT, 2) k_sweep_async(const SweepArgs a, int R, int nyb, int gz) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int nx = a.nx;
    const int64_t buf = (int64_t)Q * R * nx;  // elements of one buffer
    unsigned short* in0 = reinterpret_cast<unsigned short*>(smem);
    unsigned short* out = in0 + kIn * buf;  // odd steps only
    const long long nitems = (long long)gz * nyb;
    const uint64_t pol = evict_first_policy();
    // the copies of this CTA's first kIn - 1 items
    for (int s = 0; s < kIn - 1; ++s) {
        const long long k = blockIdx.x + (long long)s * gridDim.x;
        if (k < nitems) issue_item<P>(a, item_of(a, k, nyb), R, in0 + s * buf, pol);
        else copy_commit();
    }
    const int tpr = nx / 2;  // threads per row, two cells each
    const int r = threadIdx.x / tpr, x0 = 2 * (threadIdx.x - r * tpr);
    const bool mine = r < R;
    int j = 0;
    for (long long k = blockIdx.x; k < nitems; k += gridDim.x, ++j) {
        // the copies of item j + kIn - 1, into the buffer item j - 1 used
        const long long kn = k + (long long)(kIn - 1) * gridDim.x;
        if (kn < nitems) issue_item<P>(a, item_of(a, kn, nyb), R, in0 + ((j + kIn - 1) % kIn) * buf, pol);
        else copy_commit();
        copy_wait_older();
        __syncthreads();  // every thread's copies of item j have landed
        const Item it = item_of(a, k, nyb);
        const unsigned short* in = in0 + (j % kIn) * buf;
        const int y = mine ? item_row(a, it, R, r) : -1;
        if (y >= 0) collide_two<S, P>(a, R, r, x0, y, it.z, in, out);
        if (P == 1) {
            __syncthreads();  // the output rows are complete
            store_item(a, it, R, out);
        }
        __syncthreads();  // the input (and output) buffers are free again
    }
    copy_wait_all();
}

}  // namespace

// Whether the staged sweep applies: 16-bit storage, nx % 8 == 0 (16-byte
// chunks), nx <= kItemCells (one row per item at least), a 16-byte aligned
// array.
bool sweep_async_supported(const SweepArgs& a, int storage_bytes) {
    return storage_bytes == 2 && a.nx % 8 == 0 && a.nx <= kItemCells && (reinterpret_cast<uintptr_t>(a.F) & 15u) == 0;
}

template <int S>
static void launch_async(const SweepArgs& a, int parity, int gz, int gy, cudaStream_t st) {
    const int R = kItemCells / a.nx;  // rows per item
    const int nyb = (gy + R - 1) / R;
    const size_t smem = (size_t)(kIn + 1) * Q * R * a.nx * sizeof(unsigned short);
    // a persistent grid: as many CTAs as are resident at once (shared memory
    // carved out in full, so that two fit per SM)
    static int n_sm = 0;
    static int resident[2] = {0, 0};
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    if (!resident[parity]) {  // sized for the largest item (R * nx = kItemCells)
        const int most = (kIn + 1) * Q * kItemCells * (int)sizeof(unsigned short);
        const void* fn = parity == 0 ? (const void*)k_sweep_async<S, 0> : (const void*)k_sweep_async<S, 1>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTT, most) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        resident[parity] = per_sm;
    }
    const long long nitems = (long long)gz * nyb;
    const long long slots = (long long)n_sm * resident[parity];
    const int grid = (int)(nitems < slots ? nitems : slots);
    if (grid <= 0) return;
    if (parity == 0) k_sweep_async<S, 0><<<grid, kTT, smem, st>>>(a, R, nyb, gz);
    else k_sweep_async<S, 1><<<grid, kTT, smem, st>>>(a, R, nyb, gz);
}

void launch_sweep_async(const SweepArgs& a, int storage, int parity, int gz, int gy, cudaStream_t st) {
    if (storage == ST_F16) launch_async<ST_F16>(a, parity, gz, gy, st);
    else launch_async<ST_BF16>(a, parity, gz, gy, st);
}

}  // namespace lbsq
