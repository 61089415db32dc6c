// static_scratch.cu -- lb_fluid_totals_static: the fluid mass and momentum sum
// of a population field, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a host framework
// owns every byte of device memory through its own pool, code inside a
// latency-critical loop where an allocation would synchronise the device, or
// a monitoring hook that must not change the memory footprint of the program
// it observes.  They cannot create an lb_ctx either (lb_create allocates), so
// this entry point works on caller-owned device buffers and keeps its one
// piece of scratch -- the per-block partial sums -- in a fixed-size
// file-scope device array instead of allocated memory.
//
// The array lives in every GPU that loads the library, until the process
// exits.  In host code its name is only a host-side stand-in: the device
// address is obtained once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.  Under CUDA's lazy module
// loading (the default) that first lookup also loads this file's device code
// and array onto the device, which itself takes device memory and may
// synchronise: a caller that must never allocate makes its first call on each
// device during set-up, before its own pool takes the memory and before any
// stream capture.  Every call shares the array, so
// calls that overlap on the GPU (two streams at once) race; calls on one
// stream are ordered and safe.  Each call writes every partial it reads, so
// nothing needs clearing between calls.
#include <mutex>

#include "../../include/lbsq.h"
#include "lbsq_internal.cuh"

namespace lbsq {

namespace {

constexpr int kStaticBlocks = LB_STATIC_PARTIALS;  // partial sums per call
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

// Partial sums (mass, jx, jy, jz) of each block of one call.
static __device__ __align__(256) double g_totals_scratch[kStaticBlocks * 4];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Block b sums cells b*T + t, b*T + t + G*T, ... (a fixed assignment) and
// writes its partial.  Up to 1024 x 256 cells each thread holds one cell, as
// in the library's own mass sum; larger fields grid-stride over 1024 blocks,
// so the order of the additions (and the last bits) then differ from it.
__global__ void __launch_bounds__(kStaticThreads) k_totals_static_partial(const double* __restrict__ f,
                                                                          const int32_t* __restrict__ owner,
                                                                          int64_t N, double* scratch) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        if (owner && owner[n] != 0) continue;
        for (int i = 0; i < Q; ++i) {
            const double fi = f[(int64_t)i * N + n];
            v[0] += fi;
            v[1] += fi * cx(i);
            v[2] += fi * cy(i);
            v[3] += fi * cz(i);
        }
    }
    __shared__ double sm[kStaticThreads / 32][4];
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kStaticThreads / 32; ++w)
            for (int k = 0; k < 4; ++k) t[k] += sm[w][k];
        for (int k = 0; k < 4; ++k) scratch[(size_t)blockIdx.x * 4 + k] = t[k];
    }
}

// One block: thread j sums partials j, j + T, ...; thread 0 then sums the
// threads in order.
__global__ void __launch_bounds__(kStaticThreads) k_totals_static_final(const double* scratch, int nblocks,
                                                                        double* out) {
    __shared__ double sm[kStaticThreads][4];
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; ++k) t[k] += scratch[(size_t)b * 4 + k];
    for (int k = 0; k < 4; ++k) sm[threadIdx.x][k] = t[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < (int)blockDim.x; ++j)
            for (int k = 0; k < 4; ++k) s[k] += sm[j][k];
        for (int k = 0; k < 4; ++k) out[k] = s[k];
    }
}

// Device address of the scratch array on the current device, looked up once
// per device.
cudaError_t scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_totals_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = (double*)p;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace lbsq

extern "C" lb_status lb_fluid_totals_static(const double* f, const int32_t* owner, int64_t n_cells, double* out,
                                            void* stream) {
    using namespace lbsq;
    if (!f || !out || n_cells < 1 || n_cells > LB_STATIC_MAX_CELLS) return LB_ERR_INVALID;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return LB_ERR_CUDA;
    double* scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return LB_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // An error the calling thread already holds (from earlier, unrelated work)
    // is left for its owner to read, and nothing is launched; after the two
    // launches below, the thread's error state holds only theirs.
    if (cudaPeekAtLastError() != cudaSuccess) return LB_ERR_CUDA;
    const int64_t want = (n_cells + kStaticThreads - 1) / kStaticThreads;
    const int nblocks = (int)(want < kStaticBlocks ? want : kStaticBlocks);
    k_totals_static_partial<<<nblocks, kStaticThreads, 0, st>>>(f, owner, n_cells, scratch);
    k_totals_static_final<<<1, kStaticThreads, 0, st>>>(scratch, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
