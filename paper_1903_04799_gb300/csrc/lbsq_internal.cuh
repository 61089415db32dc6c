// lbsq_internal.cuh -- device-side building blocks shared by the CUDA
// translation units of the library (never by the CPU oracle).
//
// Population layout: one array F of 19 planes, plane i holding population i
// of every cell, x-fastest (F[i * Np + n], n = x + nx*(y + ny*z), Np = the
// cell count padded to 64).  Streaming is the in-place AA pattern:
//   even step: cell n reads F[i][n] and writes its post-collision f_i to F[ib][n];
//   odd step:  cell n reads f_i from F[ib][n - c_i] and writes f_i to F[i][n + c_i];
// (ib = opposite of i).  Both touch the same 19 slots of a cell, so the update
// is race-free in place.  Before a step of parity Q, population i of cell n
// sits in its "read slot": Q = 0: F[i][n]; Q = 1: F[ib][n - c_i].
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbsq {

constexpr int Q = 19;

// D3Q19 velocities (Sec. III): rest, 6 faces, 12 edges; opposite pairs adjacent.
// Component c+1 of velocity i is packed in bits 2i..2i+1 of a 64-bit constant,
// so cx(i) folds to a literal for a compile-time i and costs a shift for a
// run-time one.  Velocities, in order:
//   (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1)
//   (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
//   (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
constexpr unsigned long long kCX = 0x1548889549ull;
constexpr unsigned long long kCY = 0x895609495ull;
constexpr unsigned long long kCZ = 0x20a0954955ull;
__host__ __device__ constexpr int cx(int i) { return (int)((kCX >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cy(int i) { return (int)((kCY >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int cz(int i) { return (int)((kCZ >> (2 * i)) & 3ull) - 1; }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
static_assert(cx(1) == 1 && cx(2) == -1 && cy(9) == -1 && cz(13) == -1 && cz(18) == 1 && cy(17) == 1,
              "packed D3Q19 table");
// weights 1/3 (rest), 1/18 (faces), 1/36 (edges)
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

enum Storage : int { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// Population traffic of the sweeps, marked evict-first in L2 (ld/st.global.cs).
// A sweep reads and writes every population once, and a lattice larger than
// L2 would otherwise evict everything else between two steps, the body
// kernels' code and tables included.  With the hint those stay resident, and
// a sweep still reuses the planes the previous sweep wrote last.
template <class U>
__device__ __forceinline__ U ld_stream(const U* p) {
    U v;
    if constexpr (sizeof(U) == 2) {
        const unsigned short r = __ldcs(reinterpret_cast<const unsigned short*>(p));
        memcpy(&v, &r, 2);
    } else if constexpr (sizeof(U) == 4) {
        const unsigned int r = __ldcs(reinterpret_cast<const unsigned int*>(p));
        memcpy(&v, &r, 4);
    } else if constexpr (sizeof(U) == 8) {
        const uint2 r = __ldcs(reinterpret_cast<const uint2*>(p));
        memcpy(&v, &r, 8);
    } else {
        static_assert(sizeof(U) == 16, "2, 4, 8 or 16 bytes");
        const uint4 r = __ldcs(reinterpret_cast<const uint4*>(p));
        memcpy(&v, &r, 16);
    }
    return v;
}
template <class U>
__device__ __forceinline__ void st_stream(U* p, const U& v) {
    if constexpr (sizeof(U) == 2) {
        unsigned short r;
        memcpy(&r, &v, 2);
        __stcs(reinterpret_cast<unsigned short*>(p), r);
    } else if constexpr (sizeof(U) == 4) {
        unsigned int r;
        memcpy(&r, &v, 4);
        __stcs(reinterpret_cast<unsigned int*>(p), r);
    } else if constexpr (sizeof(U) == 8) {
        uint2 r;
        memcpy(&r, &v, 8);
        __stcs(reinterpret_cast<uint2*>(p), r);
    } else {
        static_assert(sizeof(U) == 16, "2, 4, 8 or 16 bytes");
        uint4 r;
        memcpy(&r, &v, 16);
        __stcs(reinterpret_cast<uint4*>(p), r);
    }
}

// Storage traits: the stored type, the arithmetic type of the collision,
// whether the store holds a deviation from w_i rho0 (every storage does), and
// the sweeps' (streaming) element access.
template <int S> struct StoreT;
template <> struct StoreT<ST_F64> {
    using T = double;
    using R = double;
    static constexpr bool dev = true;
    __device__ static R load(const T* p, R) { return ld_stream(p); }
    __device__ static void store(T* p, R v, R) { st_stream(p, v); }
};
template <> struct StoreT<ST_F32> {
    using T = float;
    using R = float;
    static constexpr bool dev = true;
    __device__ static R load(const T* p, R) { return ld_stream(p); }
    __device__ static void store(T* p, R v, R) { st_stream(p, v); }
};
template <> struct StoreT<ST_F16> {
    using T = __half;
    using R = float;
    static constexpr bool dev = true;
    __device__ static R load(const T* p, R inv_scale) { return __half2float(ld_stream(p)) * inv_scale; }
    __device__ static void store(T* p, R v, R scale) { st_stream(p, __float2half_rn(v * scale)); }
};
template <> struct StoreT<ST_BF16> {
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool dev = true;
    __device__ static R load(const T* p, R inv_scale) { return __bfloat162float(ld_stream(p)) * inv_scale; }
    __device__ static void store(T* p, R v, R scale) { st_stream(p, __float2bfloat16_rn(v * scale)); }
};

inline int storage_bytes(int s) { return s == ST_F64 ? 8 : (s == ST_F32 ? 4 : 2); }

// One lattice as seen by kernels (an array of these lives in device memory;
// a context has one, a server one per resident request).
struct Lattice {
    void* F;          // populations, storage-typed
    int nx, ny, nz;
    int64_t N, Np;    // cells, padded plane stride
    int storage;
    double rho0;
    float scale, inv_scale;  // FP16 deviation scale (1 for other storages)
    int32_t* own;       // cell owners, 0 = fluid
    int32_t* own_prev;  // owners committed at the last re-classification
    int* err;           // device error word of this lattice
    double lambda_e, lambda_o;
    double wca_sigma, wca_eps;
    int body_begin, body_count;  // this lattice's bodies in the body table
    int active;                  // 0: not stepped (a free server slot, or being set up)
    int force_avg;               // 1: F_bb and T_bb averaged over this step and the last (Ladd)
    int inc;                     // 1: incompressible equilibrium, u = j / rho0 (lb_params.equilibrium)
    int pad;
    const long long* gstep;      // server: global step counter (null for a context)
    long long stop_step;         // server: the lattice is stepped while *gstep < stop_step
    long long start_step;        // server: the global step of the lattice's first step
    int sr;                      // 1: BF16 stores of the sweeps round stochastically (lb_rounding)
    int rho_local;               // 1: the bounce-back shift takes the fluid node's density, not rho0
    float link_at;               // where on a link v_b and the lever arm are taken: 0.5 (midpoint) or 1 (node)
    int pad2;
    // context: the lattice's step count for the stochastic rounding, kept on
    // the device by the sweeps themselves (ping-pong by parity: the sweep of
    // step t reads [t & 1] = t and writes [1 - (t & 1)] = t + 1); null for a server
    unsigned long long* sr_ctr;
    // partially saturated cells (psm.cuh): spheres couple through the solid
    // fraction eps of each cell instead of links (0: off)
    int psm;
    int pad3;
    float* eps;        // [N] solid fraction
    int32_t* psm_id;   // [N] covering sphere (body index + 1), 0 = none
};

// Whether a lattice takes part in the current step.
__device__ __forceinline__ bool lattice_active(const Lattice& L) {
    return L.active && (L.gstep == nullptr || *L.gstep < L.stop_step);
}

__device__ __forceinline__ int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ int64_t cell_index(const Lattice& L, int x, int y, int z) {
    return (int64_t)x + (int64_t)L.nx * ((int64_t)y + (int64_t)L.ny * (int64_t)z);
}

__device__ __forceinline__ void cell_coords(const Lattice& L, int64_t n, int& x, int& y, int& z) {
    // cell counts stay below 2^31 (enforced at creation), so 32-bit division suffices
    const unsigned m = (unsigned)n, r = m / (unsigned)L.nx;
    x = (int)(m - r * (unsigned)L.nx);
    y = (int)(r % (unsigned)L.ny);
    z = (int)(r / (unsigned)L.ny);
}

// Flat index (plane * Np + cell) of the read slot of population i of cell
// (x,y,z) before a step of parity q.
__device__ __forceinline__ int64_t read_slot(const Lattice& L, int i, int x, int y, int z, int q) {
    if (q == 0) return (int64_t)i * L.Np + cell_index(L, x, y, z);
    int xs = wrapi(x - cx(i), L.nx), ys = wrapi(y - cy(i), L.ny), zs = wrapi(z - cz(i), L.nz);
    return (int64_t)opp(i) * L.Np + cell_index(L, xs, ys, zs);
}

// Global load; CG = true reads through L2 only (data another block of the
// same launch may have written).
template <bool CG, class T>
__device__ __forceinline__ T ld(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Absolute value f_i from a stored slot, in FP64.
template <bool CG = false>
__device__ __forceinline__ double load_abs(const Lattice& L, int64_t slot, int i) {
    switch (L.storage) {
        case ST_F64: return wgt(i) * L.rho0 + ld<CG>((const double*)L.F + slot);
        case ST_F32: return wgt(i) * L.rho0 + (double)ld<CG>((const float*)L.F + slot);
        case ST_F16: return wgt(i) * L.rho0 + (double)(__half2float(ld<CG>((const __half*)L.F + slot)) * L.inv_scale);
        default:
            return wgt(i) * L.rho0 +
                   (double)(__bfloat162float(ld<CG>((const __nv_bfloat16*)L.F + slot)) * L.inv_scale);
    }
}

// Store an absolute value f_i into a slot (every storage keeps f_i - w_i rho0).
__device__ __forceinline__ void store_abs(const Lattice& L, int64_t slot, int i, double f) {
    switch (L.storage) {
        case ST_F64: ((double*)L.F)[slot] = f - wgt(i) * L.rho0; break;
        case ST_F32: ((float*)L.F)[slot] = (float)(f - wgt(i) * L.rho0); break;
        case ST_F16: ((__half*)L.F)[slot] = __float2half_rn((float)(f - wgt(i) * L.rho0) * L.scale); break;
        default: ((__nv_bfloat16*)L.F)[slot] = __float2bfloat16_rn((float)(f - wgt(i) * L.rho0) * L.scale); break;
    }
}

// Deviation g_i = f_i - w_i rho0 of a reduced-storage slot, in FP32 (no FP64
// arithmetic), and its store.  Not for FP64 storage.
template <bool CG = false>
__device__ __forceinline__ float load_dev(const Lattice& L, int64_t slot) {
    switch (L.storage) {
        case ST_F32: return ld<CG>((const float*)L.F + slot);
        case ST_F16: return __half2float(ld<CG>((const __half*)L.F + slot)) * L.inv_scale;
        default: return __bfloat162float(ld<CG>((const __nv_bfloat16*)L.F + slot)) * L.inv_scale;
    }
}
__device__ __forceinline__ void store_dev(const Lattice& L, int64_t slot, float g) {
    switch (L.storage) {
        case ST_F32: ((float*)L.F)[slot] = g; break;
        case ST_F16: ((__half*)L.F)[slot] = __float2half_rn(g * L.scale); break;
        default: ((__nv_bfloat16*)L.F)[slot] = __float2bfloat16_rn(g * L.scale); break;
    }
}

// Minimum image of a coordinate difference into (-n/2, n/2].
__device__ __forceinline__ double min_image(double d, int n) {
    double h = 0.5 * (double)n;
    if (d > h) d = __dadd_rn(d, -(double)n);
    else if (d <= -h) d = __dadd_rn(d, (double)n);
    return d;
}

// Inside test (dx*dx + dy*dy) + dz*dz < R*R, rounded step by step (no FMA).
__device__ __forceinline__ bool inside_sphere(double dx, double dy, double dz, double R) {
    double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s < __dmul_rn(R, R);
}

// ------------------------------------------------------------------ bodies

enum BodyKind : int { BODY_WALL = 0, BODY_SPHERE = 1 };

struct BodyParams {
    int kind, mobile;
    double R, B1, B2, mass, inertia;
    double wall_vel[3];
    int wall_axis, wall_index;  // plane walls; wall_axis -1: a round tube along z
    double tube[3];             // round tube: axis (x, y) and radius
    int64_t link_off;  // first slot of this body's link segment
    int64_t link_cap;  // capacity of the segment
    int box_w[3];      // scan box extent (spheres: W = ceil(2R)+6 per axis)
    int g_links;       // blocks of the link kernel for this body (fixed by the body alone)
    int g_box;         // blocks of the box kernels for this body
    int lat;           // index of the body's lattice
    int copy_only;     // a still body whose force nobody reads: bounce-back is a plain copy
    double inv_mass, inv_inertia;
    int64_t st_off;    // first entry of the sphere's shell stencil (see k_body_fused)
    int st_count;      // stencil entries; 0 for bodies the fused kernel does not handle
    int psm;           // a sphere coupled by partially saturated cells (no links, no conversion)
    int pad_psm;
    int64_t psm_off;   // its first entry in Bodies::psm_out (a multiple of the chunk size)
};

struct BodyState {  // ping-pong by step parity
    double pos[3], vel[3], omega[3], e[3];
};

struct BodyAcc {
    double Fbb[3], Tbb[3], Sbb[6];
    double Fc[3], Tc[3];              // conversion force booked for the next update
    double Fapp[3], Tapp[3];          // force/torque that entered the last update
    double r_class[3];                // centre at the last classification
    unsigned long long margin_bits;   // min | |x - r| - R | over the box at that time
    int box_lo[3];                    // scan box origin of the current classification
    double vsum[3], vesum;            // sums over the updates of v and of v.e (mobile spheres)
    long long nsum;                   // number of updates summed
    int reclass;                      // 1: re-classify the shell this step (set by the update);
                                      // 2: classify the whole box (a body being added)
    int rel_flag;                     // queued for relinking this step
    long long link_count;
    int counter_links, counter_conv, counter_rebuild;  // last-block counters (self-resetting)
    int pad;
};

// Body table and the work lists of a step.  An item (body, block) is one
// block's share of a body; per-step lists are appended on the device:
// the update appends the box items of bodies that must re-classify, the
// classification appends the items of every body whose links must be rebuilt.
std::vector<uint32_t> shell_stencil(double R);

struct Bodies {
    const Lattice* lats;
    const BodyParams* par;
    BodyState* state[2];
    BodyAcc* acc;
    uint32_t* links;       // code = cell * 32 + i
    double* part_links;    // [body][GL][12]
    double* part_conv;     // [body][GB][6]
    int* part_count;       // [body][GB]
    int GL, GB;            // strides of the partial arrays
    const int2* link_items;
    const int* n_link_items;
    int2* box_items;
    int* n_box;
    int box_cap;
    int2* rel_items;
    int* n_rel;
    int rel_cap;
    int* done;             // blocks of the rebuild kernel that finished (self-resetting)
    int* err;              // error word for list overflow (shared)
    int* win;              // near-body window (z0, z length, y0, y length) of lattice 0 this launch writes, or null
    long long* gstep;      // server: global step counter, advanced by the rebuild kernel (or null)
    // spheres advanced by k_body_fused (body, lattice), grouped by cluster
    // class: class c holds items [fused_first[c], fused_first[c] + n_fused[c])
    const int2* fused_items;
    const int* fused_first;  // [3]
    const int* n_fused;      // [3]
    const uint32_t* stencil; // shell stencils of those spheres
    int* fused_done;         // clusters of a solo fused launch that finished (self-resetting)
    // spheres coupled by partially saturated cells: items (body, block) of
    // their boxes, and per-block partial sums [body][GB][12]
    const int2* psm_items;
    int n_psm_items;
    double* part_psm;
    // the covered fluid cells of each chunk of kBB box cells, compacted in
    // cell order: post-collision populations [Q][psm_cap], the cell within
    // the chunk [psm_cap], the count per chunk [psm_cap / kBB]; sphere k's
    // chunk q starts at entry psm_off(k) + q kBB
    double* psm_out;
    int32_t* psm_cell;
    int32_t* psm_count;
    int64_t psm_cap;
};

// Cluster class of the fused body kernel for a lattice with nf fused spheres:
// 0 (16 blocks per sphere) up to 8 spheres, 1 (8 blocks) up to 64, else 2
// (4 blocks).  Fewer blocks per sphere when there are many spheres: the
// clusters then fill the GPU in fewer waves.  A function of the lattice
// alone, so a body's result does not depend on other lattices.
inline int fused_class(int nf) { return nf <= 8 ? 0 : (nf <= 64 ? 1 : 2); }

// Largest sphere radius with a shell stencil (stencil offsets fit 10 bits).
constexpr double kStencilMaxR = 400.0;

// Cells per chunk of a sphere's box under partially saturated cells (one
// block of the box kernels per chunk).
constexpr int kPsmChunk = 256;

// Whether the fused body kernel advances a body: moving-surface spheres with
// a stencil (still obstacles are plain copies, walls never re-classify).
inline bool fused_body(const BodyParams& b) {
    return b.kind == BODY_SPHERE && !b.copy_only && !b.psm && b.R <= kStencilMaxR;
}

// Scan box of a body: origin and extent.
__device__ __forceinline__ void body_box(const Lattice& L, const BodyParams& p, const BodyState& s, int lo[3],
                                         int w[3]) {
    if (p.kind == BODY_SPHERE) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)floor(s.pos[a] - p.R) - 2;
            w[a] = p.box_w[a];
        }
    } else {
        int n[3] = {L.nx, L.ny, L.nz};
        for (int a = 0; a < 3; ++a) {
            lo[a] = 0;
            w[a] = n[a];
        }
        // a plane wall's links come from the two layers next to it (a round
        // tube's from anywhere in the lattice)
        if (p.wall_axis >= 0) {
            lo[p.wall_axis] = p.wall_index - 1;
            w[p.wall_axis] = n[p.wall_axis] < 3 ? n[p.wall_axis] : 3;
        }
    }
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Whether node (x, y) lies in the solid of the round tube q (wall_axis -1):
// (x - cx)^2 + (y - cy)^2 >= r^2 in FP64, every operation rounded as written
// (no contraction), so that the oracle's evaluation gives the same answer.
__device__ __forceinline__ bool tube_solid(const BodyParams& q, int x, int y) {
    const double dx = __dsub_rn((double)x, q.tube[0]), dy = __dsub_rn((double)y, q.tube[1]);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) >= __dmul_rn(q.tube[2], q.tube[2]);
}

}  // namespace lbsq
