// serve.cu -- the request server of include/lbsq.h: many independent squirmer
// simulations resident on one GPU, advanced together.
//
// Memory: one arena of hbm_budget_bytes is allocated at creation and carved
// per request by a first-fit free list (populations, owner fields, boundary
// links).  Body tables, partial sums, work lists and the tile list live in
// fixed-capacity arrays, so every kernel of a step reads its work from device
// memory and one captured CUDA graph (a round of steps) serves any mix of
// resident requests.
//
// A step: k_sweep_tiles (persistent; each block walks the packed list of
// z-slab tiles of all active lattices, branching per tile on the lattice's
// storage), then the body kernels of bodies.cu over all bodies (work lists),
// the last of which advances the device step counter.  A request admitted at
// global step s0 with n steps is active while s0 <= step < s0 + n, so it stops
// inside a round at its own step; every round starts on an even step, which
// keeps all resident lattices on the same streaming parity.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbsq.h"
#include "sweep_body.cuh"

namespace lbsq {
void launch_body_kernel(int which, const Bodies& B, int parity, int grid_links, int grid_box, long long* step,
                        cudaStream_t st);
void launch_fill_rest(const Lattice& L, cudaStream_t st);
void launch_plane_claim(const Lattice& L, int32_t* own, int axis, int index, int id, cudaStream_t st);
void launch_set_flags(BodyAcc* acc, int nb, int k, int reclass, cudaStream_t st);

// ---------------------------------------------------------------- tile sweep

struct TileArgs {
    const Lattice* lats;
    const SweepArgs* sargs;  // per slot, built on the host at admission (collision constants included)
    const int4* tiles;  // (lattice, first unit, end unit, paired), sorted by storage
    const int* n_tiles; // [5]: tiles of storage S are [n_tiles[S], n_tiles[S+1])
};

// A tile is the unit range [tile.y, tile.z) of one lattice, a unit being a cell
// pair (paired tiles, nx even) or a cell, numbered x-fastest over the lattice.
// A request holds fewer than 2^27 cells (validate), so every population index
// of its lattice, below 19 x 2^27 < 2^32, fits the sweeps' 32-bit offsets.
template <int P, int S>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, const int4 tile) {
    const uint32_t skey = S == ST_BF16 ? sr_step_key(a) : 0u;  // the lattice's own step (global - start)
    const unsigned nx = (unsigned)a.nx, ny = (unsigned)a.ny;
    const unsigned per_row = tile.w ? nx / 2 : nx;
    for (unsigned u = (unsigned)tile.y + threadIdx.x; u < (unsigned)tile.z; u += blockDim.x) {
        const unsigned r = u / per_row;
        const int xi = (int)(u - r * per_row);
        const int y = (int)(r % ny), z = (int)(r / ny);
        if constexpr (S != ST_F64) {
            if (tile.w) {
                sweep_two<S, P, true>(a, 2 * xi, y, z, skey);
                continue;
            }
        }
        sweep_one<S, P, false, true>(a, xi, y, z, skey);
    }
}

// One kernel per storage, so that none pays for another's registers; the
// tile list is sorted by storage and n_tiles[S .. S+1] bounds storage S.
// The sweep arguments of the tile's lattice are staged in shared memory once
// per lattice: their collision constants would otherwise be rebuilt per tile,
// in FP64, which issues at GB300's narrow FP64 rate.  The next tile's
// descriptor and its lattice's activity are fetched before the current tile
// is swept, so that their dependent loads (tile, lattice, step counter) do not
// stall the block between tiles.
template <int P, int S>
__global__ void __launch_bounds__(256, S == ST_F64 ? 1 : 2) k_sweep_tiles(const TileArgs T) {
    __shared__ __align__(16) SweepArgs s_a;
    const int t0 = T.n_tiles[S], t1 = T.n_tiles[S + 1];
    int cur = -1;
    int t = t0 + blockIdx.x;
    int4 tile = make_int4(0, 0, 0, 0);
    bool act = false;
    if (t < t1) {
        tile = T.tiles[t];
        act = lattice_active(T.lats[tile.x]);
    }
    while (t < t1) {
        const int tn = t + gridDim.x;
        int4 next = make_int4(0, 0, 0, 0);
        bool nact = false;
        if (tn < t1) {
            next = T.tiles[tn];
            nact = lattice_active(T.lats[next.x]);
        }
        if (act) {  // the same for the whole block
            if (tile.x != cur) {
                __syncthreads();  // the previous lattice's readers are done
                static_assert(sizeof(SweepArgs) % 4 == 0, "word copy");
                for (int w = threadIdx.x; w < (int)(sizeof(SweepArgs) / 4); w += blockDim.x)
                    reinterpret_cast<int*>(&s_a)[w] = __ldg(reinterpret_cast<const int*>(T.sargs + tile.x) + w);
                __syncthreads();
                cur = tile.x;
            }
            if (s_a.F != nullptr) sweep_tile<P, S>(s_a, tile);  // a slot without arguments: nothing
        }
        t = tn;
        tile = next;
        act = nact;
    }
}

template <int P>
static void launch_tiles_p(const TileArgs& T, int grid, cudaStream_t st) {
    k_sweep_tiles<P, ST_F64><<<grid, 256, 0, st>>>(T);
    k_sweep_tiles<P, ST_F32><<<grid, 256, 0, st>>>(T);
    k_sweep_tiles<P, ST_F16><<<grid, 256, 0, st>>>(T);
    k_sweep_tiles<P, ST_BF16><<<grid, 256, 0, st>>>(T);
}

static void launch_tiles(const TileArgs& T, int parity, int grid, cudaStream_t st) {
    if (parity == 0) launch_tiles_p<0>(T, grid, st);
    else launch_tiles_p<1>(T, grid, st);
}

}  // namespace lbsq

using namespace lbsq;

namespace {

constexpr int kBodiesPerSlot = 5;  // squirmer + up to four walls (or an obstacle)
constexpr int kMaxGL = 128, kMaxGB = 256;
constexpr size_t kAlign = 256;
constexpr int kMaxSkips = 4;

// First-fit allocator over one device block.
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    size_t used = 0;

    void init(char* b, size_t n) {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
        used = 0;
    }
    static size_t round(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
    bool fits(const std::vector<size_t>& sizes) const {
        // conservative: the largest free run must hold everything
        size_t need = 0, largest = 0;
        for (size_t s : sizes) need += round(s);
        for (auto& f : free_) largest = std::max(largest, f.second);
        return need <= largest;
    }
    size_t alloc(size_t n) {  // returns offset, or SIZE_MAX
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                used += n;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = round(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && off + n == nx->first) {  // merge right
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {  // merge left
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    bool used = false;
    int64_t ticket = -1;
    lb_request req{};
    Lattice L{};
    std::vector<std::pair<size_t, size_t>> blocks;  // arena (offset, size)
    int nbodies = 0;
    int squirmer = -1;  // global body index
    int64_t start = 0, stop = 0, half = 0;
    bool half_taken = false;
    double ve_half = 0.0;
    long long n_half = 0;
};

struct Queued {
    lb_request req;
    int64_t ticket;
    int skips = 0;
};

}  // namespace

struct lb_server {
    lb_server_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sm = 152;
    void* arena_mem = nullptr;
    Arena arena;
    int cap_slots = 0, cap_bodies = 0;
    // device tables
    Lattice* d_lats = nullptr;
    BodyParams* d_par = nullptr;
    BodyState* d_state[2] = {nullptr, nullptr};
    BodyAcc* d_acc = nullptr;
    double* d_part_links = nullptr;
    double* d_part_conv = nullptr;
    int* d_part_count = nullptr;
    int2* d_link_items = nullptr;
    int2* d_box_items = nullptr;
    int2* d_rel_items = nullptr;
    int* d_counts = nullptr;  // link items, box items, relink items, rebuild blocks done
    SweepArgs* d_sargs = nullptr;  // sweep arguments per slot
    int4* d_tiles = nullptr;
    int* d_ntiles = nullptr;
    long long* d_gstep = nullptr;
    int* d_errs = nullptr;  // one error word per slot
    int list_cap = 0, tile_cap = 0;
    // host state
    std::vector<Slot> slots;
    std::vector<BodyParams> par;
    std::deque<Queued> queue;
    std::map<int64_t, lb_result> done;
    int64_t next_ticket = 1;
    int64_t gstep = 0;
    double cell_updates = 0.0;
    int tile_units = 2048, blocks_per_sm = 2;
    cudaGraphExec_t graph = nullptr;
    std::string msg;
};

namespace {

lb_status sfail(lb_server* s, lb_status st, const std::string& m) {
    if (s) s->msg = m;
    return st;
}

#define SCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return sfail(s, LB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void* sv_alloc(lb_server* s, size_t bytes) {
    void* p = nullptr;
    if (s->p.allocator && s->p.allocator->alloc) p = s->p.allocator->alloc(bytes, s->p.allocator->user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void sv_free(lb_server* s, void* p, size_t bytes) {
    if (!p) return;
    if (s->p.allocator && s->p.allocator->free) s->p.allocator->free(p, bytes, s->p.allocator->user);
    else cudaFree(p);
}

// Every fixed-capacity device table, in one list for allocation and release.
struct TableSpec {
    void** ptr;
    size_t bytes;
};

std::vector<TableSpec> tables(lb_server* s) {
    const size_t B = (size_t)s->cap_bodies;
    return {
        {(void**)&s->d_lats, sizeof(Lattice) * s->cap_slots},
        {(void**)&s->d_par, sizeof(BodyParams) * B},
        {(void**)&s->d_state[0], sizeof(BodyState) * B},
        {(void**)&s->d_state[1], sizeof(BodyState) * B},
        {(void**)&s->d_acc, sizeof(BodyAcc) * B},
        {(void**)&s->d_part_links, sizeof(double) * B * kMaxGL * 12},
        {(void**)&s->d_part_conv, sizeof(double) * B * kMaxGB * 6},
        {(void**)&s->d_part_count, sizeof(int) * B * kMaxGB},
        {(void**)&s->d_link_items, sizeof(int2) * s->list_cap},
        {(void**)&s->d_box_items, sizeof(int2) * s->list_cap},
        {(void**)&s->d_rel_items, sizeof(int2) * s->list_cap},
        {(void**)&s->d_counts, sizeof(int) * 4},
        {(void**)&s->d_sargs, sizeof(SweepArgs) * s->cap_slots},
        {(void**)&s->d_tiles, sizeof(int4) * s->tile_cap},
        {(void**)&s->d_ntiles, sizeof(int) * 5},
        {(void**)&s->d_gstep, sizeof(long long)},
        {(void**)&s->d_errs, sizeof(int) * s->cap_slots},
    };
}

Bodies bodies_view(lb_server* s, bool step) {
    Bodies B;
    B.lats = s->d_lats;
    B.par = s->d_par;
    B.state[0] = s->d_state[0];
    B.state[1] = s->d_state[1];
    B.acc = s->d_acc;
    B.links = (uint32_t*)s->arena.base;
    B.part_links = s->d_part_links;
    B.part_conv = s->d_part_conv;
    B.part_count = s->d_part_count;
    B.GL = kMaxGL;
    B.GB = kMaxGB;
    B.link_items = s->d_link_items;
    B.n_link_items = s->d_counts;
    B.box_items = s->d_box_items;
    B.n_box = s->d_counts + 1;
    B.box_cap = s->list_cap;
    B.rel_items = s->d_rel_items;
    B.n_rel = s->d_counts + 2;
    B.rel_cap = s->list_cap;
    B.done = s->d_counts + 3;
    B.err = s->d_errs;  // list overflow is reported on slot 0's word
    B.win = nullptr;
    B.gstep = step ? s->d_gstep : nullptr;
    // every body takes the multi-kernel path: the fused cluster kernel for the
    // squirmers measured no faster on the serving mix (28.78k against 28.75k
    // MLUPS with 8-block clusters, slower with 16)
    B.fused_items = nullptr;
    B.n_fused = nullptr;
    B.stencil = nullptr;
    return B;
}

TileArgs tile_args(lb_server* s) { return TileArgs{s->d_lats, s->d_sargs, s->d_tiles, s->d_ntiles}; }

int storage_bytes_of(int st) { return st == LB_F64 ? 8 : (st == LB_F32 ? 4 : 2); }

int64_t sphere_link_cap(double R) {
    const double a = R + 2.3, b = std::max(R - 0.9, 0.0);
    return 18 * (int64_t)std::ceil(4.0 / 3.0 * M_PI * (a * a * a - b * b * b)) + 64;
}

// Bodies of a request (host parameters, before link segments are placed).
std::vector<BodyParams> request_bodies(const lb_request& r, std::vector<BodyState>& st) {
    std::vector<BodyParams> v;
    st.clear();
    const int n3[3] = {r.nx, r.ny, r.nz};
    const int64_t N = (int64_t)r.nx * r.ny * r.nz;
    auto wall = [&](int axis, int index) {
        BodyParams b{};
        b.kind = BODY_WALL;
        b.wall_axis = axis;
        b.wall_index = index;
        b.link_cap = 10 * (N / n3[axis]) + 64;
        for (int a = 0; a < 3; ++a) b.box_w[a] = n3[a];
        b.box_w[axis] = std::min(3, n3[axis]);
        b.g_links = (int)std::min<int64_t>(kMaxGL, std::max<int64_t>(1, (5 * (N / n3[axis]) + 127) / 128));
        v.push_back(b);
        st.push_back(BodyState{});
    };
    auto sphere = [&](const double* pos, const double* e, double R, double B1, double beta, int mobile) {
        BodyParams b{};
        b.kind = BODY_SPHERE;
        b.mobile = mobile;
        b.R = R;
        b.B1 = B1;
        b.B2 = beta * B1;
        b.mass = r.rho0 * (4.0 / 3.0) * M_PI * R * R * R;
        b.inertia = 0.4 * b.mass * R * R;
        b.inv_mass = 1.0 / b.mass;
        b.inv_inertia = 1.0 / b.inertia;
        b.link_cap = sphere_link_cap(R);
        const int W = (int)std::ceil(2.0 * R) + 6;
        b.box_w[0] = b.box_w[1] = b.box_w[2] = W;
        b.g_links = (int)std::min<int64_t>(kMaxGL, std::max<int64_t>(1, ((int64_t)std::ceil(63.0 * R * R) + 127) / 128));
        v.push_back(b);
        BodyState s{};
        const double ne = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        for (int a = 0; a < 3; ++a) {
            s.pos[a] = pos[a] - std::floor(pos[a] / n3[a]) * n3[a];
            s.e[a] = e[a] / ne;
        }
        st.push_back(s);
    };
    if (r.geometry == 1) {
        wall(0, 0);
        wall(0, r.nx - 1);
        wall(1, 0);
        wall(1, r.ny - 1);
    } else if (r.geometry == 2) {
        const double e0[3] = {0.0, 0.0, 1.0};
        sphere(r.obstacle, e0, r.obstacle[3], 0.0, 0.0, 0);
    }
    // the walls and the obstacle are still and their forces are not reported
    for (auto& b : v) b.copy_only = 1;
    sphere(r.pos, r.e, r.R, r.B1, r.beta, 1);
    for (auto& b : v) {
        const int64_t box = (int64_t)b.box_w[0] * b.box_w[1] * b.box_w[2];
        b.g_box = (int)std::min<int64_t>(kMaxGB, std::max<int64_t>(1, (box + 511) / 512));
    }
    return v;
}

size_t request_bytes(const lb_request& r, std::vector<size_t>* parts) {
    const int64_t N = (int64_t)r.nx * r.ny * r.nz, Np = (N + 63) / 64 * 64;
    std::vector<BodyState> st;
    auto bodies = request_bodies(r, st);
    int64_t links = 0;
    for (auto& b : bodies) links += b.link_cap;
    std::vector<size_t> v = {(size_t)(19 * Np * storage_bytes_of(r.storage)), (size_t)N * 4, (size_t)N * 4,
                             (size_t)links * 4};
    size_t tot = 0;
    for (size_t x : v) tot += Arena::round(x);
    if (parts) *parts = v;
    return tot;
}

lb_status validate(const lb_request& r) {
    if (r.nx < 1 || r.ny < 1 || r.nz < 1 || (int64_t)r.nx * r.ny * r.nz >= (int64_t(1) << 27)) return LB_ERR_INVALID;
    if (r.geometry < 0 || r.geometry > 2 || r.storage < LB_F64 || r.storage > LB_BF16DEV) return LB_ERR_INVALID;
    if (r.collision != LB_BGK && r.collision != LB_TRT) return LB_ERR_INVALID;
    if (!(r.lambda_e > 0.0 && r.lambda_e < 2.0) || !(r.rho0 > 0.0) || r.steps < 1) return LB_ERR_INVALID;
    if (r.collision == LB_TRT && !(r.magic > 0.0)) return LB_ERR_INVALID;
    const int nmin = std::min(r.nx, std::min(r.ny, r.nz));
    if (!(r.R > 0.0) || !(2.0 * r.R + 6.0 < (double)nmin)) return LB_ERR_INVALID;
    if (r.geometry == 2 && (!(r.obstacle[3] > 0.0) || !(2.0 * r.obstacle[3] + 6.0 < (double)nmin))) return LB_ERR_INVALID;
    const double ne = std::sqrt(r.e[0] * r.e[0] + r.e[1] * r.e[1] + r.e[2] * r.e[2]);
    if (!(ne > 0.0) || !std::isfinite(ne)) return LB_ERR_INVALID;
    return LB_OK;
}

// Set up a request in slot l: memory, populations at rest, walls, spheres
// (classification with the same kernels as a step), links, committed owners.
lb_status admit(lb_server* s, int l, const Queued& q) {
    Slot& sl = s->slots[l];
    const lb_request& r = q.req;
    std::vector<size_t> parts;
    request_bytes(r, &parts);
    std::vector<std::pair<size_t, size_t>> blocks;
    for (size_t n : parts) {
        const size_t off = s->arena.alloc(n);
        if (off == SIZE_MAX) {
            for (auto& b : blocks) s->arena.release(b.first, b.second);
            return LB_ERR_OOM;
        }
        blocks.emplace_back(off, n);
    }
    const int64_t N = (int64_t)r.nx * r.ny * r.nz;
    Lattice L{};
    L.F = s->arena.base + blocks[0].first;
    L.nx = r.nx;
    L.ny = r.ny;
    L.nz = r.nz;
    L.N = N;
    L.Np = (N + 63) / 64 * 64;
    L.storage = r.storage;
    L.rho0 = r.rho0;
    L.scale = r.storage == LB_F16DEV ? std::ldexp(1.0f, 14) : 1.0f;
    L.inv_scale = 1.0f / L.scale;
    L.own = (int32_t*)(s->arena.base + blocks[1].first);
    L.own_prev = (int32_t*)(s->arena.base + blocks[2].first);
    L.err = s->d_errs + l;
    L.lambda_e = r.lambda_e;
    L.lambda_o = r.collision == LB_BGK ? r.lambda_e : 1.0 / (0.5 + r.magic / (1.0 / r.lambda_e - 0.5));
    L.wca_sigma = r.wca_eps > 0.0 ? r.wca_sigma : 1.0;
    L.wca_eps = r.wca_eps > 0.0 ? r.wca_eps : 0.0;
    L.body_begin = l * kBodiesPerSlot;
    L.active = 0;  // not stepped until set up
    L.gstep = s->d_gstep;
    L.stop_step = s->gstep + r.steps;
    L.start_step = s->gstep;
    L.rho_local = 0;
    L.link_at = 0.5f;
    L.sr = r.storage == LB_BF16DEV ? 1 : 0;  // the default rounding of BF16 storage (lb_rounding)
    L.sr_ctr = nullptr;
    std::vector<BodyState> st;
    std::vector<BodyParams> bodies = request_bodies(r, st);
    L.body_count = (int)bodies.size();
    int64_t link_off = (int64_t)(blocks[3].first / 4);
    for (size_t j = 0; j < bodies.size(); ++j) {
        bodies[j].lat = l;
        bodies[j].link_off = link_off;
        link_off += bodies[j].link_cap;
        s->par[L.body_begin + j] = bodies[j];
    }
    cudaStream_t str = s->stream;
    SCK(cudaMemcpyAsync(s->d_lats + l, &L, sizeof(Lattice), cudaMemcpyHostToDevice, str));
    SCK(cudaMemcpyAsync(s->d_par + L.body_begin, bodies.data(), sizeof(BodyParams) * bodies.size(),
                        cudaMemcpyHostToDevice, str));
    for (int b = 0; b < 2; ++b)
        SCK(cudaMemcpyAsync(s->d_state[b] + L.body_begin, st.data(), sizeof(BodyState) * st.size(),
                            cudaMemcpyHostToDevice, str));
    SCK(cudaMemsetAsync(s->d_acc + L.body_begin, 0, sizeof(BodyAcc) * bodies.size(), str));
    SCK(cudaMemsetAsync(L.own, 0, sizeof(int32_t) * N, str));
    SCK(cudaMemsetAsync(L.own_prev, 0, sizeof(int32_t) * N, str));
    SCK(cudaMemsetAsync(L.err, 0, sizeof(int), str));
    launch_fill_rest(L, str);
    const Bodies B = bodies_view(s, false);
    // parity of the next step is that of gstep (even); set-up passes run "after
    // a step of the other parity"
    const int P = 1 - (int)(s->gstep & 1);
    for (size_t j = 0; j < bodies.size(); ++j) {
        const int k = L.body_begin + (int)j;
        if (bodies[j].kind == BODY_WALL) {
            launch_plane_claim(L, L.own, bodies[j].wall_axis, bodies[j].wall_index, k + 1, str);
        } else {
            std::vector<int2> items;
            for (int g = 0; g < bodies[j].g_box; ++g) items.push_back(make_int2(k, g));
            SCK(cudaMemcpyAsync(s->d_box_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                                str));
            const int cnt[3] = {0, (int)items.size(), 0};
            SCK(cudaMemcpyAsync(s->d_counts + 1, cnt + 1, sizeof(int) * 2, cudaMemcpyHostToDevice, str));
            launch_set_flags(s->d_acc, s->cap_bodies, k, 2, str);  // whole box
            launch_body_kernel(2, B, P, 1, std::max(1, std::min((int)items.size(), 4 * s->n_sm)), nullptr, str);
            SCK(cudaStreamSynchronize(str));  // item vector is transient
        }
    }
    // every body of the request: links from scratch, no conversion
    std::vector<int2> items;
    for (size_t j = 0; j < bodies.size(); ++j)
        for (int g = 0; g < bodies[j].g_box; ++g) items.push_back(make_int2(L.body_begin + (int)j, g));
    SCK(cudaMemcpyAsync(s->d_rel_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, str));
    const int cnt[2] = {0, (int)items.size()};
    SCK(cudaMemcpyAsync(s->d_counts + 1, cnt, sizeof(int) * 2, cudaMemcpyHostToDevice, str));
    for (size_t j = 0; j < bodies.size(); ++j) launch_set_flags(s->d_acc, s->cap_bodies, L.body_begin + (int)j, 0, str);
    const int gb = std::max(1, std::min((int)items.size(), 4 * s->n_sm));
    launch_body_kernel(3, B, P, 1, gb, nullptr, str);
    launch_body_kernel(4, B, P, 1, gb, nullptr, str);  // also empties the lists
    SCK(cudaMemcpyAsync(L.own_prev, L.own, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, str));
    L.active = 1;
    SCK(cudaMemcpyAsync(s->d_lats + l, &L, sizeof(Lattice), cudaMemcpyHostToDevice, str));
    const SweepArgs sa = sweep_args(L, L.lambda_e, L.lambda_o);
    SCK(cudaMemcpyAsync(s->d_sargs + l, &sa, sizeof(SweepArgs), cudaMemcpyHostToDevice, str));
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(str));
    int err = 0;
    SCK(cudaMemcpy(&err, L.err, sizeof(int), cudaMemcpyDeviceToHost));
    sl.used = true;
    sl.ticket = q.ticket;
    sl.req = r;
    sl.L = L;
    sl.blocks = blocks;
    sl.nbodies = (int)bodies.size();
    sl.squirmer = L.body_begin + (int)bodies.size() - 1;
    sl.start = s->gstep;
    sl.stop = L.stop_step;
    sl.half = s->gstep + r.steps / 2;
    sl.half_taken = false;
    if (err != 0) return (lb_status)err;
    return LB_OK;
}

void release_slot(lb_server* s, int l) {
    Slot& sl = s->slots[l];
    for (auto& b : sl.blocks) s->arena.release(b.first, b.second);
    sl.blocks.clear();
    sl.used = false;
    sl.L.active = 0;
    cudaMemcpyAsync(s->d_lats + l, &sl.L, sizeof(Lattice), cudaMemcpyHostToDevice, s->stream);
}

lb_status fill_result(lb_server* s, int l, lb_result* out) {
    Slot& sl = s->slots[l];
    BodyState st;
    BodyAcc acc;
    int err = 0;
    const int k = sl.squirmer;
    SCK(cudaMemcpyAsync(&st, s->d_state[sl.stop & 1] + k, sizeof(BodyState), cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaMemcpyAsync(&acc, s->d_acc + k, sizeof(BodyAcc), cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaMemcpyAsync(&err, sl.L.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    std::memset(out, 0, sizeof(*out));
    out->state = err ? LB_REQ_FAILED : LB_REQ_DONE;
    out->status = err;
    out->steps_done = sl.stop - sl.start;
    for (int a = 0; a < 3; ++a) {
        out->pos[a] = st.pos[a];
        out->vel[a] = st.vel[a];
        out->e[a] = st.e[a];
        out->omega[a] = st.omega[a];
        out->F[a] = acc.Fapp[a];
        out->T[a] = acc.Tapp[a];
        out->mean_vel[a] = acc.nsum ? acc.vsum[a] / (double)acc.nsum : 0.0;
    }
    const long long n = acc.nsum - (sl.half_taken ? sl.n_half : 0);
    out->mean_speed = n > 0 ? (acc.vesum - (sl.half_taken ? sl.ve_half : 0.0)) / (double)n : 0.0;
    return LB_OK;
}

// Upload the static work of the resident mix: link items and sweep tiles.
lb_status upload_mix(lb_server* s) {
    std::vector<int2> items;
    std::vector<int4> tiles;
    int bounds[5] = {0, 0, 0, 0, 0};
    for (int l = 0; l < s->cap_slots; ++l) {
        const Slot& sl = s->slots[l];
        if (!sl.used) continue;
        for (int j = 0; j < sl.nbodies; ++j) {
            const int k = sl.L.body_begin + j;
            for (int g = 0; g < s->par[k].g_links; ++g) items.push_back(make_int2(k, g));
        }
    }
    for (int st = 0; st < 4; ++st) {  // tiles sorted by storage
        bounds[st] = (int)tiles.size();
        for (int l = 0; l < s->cap_slots; ++l) {
            const Slot& sl = s->slots[l];
            if (!sl.used || sl.L.storage != st) continue;
            const int paired = (sl.L.nx % 2 == 0 && st != LB_F64) ? 1 : 0;
            const int64_t units = paired ? sl.L.N / 2 : sl.L.N;
            for (int64_t u0 = 0; u0 < units; u0 += s->tile_units)
                tiles.push_back(make_int4(l, (int)u0, (int)std::min<int64_t>(units, u0 + s->tile_units), paired));
        }
    }
    bounds[4] = (int)tiles.size();
    if ((int)items.size() > s->list_cap || (int)tiles.size() > s->tile_cap)
        return sfail(s, LB_ERR_CAPACITY, "work lists of the resident mix");
    if (!items.empty())
        SCK(cudaMemcpyAsync(s->d_link_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                            s->stream));
    if (!tiles.empty())
        SCK(cudaMemcpyAsync(s->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s->stream));
    const int ni = (int)items.size();
    SCK(cudaMemcpyAsync(s->d_counts, &ni, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    SCK(cudaMemcpyAsync(s->d_ntiles, bounds, sizeof(bounds), cudaMemcpyHostToDevice, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return LB_OK;
}

void enqueue_round(lb_server* s, cudaStream_t st) {
    const Bodies B = bodies_view(s, true);
    const TileArgs T = tile_args(s);
    const int grid = s->blocks_per_sm * s->n_sm;
    const int glinks = 8 * s->n_sm, gbox = 4 * s->n_sm;  // latency-bound: many blocks
    for (int k = 0; k < s->p.round_steps; ++k) {
        const int P = k & 1;  // rounds start on even steps
        launch_tiles(T, P, grid, st);
        for (int w = 1; w <= 4; ++w) launch_body_kernel(w, B, P, glinks, gbox, nullptr, st);
    }
}

lb_status build_graph(lb_server* s) {
    cudaGraph_t g = nullptr;
    SCK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_round(s, s->stream);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess) return sfail(s, LB_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph = nullptr;
        return sfail(s, LB_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

// Tile-shape autotuner: time the tile sweep on two synthetic lattices (96^3
// FP32 and FP16) for each candidate (planes per tile, blocks per SM) and keep
// the fastest.  Uses arena memory that is free at creation.
lb_status autotune(lb_server* s) {
    const int n = 96;
    Lattice Ls[2];
    std::vector<std::pair<size_t, size_t>> blocks;
    const int storages[2] = {LB_F32, LB_F16DEV};
    for (int i = 0; i < 2; ++i) {
        const int64_t N = (int64_t)n * n * n, Np = (N + 63) / 64 * 64;
        const size_t bytes = (size_t)19 * Np * storage_bytes_of(storages[i]);
        const size_t off = s->arena.alloc(bytes);
        if (off == SIZE_MAX) {
            for (auto& b : blocks) s->arena.release(b.first, b.second);
            return LB_OK;  // budget too small to tune: keep the defaults
        }
        blocks.emplace_back(off, bytes);
        Lattice L{};
        L.F = s->arena.base + off;
        L.nx = L.ny = L.nz = n;
        L.N = N;
        L.Np = Np;
        L.storage = storages[i];
        L.rho0 = 1.0;
        L.scale = storages[i] == LB_F16DEV ? std::ldexp(1.0f, 14) : 1.0f;
        L.inv_scale = 1.0f / L.scale;
        L.lambda_e = 1.0;
        L.lambda_o = 8.0 / 7.0;
        L.active = 1;
        Ls[i] = L;
        launch_fill_rest(L, s->stream);
    }
    SCK(cudaMemcpyAsync(s->d_lats, Ls, sizeof(Ls), cudaMemcpyHostToDevice, s->stream));
    const SweepArgs sa[2] = {sweep_args(Ls[0], Ls[0].lambda_e, Ls[0].lambda_o),
                             sweep_args(Ls[1], Ls[1].lambda_e, Ls[1].lambda_o)};
    SCK(cudaMemcpyAsync(s->d_sargs, sa, sizeof(sa), cudaMemcpyHostToDevice, s->stream));
    cudaEvent_t e0, e1;
    SCK(cudaEventCreate(&e0));
    SCK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_tu = s->tile_units, best_b = s->blocks_per_sm;
    const int tu_cand[4] = {512, 1024, 2048, 4096}, b_cand[2] = {2, 4};
    for (int tu : tu_cand)
        for (int bps : b_cand) {
            // lattice 0 is FP32, lattice 1 FP16: tiles [0, m) and [m, 2m)
            std::vector<int4> tiles;
            const int units = n * n * n / 2;
            for (int i = 0; i < 2; ++i)
                for (int u0 = 0; u0 < units; u0 += tu) tiles.push_back(make_int4(i, u0, std::min(units, u0 + tu), 1));
            const int m = (int)tiles.size() / 2;
            const int bounds[5] = {0, 0, m, 2 * m, 2 * m};
            SCK(cudaMemcpyAsync(s->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                s->stream));
            SCK(cudaMemcpyAsync(s->d_ntiles, bounds, sizeof(bounds), cudaMemcpyHostToDevice, s->stream));
            const TileArgs T = tile_args(s);
            for (int w = 0; w < 2; ++w) launch_tiles(T, w & 1, bps * s->n_sm, s->stream);
            SCK(cudaEventRecord(e0, s->stream));
            for (int w = 0; w < 6; ++w) launch_tiles(T, w & 1, bps * s->n_sm, s->stream);
            SCK(cudaEventRecord(e1, s->stream));
            SCK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            SCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_tu = tu;
                best_b = bps;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto& b : blocks) s->arena.release(b.first, b.second);
    Lattice zero[2] = {};
    SCK(cudaMemcpyAsync(s->d_lats, zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream));
    SCK(cudaMemsetAsync(s->d_sargs, 0, sizeof(sa), s->stream));
    const int nt0[5] = {0, 0, 0, 0, 0};
    SCK(cudaMemcpyAsync(s->d_ntiles, nt0, sizeof(nt0), cudaMemcpyHostToDevice, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    s->tile_units = best_tu;
    s->blocks_per_sm = best_b;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_server_params_default(lb_server_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->device = 0;
    p->hbm_budget_bytes = (size_t)8 << 30;
    p->max_resident = 64;
    p->round_steps = 64;
    p->tile_units = 0;
}

lb_status lb_server_create(const lb_server_params* p, lb_server** out) {
    if (!p || !out) return LB_ERR_INVALID;
    if (p->max_resident < 1 || p->max_resident > 256 || p->round_steps < 2 || (p->round_steps & 1) ||
        p->hbm_budget_bytes < ((size_t)1 << 20) || p->tile_units < 0)
        return LB_ERR_INVALID;
    lb_server* s = new (std::nothrow) lb_server();
    if (!s) return LB_ERR_OOM;
    s->p = *p;
    auto bail = [&](lb_status st) {
        lb_server_destroy(s);
        return st;
    };
    if (cudaSetDevice(p->device) != cudaSuccess) return bail(LB_ERR_CUDA);
    if (p->stream) s->stream = (cudaStream_t)p->stream;
    else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(LB_ERR_CUDA);
        s->own_stream = true;
    }
    cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, p->device);
    s->cap_slots = p->max_resident;
    s->cap_bodies = s->cap_slots * kBodiesPerSlot;
    s->list_cap = s->cap_bodies * kMaxGB;
    s->tile_cap = 1 << 20;
    s->arena_mem = sv_alloc(s, p->hbm_budget_bytes);
    if (!s->arena_mem) return bail(LB_ERR_OOM);
    s->arena.init((char*)s->arena_mem, p->hbm_budget_bytes);
    for (auto& t : tables(s)) {
        *t.ptr = sv_alloc(s, t.bytes);
        if (!*t.ptr) return bail(LB_ERR_OOM);
        if (cudaMemsetAsync(*t.ptr, 0, t.bytes, s->stream) != cudaSuccess) return bail(LB_ERR_CUDA);
    }
    s->slots.resize(s->cap_slots);
    s->par.resize(s->cap_bodies);
    if (p->tile_units > 0) s->tile_units = p->tile_units;
    else if (autotune(s) != LB_OK) return bail(LB_ERR_CUDA);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bail(LB_ERR_CUDA);
    *out = s;
    return LB_OK;
}

lb_status lb_server_destroy(lb_server* s) {
    if (!s) return LB_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (auto& t : tables(s)) sv_free(s, *t.ptr, t.bytes);
    sv_free(s, s->arena_mem, s->p.hbm_budget_bytes);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return LB_OK;
}

const char* lb_server_last_error(const lb_server* s) { return s ? s->msg.c_str() : "null server"; }

lb_status lb_server_submit(lb_server* s, const lb_request* r, int64_t* ticket) {
    if (!s || !r || !ticket) return LB_ERR_INVALID;
    if (validate(*r) != LB_OK) return sfail(s, LB_ERR_INVALID, "request parameters");
    if (request_bytes(*r, nullptr) > s->p.hbm_budget_bytes) return sfail(s, LB_ERR_INVALID, "request exceeds the budget");
    Queued q;
    q.req = *r;
    q.ticket = s->next_ticket++;
    s->queue.push_back(q);
    *ticket = q.ticket;
    return LB_OK;
}

lb_status lb_server_advance(lb_server* s, int32_t* running, int32_t* queued) {
    if (!s) return LB_ERR_INVALID;
    SCK(cudaSetDevice(s->p.device));
    bool changed = false;
    // 1. retire requests that reached their last step
    for (int l = 0; l < s->cap_slots; ++l) {
        Slot& sl = s->slots[l];
        if (!sl.used || s->gstep < sl.stop) continue;
        lb_result res;
        lb_status st = fill_result(s, l, &res);
        if (st != LB_OK) return st;
        s->done[sl.ticket] = res;
        release_slot(s, l);
        changed = true;
    }
    // 2. admit in arrival order; later requests may pass one that does not fit
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        int free_slot = -1;
        for (int l = 0; l < s->cap_slots && free_slot < 0; ++l)
            if (!s->slots[l].used) free_slot = l;
        if (free_slot < 0) break;
        std::vector<size_t> parts;
        request_bytes(it->req, &parts);
        if (!s->arena.fits(parts)) {
            if (++it->skips > kMaxSkips) break;  // stop passing it
            ++it;
            continue;
        }
        lb_status st = admit(s, free_slot, *it);
        if (st == LB_ERR_OOM) {  // fragmented: try later
            if (++it->skips > kMaxSkips) break;
            ++it;
            continue;
        }
        if (st != LB_OK) {
            if (st == LB_ERR_CUDA) return st;
            lb_result res{};
            res.state = LB_REQ_FAILED;
            res.status = st;
            s->done[it->ticket] = res;
            release_slot(s, free_slot);
        }
        it = s->queue.erase(it);
        changed = true;
    }
    if (changed) {
        lb_status st = upload_mix(s);
        if (st != LB_OK) return st;
    }
    // 3. one round for every resident request
    int n_run = 0;
    for (auto& sl : s->slots) n_run += sl.used ? 1 : 0;
    if (n_run > 0) {
        if (!s->graph) {
            lb_status st = build_graph(s);
            if (st != LB_OK) return st;
        }
        SCK(cudaMemcpyAsync(s->d_gstep, &s->gstep, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
        SCK(cudaGraphLaunch(s->graph, s->stream));
        for (auto& sl : s->slots)
            if (sl.used) {
                const int64_t a = std::max(s->gstep, sl.start), b = std::min(s->gstep + s->p.round_steps, sl.stop);
                if (b > a) s->cell_updates += (double)sl.L.N * (double)(b - a);
            }
        s->gstep += s->p.round_steps;
        SCK(cudaStreamSynchronize(s->stream));
        // mean-speed window: snapshot the sums at the first round end past half-way
        for (auto& sl : s->slots) {
            if (!sl.used || sl.half_taken || s->gstep < sl.half) continue;
            BodyAcc acc;
            SCK(cudaMemcpy(&acc, s->d_acc + sl.squirmer, sizeof(BodyAcc), cudaMemcpyDeviceToHost));
            sl.ve_half = acc.vesum;
            sl.n_half = acc.nsum;
            sl.half_taken = true;
        }
    }
    if (running) *running = n_run;
    if (queued) *queued = (int32_t)s->queue.size();
    return LB_OK;
}

lb_status lb_server_poll(lb_server* s, int64_t ticket, lb_result* out) {
    if (!s || !out) return LB_ERR_INVALID;
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
        *out = it->second;
        s->done.erase(it);
        return LB_OK;
    }
    for (auto& sl : s->slots)
        if (sl.used && sl.ticket == ticket) {
            std::memset(out, 0, sizeof(*out));
            out->state = LB_REQ_RUNNING;
            out->steps_done = std::min(s->gstep, sl.stop) - sl.start;
            return LB_OK;
        }
    for (auto& q : s->queue)
        if (q.ticket == ticket) {
            std::memset(out, 0, sizeof(*out));
            out->state = LB_REQ_QUEUED;
            return LB_OK;
        }
    return sfail(s, LB_ERR_INVALID, "unknown ticket");
}

lb_status lb_server_info(const lb_server* s, int32_t* tile_units, int32_t* blocks_per_sm, size_t* bytes_used,
                         double* cell_updates) {
    if (!s) return LB_ERR_INVALID;
    if (tile_units) *tile_units = s->tile_units;
    if (blocks_per_sm) *blocks_per_sm = s->blocks_per_sm;
    if (bytes_used) *bytes_used = s->arena.used;
    if (cell_updates) *cell_updates = s->cell_updates;
    return LB_OK;
}

}  // extern "C"
