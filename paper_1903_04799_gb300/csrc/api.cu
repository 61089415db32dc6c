// api.cu -- the C ABI of include/lbsq.h: context life cycle, validation,
// device memory, body set-up and the per-step launch sequence (replayed from
// a CUDA graph of eight steps, starting on an even step, once the body set is
// fixed).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbsq.h"
#include "lbsq_internal.cuh"

namespace lbsq {
void launch_sweep(const Lattice& L, double lambda_e, double lambda_o, int parity, int variant, int zmode,
                  const int* win, int gz, int gy, cudaStream_t st);
void launch_body_kernel(int which, const Bodies& B, int parity, int grid_links, int grid_box, long long* step,
                        cudaStream_t st);
void launch_body_step(const Bodies& B, int parity, int grid_links, int grid_box, long long* step, cudaStream_t st);
void launch_body_fused(const Bodies& B, int parity, int cls, int clusters, cudaStream_t st, int tail,
                       cudaEvent_t started = nullptr);
cudaError_t prepare_body_kernels();
void launch_fill_rest(const Lattice& L, cudaStream_t st);
void launch_set_eq(const Lattice& L, const double* rho, const double* u, int q, cudaStream_t st);
void launch_set_pop(const Lattice& L, const double* f, int q, cudaStream_t st);
void launch_get_pop(const Lattice& L, double* f, int q, cudaStream_t st);
void launch_fields(const Lattice& L, const int32_t* own, double* rho, double* u, int q, cudaStream_t st);
int mass_partial_blocks(const Lattice& L);
void launch_mass(const Lattice& L, const int32_t* own, double* part, double* out, int q, cudaStream_t st);
void launch_sphere_overlap(const Lattice& L, const int32_t* own, const double* pos, double R, int W, int* count,
                           cudaStream_t st);
void launch_plane_overlap(const Lattice& L, const int32_t* own, const int* kind, int axis, int index, int* count,
                          cudaStream_t st);
void launch_plane_claim(const Lattice& L, int32_t* own, int axis, int index, int id, cudaStream_t st);
void launch_tube_overlap(const Lattice& L, const int32_t* own, const int* kind, const BodyParams& q, int* count,
                         cudaStream_t st);
void launch_tube_claim(const Lattice& L, int32_t* own, const BodyParams& q, int id, cudaStream_t st);
void launch_set_flags(BodyAcc* acc, int nb, int k, int reclass, cudaStream_t st);
void launch_psm_cover(const Bodies& B, int parity, int grid, bool f64, cudaStream_t st);
void launch_psm_scatter(const Bodies& B, int parity, int grid, cudaStream_t st);
}  // namespace lbsq

using namespace lbsq;

struct lb_ctx {
    lb_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Lattice L{};
    double lambda_e = 1.0, lambda_o = 1.0;
    int32_t* own = nullptr;
    int32_t* own_prev = nullptr;
    // bodies
    std::vector<BodyParams> par;
    std::vector<int> kind;
    int cap = 0;
    BodyParams* d_par = nullptr;
    BodyState* d_state[2] = {nullptr, nullptr};
    BodyAcc* d_acc = nullptr;
    int* d_kind = nullptr;
    uint32_t* d_links = nullptr;
    int64_t links_total = 0;
    double* d_part_links = nullptr;
    double* d_part_conv = nullptr;
    int* d_part_count = nullptr;
    int G_links = 1, G_box = 1;
    // work lists: static link items, device-built box and relink items
    int2* d_link_items = nullptr;
    int2* d_box_items = nullptr;
    int2* d_rel_items = nullptr;
    int* d_counts = nullptr;  // [0] link items, [1] box items, [2] relink items, [3] rebuild blocks done,
                              // [4..6] fused spheres per class, [7..9] first fused item per class,
                              // [10] clusters of a solo fused launch done
    int n_link_items = 0, list_cap = 0, list_alloc = 0;
    // spheres advanced by the fused cluster kernel, and their shell stencils
    int2* d_fused_items = nullptr;
    uint32_t* d_stencil = nullptr;
    int n_fused = 0, fused_cls = 0, fused_alloc = 0;
    // the lattice holds one fused sphere and no other body: its step needs
    // only the fused kernel (no body can come near another)
    bool solo = false;
    int64_t stencil_alloc = 0;
    int grid_box = 1;
    int n_sm = 152;
    Lattice* d_lat = nullptr;  // the one lattice descriptor on the device
    double wca_sigma = 1.0, wca_eps = 0.0;
    int force_avg = 0;  // lb_set_force_average
    // spheres coupled by partially saturated cells (lb_set_coupling): the
    // solid fraction and covering sphere per cell, the (body, block) items of
    // the spheres' boxes, their per-block force partials and the covered
    // cells' post-collision populations
    bool psm = false;
    float* d_eps = nullptr;
    int32_t* d_psm_id = nullptr;
    int2* d_psm_items = nullptr;
    double* d_part_psm = nullptr;
    double* d_psm_out = nullptr;
    int32_t* d_psm_cell = nullptr;
    int32_t* d_psm_count = nullptr;
    int64_t psm_cap = 0, psm_out_alloc = 0;
    int n_psm_items = 0, psm_alloc = 0, grid_psm = 1;
    // scratch
    double* d_mass_part = nullptr;
    double* d_small = nullptr;  // 8 doubles
    int* d_err = nullptr;
    int* d_count = nullptr;
    double* d_fields = nullptr;  // 4 N doubles, allocated on first host export
    double* d_pop = nullptr;     // 19 N doubles, allocated on first population I/O
    // bookkeeping
    int64_t step = 0;
    int64_t launches = 0;
    int sticky = 0;
    std::string msg;
    std::vector<std::pair<void*, size_t>> allocs;
    // graph of two steps (even then odd)
    // graphs of 8 steps: [0] whole steps, or (split lattices) 8 units from t =
    // 1 (mod 4); [1] split lattices, 8 units from t = 3 (mod 4)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_launches = 0;  // kernel launches in one replay
    int sweep_variant = 0;
    // overlap of the body kernels of step t with the far sweep of step t+1:
    // the far sweep on `side`, the body kernels on `hi` (highest priority, so
    // that SM slots freed by sweep blocks go to the short body kernels first)
    cudaStream_t side = nullptr, hi = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    cudaEvent_t ev_started = nullptr;  // every block of the fused body kernel has begun (see enqueue_unit)
    int* d_win = nullptr;  // [4][4] near-body windows (z0, z length, y0, y length) by step (mod 4)
    bool split = false;    // whether steps are split into far and near sweeps
    int win_max = 0;       // upper bound of the window's z length (planes)
    int ywin_max = 0;      // upper bound of its y length (rows)
    bool pending = false;  // split steps: the body step of step `step - 1` is not issued yet (see settle)
    // kernel tracing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_used;  // (kernel kind, index of the start event)
};

namespace {

lb_status fail(lb_ctx* c, lb_status s, const std::string& m) {
    if (c) c->msg = m;
    return s;
}

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

void* dalloc(lb_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->p.allocator && c->p.allocator->alloc) {
        p = c->p.allocator->alloc(bytes, c->p.allocator->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.emplace_back(p, bytes);
    return p;
}

void dfree(lb_ctx* c, void* p) {
    if (!p) return;
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (c->allocs[k].first == p) {
            if (c->p.allocator && c->p.allocator->free) c->p.allocator->free(p, c->allocs[k].second, c->p.allocator->user);
            else cudaFree(p);
            c->allocs.erase(c->allocs.begin() + k);
            return;
        }
    }
}

template <class T>
T* dalloc_t(lb_ctx* c, size_t n) {
    return (T*)dalloc(c, n * sizeof(T));
}

void drop_graph(lb_ctx* c) {
    for (auto& g : c->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

Bodies bodies_view(const lb_ctx* c) {
    Bodies B;
    B.lats = c->d_lat;
    B.par = c->d_par;
    B.state[0] = c->d_state[0];
    B.state[1] = c->d_state[1];
    B.acc = c->d_acc;
    B.links = c->d_links;
    B.part_links = c->d_part_links;
    B.part_conv = c->d_part_conv;
    B.part_count = c->d_part_count;
    B.GL = c->G_links;
    B.GB = c->G_box;
    B.link_items = c->d_link_items;
    B.n_link_items = c->d_counts;
    B.box_items = c->d_box_items;
    B.n_box = c->d_counts + 1;
    B.box_cap = c->list_cap;
    B.rel_items = c->d_rel_items;
    B.n_rel = c->d_counts + 2;
    B.rel_cap = c->list_cap;
    B.done = c->d_counts + 3;
    B.err = c->d_err;
    B.win = nullptr;  // see bodies_for_step
    B.gstep = nullptr;
    B.fused_items = c->d_fused_items;
    B.n_fused = c->d_counts + 4;
    B.fused_first = c->d_counts + 7;
    B.stencil = c->d_stencil;
    B.fused_done = c->d_counts + 10;
    B.psm_items = c->d_psm_items;
    B.n_psm_items = c->n_psm_items;
    B.part_psm = c->d_part_psm;
    B.psm_out = c->d_psm_out;
    B.psm_cell = c->d_psm_cell;
    B.psm_count = c->d_psm_count;
    B.psm_cap = c->psm_cap;
    return B;
}

// Window slot of the sweeps of step s.  Four slots by step: the body kernels
// of step t write slot t + 2 while the far sweep of step t, which reads slot t,
// may still run beside them (see enqueue_unit).
int* win_slot(const lb_ctx* c, int64_t s) { return c->d_win + 4 * (int)(s & 3); }

// The view for the body kernels of step t: they write the window of step t + 2.
Bodies bodies_for_step(const lb_ctx* c, int64_t t) {
    Bodies B = bodies_view(c);
    if (c->split) B.win = win_slot(c, t + 2);
    return B;
}

// The lattice descriptor the body kernels read, rebuilt from the context.
lb_status upload_lattice(lb_ctx* c) {
    Lattice L = c->L;
    L.lambda_e = c->lambda_e;
    L.lambda_o = c->lambda_o;
    L.wca_sigma = c->wca_sigma;
    L.wca_eps = c->wca_eps;
    L.force_avg = c->force_avg;
    L.body_begin = 0;
    L.body_count = (int)c->par.size();
    L.active = 1;
    L.gstep = nullptr;
    L.stop_step = 0;
    c->L = L;
    CK(cudaMemcpyAsync(c->d_lat, &L, sizeof(Lattice), cudaMemcpyHostToDevice, c->stream));
    return LB_OK;
}

// Upper bound on the boundary links of a sphere of radius R: 18 per lattice
// node within the shell R - 0.9 < |d| < R + 2.3 (covers any centre offset).
int64_t sphere_link_cap(double R) {
    double a = R + 2.3, b = std::max(R - 0.9, 0.0);
    double v = 4.0 / 3.0 * M_PI * (a * a * a - b * b * b);
    return 18 * (int64_t)std::ceil(v) + 64;
}

bool check_device_error(lb_ctx* c, lb_status* out) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        *out = cuda_fail(c, e, "synchronise");
        return true;
    }
    if (h != 0) {
        c->sticky = h;
        const char* what = h == LB_ERR_OVERLAP    ? "a body overlaps another body or a wall"
                           : h == LB_ERR_DIVERGED ? "a body reached |v| >= 1/2"
                           : h == LB_ERR_CAPACITY ? "a boundary-link list outgrew its capacity"
                           : h == LB_ERR_TIMEOUT  ? "a bounded device wait ran out"
                                                  : "device error";
        *out = fail(c, (lb_status)h, what);
        return true;
    }
    return false;
}

lb_status sync_checked(lb_ctx* c) {
    lb_status s;
    if (check_device_error(c, &s)) return s;
    return LB_OK;
}

// Grow the body arrays to hold at least n bodies, keeping their contents.
lb_status ensure_body_capacity(lb_ctx* c, int n) {
    if (n <= c->cap) return LB_OK;
    int nc = std::max(8, c->cap * 2);
    while (nc < n) nc *= 2;
    BodyParams* par = dalloc_t<BodyParams>(c, nc);
    BodyState* s0 = dalloc_t<BodyState>(c, nc);
    BodyState* s1 = dalloc_t<BodyState>(c, nc);
    BodyAcc* acc = dalloc_t<BodyAcc>(c, nc);
    int* kind = dalloc_t<int>(c, nc);
    if (!par || !s0 || !s1 || !acc || !kind) return fail(c, LB_ERR_OOM, "body arrays");
    CK(cudaMemsetAsync(acc, 0, sizeof(BodyAcc) * nc, c->stream));
    int nb = (int)c->par.size();
    if (nb > 0) {
        CK(cudaMemcpyAsync(par, c->d_par, sizeof(BodyParams) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(s0, c->d_state[0], sizeof(BodyState) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(s1, c->d_state[1], sizeof(BodyState) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(acc, c->d_acc, sizeof(BodyAcc) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(kind, c->d_kind, sizeof(int) * nb, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, c->d_par);
    dfree(c, c->d_state[0]);
    dfree(c, c->d_state[1]);
    dfree(c, c->d_acc);
    dfree(c, c->d_kind);
    c->d_par = par;
    c->d_state[0] = s0;
    c->d_state[1] = s1;
    c->d_acc = acc;
    c->d_kind = kind;
    c->cap = nc;
    return LB_OK;
}

// After the body set changed: assign link segments, size the partial-sum
// buffers and work lists, and upload the body parameters.
lb_status relayout(lb_ctx* c) {
    const int nb = (int)c->par.size();
    int64_t off = 0;
    int gl = 1, gb = 1, sum_gb = 0;
    std::vector<int2> items;
    std::vector<int2> fused;
    std::vector<int2> psm_items;
    std::vector<uint32_t> stencil;
    int64_t psm_cap = 0;
    for (int k = 0; k < nb; ++k) {
        BodyParams& b = c->par[k];
        b.link_off = off;
        off += b.link_cap;
        b.lat = 0;
        b.st_off = 0;
        b.st_count = 0;
        if (fused_body(b)) {
            const std::vector<uint32_t> v = shell_stencil(b.R);
            b.st_off = (int64_t)stencil.size();
            b.st_count = (int)v.size();
            stencil.insert(stencil.end(), v.begin(), v.end());
            fused.push_back(make_int2(k, 0));
        }
        // block counts depend on the body alone (so do its fixed-order
        // reductions): about one link per thread of the link kernel, two box
        // cells per thread of the box kernels; capped by the shared staging
        // buffers of the final sums (128 and 256 partials)
        const int64_t box = (int64_t)b.box_w[0] * b.box_w[1] * b.box_w[2];
        int64_t expect;
        if (b.kind == BODY_SPHERE) {
            expect = (int64_t)std::ceil(63.0 * b.R * b.R);  // about 5 links per node of 4 pi R^2
        } else if (b.wall_axis < 0) {
            // round tube: about 5 links per wall node of the circumference, on every plane
            expect = (int64_t)std::ceil(5.0 * 6.2832 * b.tube[2]) * c->L.nz;
        } else {
            const int n3[3] = {c->L.nx, c->L.ny, c->L.nz};
            expect = 5 * (c->L.N / n3[b.wall_axis]);
        }
        b.g_links = (int)std::min<int64_t>(128, std::max<int64_t>(1, (expect + 127) / 128));
        b.g_box = (int)std::min<int64_t>(256, std::max<int64_t>(1, (box + 511) / 512));
        gl = std::max(gl, b.g_links);
        gb = std::max(gb, b.g_box);
        sum_gb += b.g_box;
        b.psm_off = psm_cap;
        if (b.psm) {  // one item per chunk of the box
            const int64_t nq = (box + kPsmChunk - 1) / kPsmChunk;
            for (int64_t q = 0; q < nq; ++q) psm_items.push_back(make_int2(k, (int)q));
            psm_cap += nq * kPsmChunk;
        }
        else if (!fused_body(b))
            for (int g = 0; g < b.g_links; ++g) items.push_back(make_int2(k, g));
    }
    if ((int)fused.size() > c->fused_alloc) {
        dfree(c, c->d_fused_items);
        c->d_fused_items = dalloc_t<int2>(c, fused.size());
        if (!c->d_fused_items) return fail(c, LB_ERR_OOM, "fused body list");
        c->fused_alloc = (int)fused.size();
    }
    if ((int64_t)stencil.size() > c->stencil_alloc) {
        dfree(c, c->d_stencil);
        c->d_stencil = dalloc_t<uint32_t>(c, stencil.size());
        if (!c->d_stencil) return fail(c, LB_ERR_OOM, "shell stencils");
        c->stencil_alloc = (int64_t)stencil.size();
    }
    c->n_fused = (int)fused.size();
    c->fused_cls = fused_class(c->n_fused);
    c->solo = c->n_fused == 1 && nb == 1;
    if (!fused.empty()) {
        CK(cudaMemcpyAsync(c->d_fused_items, fused.data(), sizeof(int2) * fused.size(), cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_stencil, stencil.data(), sizeof(uint32_t) * stencil.size(), cudaMemcpyHostToDevice,
                           c->stream));
    }
    if (off > c->links_total) {
        dfree(c, c->d_links);
        c->d_links = dalloc_t<uint32_t>(c, (size_t)off);
        if (!c->d_links) return fail(c, LB_ERR_OOM, "link lists");
        c->links_total = off;
    }
    c->G_links = gl;
    c->G_box = gb;
    dfree(c, c->d_part_links);
    dfree(c, c->d_part_conv);
    dfree(c, c->d_part_count);
    c->d_part_links = dalloc_t<double>(c, (size_t)nb * c->G_links * 12);
    c->d_part_conv = dalloc_t<double>(c, (size_t)nb * c->G_box * 6);
    c->d_part_count = dalloc_t<int>(c, (size_t)nb * c->G_box);
    if (!c->d_part_links || !c->d_part_conv || !c->d_part_count) return fail(c, LB_ERR_OOM, "partials");
    if (!psm_items.empty()) {
        dfree(c, c->d_part_psm);
        c->d_part_psm = dalloc_t<double>(c, (size_t)(psm_cap / kPsmChunk) * 12);
        if ((int)psm_items.size() > c->psm_alloc) {
            dfree(c, c->d_psm_items);
            c->d_psm_items = dalloc_t<int2>(c, psm_items.size());
            c->psm_alloc = c->d_psm_items ? (int)psm_items.size() : 0;
        }
        if (psm_cap > c->psm_out_alloc) {
            dfree(c, c->d_psm_out);
            dfree(c, c->d_psm_cell);
            dfree(c, c->d_psm_count);
            c->d_psm_out = dalloc_t<double>(c, (size_t)Q * psm_cap);
            c->d_psm_cell = dalloc_t<int32_t>(c, (size_t)psm_cap);
            c->d_psm_count = dalloc_t<int32_t>(c, (size_t)(psm_cap / kPsmChunk));
            c->psm_out_alloc = c->d_psm_out && c->d_psm_cell && c->d_psm_count ? psm_cap : 0;
        }
        if (!c->d_part_psm || !c->d_psm_items || !c->d_psm_out || !c->d_psm_cell || !c->d_psm_count)
            return fail(c, LB_ERR_OOM, "partially saturated cells");
        CK(cudaMemcpyAsync(c->d_psm_items, psm_items.data(), sizeof(int2) * psm_items.size(),
                           cudaMemcpyHostToDevice, c->stream));
    }
    c->n_psm_items = (int)psm_items.size();
    c->psm_cap = psm_cap;
    c->grid_psm = std::max(1, std::min(c->n_psm_items, 4 * c->n_sm));
    // work lists: every body appears at most once per step in each list
    const int need = std::max<int>((int)items.size(), sum_gb);
    if (need > c->list_alloc) {
        dfree(c, c->d_link_items);
        dfree(c, c->d_box_items);
        dfree(c, c->d_rel_items);
        c->d_link_items = dalloc_t<int2>(c, need);
        c->d_box_items = dalloc_t<int2>(c, need);
        c->d_rel_items = dalloc_t<int2>(c, need);
        if (!c->d_link_items || !c->d_box_items || !c->d_rel_items) return fail(c, LB_ERR_OOM, "work lists");
        c->list_alloc = need;
    }
    c->list_cap = sum_gb;
    c->n_link_items = (int)items.size();
    c->grid_box = std::max(1, std::min(sum_gb, 4 * c->n_sm));
    CK(cudaMemcpyAsync(c->d_link_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice,
                       c->stream));
    int counts[11] = {c->n_link_items, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    counts[4 + c->fused_cls] = c->n_fused;  // one lattice: one class, starting at item 0
    CK(cudaMemcpyAsync(c->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_par, c->par.data(), sizeof(BodyParams) * nb, cudaMemcpyHostToDevice, c->stream));
    // both state buffers hold the current state
    const int cur = (int)(c->step & 1);
    CK(cudaMemcpyAsync(c->d_state[1 - cur], c->d_state[cur], sizeof(BodyState) * nb, cudaMemcpyDeviceToDevice,
                       c->stream));
    lb_status s = upload_lattice(c);
    if (s != LB_OK) return s;
    // near-body window: upper bounds of its z and y lengths, which size the
    // near sweep's grid.  The window is one periodic box around every body's
    // range (near_window), so with one body it is that body's range; with
    // several it also spans the gaps between them and may be any length up
    // to the whole lattice.  The split pays only when the summed ranges leave
    // most of the planes outside (a z-normal wall spans every row).
    int wmax = 0, ymax = 0, ranges = 0;
    bool across = false;
    for (auto& b : c->par) {
        if (b.kind == BODY_SPHERE) {
            wmax += b.box_w[2] + 5;
            ymax += b.box_w[1] + 5;
            ++ranges;
        } else if (b.wall_axis == 2) {
            wmax += 3 + 5;
            ymax += c->L.ny;
            ++ranges;
        } else {
            across = true;
        }
    }
    // (partially saturated cells: every step sweeps the whole lattice)
    c->split = !c->psm && !across && nb > 0 && wmax * 5 < 3 * c->L.nz;
    if (ranges > 1) {
        wmax = c->L.nz;
        ymax = c->L.ny;
    }
    c->win_max = std::min(wmax, c->L.nz);
    // the device takes every row once the extent may reach 3/5 of them
    c->ywin_max = ymax * 5 < 3 * c->L.ny ? ymax : c->L.ny;
    // whole lattice until the first rebuild
    int win_init[16];
    for (int k = 0; k < 4; ++k) {
        win_init[4 * k] = 0;
        win_init[4 * k + 1] = c->L.nz;
        win_init[4 * k + 2] = 0;
        win_init[4 * k + 3] = c->L.ny;
    }
    CK(cudaMemcpyAsync(c->d_win, win_init, sizeof(win_init), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // host vectors above are transient
    drop_graph(c);
    return LB_OK;
}

// Upload a host-built item list as the relink (which = 2) or box (1) list.
lb_status set_list(lb_ctx* c, int which, const std::vector<int2>& items) {
    int2* dst = which == 1 ? c->d_box_items : c->d_rel_items;
    if ((int)items.size() > c->list_cap) return fail(c, LB_ERR_CAPACITY, "work list");
    if (!items.empty())
        CK(cudaMemcpyAsync(dst, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, c->stream));
    const int n = (int)items.size();
    CK(cudaMemcpyAsync(c->d_counts + which, &n, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

std::vector<int2> box_items_of(const lb_ctx* c, int k) {
    std::vector<int2> v;
    for (int g = 0; g < c->par[k].g_box; ++g) v.push_back(make_int2(k, g));
    return v;
}

// Rebuild every link list (no conversion) and commit the owners, as if after a
// step of parity 1 - cur (the next sweep has parity cur).
lb_status relink_all(lb_ctx* c) {
    const int nb = (int)c->par.size();
    const int cur = (int)(c->step & 1);
    std::vector<int2> all;
    for (int k = 0; k < nb; ++k) {
        auto v = box_items_of(c, k);
        all.insert(all.end(), v.begin(), v.end());
    }
    lb_status s = set_list(c, 2, all);
    if (s != LB_OK) return s;
    Bodies B = bodies_view(c);
    if (c->split) B.win = win_slot(c, c->step + 1);  // the first split sweep, of step + 1
    launch_set_flags(c->d_acc, nb, -1, 0, c->stream);
    launch_body_kernel(3, B, 1 - cur, 1, c->grid_box, nullptr, c->stream);
    launch_body_kernel(4, B, 1 - cur, 1, c->grid_box, nullptr, c->stream);
    c->launches += 3;
    CK(cudaMemcpyAsync(c->own_prev, c->own, sizeof(int32_t) * c->L.N, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaGetLastError());
    return sync_checked(c);
}

lb_status new_body(lb_ctx* c, const BodyParams& bp, const BodyState& st, int kind_code, int32_t* id_out) {
    const int nb = (int)c->par.size();
    lb_status s = ensure_body_capacity(c, nb + 1);
    if (s != LB_OK) return s;
    CK(cudaMemcpyAsync(c->d_par + nb, &bp, sizeof(BodyParams), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_state[0] + nb, &st, sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_state[1] + nb, &st, sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_acc + nb, 0, sizeof(BodyAcc), c->stream));
    CK(cudaMemcpyAsync(c->d_kind + nb, &kind_code, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    c->par.push_back(bp);
    c->kind.push_back(kind_code);
    *id_out = nb + 1;
    return LB_OK;
}

// Round tube along z (lb_add_wall kind 3).
lb_status add_round_tube(lb_ctx* c, const double* params, int32_t nparams, int32_t* id) {
    if (!params || nparams != 3) return fail(c, LB_ERR_INVALID, "round tube needs cx, cy, radius");
    const double cx = params[0], cy = params[1], r = params[2];
    if (!(r > 1.0) || !(cx >= 0.0) || !(cy >= 0.0) || !(cx <= c->L.nx - 1) || !(cy <= c->L.ny - 1))
        return fail(c, LB_ERR_INVALID, "round tube: radius > 1 and the axis inside the box");
    BodyParams bp{};
    bp.kind = BODY_WALL;
    bp.mobile = 0;
    bp.wall_axis = -1;
    bp.tube[0] = cx;
    bp.tube[1] = cy;
    bp.tube[2] = r;
    CK(cudaMemsetAsync(c->d_count, 0, sizeof(int), c->stream));
    if (!c->par.empty()) {
        launch_tube_overlap(c->L, c->own, c->d_kind, bp, c->d_count, c->stream);
        c->launches += 1;
    }
    int hcount = 0;
    CK(cudaMemcpyAsync(&hcount, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hcount != 0) return fail(c, LB_ERR_OVERLAP, "the tube overlaps a sphere");
    // links: the fluid nodes next to the solid, about 10 per unit of
    // circumference and plane at most
    bp.link_cap = (int64_t)(10.0 * (6.2832 * r + 16.0)) * c->L.nz + 64;
    bp.box_w[0] = c->L.nx;
    bp.box_w[1] = c->L.ny;
    bp.box_w[2] = c->L.nz;
    BodyState st{};  // a tube has no position, velocity or orientation of its own
    int32_t nid = 0;
    lb_status s = new_body(c, bp, st, BODY_WALL, &nid);
    if (s != LB_OK) return s;
    launch_tube_claim(c->L, c->own, bp, nid, c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    s = relayout(c);
    if (s == LB_OK) s = relink_all(c);
    if (s != LB_OK) return s;
    *id = nid;
    return LB_OK;
}

}  // namespace

extern "C" {

static void settle(lb_ctx* c);  // issues pending body kernels (defined with lb_step)

void lb_params_default(lb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 32;
    p->collision = LB_BGK;
    p->lambda_e = 1.0;
    p->magic = 3.0 / 16.0;
    p->rho0 = 1.0;
    p->storage = LB_F64;
    p->dev_scale_log2 = -1;
    p->device = 0;
    p->stream = nullptr;
    p->allocator = nullptr;
    p->equilibrium = LB_EQ_COMPRESSIBLE;
    p->rounding = LB_ROUND_DEFAULT;
}

lb_status lb_create(const lb_params* p, lb_ctx** out) {
    if (!p || !out) return LB_ERR_INVALID;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || N >= (int64_t(1) << 27)) return LB_ERR_INVALID;
    if (!(p->lambda_e > 0.0 && p->lambda_e < 2.0) || !(p->rho0 > 0.0)) return LB_ERR_INVALID;
    if (p->collision != LB_BGK && p->collision != LB_TRT) return LB_ERR_INVALID;
    if (p->storage < LB_F64 || p->storage > LB_BF16DEV) return LB_ERR_INVALID;
    if (p->collision == LB_TRT && !(p->magic > 0.0)) return LB_ERR_INVALID;
    if (p->dev_scale_log2 < -1 || p->dev_scale_log2 > 40) return LB_ERR_INVALID;
    if (p->equilibrium != LB_EQ_COMPRESSIBLE && p->equilibrium != LB_EQ_INCOMPRESSIBLE) return LB_ERR_INVALID;
    if (p->rounding < LB_ROUND_DEFAULT || p->rounding > LB_ROUND_STOCHASTIC) return LB_ERR_INVALID;
    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ERR_OOM;
    c->p = *p;
    auto bail = [&](lb_status s) {
        lb_destroy(c);
        return s;
    };
    if (cudaSetDevice(p->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(LB_ERR_CUDA);
    }
    if (prepare_body_kernels() != cudaSuccess) {
        cudaGetLastError();
        return bail(LB_ERR_CUDA);
    }
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(LB_ERR_CUDA);
        c->own_stream = true;
    }
    c->lambda_e = p->lambda_e;
    // TRT odd rate from the magic parameter (1/le - 1/2)(1/lo - 1/2) = magic (Sec. III)
    c->lambda_o = p->collision == LB_BGK ? p->lambda_e : 1.0 / (0.5 + p->magic / (1.0 / p->lambda_e - 0.5));
    Lattice& L = c->L;
    L.nx = p->nx;
    L.ny = p->ny;
    L.nz = p->nz;
    L.N = N;
    L.Np = (N + 63) / 64 * 64;
    L.storage = p->storage;
    L.inc = p->equilibrium == LB_EQ_INCOMPRESSIBLE ? 1 : 0;
    L.rho0 = p->rho0;
    // FP16 deviation scale: 2^14 keeps deviations up to 4 representable and
    // the usual 1e-5 .. 1e-2 in FP16's normal range
    const int k = p->dev_scale_log2 < 0 ? 14 : p->dev_scale_log2;
    L.scale = p->storage == LB_F16DEV ? std::ldexp(1.0f, k) : 1.0f;
    L.inv_scale = 1.0f / L.scale;
    L.sr = p->storage == LB_BF16DEV && p->rounding != LB_ROUND_NEAREST ? 1 : 0;
    L.rho_local = 0;
    L.link_at = 0.5f;
    L.F = dalloc(c, (size_t)Q * L.Np * storage_bytes(p->storage));
    L.sr_ctr = dalloc_t<unsigned long long>(c, 2);
    c->own = dalloc_t<int32_t>(c, (size_t)N);
    c->own_prev = dalloc_t<int32_t>(c, (size_t)N);
    c->d_mass_part = dalloc_t<double>(c, (size_t)mass_partial_blocks(L) * 4);
    c->d_small = dalloc_t<double>(c, 8);
    c->d_err = dalloc_t<int>(c, 2);
    c->d_count = dalloc_t<int>(c, 2);
    c->d_lat = dalloc_t<Lattice>(c, 1);
    c->d_counts = dalloc_t<int>(c, 11);
    c->d_win = dalloc_t<int>(c, 16);
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) return bail(LB_ERR_CUDA);
    if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_started, cudaEventDisableTiming) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    if (!L.F || !c->own || !c->own_prev || !c->d_mass_part || !c->d_small || !c->d_err || !c->d_count ||
        !c->d_lat || !c->d_counts || !c->d_win)
        return bail(LB_ERR_OOM);
    L.own = c->own;
    L.own_prev = c->own_prev;
    L.err = c->d_err;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) c->n_sm = 152;
    if (cudaMemsetAsync(c->d_counts, 0, sizeof(int) * 4, c->stream) != cudaSuccess) return bail(LB_ERR_CUDA);
    if (upload_lattice(c) != LB_OK) return bail(LB_ERR_CUDA);
    if (cudaMemsetAsync(c->own, 0, sizeof(int32_t) * N, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->own_prev, 0, sizeof(int32_t) * N, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_err, 0, sizeof(int) * 2, c->stream) != cudaSuccess ||
        cudaMemsetAsync(L.sr_ctr, 0, sizeof(unsigned long long) * 2, c->stream) != cudaSuccess)
        return bail(LB_ERR_CUDA);
    launch_fill_rest(L, c->stream);
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(LB_ERR_CUDA);
    *out = c;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx* c) {
    if (!c) return LB_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    if (c->ev_started) cudaEventDestroy(c->ev_started);
    for (cudaStream_t st : {c->side, c->hi})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    while (!c->allocs.empty()) dfree(c, c->allocs.back().first);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->msg.c_str() : "null context"; }
int64_t lb_step_count(const lb_ctx* c) { return c ? c->step : -1; }
int64_t lb_kernel_launches(const lb_ctx* c) { return c ? c->launches : -1; }

lb_status lb_add_squirmer(lb_ctx* c, const double pos[3], const double e[3], double R, double B1, double beta,
                          int32_t mobile, double density, int32_t* id) {
    if (!c || !pos || !e || !id) return LB_ERR_INVALID;
    if (c->sticky) return fail(c, LB_ERR_STATE, "context holds a device error");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const int nmin = std::min(c->L.nx, std::min(c->L.ny, c->L.nz));
    const double ne = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (!(R > 0.0) || !(2.0 * R + 6.0 < (double)nmin)) return fail(c, LB_ERR_INVALID, "radius vs box");
    if (!(ne > 0.0) || !std::isfinite(ne)) return fail(c, LB_ERR_INVALID, "orientation");
    if (!(density > 0.0) || !std::isfinite(B1) || !std::isfinite(beta)) return fail(c, LB_ERR_INVALID, "parameters");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(pos[a])) return fail(c, LB_ERR_INVALID, "position");
    CK(cudaSetDevice(c->p.device));
    const int n3[3] = {c->L.nx, c->L.ny, c->L.nz};
    BodyState st{};
    for (int a = 0; a < 3; ++a) {
        st.pos[a] = pos[a] - std::floor(pos[a] / n3[a]) * n3[a];
        st.e[a] = e[a] / ne;
    }
    const int W = (int)std::ceil(2.0 * R) + 6;
    if (c->psm) {
        // partially saturated cells: the sphere claims no cell and has no
        // links; its cells are found at the start of every step
        BodyParams bp{};
        bp.kind = BODY_SPHERE;
        bp.psm = 1;
        bp.mobile = mobile ? 1 : 0;
        bp.R = R;
        bp.B1 = B1;
        bp.B2 = beta * B1;
        bp.mass = density * (4.0 / 3.0) * M_PI * R * R * R;
        bp.inertia = 0.4 * bp.mass * R * R;
        bp.inv_mass = 1.0 / bp.mass;
        bp.inv_inertia = 1.0 / bp.inertia;
        bp.link_cap = 0;
        bp.box_w[0] = bp.box_w[1] = bp.box_w[2] = W;
        int32_t nid = 0;
        lb_status s = new_body(c, bp, st, BODY_SPHERE, &nid);
        if (s == LB_OK) s = relayout(c);
        if (s != LB_OK) return s;
        *id = nid;
        return LB_OK;
    }
    // overlap check before anything changes
    CK(cudaMemsetAsync(c->d_count, 0, sizeof(int), c->stream));
    CK(cudaMemcpyAsync(c->d_small, st.pos, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_sphere_overlap(c->L, c->own, st.pos, R, W, c->d_count, c->stream);
    c->launches += 1;
    int hcount = 0;
    CK(cudaMemcpyAsync(&hcount, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hcount != 0) return fail(c, LB_ERR_OVERLAP, "the sphere overlaps a solid cell");
    BodyParams bp{};
    bp.kind = BODY_SPHERE;
    bp.mobile = mobile ? 1 : 0;
    bp.R = R;
    bp.B1 = B1;
    bp.B2 = beta * B1;
    bp.mass = density * (4.0 / 3.0) * M_PI * R * R * R;
    bp.inertia = 0.4 * bp.mass * R * R;
    bp.inv_mass = 1.0 / bp.mass;
    bp.inv_inertia = 1.0 / bp.inertia;
    bp.link_cap = sphere_link_cap(R);
    bp.box_w[0] = bp.box_w[1] = bp.box_w[2] = W;
    int32_t nid = 0;
    lb_status s = new_body(c, bp, st, BODY_SPHERE, &nid);
    if (s != LB_OK) return s;
    s = relayout(c);
    if (s != LB_OK) return s;
    // claim the covered cells and record the node margin with a classify pass
    // "after a step of parity 1 - cur" (it reads state[cur])
    const int nb = (int)c->par.size();
    const int cur = (int)(c->step & 1);
    s = set_list(c, 1, box_items_of(c, nid - 1));
    if (s != LB_OK) return s;
    launch_set_flags(c->d_acc, nb, -1, 0, c->stream);
    launch_set_flags(c->d_acc, nb, nid - 1, 2, c->stream);  // whole box
    Bodies B = bodies_view(c);
    launch_body_kernel(2, B, 1 - cur, 1, c->grid_box, nullptr, c->stream);
    launch_body_kernel(5, B, 1 - cur, 1, 1, nullptr, c->stream);
    c->launches += 4;
    CK(cudaGetLastError());
    s = relink_all(c);
    if (s != LB_OK) return s;
    *id = nid;
    return LB_OK;
}

lb_status lb_add_wall(lb_ctx* c, int32_t kind, const double* params, int32_t nparams, int32_t* id) {
    if (!c || !id) return LB_ERR_INVALID;
    if (c->sticky) return fail(c, LB_ERR_STATE, "context holds a device error");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const int n3[3] = {c->L.nx, c->L.ny, c->L.nz};
    if (kind == 2) {
        if (!params || nparams < 4) return fail(c, LB_ERR_INVALID, "obstacle needs x, y, z, radius");
        const double e[3] = {0.0, 0.0, 1.0};
        return lb_add_squirmer(c, params, e, params[3], 0.0, 0.0, 0, 1.0, id);
    }
    if (kind == 3) return add_round_tube(c, params, nparams, id);
    if (kind == 1) {
        // square tube along z: plane walls x = 0, x = nx-1, y = 0, y = ny-1
        const double walls[4][2] = {{0, 0}, {0, (double)(n3[0] - 1)}, {1, 0}, {1, (double)(n3[1] - 1)}};
        int32_t first = 0;
        for (int w = 0; w < 4; ++w) {
            int32_t wid = 0;
            lb_status s = lb_add_wall(c, 0, walls[w], 2, &wid);
            if (s != LB_OK) return s;
            if (w == 0) first = wid;
        }
        *id = first;
        return LB_OK;
    }
    if (kind != 0 || !params || (nparams != 2 && nparams != 5)) return fail(c, LB_ERR_INVALID, "wall kind/params");
    const int axis = (int)params[0], index = (int)params[1];
    if (params[0] != axis || params[1] != index || axis < 0 || axis > 2 || index < 0 || index >= n3[axis])
        return fail(c, LB_ERR_INVALID, "plane wall axis/index");
    CK(cudaMemsetAsync(c->d_count, 0, sizeof(int), c->stream));
    if (!c->par.empty()) {
        launch_plane_overlap(c->L, c->own, c->d_kind, axis, index, c->d_count, c->stream);
        c->launches += 1;
    }
    int hcount = 0;
    CK(cudaMemcpyAsync(&hcount, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hcount != 0) return fail(c, LB_ERR_OVERLAP, "the wall overlaps a sphere");
    BodyParams bp{};
    bp.kind = BODY_WALL;
    bp.mobile = 0;
    bp.wall_axis = axis;
    bp.wall_index = index;
    if (nparams == 5)
        for (int a = 0; a < 3; ++a) bp.wall_vel[a] = params[2 + a];
    const int64_t area = c->L.N / n3[axis];
    bp.link_cap = 10 * area + 64;
    for (int a = 0; a < 3; ++a) bp.box_w[a] = n3[a];
    bp.box_w[axis] = std::min(3, n3[axis]);
    BodyState st{};  // a wall has no position, velocity or orientation of its own
    int32_t nid = 0;
    lb_status s = new_body(c, bp, st, BODY_WALL, &nid);
    if (s != LB_OK) return s;
    launch_plane_claim(c->L, c->own, axis, index, nid, c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    s = relayout(c);
    if (s == LB_OK) s = relink_all(c);
    if (s != LB_OK) return s;
    *id = nid;
    return LB_OK;
}

lb_status lb_set_contact(lb_ctx* c, double sigma, double eps) {
    if (!c || !(sigma > 0.0) || !(eps >= 0.0)) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    c->wca_sigma = sigma;
    c->wca_eps = eps;
    drop_graph(c);
    CK(cudaSetDevice(c->p.device));
    lb_status s = upload_lattice(c);
    if (s != LB_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_coupling(lb_ctx* c, int32_t coupling) {
    if (!c || (coupling != LB_COUPLE_LINKS && coupling != LB_COUPLE_PSM)) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const bool want = coupling == LB_COUPLE_PSM;
    if (want == c->psm) return LB_OK;
    for (const BodyParams& b : c->par)
        if (b.kind == BODY_SPHERE) return fail(c, LB_ERR_INVALID, "set the coupling before adding spheres");
    if (want && !c->d_eps) {
        c->d_eps = dalloc_t<float>(c, (size_t)c->L.N);
        c->d_psm_id = dalloc_t<int32_t>(c, (size_t)c->L.N);
        if (!c->d_eps || !c->d_psm_id) return fail(c, LB_ERR_OOM, "solid fractions");
        CK(cudaMemsetAsync(c->d_eps, 0, sizeof(float) * c->L.N, c->stream));
        CK(cudaMemsetAsync(c->d_psm_id, 0, sizeof(int32_t) * c->L.N, c->stream));
    }
    c->psm = want;
    c->L.psm = want ? 1 : 0;
    c->L.eps = c->d_eps;
    c->L.psm_id = c->d_psm_id;
    lb_status s = relayout(c);
    if (s != LB_OK) return s;
    return LB_OK;
}

lb_status lb_get_solid_fraction(lb_ctx* c, double* eps) {
    if (!c || !eps) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    const size_t N = (size_t)c->L.N;
    if (!c->psm) {
        std::fill(eps, eps + N, 0.0);
        return LB_OK;
    }
    std::vector<float> h(N);
    CK(cudaMemcpyAsync(h.data(), c->d_eps, sizeof(float) * N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t n = 0; n < N; ++n) eps[n] = (double)h[n];
    return LB_OK;
}

lb_status lb_set_link_options(lb_ctx* c, int32_t density_of_node, int32_t velocity_at_node) {
    if (!c || (density_of_node != 0 && density_of_node != 1) || (velocity_at_node != 0 && velocity_at_node != 1))
        return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    c->L.rho_local = density_of_node;
    c->L.link_at = velocity_at_node ? 1.0f : 0.5f;
    drop_graph(c);
    lb_status s = upload_lattice(c);
    if (s != LB_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_force_average(lb_ctx* c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    c->force_avg = on;
    drop_graph(c);
    lb_status s = upload_lattice(c);
    if (s != LB_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

static lb_status ensure_scratch(lb_ctx* c, double** buf, size_t n) {
    if (*buf) return LB_OK;
    *buf = dalloc_t<double>(c, n);
    return *buf ? LB_OK : fail(c, LB_ERR_OOM, "export buffer");
}

lb_status lb_set_fields(lb_ctx* c, const double* rho, const double* u) {
    if (!c || !rho || !u) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const size_t N = (size_t)c->L.N;
    lb_status s = ensure_scratch(c, &c->d_fields, 4 * N);
    if (s != LB_OK) return s;
    CK(cudaMemcpyAsync(c->d_fields, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fields + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_set_eq(c->L, c->d_fields, c->d_fields + N, (int)(c->step & 1), c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_populations(lb_ctx* c, const double* f) {
    if (!c || !f) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const size_t N = (size_t)c->L.N;
    lb_status s = ensure_scratch(c, &c->d_pop, Q * N);
    if (s != LB_OK) return s;
    CK(cudaMemcpyAsync(c->d_pop, f, Q * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_set_pop(c->L, c->d_pop, (int)(c->step & 1), c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_get_populations(lb_ctx* c, double* f) {
    if (!c || !f) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const size_t N = (size_t)c->L.N;
    lb_status s = ensure_scratch(c, &c->d_pop, Q * N);
    if (s != LB_OK) return s;
    launch_get_pop(c->L, c->d_pop, (int)(c->step & 1), c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(f, c->d_pop, Q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sync_checked(c);
}

static cudaEvent_t pool_event(lb_ctx* c, size_t k) {
    while (c->ev_pool.size() <= k) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[k];
}

static void sweep_all(lb_ctx* c, int parity, cudaStream_t st) {
    launch_sweep(c->L, c->lambda_e, c->lambda_o, parity, c->sweep_variant, 0, nullptr, c->L.nz, c->L.ny, st);
}

// The sweep of a lattice with partially saturated cells: before it the
// solid fractions, the covered cells' collisions and each sphere's force and
// update (from the populations the step starts from); after it the covered
// cells' results over the sweep's.  Returns the launch count.
static int psm_sweep(lb_ctx* c, const Bodies& B, int parity, cudaStream_t st) {
    if (c->n_psm_items == 0) {
        sweep_all(c, parity, st);
        return 1;
    }
    launch_psm_cover(B, parity, c->grid_psm, c->p.storage == LB_F64, st);
    sweep_all(c, parity, st);
    launch_psm_scatter(B, parity, c->grid_psm, st);
    return 4;
}

// The body kernels of one step on stream st: the fused kernel (spheres), the
// link kernel (walls and still obstacles, if any), then classify, convert and
// rebuild, which re-classify the spheres queued by the other two (bodies near
// another body) and end the step; for a lattice with a single sphere and no
// other body, the fused kernel alone.  Returns the launch count.
// started: recorded when every block of the fused kernel has begun (if it is
// launched: c->solo or c->n_fused > 0).
static int body_step(lb_ctx* c, const Bodies& B, int parity, cudaStream_t st, cudaEvent_t started = nullptr) {
    if (c->solo) {  // the fused kernel is the whole body step
        launch_body_fused(B, parity, c->fused_cls, 1, st, 1, started);
        return 1;
    }
    int n = 0;
    if (c->n_fused > 0) {
        launch_body_fused(B, parity, c->fused_cls, c->n_fused, st, 0, started);
        n++;
    }
    if (c->n_link_items > 0) {
        launch_body_kernel(1, B, parity, c->n_link_items, c->grid_box, nullptr, st);
        n++;
    }
    for (int which = 2; which <= 4; ++which) launch_body_kernel(which, B, parity, c->n_link_items, c->grid_box, nullptr, st);
    return n + 3;
}

// Traced step: each kernel between its own pair of events, no overlap.
static void enqueue_traced_step(lb_ctx* c) {
    const int parity = (int)(c->step & 1);
    const int nk = c->par.empty() ? 1 : 5;
    const bool psm = c->psm && c->n_psm_items > 0;
    if (psm) {  // kind 1: solid fractions, covered cells, sphere forces
        const size_t e0 = 2 * c->ev_used.size();
        cudaEventRecord(pool_event(c, e0), c->stream);
        launch_psm_cover(bodies_view(c), parity, c->grid_psm, c->p.storage == LB_F64, c->stream);
        c->launches += 2;
        cudaEventRecord(pool_event(c, e0 + 1), c->stream);
        c->ev_used.emplace_back(1, (int)e0);
    }
    for (int k = 0; k < nk; ++k) {
        if (k == 1 && psm) {  // kind 1: the covered cells' results
            const size_t e0 = 2 * c->ev_used.size();
            cudaEventRecord(pool_event(c, e0), c->stream);
            launch_psm_scatter(bodies_view(c), parity, c->grid_psm, c->stream);
            c->launches += 1;
            cudaEventRecord(pool_event(c, e0 + 1), c->stream);
            c->ev_used.emplace_back(1, (int)e0);
        }
        const size_t e0 = 2 * c->ev_used.size();
        cudaEventRecord(pool_event(c, e0), c->stream);
        if (k == 0) {
            sweep_all(c, parity, c->stream);
            c->launches += 1;
        } else if (k == 1) {
            const Bodies B = bodies_for_step(c, c->step);
            if (c->n_fused > 0) {
                launch_body_fused(B, parity, c->fused_cls, c->n_fused, c->stream, 0);
                c->launches += 1;
            }
            if (c->n_link_items > 0) {
                launch_body_kernel(1, B, parity, c->n_link_items, c->grid_box, nullptr, c->stream);
                c->launches += 1;
            }
        } else {
            launch_body_kernel(k, bodies_for_step(c, c->step), parity, c->n_link_items, c->grid_box, nullptr,
                               c->stream);
            c->launches += 1;
        }
        cudaEventRecord(pool_event(c, e0 + 1), c->stream);
        c->ev_used.emplace_back(k, (int)e0);
    }
    c->step++;
}

// n whole steps on the context's stream (the sweep, then the body kernels).
static void enqueue_steps(lb_ctx* c, int64_t n) {
    const bool bodies = !c->par.empty();
    const Bodies B = bodies_view(c);
    for (int64_t k = 0; k < n; ++k) {
        const int parity = (int)(c->step & 1);
        if (c->psm) {
            c->launches += psm_sweep(c, B, parity, c->stream);
        } else {
            sweep_all(c, parity, c->stream);
            c->launches += 1;
        }
        if (bodies) c->launches += body_step(c, B, parity, c->stream);
        c->step++;
    }
}

// When the bodies occupy a thin box of rows, steps run as a pipeline of
// units on two chains.  Unit t issues the body kernels of step t (whose sweep
// is done) and the near sweep of step t+1 (the window) on `hi`, and the far
// sweep of step t+1 (every cell outside the window) on `side`.
//   - near(t+1) waits for body(t) (stream order) and far(t): a sweep's cells
//     touch only their own slots, so it does not wait for far(t+1);
//   - far(t+1) waits for far(t) (stream order) and near(t), and for the
//     clusters of body(t) to be placed (see below), not for body(t) to end:
//     the window of step t+1, computed two steps ahead with two cells to
//     spare, holds every cell the body kernels of steps t and t+1 touch.
// The far sweeps run back to back and set the pace; body and near sweep run
// beside them.  After a unit the body kernels of step t+1 are pending:
// lb_step returns with them pending, so that consecutive calls keep the
// overlap, and every call that reads or changes the context issues them
// first (settle).

// Start of a run of units: both chains wait for everything issued so far.
static void begin_units(lb_ctx* c) {
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    cudaStreamWaitEvent(c->hi, c->ev_fork, 0);
    cudaEventRecord(c->ev_join, c->stream);   // "the last far sweep"
    cudaEventRecord(c->ev_join2, c->stream);  // "the last near sweep"
}

static void enqueue_unit(lb_ctx* c) {
    const int64_t t = c->step - 1;
    const int parity = (int)(t & 1), q = 1 - parity;
    const int* win = win_slot(c, t + 1);
    // the far sweep starts once the fused kernel's clusters are placed: started
    // first, it would fill every SM, and a cluster waits for SMs of one GPC to
    // drain together
    const bool fused = c->solo || c->n_fused > 0;
    c->launches += body_step(c, bodies_for_step(c, t), parity, c->hi, fused ? c->ev_started : nullptr);
    cudaStreamWaitEvent(c->hi, c->ev_join, 0);  // far(t), before near(t+1)
    if (fused) cudaStreamWaitEvent(c->side, c->ev_started, 0);
    cudaStreamWaitEvent(c->side, c->ev_join2, 0);  // near(t), before far(t+1)
    launch_sweep(c->L, c->lambda_e, c->lambda_o, q, c->sweep_variant, 1, win, c->L.nz, c->L.ny, c->side);
    cudaEventRecord(c->ev_join, c->side);
    launch_sweep(c->L, c->lambda_e, c->lambda_o, q, c->sweep_variant, 2, win, c->win_max, c->ywin_max, c->hi);
    cudaEventRecord(c->ev_join2, c->hi);
    c->launches += 2;
    c->step++;
}

// End of a run of units: the context's stream waits for both chains.
static void end_units(lb_ctx* c) {
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    cudaStreamWaitEvent(c->stream, c->ev_join2, 0);
}

// Issue the pending body kernels, if any: the context then holds whole steps.
static void settle(lb_ctx* c) {
    if (!c->pending) return;
    c->launches += body_step(c, bodies_for_step(c, c->step - 1), (int)((c->step - 1) & 1), c->stream);
    c->pending = false;
}

constexpr int kGraphSteps = 8;

static lb_status build_graph(lb_ctx* c, int which) {
    cudaGraph_t g = nullptr;
    const int64_t saved_launches = c->launches, saved_step = c->step;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    if (c->split) {
        c->step = 2 + 2 * which;  // 8 units from t = 1 or 3 (the window slots repeat every 4 steps)
        begin_units(c);
        for (int k = 0; k < kGraphSteps; ++k) enqueue_unit(c);
        end_units(c);
    } else {
        c->step = 0;  // 8 steps from an even step
        enqueue_steps(c, kGraphSteps);
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->graph_launches = c->launches - saved_launches;
    c->launches = saved_launches;
    c->step = saved_step;
    if (e != cudaSuccess) return cuda_fail(c, e, "capture");
    e = cudaGraphInstantiate(&c->graph[which], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[which] = nullptr;
        return cuda_fail(c, e, "instantiate");
    }
    return LB_OK;
}

lb_status lb_step(lb_ctx* c, int64_t nsteps) {
    if (!c || nsteps < 0) return LB_ERR_INVALID;
    if (c->sticky) return fail(c, LB_ERR_STATE, "context holds a device error");
    CK(cudaSetDevice(c->p.device));
    if (c->profiling) {
        for (int64_t k = 0; k < nsteps; ++k) enqueue_traced_step(c);
        CK(cudaGetLastError());
        return LB_OK;
    }
    int64_t left = nsteps;
    if (c->split) {
        if (left > 0 && !c->pending) {
            sweep_all(c, (int)(c->step & 1), c->stream);
            c->launches += 1;
            c->step++;
            c->pending = true;
            left--;
        }
        if (left > 0 && ((c->step - 1) & 1) == 0) {  // graphs start on a unit of odd t
            begin_units(c);
            enqueue_unit(c);
            end_units(c);
            left--;
        }
    } else if (left > 0 && (c->step & 1)) {  // graphs start on even steps
        enqueue_steps(c, 1);
        left--;
    }
    if (left >= kGraphSteps) {
        // split lattices: t = step - 1 is odd here; t = 3 (mod 4) takes graph 1
        const int which = c->split ? (int)(((c->step - 1) >> 1) & 1) : 0;
        if (!c->graph[which]) {
            lb_status s = build_graph(c, which);
            if (s != LB_OK) return s;
        }
        while (left >= kGraphSteps) {
            CK(cudaGraphLaunch(c->graph[which], c->stream));
            c->launches += c->graph_launches;
            c->step += kGraphSteps;
            left -= kGraphSteps;
        }
    }
    if (c->split && left > 0) {
        begin_units(c);
        for (; left > 0; --left) enqueue_unit(c);
        end_units(c);
    } else if (left > 0) {
        enqueue_steps(c, left);
    }
    CK(cudaGetLastError());
    return LB_OK;
}

lb_status lb_set_sweep_variant(lb_ctx* c, int32_t variant) {
    if (!c || variant < 0 || variant > 3) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    c->sweep_variant = variant;
    drop_graph(c);
    return LB_OK;
}

lb_status lb_profile_begin(lb_ctx* c) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    c->profiling = true;
    c->ev_used.clear();
    return LB_OK;
}

lb_status lb_profile_end(lb_ctx* c, double total_ms[6], int64_t launches[6]) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    c->profiling = false;
    lb_status s = sync_checked(c);
    double t[6] = {0, 0, 0, 0, 0, 0};
    int64_t n[6] = {0, 0, 0, 0, 0, 0};
    for (auto& u : c->ev_used) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[u.second], c->ev_pool[u.second + 1]) == cudaSuccess) {
            t[u.first] += ms;
            n[u.first] += 1;
        }
    }
    c->ev_used.clear();
    if (s != LB_OK) return s;
    for (int k = 0; k < 6; ++k) {
        if (total_ms) total_ms[k] = t[k];
        if (launches) launches[k] = n[k];
    }
    return LB_OK;
}

lb_status lb_sync(lb_ctx* c) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    return sync_checked(c);
}

lb_status lb_get_fields_device(lb_ctx* c, double* rho_dev, double* u_dev) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    launch_fields(c->L, c->own, rho_dev, u_dev, (int)(c->step & 1), c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    return LB_OK;
}

lb_status lb_get_fields(lb_ctx* c, double* rho, double* u) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    const size_t N = (size_t)c->L.N;
    lb_status s = ensure_scratch(c, &c->d_fields, 4 * N);
    if (s != LB_OK) return s;
    launch_fields(c->L, c->own, c->d_fields, c->d_fields + N, (int)(c->step & 1), c->stream);
    c->launches += 1;
    CK(cudaGetLastError());
    s = sync_checked(c);
    if (s != LB_OK) return s;
    if (rho) CK(cudaMemcpyAsync(rho, c->d_fields, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u) CK(cudaMemcpyAsync(u, c->d_fields + N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_get_owner(lb_ctx* c, int32_t* owner) {
    if (!c || !owner) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    CK(cudaMemcpyAsync(owner, c->own, sizeof(int32_t) * c->L.N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

static lb_status read_acc(lb_ctx* c, int32_t id, BodyAcc* a) {
    if (id < 1 || id > (int32_t)c->par.size()) return fail(c, LB_ERR_INVALID, "bad body id");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    CK(cudaMemcpyAsync(a, c->d_acc + (id - 1), sizeof(BodyAcc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_get_force_torque(lb_ctx* c, int32_t id, double F[3], double T[3]) {
    if (!c || !F || !T) return LB_ERR_INVALID;
    BodyAcc a;
    lb_status s = read_acc(c, id, &a);
    if (s != LB_OK) return s;
    for (int k = 0; k < 3; ++k) {
        F[k] = a.Fapp[k];
        T[k] = a.Tapp[k];
    }
    return LB_OK;
}

lb_status lb_get_stresslet(lb_ctx* c, int32_t id, double S[6]) {
    if (!c || !S) return LB_ERR_INVALID;
    BodyAcc a;
    lb_status s = read_acc(c, id, &a);
    if (s != LB_OK) return s;
    for (int k = 0; k < 6; ++k) S[k] = a.Sbb[k];
    return LB_OK;
}

lb_status lb_get_object_state(lb_ctx* c, int32_t id, double pos[3], double vel[3], double e[3], double omega[3]) {
    if (!c) return LB_ERR_INVALID;
    if (id < 1 || id > (int32_t)c->par.size()) return fail(c, LB_ERR_INVALID, "bad body id");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    BodyState st;
    CK(cudaMemcpyAsync(&st, c->d_state[c->step & 1] + (id - 1), sizeof(BodyState), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) {
        if (pos) pos[k] = st.pos[k];
        if (vel) vel[k] = st.vel[k];
        if (e) e[k] = st.e[k];
        if (omega) omega[k] = st.omega[k];
    }
    return LB_OK;
}

lb_status lb_get_mass(lb_ctx* c, double* mass, double mom[3]) {
    if (!c) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    launch_mass(c->L, c->own, c->d_mass_part, c->d_small, (int)(c->step & 1), c->stream);
    c->launches += 2;
    CK(cudaGetLastError());
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    double h[4];
    CK(cudaMemcpyAsync(h, c->d_small, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (mass) *mass = h[0];
    if (mom)
        for (int k = 0; k < 3; ++k) mom[k] = h[1 + k];
    return LB_OK;
}

lb_status lb_get_links(lb_ctx* c, int32_t id, int64_t* out, int64_t cap, int64_t* count) {
    if (!c || !count || cap < 0 || (cap > 0 && !out)) return LB_ERR_INVALID;
    if (id < 0 || id > (int32_t)c->par.size()) return fail(c, LB_ERR_INVALID, "bad body id");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    const int nb = (int)c->par.size();
    std::vector<BodyAcc> acc(nb);
    if (nb) CK(cudaMemcpyAsync(acc.data(), c->d_acc, sizeof(BodyAcc) * nb, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t n = 0;
    std::vector<uint32_t> buf;
    for (int k = 0; k < nb; ++k) {
        if (id != 0 && k != id - 1) continue;
        const int64_t m = acc[k].link_count;
        buf.resize((size_t)m);
        if (m) {
            CK(cudaMemcpyAsync(buf.data(), c->d_links + c->par[k].link_off, m * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        for (int64_t l = 0; l < m; ++l, ++n)
            if (n < cap) out[n] = (int64_t)buf[(size_t)l];
    }
    *count = n;
    return LB_OK;
}


// ---------------------------------------------------------------- checkpoint

namespace {

constexpr char kCkptMagic[8] = {'L', 'B', 'S', 'Q', 'C', 'K', 'P', '1'};

struct CkptHeader {
    char magic[8];
    uint32_t version, storage;
    int32_t nx, ny, nz, nbodies;
    int32_t equilibrium, reserved;  // reserved: Lattice::sr (the rounding of BF16 stores)
    double lambda_e, lambda_o, rho0;
    double scale;
    int64_t step;
    uint64_t bodies_hash;  // the bodies' defining parameters (see bodies_hash)
    uint64_t bytes;        // the whole checkpoint
};

// FNV-1a over the parameters that define the bodies (not the derived layout).
uint64_t bodies_hash(const lb_ctx* c) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ull;
    };
    for (size_t k = 0; k < c->par.size(); ++k) {
        const BodyParams& q = c->par[k];
        mix(&c->kind[k], sizeof(int));
        mix(&q.kind, sizeof(q.kind));
        mix(&q.mobile, sizeof(q.mobile));
        mix(&q.R, sizeof(q.R));
        mix(&q.B1, sizeof(q.B1));
        mix(&q.B2, sizeof(q.B2));
        mix(&q.mass, sizeof(q.mass));
        mix(&q.inertia, sizeof(q.inertia));
        mix(q.wall_vel, sizeof(q.wall_vel));
        mix(&q.wall_axis, sizeof(q.wall_axis));
        mix(&q.wall_index, sizeof(q.wall_index));
        mix(q.tube, sizeof(q.tube));
        mix(&q.psm, sizeof(q.psm));
    }
    mix(&c->wca_sigma, sizeof(double));
    mix(&c->wca_eps, sizeof(double));
    return h;
}

size_t pop_bytes(const lb_ctx* c) { return (size_t)Q * c->L.Np * storage_bytes(c->p.storage); }

// The bodies' accumulators (link counts included), read after the step work.
lb_status read_accs(lb_ctx* c, std::vector<BodyAcc>& acc) {
    acc.resize(c->par.size());
    if (!acc.empty())
        CK(cudaMemcpyAsync(acc.data(), c->d_acc, sizeof(BodyAcc) * acc.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

size_t ckpt_bytes(const lb_ctx* c, const std::vector<BodyAcc>& acc) {
    size_t n = sizeof(CkptHeader) + pop_bytes(c) + 2 * sizeof(int32_t) * (size_t)c->L.N + 16 * sizeof(int);
    for (const BodyAcc& a : acc) n += 2 * sizeof(BodyState) + sizeof(BodyAcc) + sizeof(uint32_t) * (size_t)a.link_count;
    return n;
}

}  // namespace

lb_status lb_checkpoint_size(lb_ctx* c, size_t* bytes) {
    if (!c || !bytes) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    std::vector<BodyAcc> acc;
    s = read_accs(c, acc);
    if (s != LB_OK) return s;
    *bytes = ckpt_bytes(c, acc);
    return LB_OK;
}

lb_status lb_checkpoint(lb_ctx* c, void* buf, size_t bytes) {
    if (!c || !buf) return LB_ERR_INVALID;
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    std::vector<BodyAcc> acc;
    s = read_accs(c, acc);
    if (s != LB_OK) return s;
    const size_t need = ckpt_bytes(c, acc);
    if (bytes < need) return fail(c, LB_ERR_INVALID, "checkpoint buffer too small (see lb_checkpoint_size)");
    unsigned char* o = static_cast<unsigned char*>(buf);
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 3;  // 3: FP64 populations are stored as deviations f - w rho0
    h.storage = (uint32_t)c->p.storage;
    h.equilibrium = c->L.inc;
    h.reserved = c->L.sr;  // rounding of the BF16 stores
    h.nx = c->L.nx;
    h.ny = c->L.ny;
    h.nz = c->L.nz;
    h.nbodies = (int32_t)c->par.size();
    h.lambda_e = c->lambda_e;
    h.lambda_o = c->lambda_o;
    h.rho0 = c->L.rho0;
    h.scale = c->L.scale;
    h.step = c->step;
    h.bodies_hash = bodies_hash(c);
    h.bytes = need;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const size_t N = (size_t)c->L.N;
    CK(cudaMemcpyAsync(o, c->L.F, pop_bytes(c), cudaMemcpyDeviceToHost, c->stream));
    o += pop_bytes(c);
    CK(cudaMemcpyAsync(o, c->own, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, c->stream));
    o += sizeof(int32_t) * N;
    CK(cudaMemcpyAsync(o, c->own_prev, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, c->stream));
    o += sizeof(int32_t) * N;
    CK(cudaMemcpyAsync(o, c->d_win, 16 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    o += 16 * sizeof(int);
    for (size_t k = 0; k < acc.size(); ++k) {
        CK(cudaMemcpyAsync(o, c->d_state[0] + k, sizeof(BodyState), cudaMemcpyDeviceToHost, c->stream));
        o += sizeof(BodyState);
        CK(cudaMemcpyAsync(o, c->d_state[1] + k, sizeof(BodyState), cudaMemcpyDeviceToHost, c->stream));
        o += sizeof(BodyState);
        std::memcpy(o, &acc[k], sizeof(BodyAcc));
        o += sizeof(BodyAcc);
        const size_t nl = (size_t)acc[k].link_count;
        if (nl)
            CK(cudaMemcpyAsync(o, c->d_links + c->par[k].link_off, sizeof(uint32_t) * nl, cudaMemcpyDeviceToHost,
                               c->stream));
        o += sizeof(uint32_t) * nl;
    }
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_restore(lb_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf || bytes < sizeof(CkptHeader)) return LB_ERR_INVALID;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 3) return fail(c, LB_ERR_INVALID, "not a checkpoint");
    if (h.bytes != bytes) return fail(c, LB_ERR_INVALID, "checkpoint size differs from its header");
    if (h.storage != (uint32_t)c->p.storage || h.nx != c->L.nx || h.ny != c->L.ny || h.nz != c->L.nz ||
        h.lambda_e != c->lambda_e || h.lambda_o != c->lambda_o || h.rho0 != c->L.rho0 ||
        h.scale != (double)c->L.scale || h.equilibrium != c->L.inc || h.reserved != c->L.sr)
        return fail(c, LB_ERR_INVALID, "checkpoint of a lattice with other parameters");
    if (h.nbodies != (int32_t)c->par.size() || h.bodies_hash != bodies_hash(c))
        return fail(c, LB_ERR_INVALID, "checkpoint of other bodies (add the same bodies in the same order)");
    CK(cudaSetDevice(c->p.device));
    settle(c);
    lb_status s = sync_checked(c);
    if (s != LB_OK) return s;
    // walk the sections once to check the link counts before anything is written
    const unsigned char* base = static_cast<const unsigned char*>(buf);
    const size_t N = (size_t)c->L.N;
    const size_t fixed = sizeof(CkptHeader) + pop_bytes(c) + 2 * sizeof(int32_t) * N + 16 * sizeof(int);
    std::vector<BodyAcc> acc(c->par.size());
    std::vector<size_t> at(c->par.size());
    size_t off = fixed;
    for (size_t k = 0; k < acc.size(); ++k) {
        if (off + 2 * sizeof(BodyState) + sizeof(BodyAcc) > bytes) return fail(c, LB_ERR_INVALID, "truncated checkpoint");
        at[k] = off;
        std::memcpy(&acc[k], base + off + 2 * sizeof(BodyState), sizeof(BodyAcc));
        if (acc[k].link_count < 0 || acc[k].link_count > c->par[k].link_cap)
            return fail(c, LB_ERR_INVALID, "checkpoint link list larger than this context holds");
        off += 2 * sizeof(BodyState) + sizeof(BodyAcc) + sizeof(uint32_t) * (size_t)acc[k].link_count;
    }
    if (off != bytes) return fail(c, LB_ERR_INVALID, "checkpoint size differs from its sections");
    const unsigned char* o = base + sizeof(CkptHeader);
    CK(cudaMemcpyAsync(c->L.F, o, pop_bytes(c), cudaMemcpyHostToDevice, c->stream));
    o += pop_bytes(c);
    CK(cudaMemcpyAsync(c->own, o, sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->stream));
    o += sizeof(int32_t) * N;
    CK(cudaMemcpyAsync(c->own_prev, o, sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->stream));
    o += sizeof(int32_t) * N;
    CK(cudaMemcpyAsync(c->d_win, o, 16 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    for (size_t k = 0; k < acc.size(); ++k) {
        const unsigned char* b = base + at[k];
        CK(cudaMemcpyAsync(c->d_state[0] + k, b, sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->d_state[1] + k, b + sizeof(BodyState), sizeof(BodyState), cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_acc + k, b + 2 * sizeof(BodyState), sizeof(BodyAcc), cudaMemcpyHostToDevice,
                           c->stream));
        const size_t nl = (size_t)acc[k].link_count;
        if (nl)
            CK(cudaMemcpyAsync(c->d_links + c->par[k].link_off, b + 2 * sizeof(BodyState) + sizeof(BodyAcc),
                               sizeof(uint32_t) * nl, cudaMemcpyHostToDevice, c->stream));
    }
    // the step count the sweeps keep for the stochastic rounding: the next
    // sweep (of parity step & 1) reads it
    const unsigned long long st = (unsigned long long)h.step;
    CK(cudaMemcpyAsync(c->L.sr_ctr + (st & 1), &st, sizeof(st), cudaMemcpyHostToDevice, c->stream));
    // solid fractions are found afresh at the start of the next step; the
    // spheres may sit elsewhere than when they were last found
    if (c->psm) {
        CK(cudaMemsetAsync(c->d_eps, 0, sizeof(float) * N, c->stream));
        CK(cudaMemsetAsync(c->d_psm_id, 0, sizeof(int32_t) * N, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));  // the caller's buffer may go once we return
    c->step = h.step;
    c->pending = false;
    drop_graph(c);
    return LB_OK;
}

}  // extern "C"
