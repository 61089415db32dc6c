// bodies.cu -- everything of a time step that concerns the bodies, after the
// lattice sweep of step t (parity P = t & 1):
//
//   k_links<P>     shifted bounce-back on every boundary link (Sec. III), with
//                  the wall velocity of Eq. "vb" plus the slip of Eq.
//                  "squirmer" taken at the link midpoint; momentum exchange
//                  force, torque and stresslet (Eqs. "bbforce", "bbtorque")
//                  reduced per body in FP64 in a fixed order; the last block
//                  of each body then does the symplectic Euler update (with
//                  the conversion force of the previous remap, Eq.
//                  "consforce", and the WCA force of Eq. "wca") and, when a
//                  lattice node can cross the body surface, queues the body
//                  for re-classification;
//   k_classify<P>  new owner of every cell in the scan box of each queued
//                  body; queues every body whose links the change touches;
//   k_convert<P>   Aidun conversion of covered / uncovered cells, booking the
//                  conversion force; counts the new boundary links;
//   k_rebuild<P>   compacts the new link lists (block scan, canonical order
//                  within each body's scan box), commits the new owners and
//                  empties the step's work lists.
//
// All kernels walk work lists of (body, block) items with a fixed grid, so one
// launch serves any number of bodies on any number of lattices (a context has
// one lattice, a server many), and a captured CUDA graph stays valid when the
// set of bodies changes.  A body's block count is a function of the body
// alone, and every reduction is a fixed tree (shared memory, then per-block
// partials summed in block order by the last block of the body), so a body's
// results do not depend on scheduling or on the other bodies present.
//
// Body state is double-buffered by step parity: the step of parity P reads
// state[P] and writes state[1-P], so a body's update never races with another
// body reading its position.
//
// FP64 throughput is low on this GPU (about 2 FP64 operations per clock per
// SM), so the FP64 work per link is kept to the arithmetic of the method and
// reductions add each value once (no shuffle trees over idle lanes).
#include <cfloat>

#include <cooperative_groups.h>

#include "lbsq_internal.cuh"
#include "psm.cuh"

namespace lbsq {

constexpr int kLB = 128;  // threads of the link kernel
constexpr int kBB = 256;  // threads of the box kernels
static_assert(kBB == kPsmChunk, "a chunk of partially saturated cells is one block of the box kernels");

// ---------------------------------------------------------------- reductions

// Sum K doubles over a block of T threads in a fixed order: each value is
// added once, by many lanes at a time (one FP64 warp instruction costs the
// pipe the same with 1 or 32 active lanes).  Stage 1: K*8 threads each sum a
// segment of T/8 values of one component; stage 2: K threads sum the 8
// segments.  Result in out[K] (shared), valid for all threads on return.
// Uses the shared buffer sm[K*T + K*8].
template <int K, int T>
__device__ __forceinline__ void block_sum_fixed(const double (&v)[K], double* sm, double* out) {
    constexpr int SEG = 8, LEN = T / SEG;
#pragma unroll
    for (int c = 0; c < K; ++c) sm[c * T + threadIdx.x] = v[c];
    __syncthreads();
    double* sm2 = sm + K * T;
    for (int t = threadIdx.x; t < K * SEG; t += T) {
        const int c = t / SEG, sg = t % SEG;
        double a = 0.0;
        for (int q = 0; q < LEN; ++q) a += sm[c * T + sg * LEN + q];
        sm2[c * SEG + sg] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double a = 0.0;
        for (int sg = 0; sg < SEG; ++sg) a += sm2[threadIdx.x * SEG + sg];
        out[threadIdx.x] = a;
    }
    __syncthreads();
}

// Integer block sum (exact, so any order gives the same result): warp
// shuffles, then one warp over the warp totals.
template <int T>
__device__ __forceinline__ long long block_sum_ll(long long v, long long* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < T / 32 ? sm[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sm[0] = v;
    }
    __syncthreads();
    const long long r = sm[0];
    __syncthreads();
    return r;
}

// Exclusive scan of one int per thread over the block; returns the thread's
// offset and writes the block total to *total.
template <int T>
__device__ __forceinline__ int block_scan(int v, int* total, int* sm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int nw = T / 32;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < nw; ++w) {
            const int t = sm[w];
            sm[w] = acc;
            acc += t;
        }
        sm[nw] = acc;
    }
    __syncthreads();
    const int res = sm[warp] + inc - v;
    *total = sm[nw];
    __syncthreads();
    return res;
}

// Last-block election among the nblocks blocks of one body: every block calls
// it once after writing its partial; it returns true in the last to arrive,
// which may then read all partials.  The counter resets itself.
__device__ __forceinline__ bool last_block(int* counter, int nblocks, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(counter, 1);
        *flag = (t == nblocks - 1);
        if (*flag) *counter = 0;
    }
    __syncthreads();
    const bool last = *flag != 0;
    if (last) __threadfence();
    __syncthreads();
    return last;
}

// The G partials of one body summed in a fixed order, staged in shared memory
// with cache-global loads (no stale L1 line): K*8 lanes each sum a run of
// consecutive partials of one component, K lanes then sum the 8 runs.  The
// grouping depends on G only (a property of the body).  Result in out[K]
// (shared).  Uses sm[G*K + K*8].
template <int K>
__device__ __forceinline__ void ordered_partial_sum(const double* part, int G, double* sm, double* out) {
    constexpr int SEG = 8;
    for (int t = threadIdx.x; t < G * K; t += blockDim.x) sm[t] = __ldcg(part + t);
    __syncthreads();
    double* sm2 = sm + G * K;
    const int run = (G + SEG - 1) / SEG;
    for (int t = threadIdx.x; t < K * SEG; t += blockDim.x) {
        const int c = t / SEG, sg = t % SEG;
        double a = 0.0;
        for (int g = sg * run; g < (sg + 1) * run && g < G; ++g) a += sm[g * K + c];
        sm2[c * SEG + sg] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double a = 0.0;
        for (int sg = 0; sg < SEG; ++sg) a += sm2[threadIdx.x * SEG + sg];
        out[threadIdx.x] = a;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- geometry

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ int step_wrap(int a, int c, int n) {
    a += c;
    if (a < 0) a += n;
    else if (a >= n) a -= n;
    return a;
}

// c * v for a lattice component c in {-1, 0, 1}, without a multiplication
__device__ __forceinline__ double csel(int c, double v) { return c > 0 ? v : (c < 0 ? -v : 0.0); }

__device__ __forceinline__ double wca_force(double r, double sigma, double eps) {
    if (eps == 0.0 || r >= 1.122462048309373 * sigma) return 0.0;  // 2^(1/6)
    if (r < 0.05 * sigma) r = 0.05 * sigma;
    const double sr = sigma / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
    return 24.0 * eps / r * (2.0 * sr6 * sr6 - sr6);
}

__device__ __forceinline__ int wrap_pos(int a, int n) { return ((a % n) + n) % n; }

__device__ __forceinline__ bool axis_overlap(int a, int wa, int b, int wb, int n) {
    if (wa >= n || wb >= n) return true;
    return wrap_pos(b - a, n) < wa || wrap_pos(a - b, n) < wb;
}

// Whether a box (origin lo, extent w, in nodes), grown by g cells, can hold a
// node that neighbours a wall node of round tube q: nodes at distance r or
// more from the axis are wall, their lattice neighbours lie at r - sqrt(2) or
// more (in the cross-section), so a box whose corners (grown) all lie within
// r - 2 - g of the axis holds none.  Conservative: a box across the periodic
// edge of the cross-section lies in the wall anyway.
__device__ __forceinline__ bool box_meets_tube(const BodyParams& q, const int lo[3], const int w[3], int g) {
    double far2 = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const double dx = (double)(i ? lo[0] + w[0] - 1 + g : lo[0] - g) - q.tube[0];
            const double dy = (double)(j ? lo[1] + w[1] - 1 + g : lo[1] - g) - q.tube[1];
            far2 = fmax(far2, dx * dx + dy * dy);
        }
    const double rr = q.tube[2] - 2.0 - (double)g;
    return rr <= 0.0 || far2 >= rr * rr;
}
__device__ __forceinline__ bool round_tube(const BodyParams& q) { return q.kind == BODY_WALL && q.wall_axis < 0; }

__device__ __forceinline__ bool boxes_intersect(const Lattice& L, const BodyParams& pa, const BodyState& sa,
                                                const BodyParams& pb, const BodyState& sb) {
    int la[3], wa[3], lb[3], wb[3];
    body_box(L, pa, sa, la, wa);
    body_box(L, pb, sb, lb, wb);
    // a round tube's box is the whole lattice; its links sit along its wall
    if (round_tube(pb) && !round_tube(pa)) return box_meets_tube(pb, la, wa, 0);
    if (round_tube(pa) && !round_tube(pb)) return box_meets_tube(pa, lb, wb, 0);
    return axis_overlap(la[0], wa[0], lb[0], wb[0], L.nx) && axis_overlap(la[1], wa[1], lb[1], wb[1], L.ny) &&
           axis_overlap(la[2], wa[2], lb[2], wb[2], L.nz);
}

// Box-partition helper: block g of G covers box cells [b0, b1).
__device__ __forceinline__ void box_range(long long total, int g, int G, long long& b0, long long& b1) {
    const long long chunk = (total + G - 1) / G;
    b0 = (long long)g * chunk;
    b1 = b0 + chunk < total ? b0 + chunk : total;
}

__device__ __forceinline__ void box_cell(const Lattice& L, const int lo[3], const int w[3], long long b, int& x,
                                         int& y, int& z) {
    // box sizes stay below 2^31 cells: 32-bit division
    const unsigned ub = (unsigned)b, r = ub / (unsigned)w[0];
    const int bx = (int)(ub - r * (unsigned)w[0]);
    const int by = (int)(r % (unsigned)w[1]), bz = (int)(r / (unsigned)w[1]);
    x = wrapi(lo[0] + bx, L.nx);
    y = wrapi(lo[1] + by, L.ny);
    z = wrapi(lo[2] + bz, L.nz);
}

// FP32 view of a sphere's centre relative to nodes: integer part and fraction
// of each coordinate, so that node offsets keep full precision.
struct CentreF {
    int ip[3];
    float fp[3];
};

__device__ __forceinline__ CentreF centre_f(const BodyState& s) {
    CentreF c;
    for (int a = 0; a < 3; ++a) {
        c.ip[a] = (int)floor(s.pos[a]);
        c.fp[a] = (float)(s.pos[a] - (double)c.ip[a]);
    }
    return c;
}

// |d|^2 of node (x,y,z) from the centre in FP32 (minimum image).  The node
// offset k = x - floor(r) is wrapped as an integer first, so t = k - frac(r)
// carries only the rounding of frac(r) to FP32 (2^-25) and of the difference
// (|t| 2^-24): for nodes with every |t| <= T the error of |d|^2 is below
// (15 T^2 + 3 T) 2^-24 (two roundings per square and sum, FMA or not).
__device__ __forceinline__ float dist2_f(const Lattice& L, const CentreF& c, int x, int y, int z) {
    const int xi[3] = {x, y, z}, n3[3] = {L.nx, L.ny, L.nz};
    float s2 = 0.0f;
    for (int a = 0; a < 3; ++a) {
        int k = xi[a] - c.ip[a];
        if (2 * k > n3[a]) k -= n3[a];
        else if (2 * k <= -n3[a]) k += n3[a];
        float t = (float)k - c.fp[a];
        if (2.0f * t <= -(float)n3[a]) t += (float)n3[a];
        s2 += t * t;
    }
    return s2;
}

// Whether a node of a sphere's box can hold a boundary link of the sphere or
// change owner in one step: only nodes with R - 1.5 < |d| < R + 2 can (a
// link joins a fluid node to a solid neighbour at most sqrt(2) away; a body
// moves less than half a node per step).  Generous bounds cover the FP32
// error of dist2_f.
__device__ __forceinline__ bool in_shell(float d2, float R) {
    const float lo = R > 1.5f ? (R - 1.5f) * (R - 1.5f) - 0.25f : -1.0f;
    const float hi = (R + 2.0f) * (R + 2.0f) + 0.25f;
    return d2 > lo && d2 < hi;
}

// Append n consecutive items (k, 0..n-1) to a list, by the calling block.
__device__ __forceinline__ void append_items(int2* items, int* count, int cap, int k, int n, int* err,
                                             int* sm_base) {
    __syncthreads();
    if (threadIdx.x == 0) *sm_base = atomicAdd(count, n);
    __syncthreads();
    const int base = *sm_base;
    if (base + n > cap) {
        if (threadIdx.x == 0) set_error(err, 8);
    } else {
        for (int g = threadIdx.x; g < n; g += blockDim.x) items[base + g] = make_int2(k, g);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- Newton-Euler

// Rare or long paths of the update, kept out of line so that the code a step
// runs stays short (it is fetched cold every step).
__device__ __noinline__ void rot_coeffs(double t2, double& sa, double& c1, double& c) {
    const double th = sqrt(t2);
    double sn;
    sincos(th, &sn, &c);
    sa = sn / th;
    c1 = (1.0 - c) / t2;
}

__device__ __noinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }

// WCA force on sphere k from the other bodies of its lattice (Eq. "wca").
template <int P>
__device__ __noinline__ void wca_sum(const Lattice& L, const Bodies& B, int k, const BodyParams& p,
                                     const BodyState& s, double* fw) {
    const int n3[3] = {L.nx, L.ny, L.nz};
    for (int j = L.body_begin; j < L.body_begin + L.body_count; ++j) {
        if (j == k) continue;
        const BodyParams& q = B.par[j];
        const BodyState& t = B.state[P][j];
        if (q.kind == BODY_SPHERE) {
            double dd[3];
            for (int b = 0; b < 3; ++b) dd[b] = min_image(s.pos[b] - t.pos[b], n3[b]);
            const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            const double f = wca_force(dist - p.R - q.R, L.wca_sigma, L.wca_eps);
            if (f != 0.0)
                for (int b = 0; b < 3; ++b) fw[b] += f * dd[b] / dist;
        } else if (q.wall_axis < 0) {
            // round tube: its surface half a cell inside the first solid
            // radius, as for a plane wall; the force points to the axis
            const double dx = s.pos[0] - q.tube[0], dy = s.pos[1] - q.tube[1];
            const double rho = sqrt(dx * dx + dy * dy);
            const double f = wca_force((q.tube[2] - 0.5) - rho - p.R, L.wca_sigma, L.wca_eps);
            if (f != 0.0 && rho > 0.0) {
                fw[0] -= f * dx / rho;
                fw[1] -= f * dy / rho;
            }
        } else {
            const int ax = q.wall_axis;
            const double dd = min_image(s.pos[ax] - (double)q.wall_index, n3[ax]);
            const double f = wca_force(fabs(dd) - 0.5 - p.R, L.wca_sigma, L.wca_eps);
            if (f != 0.0) fw[ax] += dd > 0.0 ? f : -f;
        }
    }
}

// Sum over lanes 0..2 of a value held per lane, as (x0 + x1) + x2 on every
// lane (the same bits everywhere).
__device__ __forceinline__ double sum3(double v) {
    const double v0 = __shfl_sync(0xffffffffu, v, 0), v1 = __shfl_sync(0xffffffffu, v, 1),
                 v2 = __shfl_sync(0xffffffffu, v, 2);
    return (v0 + v1) + v2;
}

// Component b of a vector held as one component per lane 0..2.
__device__ __forceinline__ double comp(double v, int b) { return __shfl_sync(0xffffffffu, v, b); }

// Symplectic Euler of body k, by one whole warp (lane a < 3 holds vector
// component a): applies the momentum exchange of this step plus the
// conversion force booked by the last remap, writes state[1-P], and decides
// whether a node can cross the surface.  Splitting the vectors over lanes
// shortens the serial FP64 chain, which this GPU issues at a low rate.
// p, s, Ai: the body's parameters, state of this step and accumulators (the
// tables of B or copies of them); the results go to the tables of B.
// Results go to *Ao (accumulators) and *So (the state of the next step); if
// `out` is given, the new state and the re-classification flag are also
// written there (lane a < 3: components a; lane 0: *out_reclass).  Out of
// line, with its outputs behind pointers: a call with the outputs pointed at
// scratch runs the same instructions (see k_body_fused).
template <int P>
__device__ __noinline__ void update_body(const Lattice& L, const Bodies& B, int k, const BodyParams& p,
                                         const BodyState& s, const BodyAcc& Ai, const double* tot, BodyAcc* Ao,
                                         BodyState* So, BodyState* out = nullptr, int* out_reclass = nullptr) {
    const int lane = threadIdx.x & 31;
    const int a = lane < 3 ? lane : 0;  // lanes >= 3 shadow component 0 and store nothing
    const bool own = lane < 3;
    BodyAcc& A = *Ao;
    // Ladd's coupling averages the momentum exchange over this step and the
    // last (Sec. III names the option; the paper's runs leave it off).  Ai.Fbb
    // and Ai.Tbb still hold the last step's values here (0 before a body's
    // first step).
    const double Fh = L.force_avg ? 0.5 * (tot[a] + Ai.Fbb[a]) : tot[a];
    const double Th = L.force_avg ? 0.5 * (tot[3 + a] + Ai.Tbb[a]) : tot[3 + a];
    const double Fa = Fh + Ai.Fc[a], Ta = Th + Ai.Tc[a];
    const double rc = Ai.r_class[a], vs = Ai.vsum[a], ves = Ai.vesum;
    const long long ns = Ai.nsum;
    const unsigned long long mbits = Ai.margin_bits;
    double v = s.vel[a], w = s.omega[a], x = s.pos[a], e = s.e[a];
    __syncwarp();
    if (own) {
        A.Fbb[a] = tot[a];
        A.Tbb[a] = tot[3 + a];
        A.Sbb[a] = tot[6 + a];
        A.Sbb[3 + a] = tot[9 + a];
        A.Fapp[a] = Fa;
        A.Tapp[a] = Ta;
        A.Fc[a] = 0.0;
        A.Tc[a] = 0.0;
    }
    int reclass = 0;
    if (p.kind == BODY_SPHERE && p.mobile) {
        const int n3[3] = {L.nx, L.ny, L.nz};
        double Fw = 0.0;  // WCA contact force, component a
        if (L.wca_eps != 0.0) {
            double fw[3] = {0.0, 0.0, 0.0};
            if (lane == 0) wca_sum<P>(L, B, k, p, s, fw);
            const double f0 = __shfl_sync(0xffffffffu, fw[0], 0), f1 = __shfl_sync(0xffffffffu, fw[1], 0),
                         f2 = __shfl_sync(0xffffffffu, fw[2], 0);
            Fw = a == 0 ? f0 : (a == 1 ? f1 : f2);
        }
        v = v + (Fa + Fw) * p.inv_mass;
        w = w + Ta * p.inv_inertia;
        const double sp = sum3(v * v);
        // The geometry of the next step (node-crossing stencils, the near
        // window) assumes a move of under half a cell.  A body at |v| >= 1/2
        // (or NaN) has left the scheme: the error is flagged and the body
        // stays where it is, so no later kernel indexes outside its tables.
        const bool ok = sp < 0.25;
        if (ok) {
            x = x + v;
            if (x >= (double)n3[a]) x -= (double)n3[a];
            else if (x < 0.0) x += (double)n3[a];
        } else {
            v = 0.0;
            w = 0.0;
        }
        // Rotation of e about w by the angle th = |w| (Rodrigues), renormalised:
        //   e' = e cos(th) + (w x e) sin(th)/th + w (w.e) (1 - cos(th))/th^2.
        // A body turns by far less than 0.01 rad per step, where the Taylor
        // series of sin(th)/th and (1 - cos(th))/th^2 to th^8 are exact in
        // FP64 (the first omitted terms are below 3e-28); larger angles use
        // sincos.  1/sqrt(n2) for n2 within 1e-8 of 1 is one Newton step from 1
        // (relative error 3/8 (n2 - 1)^2, below 4e-17).
        const double t2 = sum3(w * w);
        if (t2 != 0.0) {
            double sa, c1, c;
            if (t2 < 1e-4) {
                sa = 1.0 + t2 * (-1.0 / 6.0 + t2 * (1.0 / 120.0 + t2 * (-1.0 / 5040.0 + t2 * (1.0 / 362880.0))));
                c1 = 0.5 + t2 * (-1.0 / 24.0 + t2 * (1.0 / 720.0 + t2 * (-1.0 / 40320.0 + t2 * (1.0 / 3628800.0))));
                c = 1.0 - t2 * c1;
            } else {
                rot_coeffs(t2, sa, c1, c);
            }
            const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
            const double wxe = comp(w, a1) * comp(e, a2) - comp(w, a2) * comp(e, a1);
            const double we = sum3(w * e);
            const double r = e * c + wxe * sa + w * (we * c1);
            const double n2 = sum3(r * r);
            const double inr = fabs(n2 - 1.0) < 1e-8 ? 1.5 - 0.5 * n2 : inv_sqrt(n2);
            e = r * inr;
        }
        const double ve = sum3(v * e);
        const double dd = min_image(x - rc, n3[a]);
        const double disp2 = sum3(dd * dd);
        __syncwarp();
        if (own) A.vsum[a] = vs + v;
        if (lane == 0) {
            A.vesum = ves + ve;
            A.nsum = ns + 1;
            if (!ok) set_error(L.err, 5);
        }
        // Node crossing test: every node of the box kept its side of the surface
        // if the centre moved less than the distance of the nearest node to the
        // surface at the last classification (less a 1e-9 guard, far above the
        // FP64 error of the inside test).
        const double mg = __longlong_as_double((long long)mbits) - 1e-9;
        reclass = !(mg > 0.0 && disp2 < mg * mg);
        __syncwarp();
        if (reclass && lane == 0) A.margin_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
    }
    BodyState& so = *So;
    if (own) {
        so.pos[a] = x;
        so.vel[a] = v;
        so.omega[a] = w;
        so.e[a] = e;
        if (out) {
            out->pos[a] = x;
            out->vel[a] = v;
            out->omega[a] = w;
            out->e[a] = e;
        }
    }
    if (lane == 0) {
        A.reclass = reclass;
        if (out_reclass) *out_reclass = reclass;
    }
    __syncwarp();
}

// ---------------------------------------------------------------- k_links

// One block's share of one body's links.  FP64 storage: every quantity in
// FP64 (parity with the FP64 reference to roundoff).  Reduced storages: the
// wall velocity and the reflected deviation in FP32 (the stored populations
// carry FP32 or coarser precision anyway), the momentum exchange accumulated
// in FP64 from per-thread FP32 terms.  For spheres the rest part 2 w_i rho0 of
// each exchanged pair is dropped from the sums: over the links of a closed
// solid it adds exactly zero to the force, the torque and the stresslet (each
// solid-solid neighbour pair cancels).  Walls keep it (a wall's force
// includes the rest pressure) and have no torque or stresslet.
// Density of fluid node n = (x, y, z) from the post-collision populations
// sweep P left: P = 0 in F[j][n] for every j, P = 1 in F[j][n + c_j].  The
// link work writes only slots that solid cells' sweeps produced, so these are
// stable while the links run.  FP64 storage sums in FP64, reduced storages in
// FP32 (their own precision), both plus rho0.
template <int P>
__device__ __noinline__ double post_density(const Lattice& L, int64_t n, int x, int y, int z) {
    if (L.storage == ST_F64) {
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int64_t c = P == 0 ? n
                                     : cell_index(L, step_wrap(x, cx(j), L.nx), step_wrap(y, cy(j), L.ny),
                                                  step_wrap(z, cz(j), L.nz));
            r += ((const double*)L.F)[(int64_t)j * L.Np + c];
        }
        return L.rho0 + r;
    }
    float r = 0.0f;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t c = P == 0 ? n
                                 : cell_index(L, step_wrap(x, cx(j), L.nx), step_wrap(y, cy(j), L.ny),
                                              step_wrap(z, cz(j), L.nz));
        r += load_dev(L, (int64_t)j * L.Np + c);
    }
    return L.rho0 + (double)r;
}

template <int P, bool DP>
__device__ __forceinline__ void link_terms(const Lattice& L, const BodyParams& p, const BodyState& s, long long cnt,
                                           const uint32_t* links, int g, int G, double (&acc)[12]) {
    const int64_t Np = L.Np;
    const bool sphere = p.kind == BODY_SPHERE;
    // body position split into integer and fraction, so that FP32 link
    // offsets keep full precision far from the origin
    int ip[3];
    float fp[3], e32[3], v32[3], w32[3];
    if (!DP) {
        for (int a = 0; a < 3; ++a) {
            ip[a] = (int)floor(s.pos[a]);
            fp[a] = (float)(s.pos[a] - (double)ip[a]);
            e32[a] = (float)s.e[a];
            v32[a] = (float)s.vel[a];
            w32[a] = (float)s.omega[a];
        }
    }
    const float B1f = (float)p.B1, B2f = (float)p.B2, shf0 = (float)(6.0 * L.rho0), lat = L.link_at;
    // A thread's links are taken kU at a time: the link codes, then the
    // outgoing populations of all kU are loaded before any arithmetic or
    // store, so their memory latencies overlap.
    constexpr int kU = 2;
    const long long stride = (long long)G * blockDim.x;
    for (long long l0 = (long long)g * blockDim.x + threadIdx.x; l0 < cnt; l0 += kU * stride) {
    uint32_t codes[kU];
    double fouts[kU];
    float gouts[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) codes[u] = l0 + u * stride < cnt ? links[l0 + u * stride] : 0u;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        if (l0 + u * stride >= cnt) continue;
        const int64_t n = codes[u] >> 5;
        const int i = codes[u] & 31;
        int x, y, z;
        cell_coords(L, n, x, y, z);
        const int64_t ns =
            cell_index(L, step_wrap(x, cx(i), L.nx), step_wrap(y, cy(i), L.ny), step_wrap(z, cz(i), L.nz));
        const int64_t out_slot = P == 0 ? (int64_t)opp(i) * Np + n : (int64_t)i * Np + ns;
        if (DP || !sphere) fouts[u] = load_abs(L, out_slot, i);
        else gouts[u] = load_dev(L, out_slot);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        if (l0 + u * stride >= cnt) continue;
        const uint32_t code = codes[u];
        const int64_t n = code >> 5;
        const int i = code & 31, ib = opp(i);
        const int ci[3] = {cx(i), cy(i), cz(i)};
        int x, y, z;
        cell_coords(L, n, x, y, z);
        const int64_t ns =
            cell_index(L, step_wrap(x, ci[0], L.nx), step_wrap(y, ci[1], L.ny), step_wrap(z, ci[2], L.nz));
        // where sweep P left f*_i of the fluid node (loaded above), and where
        // the next sweep reads the reflected population f_ib of the fluid node
        const int64_t in_slot = P == 0 ? (int64_t)i * Np + ns : (int64_t)ib * Np + n;
        if (DP || !sphere) {
            const double fout = fouts[u];
            double vb[3], d[3];
            if (sphere) {
                // link midpoint (or boundary node) relative to the centre; rigid motion + slip there
                const double la = (double)L.link_at;
                d[0] = min_image(((double)x + la * ci[0]) - s.pos[0], L.nx);
                d[1] = min_image(((double)y + la * ci[1]) - s.pos[1], L.ny);
                d[2] = min_image(((double)z + la * ci[2]) - s.pos[2], L.nz);
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double sl[3] = {0.0, 0.0, 0.0};
                if (r2 > 0.0) {
                    const double ir = 1.0 / sqrt(r2);
                    const double n0 = d[0] * ir, n1 = d[1] * ir, n2 = d[2] * ir;
                    const double ct = s.e[0] * n0 + s.e[1] * n1 + s.e[2] * n2;
                    const double a = p.B1 + p.B2 * ct;
                    sl[0] = a * (ct * n0 - s.e[0]);
                    sl[1] = a * (ct * n1 - s.e[1]);
                    sl[2] = a * (ct * n2 - s.e[2]);
                }
                double w[3];
                cross3(s.omega, d, w);
                for (int a = 0; a < 3; ++a) vb[a] = s.vel[a] + w[a] + sl[a];
            } else {
                for (int a = 0; a < 3; ++a) vb[a] = p.wall_vel[a];
            }
            const double cv = csel(ci[0], vb[0]) + csel(ci[1], vb[1]) + csel(ci[2], vb[2]);
            const double rs = L.rho_local ? post_density<P>(L, n, x, y, z) : L.rho0;
            const double fin = fout - 6.0 * rs * wgt(i) * cv;
            store_abs(L, in_slot, ib, fin);
            // momentum given to the body, c_i (f_out + f_in); torque, stresslet
            const double sf = fout + fin;
            const double dF[3] = {csel(ci[0], sf), csel(ci[1], sf), csel(ci[2], sf)};
            acc[0] += dF[0];
            acc[1] += dF[1];
            acc[2] += dF[2];
            if (sphere) {
                acc[3] += d[1] * dF[2] - d[2] * dF[1];
                acc[4] += d[2] * dF[0] - d[0] * dF[2];
                acc[5] += d[0] * dF[1] - d[1] * dF[0];
                const double tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) * (1.0 / 3.0);
                acc[6] -= d[0] * dF[0] - tr;
                acc[7] -= d[1] * dF[1] - tr;
                acc[8] -= d[2] * dF[2] - tr;
                acc[9] -= 0.5 * (d[0] * dF[1] + d[1] * dF[0]);
                acc[10] -= 0.5 * (d[0] * dF[2] + d[2] * dF[0]);
                acc[11] -= 0.5 * (d[1] * dF[2] + d[2] * dF[1]);
            }
        } else {
            // FP32 path (reduced storage, sphere): deviations g = f - w rho0
            const float gout = gouts[u];
            float d[3];
            const int xi[3] = {x, y, z};
            const int n3[3] = {L.nx, L.ny, L.nz};
            for (int a = 0; a < 3; ++a) {
                float t = (float)(xi[a] - ip[a]) + (lat * (float)ci[a] - fp[a]);
                const float h = 0.5f * (float)n3[a];
                if (t > h) t -= (float)n3[a];
                else if (t <= -h) t += (float)n3[a];
                d[a] = t;
            }
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            float sl[3] = {0.0f, 0.0f, 0.0f};
            if (r2 > 0.0f) {
                const float ir = rsqrtf(r2);
                const float n0 = d[0] * ir, n1 = d[1] * ir, n2 = d[2] * ir;
                const float ct = e32[0] * n0 + e32[1] * n1 + e32[2] * n2;
                const float a = B1f + B2f * ct;
                sl[0] = a * (ct * n0 - e32[0]);
                sl[1] = a * (ct * n1 - e32[1]);
                sl[2] = a * (ct * n2 - e32[2]);
            }
            const float vb0 = v32[0] + (w32[1] * d[2] - w32[2] * d[1]) + sl[0];
            const float vb1 = v32[1] + (w32[2] * d[0] - w32[0] * d[2]) + sl[1];
            const float vb2 = v32[2] + (w32[0] * d[1] - w32[1] * d[0]) + sl[2];
            const float cv = (ci[0] > 0 ? vb0 : (ci[0] < 0 ? -vb0 : 0.0f)) +
                             (ci[1] > 0 ? vb1 : (ci[1] < 0 ? -vb1 : 0.0f)) +
                             (ci[2] > 0 ? vb2 : (ci[2] < 0 ? -vb2 : 0.0f));
            const float shf = L.rho_local ? (float)(6.0 * post_density<P>(L, n, x, y, z)) : shf0;
            const float gin = gout - shf * (float)wgt(i) * cv;
            store_dev(L, in_slot, gin);
            const float sf = gout + gin;
            const float dF[3] = {ci[0] > 0 ? sf : (ci[0] < 0 ? -sf : 0.0f), ci[1] > 0 ? sf : (ci[1] < 0 ? -sf : 0.0f),
                                 ci[2] > 0 ? sf : (ci[2] < 0 ? -sf : 0.0f)};
            const float tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) * (1.0f / 3.0f);
            const float t12[12] = {dF[0],
                                   dF[1],
                                   dF[2],
                                   d[1] * dF[2] - d[2] * dF[1],
                                   d[2] * dF[0] - d[0] * dF[2],
                                   d[0] * dF[1] - d[1] * dF[0],
                                   -(d[0] * dF[0] - tr),
                                   -(d[1] * dF[1] - tr),
                                   -(d[2] * dF[2] - tr),
                                   -0.5f * (d[0] * dF[1] + d[1] * dF[0]),
                                   -0.5f * (d[0] * dF[2] + d[2] * dF[0]),
                                   -0.5f * (d[1] * dF[2] + d[2] * dF[1])};
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] += (double)t12[c];
        }
    }
    }
}

// Links of a still body with no force readout: out slot copied to in slot in
// the storage format (f_in = f_out when the wall velocity is zero).
template <int P>
__device__ __forceinline__ void copy_links(const Lattice& L, long long cnt, const uint32_t* links, int g, int G) {
    const int64_t Np = L.Np;
    const int bytes = L.storage == ST_F64 ? 8 : (L.storage == ST_F32 ? 4 : 2);
    for (long long l = (long long)g * blockDim.x + threadIdx.x; l < cnt; l += (long long)G * blockDim.x) {
        const uint32_t code = links[l];
        const int64_t n = code >> 5;
        const int i = code & 31, ib = opp(i);
        int x, y, z;
        cell_coords(L, n, x, y, z);
        const int64_t ns =
            cell_index(L, step_wrap(x, cx(i), L.nx), step_wrap(y, cy(i), L.ny), step_wrap(z, cz(i), L.nz));
        const int64_t out_slot = P == 0 ? (int64_t)ib * Np + n : (int64_t)i * Np + ns;
        const int64_t in_slot = P == 0 ? (int64_t)i * Np + ns : (int64_t)ib * Np + n;
        if (bytes == 8) ((double*)L.F)[in_slot] = ((const double*)L.F)[out_slot];
        else if (bytes == 4) ((float*)L.F)[in_slot] = ((const float*)L.F)[out_slot];
        else ((unsigned short*)L.F)[in_slot] = ((const unsigned short*)L.F)[out_slot];
    }
}

template <int P>
__global__ void __launch_bounds__(kLB) k_links(const Bodies B) {
    __shared__ double sm[12 * kLB + 12 * 8];
    __shared__ double s_tot[12];
    __shared__ int s_flag;
    const int nitems = *B.n_link_items;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = B.link_items[it];
        const int k = item.x, g = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        if (!lattice_active(L)) continue;
        const int G = p.g_links;
        BodyAcc& A = B.acc[k];
        if (p.copy_only) {
            // still wall or obstacle (v_b = 0): the reflected population equals the
            // outgoing one bit for bit; no momentum is summed and nothing moves
            copy_links<P>(L, A.link_count, B.links + p.link_off, g, G);
            continue;
        }
        double acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = 0.0;
        if (L.storage == ST_F64)
            link_terms<P, true>(L, p, B.state[P][k], A.link_count, B.links + p.link_off, g, G, acc);
        else
            link_terms<P, false>(L, p, B.state[P][k], A.link_count, B.links + p.link_off, g, G, acc);
        block_sum_fixed<12, kLB>(acc, sm, s_tot);
        double* part = B.part_links + ((size_t)k * B.GL + g) * 12;
        if (threadIdx.x < 12) part[threadIdx.x] = s_tot[threadIdx.x];
        if (!last_block(&A.counter_links, G, &s_flag)) continue;
        ordered_partial_sum<12>(B.part_links + (size_t)k * B.GL * 12, G, sm, s_tot);
        if (threadIdx.x < 32) update_body<P>(L, B, k, p, B.state[P][k], A, s_tot, &A, &B.state[1 - P][k]);
        __syncthreads();
        if (threadIdx.x == 0) s_flag = A.reclass;
        __syncthreads();
        if (s_flag) append_items(B.box_items, B.n_box, B.box_cap, k, p.g_box, B.err, (int*)sm);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- per-cell steps
// Shared by the multi-kernel path (k_classify, k_convert, k_rebuild) and the
// fused cluster kernel, so that both take the same decisions cell by cell.
// CG = true: owner and population reads go through L2 (another block of the
// same launch may have written them).

// New owner of shell node (x, y, z) of sphere id (s = its new state; s32 its
// FP32 |d|^2).  Nodes farther than `band` from the surface in FP32 are
// decided in FP32, the rest by the exact FP64 test.  Returns a lower bound of
// the node's distance to the surface: FP32 offsets and square root (absolute
// error below 1e-4 for |d| < 2^10) minus 1e-3.
// Whether node (x, y, z) is inside the sphere of radius R centred at pos
// (s32: the node's FP32 |d|^2 from dist2_f, band: band_of(R)).  Nodes
// farther than the band from the surface are decided in FP32 (the FP32 error
// is less than half the band there), the rest by the exact FP64 test, so the
// result equals the exact test for every node.
__device__ __noinline__ bool inside_exact(int nx, int ny, int nz, const double* pos, double R, int x, int y, int z) {
    const double dx = min_image((double)x - pos[0], nx);
    const double dy = min_image((double)y - pos[1], ny);
    const double dz = min_image((double)z - pos[2], nz);
    return inside_sphere(dx, dy, dz, R);
}

__device__ __forceinline__ bool inside_node(const Lattice& L, const double pos[3], double R, float s32, float R2f,
                                            float band, int x, int y, int z) {
    if (fabsf(s32 - R2f) > band) return s32 < R2f;
    return inside_exact(L.nx, L.ny, L.nz, pos, R, x, y, z);  // rare: out of line
}

// Half-width of the band around R^2 in which inside_node falls back to the
// exact test, for a sphere of radius R: twice the dist2_f error bound for
// nodes with |t| <= R + 3 plus the rounding of R^2 to FP32.  Nodes farther
// out are outside the sphere whatever the rounding.
__device__ __forceinline__ float band_of(float R) {
    const float T = R + 3.0f;
    return 3e-6f * T * T + 1e-5f;
}

template <bool CG>
__device__ __forceinline__ float classify_cell(const Lattice& L, const BodyParams& p, const BodyState& s, int id,
                                               int x, int y, int z, float s32, float R2f, float band) {
    const int64_t n = cell_index(L, x, y, z);
    const bool in = inside_node(L, s.pos, p.R, s32, R2f, band, x, y, z);
    const int old = ld<CG>(L.own_prev + n);
    if (in) {
        if (old == 0) {
            const int r = atomicCAS(&L.own[n], 0, id);
            if (r != 0 && r != id) set_error(L.err, 4);
        } else if (old != id) {
            set_error(L.err, 4);
        }
    } else if (old == id) {
        L.own[n] = 0;
    }
    const float dist = sqrtf(s32);
    return fmaxf(fabsf(dist - (float)p.R) - 1e-3f, 0.0f);
}

// Momentum of the populations of node (x, y, z) (read slots of parity q)
// and its moment about the centre, added to acc: what a node the body covers
// gives to the body.  Out of line: rare, and long in FP64.
template <bool CG>
__device__ __noinline__ void covered_momentum(const Lattice& L, const BodyState& s, int x, int y, int z, int q,
                                              double* acc) {
    // all 19 loads before the first add (one memory latency, not 19); the
    // sums run in direction order
    double m[3] = {0.0, 0.0, 0.0};
    if (L.storage == ST_F64) {
        // sum_i c_i w_i rho0 = 0: the momentum is that of the stored deviations
        double f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = ld<CG>((const double*)L.F + read_slot(L, i, x, y, z, q));
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            m[0] += f[i] * cx(i);
            m[1] += f[i] * cy(i);
            m[2] += f[i] * cz(i);
        }
    } else {
        // sum_i c_i w_i rho0 = 0: the momentum is that of the stored deviations,
        // summed in FP32 (their own precision)
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = load_dev<CG>(L, read_slot(L, i, x, y, z, q));
        float mf[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            mf[0] += g[i] * (float)cx(i);
            mf[1] += g[i] * (float)cy(i);
            mf[2] += g[i] * (float)cz(i);
        }
        for (int a = 0; a < 3; ++a) m[a] = (double)mf[a];
    }
    const double d[3] = {min_image((double)x - s.pos[0], L.nx), min_image((double)y - s.pos[1], L.ny),
                         min_image((double)z - s.pos[2], L.nz)};
    double t[3];
    cross3(d, m, t);
    for (int a = 0; a < 3; ++a) {
        acc[a] += m[a];
        acc[3 + a] += t[a];
    }
}

// Conversion at node (x, y, z) after the re-classification of sphere id
// (conv: whether it re-classified; q: parity of the next sweep).  A node the
// sphere covered gives its momentum (and its torque about the centre) to acc;
// returns 1 for a node it uncovered (refilled by the caller).  Counts into
// lcount the links from this node, if fluid, to the sphere.
template <bool CG>
__device__ __forceinline__ int convert_cell(const Lattice& L, const BodyState& s, int id, int x, int y, int z, int q,
                                            bool conv, double (&acc)[6], long long& lcount) {
    const int64_t n = cell_index(L, x, y, z);
    const int now = ld<CG>(L.own + n);
    int uncover = 0;
    if (conv) {
        const int was = ld<CG>(L.own_prev + n);
        if (was == 0 && now == id) {
            covered_momentum<CG>(L, s, x, y, z, q, acc);  // fluid -> solid: to the body
        } else if (was == id && now == 0) {
            uncover = 1;
        }
    }
    if (now == 0)
        for (int i = 1; i < Q; ++i) {
            const int64_t nn =
                cell_index(L, step_wrap(x, cx(i), L.nx), step_wrap(y, cy(i), L.ny), step_wrap(z, cz(i), L.nz));
            lcount += ld<CG>(L.own + nn) == id;
        }
    return uncover;
}

// Directions i of the links from fluid node (x, y, z) (owner `now`) to
// sphere id, as a bit mask.
template <bool CG>
__device__ __forceinline__ uint32_t link_mask(const Lattice& L, int x, int y, int z, int id, int now) {
    uint32_t mask = 0;
    if (now == 0) {
        for (int i = 1; i < Q; ++i) {
            const int64_t nn =
                cell_index(L, step_wrap(x, cx(i), L.nx), step_wrap(y, cy(i), L.ny), step_wrap(z, cz(i), L.nz));
            if (ld<CG>(L.own + nn) == id) mask |= 1u << i;
        }
    }
    return mask;
}

// ---------------------------------------------------------------- k_classify

template <int P>
__global__ void __launch_bounds__(kBB) k_classify(const Bodies B) {
    __shared__ double smd[kBB / 32];
    __shared__ int s_base, s_scan[kBB / 32 + 1];
    const int nitems = *B.n_box;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = B.box_items[it];
        const int k = item.x, g = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        BodyAcc& A = B.acc[k];
        const BodyState& s = B.state[1 - P][k];
        if (g == 0) {
            // queue every body of this lattice whose links the change can touch:
            // this body and every body whose scan box meets this body's box
            // (one thread per candidate body, in rounds of the block size)
            for (int j0 = L.body_begin; j0 < L.body_begin + L.body_count; j0 += kBB) {
                const int j = j0 + threadIdx.x;
                int take = 0, nb = 0;
                if (j < L.body_begin + L.body_count &&
                    (j == k || boxes_intersect(L, p, s, B.par[j], B.state[1 - P][j]))) {
                    take = atomicExch(&B.acc[j].rel_flag, 1) == 0;
                    nb = take ? B.par[j].g_box : 0;
                }
                int total;
                const int off = block_scan<kBB>(nb, &total, s_scan);
                if (threadIdx.x == 0 && total > 0) s_base = atomicAdd(B.n_rel, total);
                __syncthreads();
                if (take) {
                    if (s_base + off + nb > B.rel_cap) set_error(B.err, 8);
                    else
                        for (int gg = 0; gg < nb; ++gg) B.rel_items[s_base + off + gg] = make_int2(j, gg);
                }
                __syncthreads();
            }
        }
        int lo[3], w[3];
        body_box(L, p, s, lo, w);
        if (g == 0 && threadIdx.x == 0)
            for (int a = 0; a < 3; ++a) {
                A.box_lo[a] = lo[a];
                A.r_class[a] = s.pos[a];
            }
        const int id = k + 1;
        long long b0, b1;
        box_range((long long)w[0] * w[1] * w[2], g, p.g_box, b0, b1);
        const CentreF cf = centre_f(s);
        const float R2f = (float)(p.R * p.R), Rf = (float)p.R;
        const bool full = A.reclass == 2;  // first classification of a new body
        // nodes farther than the band from the surface are decided in FP32,
        // the rest by the exact FP64 test (see inside_node)
        const float band = band_of(Rf);
        float mloc = FLT_MAX;
        for (long long b = b0 + threadIdx.x; b < b1; b += kBB) {
            int x, y, z;
            box_cell(L, lo, w, b, x, y, z);
            const float s32 = dist2_f(L, cf, x, y, z);
            // nodes well inside or well outside kept their side since the last
            // classification (a body moves less than half a node per step)
            if (!full && !in_shell(s32, Rf)) continue;
            mloc = fminf(mloc, classify_cell<false>(L, p, s, id, x, y, z, s32, R2f, band));
        }
        // block minimum (FP32 values, exact)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mloc = fminf(mloc, __shfl_down_sync(0xffffffffu, mloc, o));
        if ((threadIdx.x & 31) == 0) smd[threadIdx.x >> 5] = (double)mloc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = DBL_MAX;
            for (int q = 0; q < kBB / 32; ++q) m = fmin(m, smd[q]);
            atomicMin(&A.margin_bits, (unsigned long long)__double_as_longlong(m));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- k_convert

// Sum of one double per lane over the warp, in a fixed tree order (lane 0
// holds the result): five shuffle levels instead of a serial chain, each
// level one FP64 add for the whole warp.
__device__ __forceinline__ double warp_tree_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Density of node (x, y, z) from its populations in the read slots of parity
// q.  Reduced storages: rho0 plus the FP32 sum of the stored deviations (the
// stored values carry FP32 precision or less), one FP64 add in all.  All 19
// loads are issued before the first add (one memory latency, not 19); the
// sum runs in direction order.
template <bool CG>
__device__ __forceinline__ double node_density(const Lattice& L, int x, int y, int z, int q) {
    if (L.storage == ST_F64) {
        // rho0 plus the sum of the stored deviations
        double f[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) f[j] = ld<CG>((const double*)L.F + read_slot(L, j, x, y, z, q));
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < Q; ++j) r += f[j];
        return L.rho0 + r;
    }
    float g[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) g[j] = load_dev<CG>(L, read_slot(L, j, x, y, z, q));
    float t = 0.0f;
#pragma unroll
    for (int j = 0; j < Q; ++j) t += g[j];
    return L.rho0 + (double)t;
}

// 1/k for k = 1..18, correctly rounded (the mean of k neighbour densities is
// their sum times 1/k, within an ulp of the quotient).
__constant__ double kInvCount[19] = {0.0,       1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,
                                     1.0 / 7,   1.0 / 8,    1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13,
                                     1.0 / 14,  1.0 / 15,   1.0 / 16, 1.0 / 17, 1.0 / 18};

// Second half of a refill (shared by refill_cell and geo_refill): lane l
// holds the density r of neighbour l and whether it counts (valid).  The
// neighbour densities are summed in lane order; lanes 0..18 write the
// equilibrium of population l at the mean density and the rigid-body
// velocity there.  The created momentum (taken from the body) is added to acc
// of lane 0.
__device__ __noinline__ void refill_finish(const Lattice& L, const BodyState& s, int x, int y, int z, int q,
                                              double r, int valid, double* acc) {
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(__ballot_sync(0xffffffffu, valid != 0));
    const double sum = __shfl_sync(0xffffffffu, warp_tree_sum(valid ? r : 0.0), 0);
    const double rb = cnt > 0 ? sum * kInvCount[cnt] : L.rho0;
    const double d[3] = {min_image((double)x - s.pos[0], L.nx), min_image((double)y - s.pos[1], L.ny),
                         min_image((double)z - s.pos[2], L.nz)};
    double wd[3];
    cross3(s.omega, d, wd);
    const double u[3] = {s.vel[0] + wd[0], s.vel[1] + wd[1], s.vel[2] + wd[2]};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double fi = 0.0;
    if (lane < Q) {
        const double cu = cx(lane) * u[0] + cy(lane) * u[1] + cz(lane) * u[2];
        fi = L.inc ? wgt(lane) * (rb + L.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu))
                   : wgt(lane) * rb * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        store_abs(L, read_slot(L, lane, x, y, z, q), lane, fi);
    }
    // created momentum sum_l c_l f_l: lane l holds its term (zero beyond Q)
    const double m[3] = {warp_tree_sum(lane < Q ? fi * cx(lane) : 0.0), warp_tree_sum(lane < Q ? fi * cy(lane) : 0.0),
                         warp_tree_sum(lane < Q ? fi * cz(lane) : 0.0)};
    if (lane == 0) {
        double t[3];
        cross3(d, m, t);
        for (int a = 0; a < 3; ++a) {
            acc[a] -= m[a];
            acc[3 + a] -= t[a];
        }
    }
}

// Refill of one uncovered cell by one warp: lane l = 1..18 reads the density of
// neighbour l (if fluid now and before); see refill_finish.
template <bool CG>
__device__ __noinline__ void refill_cell(const Lattice& L, const BodyState& s, int x, int y, int z, int q,
                                            double* acc) {
    const int lane = threadIdx.x & 31;
    double r = 0.0;
    int valid = 0;
    if (lane >= 1 && lane < Q) {
        const int xn = step_wrap(x, cx(lane), L.nx), yn = step_wrap(y, cy(lane), L.ny),
                  zn = step_wrap(z, cz(lane), L.nz);
        const int64_t nn = cell_index(L, xn, yn, zn);
        if (ld<CG>(L.own + nn) == 0 && ld<CG>(L.own_prev + nn) == 0) {
            valid = 1;
            r = node_density<CG>(L, xn, yn, zn, q);
        }
    }
    refill_finish(L, s, x, y, z, q, r, valid, acc);
}

template <int P>
__global__ void __launch_bounds__(kBB) k_convert(const Bodies B) {
    __shared__ double sm[6 * kBB + 6 * 8];
    __shared__ double s_tot[6];
    __shared__ long long sml[kBB];
    __shared__ int s_list[kBB], s_scan[kBB / 32 + 1], s_flag;
    const int nitems = *B.n_rel;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = B.rel_items[it];
        const int k = item.x, g = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        BodyAcc& A = B.acc[k];
        const int G = p.g_box;
        const BodyState& s = B.state[1 - P][k];
        const int q = 1 - P;  // parity of the next sweep
        const int id = k + 1;
        const bool conv = A.reclass != 0;
        int lo[3], w[3];
        body_box(L, p, s, lo, w);
        long long b0, b1;
        box_range((long long)w[0] * w[1] * w[2], g, G, b0, b1);
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        long long lcount = 0;
        const bool sphere = p.kind == BODY_SPHERE;
        const CentreF cf = centre_f(s);
        const float Rf = (float)p.R;
        for (long long r0 = b0; r0 < b1; r0 += kBB) {
            const long long b = r0 + threadIdx.x;
            int uncover = 0, x = 0, y = 0, z = 0;
            bool take = b < b1;
            if (take) {
                box_cell(L, lo, w, b, x, y, z);
                if (sphere) take = in_shell(dist2_f(L, cf, x, y, z), Rf);
            }
            if (take) uncover = convert_cell<false>(L, s, id, x, y, z, q, conv, acc, lcount);
            // solid -> fluid cells of this round, in thread order, refilled by warps
            int nu;
            const int pos = block_scan<kBB>(uncover, &nu, s_scan);
            if (uncover) s_list[pos] = (int)(b - b0);
            __syncthreads();
            for (int u = threadIdx.x >> 5; u < nu; u += kBB / 32) {
                int ux, uy, uz;
                box_cell(L, lo, w, b0 + s_list[u], ux, uy, uz);
                refill_cell<false>(L, s, ux, uy, uz, q, acc);
            }
            __syncthreads();
        }
        // conversions are rare: blocks without one skip the FP64 block sum
        const int had = acc[0] != 0.0 || acc[1] != 0.0 || acc[2] != 0.0 || acc[3] != 0.0 || acc[4] != 0.0 ||
                        acc[5] != 0.0;
        if (__syncthreads_or(had)) {
            block_sum_fixed<6, kBB>(acc, sm, s_tot);
        } else if (threadIdx.x < 6) {
            s_tot[threadIdx.x] = 0.0;
        }
        lcount = block_sum_ll<kBB>(lcount, sml);
        if (threadIdx.x < 6) B.part_conv[((size_t)k * B.GB + g) * 6 + threadIdx.x] = s_tot[threadIdx.x];
        if (threadIdx.x == 0) B.part_count[(size_t)k * B.GB + g] = (int)lcount;
        if (!last_block(&A.counter_conv, G, &s_flag)) continue;
        if (!conv) continue;
        ordered_partial_sum<6>(B.part_conv + (size_t)k * B.GB * 6, G, sm, s_tot);
        if (threadIdx.x < 3) {
            A.Fc[threadIdx.x] += s_tot[threadIdx.x];
            A.Tc[threadIdx.x] += s_tot[3 + threadIdx.x];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- k_rebuild

// Periodic extent [lo, hi) along one axis of n cells that holds the ranges
// [lo_j, lo_j + w_j) added to it, each unwrapped to within half a lattice of
// the first one's centre.
struct Extent {
    int lo = 0, hi = 0, ref = 0;
    bool first = true;
    __device__ void add(int lo_j, int w, int n) {
        int c = lo_j + w / 2;
        if (first) ref = c;
        while (c - ref > n / 2) {
            lo_j -= n;
            c -= n;
        }
        while (c - ref < -n / 2) {
            lo_j += n;
            c += n;
        }
        if (first || lo_j < lo) lo = lo_j;
        if (first || lo_j + w > hi) hi = lo_j + w;
        first = false;
    }
    // (start, length) in [0, n) x [1, n]: the whole axis when the extent
    // covers more than 3/5 of it
    __device__ void window(int n, int* out) const {
        if ((hi - lo) * 5 < 3 * n) {
            out[0] = ((lo % n) + n) % n;
            out[1] = hi - lo;
        } else {
            out[0] = 0;
            out[1] = n;
        }
    }
};

// Window of lattice 0 that holds every cell the body kernels of the next two
// steps can touch: the z- and y-extent of every body's scan box at the new
// positions, two more cells on each side (a body moves less than half a cell
// per step).  A z-normal wall spans every row.  Stored at B.win, the slot of
// the sweeps two steps later (see api.cu); the whole lattice when the bodies
// spread over more than 3/5 of the planes.
__device__ __forceinline__ void add_sphere_extent(const Lattice& L, const BodyParams& q, const double* pos, Extent& ez,
                                                  Extent& ey) {
    ez.add((int)floor(pos[2] - q.R) - 4, q.box_w[2] + 4, L.nz);
    ey.add((int)floor(pos[1] - q.R) - 4, q.box_w[1] + 4, L.ny);
}

// The window when the lattice's only body is the sphere q at pos (as
// near_window computes it then).
__device__ void sphere_window(const Lattice& L, const BodyParams& q, const double* pos, int* win) {
    Extent ez, ey;
    add_sphere_extent(L, q, pos, ez, ey);
    int w[4] = {0, L.nz, 0, L.ny};
    ez.window(L.nz, w);
    if (w[1] < L.nz) ey.window(L.ny, w + 2);
    for (int i = 0; i < 4; ++i) win[i] = w[i];
}

template <int P>
__device__ void near_window(const Bodies& B) {
    const Lattice& L = B.lats[0];
    Extent ez, ey;
    bool full = L.body_count == 0, all_rows = false;
    for (int j = L.body_begin; j < L.body_begin + L.body_count && !full; ++j) {
        const BodyParams& q = B.par[j];
        if (q.kind == BODY_SPHERE) {
            add_sphere_extent(L, q, B.state[1 - P][j].pos, ez, ey);
        } else if (q.wall_axis == 2) {
            ez.add(q.wall_index - 3, 3 + 4, L.nz);
            all_rows = true;
        } else {
            full = true;  // a wall across every plane
        }
    }
    int w[4] = {0, L.nz, 0, L.ny};
    if (!full) {
        ez.window(L.nz, w);
        if (w[1] < L.nz && !all_rows) ey.window(L.ny, w + 2);
    }
    for (int i = 0; i < 4; ++i) B.win[i] = w[i];
}

template <int P>
__global__ void __launch_bounds__(kBB) k_rebuild(const Bodies B) {
    __shared__ long long sml[kBB];
    __shared__ int s_scan[kBB / 32 + 1], s_flag;
    __shared__ long long s_base;
    const int nitems = *B.n_rel;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = B.rel_items[it];
        const int k = item.x, g = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        BodyAcc& A = B.acc[k];
        const int G = p.g_box;
        const BodyState& s = B.state[1 - P][k];
        const int id = k + 1;
        int lo[3], w[3];
        body_box(L, p, s, lo, w);
        // offset of this block's links: the counts of the blocks before it
        {
            const int* pc = B.part_count + (size_t)k * B.GB;
            long long before = 0, all = 0;
            for (int gg = threadIdx.x; gg < G; gg += kBB) {
                const long long v = __ldcg(pc + gg);
                all += v;
                if (gg < g) before += v;
            }
            before = block_sum_ll<kBB>(before, sml);
            all = block_sum_ll<kBB>(all, sml);
            if (threadIdx.x == 0) {
                s_base = before;
                if (g == 0) {
                    if (all > p.link_cap) set_error(L.err, 8);
                    A.link_count = all < p.link_cap ? all : p.link_cap;
                }
            }
            __syncthreads();
        }
        long long base = s_base;
        uint32_t* links = B.links + p.link_off;
        const bool commit = A.reclass != 0;
        const bool sphere = p.kind == BODY_SPHERE;
        const CentreF cf = centre_f(s);
        const float Rf = (float)p.R;
        long long b0, b1;
        box_range((long long)w[0] * w[1] * w[2], g, G, b0, b1);
        for (long long r0 = b0; r0 < b1; r0 += kBB) {
            const long long b = r0 + threadIdx.x;
            uint32_t mask = 0;
            int64_t n = 0;
            int x = 0, y = 0, z = 0;
            bool take = b < b1;
            if (take) {
                box_cell(L, lo, w, b, x, y, z);
                // same predicate as the count in k_convert (only shell nodes can
                // hold links; only they changed owner)
                if (sphere) take = in_shell(dist2_f(L, cf, x, y, z), Rf);
            }
            if (take) {
                n = cell_index(L, x, y, z);
                const int now = L.own[n];
                mask = link_mask<false>(L, x, y, z, id, now);
                if (commit) L.own_prev[n] = now;
            }
            int tot;
            const int off = block_scan<kBB>(__popc(mask), &tot, s_scan);
            long long pos = base + off;
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                if (pos < p.link_cap) links[pos] = (uint32_t)(n * 32 + i);
                pos++;
            }
            base += tot;
        }
        if (!last_block(&A.counter_rebuild, G, &s_flag)) continue;
        if (threadIdx.x == 0) A.rel_flag = 0;
        __syncthreads();
    }
    // the last block of the launch empties the step's work lists (every block
    // has read the counts by now)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(B.done, 1) == (int)gridDim.x - 1) {
            *B.n_box = 0;
            *B.n_rel = 0;
            *B.done = 0;
            if (B.win) near_window<P>(B);
            if (B.gstep) *B.gstep += 1;
        }
    }
}

__global__ void k_tick(int* n_box, int* n_rel, long long* step) {
    *n_box = 0;
    *n_rel = 0;
    if (step) *step += 1;
}

// ---------------------------------------------------------------- k_body_fused

// The whole body step of one sphere in one launch: one thread-block cluster
// per sphere runs the phases of k_links, k_classify, k_convert and k_rebuild
// back to back, separated by cluster barriers, and combines its blocks'
// partial sums through distributed shared memory (rank order, fixed).  The
// scan covers the sphere's shell stencil instead of its whole box: the
// offsets o from the centre's node floor(r) for which some centre fraction
// f in [0,1]^3 puts |o - f| within the shell R - 1.5 .. R + 2 (with margin),
// in box order (z, y, x), so the link list comes out in the same canonical
// order as from the box scan.
//
// A sphere whose box, grown by one cell, meets another body's grown box at
// the start of the step (the cells and links of both can change together)
// re-classifies through the multi-kernel path instead: the cluster queues its
// box items, as k_links does.  Its force, torque and update stay here.
constexpr int kFT = 256;  // threads per block

namespace cg = cooperative_groups;

__device__ __forceinline__ bool boxes_near(const Lattice& L, const BodyParams& pa, const BodyState& sa,
                                           const BodyParams& pb, const BodyState& sb) {
    int la[3], wa[3], lb[3], wb[3];
    body_box(L, pa, sa, la, wa);
    body_box(L, pb, sb, lb, wb);
    if (round_tube(pb) && !round_tube(pa)) return box_meets_tube(pb, la, wa, 2);
    if (round_tube(pa) && !round_tube(pb)) return box_meets_tube(pa, lb, wb, 2);
    const int n3[3] = {L.nx, L.ny, L.nz};
    for (int a = 0; a < 3; ++a)
        if (!axis_overlap(la[a] - 1, wa[a] + 2, lb[a] - 1, wb[a] + 2, n3[a])) return false;
    return true;
}

// Geometry of one step's shell scan of an isolated sphere, in offsets from
// the node ip = floor(r) of the new centre r.  Stencil offset o is the node
// ip + o; its FP32 offset from the new centre is t = o - frac(r), the value
// dist2_f computes, and from the centre r_old of the last classification
// t = (o + sh) - frac(r_old), sh = ip - floor(r_old) (minimum image).  Both
// are within the error bound of dist2_f, so inside tests decide exactly (see
// inside_node).
struct ShellGeo {
    int ip[3], sh[3], lrel[3], w[3], n3[3];
    float fn[3], fo[3];
    float R2f, band, Rf;
    double R, pos[3], old[3];
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ float d2_off(int ox, int oy, int oz, const float f[3]) {
    const float tx = (float)ox - f[0], ty = (float)oy - f[1], tz = (float)oz - f[2];
    return tx * tx + ty * ty + tz * tz;
}

// Whether node ip + o is inside the sphere centred at c (G.pos or G.old);
// s: its FP32 |d|^2 from c.
__device__ __forceinline__ bool geo_inside(const ShellGeo& G, float s, const double* c, int ox, int oy, int oz) {
    if (fabsf(s - G.R2f) > G.band) return s < G.R2f;
    return inside_exact(G.n3[0], G.n3[1], G.n3[2], c, G.R, wrap1(G.ip[0] + ox, G.n3[0]),
                        wrap1(G.ip[1] + oy, G.n3[1]), wrap1(G.ip[2] + oz, G.n3[2]));
}

__device__ __forceinline__ void decode_off(uint32_t code, int& ox, int& oy, int& oz) {
    ox = (int)(code & 1023u) - 512;
    oy = (int)((code >> 10) & 1023u) - 512;
    oz = (int)(code >> 20) - 512;
}

// Whether offset o lies in the scan box and in the shell; s: its FP32 |d|^2.
__device__ __forceinline__ bool geo_take(const ShellGeo& G, int ox, int oy, int oz, float& s) {
    if ((unsigned)(ox - G.lrel[0]) >= (unsigned)G.w[0] || (unsigned)(oy - G.lrel[1]) >= (unsigned)G.w[1] ||
        (unsigned)(oz - G.lrel[2]) >= (unsigned)G.w[2])
        return false;
    s = d2_off(ox, oy, oz, G.fn);
    return in_shell(s, G.Rf);
}

__device__ __forceinline__ int64_t geo_cell(const Lattice& L, const ShellGeo& G, int ox, int oy, int oz, int& x,
                                            int& y, int& z) {
    x = wrap1(G.ip[0] + ox, L.nx);
    y = wrap1(G.ip[1] + oy, L.ny);
    z = wrap1(G.ip[2] + oz, L.nz);
    return cell_index(L, x, y, z);
}

// Links from the fluid node ip + o to the sphere at its new centre, as a bit
// mask over directions.  The 18 FP32 tests are independent and unrolled, so
// they overlap; the neighbours in the band, for which geo_inside takes the
// exact test, follow one by one (rare).
__device__ __forceinline__ uint32_t geo_mask(const ShellGeo& G, int ox, int oy, int oz) {
    const float f[3] = {G.fn[0], G.fn[1], G.fn[2]};
    const float R2f = G.R2f, band = G.band;
    uint32_t mask = 0, amb = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float s = d2_off(ox + cx(i), oy + cy(i), oz + cz(i), f);
        if (fabsf(s - R2f) > band) mask |= s < R2f ? 1u << i : 0u;
        else amb |= 1u << i;
    }
    while (amb) {
        const int i = __ffs(amb) - 1;
        amb &= amb - 1;
        const int a = ox + cx(i), b = oy + cy(i), c = oz + cz(i);
        if (inside_exact(G.n3[0], G.n3[1], G.n3[2], G.pos, G.R, wrap1(G.ip[0] + a, G.n3[0]),
                         wrap1(G.ip[1] + b, G.n3[1]), wrap1(G.ip[2] + c, G.n3[2])))
            mask |= 1u << i;
    }
    return mask;
}

// Refill of the uncovered node ip + o (see refill_cell): the neighbours that
// are fluid now and were fluid at the last classification are those outside
// the sphere at both centres, so the owner field is not read.
__device__ __noinline__ void geo_refill(const Lattice& L, const ShellGeo& G, const BodyState& s, int ox, int oy,
                                        int oz, int q, double* acc) {
    const int lane = threadIdx.x & 31;
    double r = 0.0;
    int valid = 0;
    if (lane >= 1 && lane < Q) {
        const int a = ox + cx(lane), b = oy + cy(lane), c = oz + cz(lane);
        if (!geo_inside(G, d2_off(a, b, c, G.fn), G.pos, a, b, c) &&
            !geo_inside(G, d2_off(a + G.sh[0], b + G.sh[1], c + G.sh[2], G.fo), G.old, a, b, c)) {
            valid = 1;
            int xn, yn, zn;
            geo_cell(L, G, a, b, c, xn, yn, zn);
            r = node_density<true>(L, xn, yn, zn, q);
        }
    }
    int x, y, z;
    geo_cell(L, G, ox, oy, oz, x, y, z);
    refill_finish(L, s, x, y, z, q, r, valid, acc);
}

// Copy n bytes (a multiple of 8) from global to shared memory, by the block.
__device__ __forceinline__ void copy_words(void* dst, const void* src, int n) {
    for (int t = threadIdx.x; t < n / 8; t += blockDim.x)
        reinterpret_cast<long long*>(dst)[t] = __ldcg(reinterpret_cast<const long long*>(src) + t);
}

constexpr int kStcBuf = 2048;  // stencil entries a block keeps in shared memory

template <int P>
__global__ void __launch_bounds__(kFT, 2) k_body_fused(const Bodies B, int cls, int tail) {
    cg::cluster_group cl = cg::this_cluster();
    const int KC = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int cid = blockIdx.x / KC, ncl = gridDim.x / KC;
    __shared__ double sm[12 * kFT + 12 * 8];
    __shared__ double s_tot[12], s_conv[6];
    __shared__ Lattice s_L;
    __shared__ BodyParams s_p;
    __shared__ BodyState s_s0, s_new, s_cur;
    __shared__ BodyAcc s_A, s_dryA;
    __shared__ BodyState s_dryS, s_dryS2;
    __shared__ double s_zero[12];
    __shared__ int s_dryMode;
    __shared__ ShellGeo s_geo;
    __shared__ uint32_t s_stc[kStcBuf];
    __shared__ uint32_t s_emask[kStcBuf];  // phase A's link mask of each stencil entry, for phase B
    __shared__ int s_updated;              // rank 0: s_new holds this launch's new state
    __shared__ int s_lo[3];
    __shared__ long long sml[kFT / 32];
    __shared__ long long s_count, s_before;
    __shared__ int s_scan[kFT / 32 + 1], s_list[kFT], s_mode, s_base;
    __shared__ float s_min[kFT / 32], s_margin;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = B.fused_first[cls], nitems = B.n_fused[cls];
    if (threadIdx.x < 12) s_zero[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) s_updated = 0;
    for (int it = cid; it < nitems; it += ncl) {
        // everything of this body and lattice that the step reads, in one go
        // (the sweep streams the whole lattice through L2 between two steps,
        // so these tables come from HBM)
        const int2 item = B.fused_items[i0 + it];
        const int k = item.x;
        __syncthreads();  // the previous item's readers of the copies are done
        copy_words(&s_L, B.lats + item.y, sizeof(Lattice));
        copy_words(&s_p, B.par + k, sizeof(BodyParams));
        copy_words(&s_s0, B.state[P] + k, sizeof(BodyState));
        copy_words(&s_A, B.acc + k, sizeof(BodyAcc));
        __syncthreads();
        const Lattice& L = s_L;
        const BodyParams& p = s_p;
        const BodyState& s0 = s_s0;
        if (!lattice_active(L)) continue;  // the same in every block of the cluster
        // this block's share of the shell stencil, fetched while the links run
        const uint32_t* stc = B.stencil + p.st_off;
        long long b0, b1;
        box_range(p.st_count, rank, KC, b0, b1);
        for (long long b = b0 + threadIdx.x; b < b1 && b < b0 + kStcBuf; b += kFT) s_stc[b - b0] = __ldg(stc + b);

        // ---- bounce-back and momentum exchange on the links (as k_links), by
        // ranks 1 .. KC-1.  Meanwhile warp 0 of rank 0 runs the update once on
        // scratch: its code is cold every step (the sweep streams the lattice
        // through L2 between steps), and the real update after the reduction
        // then runs warm.  The scratch call writes only shared memory.
        double acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = 0.0;
        if (rank == 0) {
            if (threadIdx.x < 32)
                update_body<P>(L, B, k, p, s0, s_A, s_zero, &s_dryA, &s_dryS, &s_dryS2, &s_dryMode);
        } else if (L.storage == ST_F64) {
            link_terms<P, true>(L, p, s0, s_A.link_count, B.links + p.link_off, rank - 1, KC - 1, acc);
        } else {
            link_terms<P, false>(L, p, s0, s_A.link_count, B.links + p.link_off, rank - 1, KC - 1, acc);
        }
        block_sum_fixed<12, kFT>(acc, sm, s_tot);
        int near = 0;
        if (rank == 0)
            for (int j = L.body_begin + threadIdx.x; j < L.body_begin + L.body_count; j += kFT)
                if (j != k && boxes_near(L, p, s0, B.par[j], B.state[P][j])) near = 1;
        near = __syncthreads_or(near);
        cl.sync();
        if (rank == 0) {
            // the blocks' partial sums, all fetched at once, then summed in rank order
            if (threadIdx.x < 12 * KC) sm[threadIdx.x] = cl.map_shared_rank(s_tot, threadIdx.x / 12)[threadIdx.x % 12];
            __syncthreads();
            if (threadIdx.x < 12) {
                double t = 0.0;
                for (int r = 0; r < KC; ++r) t += sm[r * 12 + threadIdx.x];
                sm[12 * KC + threadIdx.x] = t;
            }
            __syncthreads();
            if (threadIdx.x < 32)
                update_body<P>(L, B, k, p, s0, s_A, sm + 12 * KC, &B.acc[k], &B.state[1 - P][k], &s_new, &s_mode);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_mode = s_mode ? (near ? 2 : 1) : 0;
                s_updated = 1;
            }
            __syncthreads();
            if (s_mode == 2) append_items(B.box_items, B.n_box, B.box_cap, k, p.g_box, B.err, &s_base);
        }
        cl.sync();
        if (*cl.map_shared_rank(&s_mode, 0) != 1) continue;
        BodyAcc& A = B.acc[k];

        // ---- phase A: re-classification of the shell, conversions, link count
        // (as k_classify + k_convert).  No other body owns a cell of the box, so
        // the owner of a node is whether it is inside the sphere: now at the new
        // centre, before at the centre of the last classification.
        if (threadIdx.x < 12) {  // the new state, one double per thread
            const double* src = reinterpret_cast<const double*>(cl.map_shared_rank(&s_new, 0));
            reinterpret_cast<double*>(&s_cur)[threadIdx.x] = src[threadIdx.x];
        }
        if (threadIdx.x < 3) {  // geometry of axis a
            const int a = threadIdx.x;
            ShellGeo& G = s_geo;
            const int n = a == 0 ? L.nx : (a == 1 ? L.ny : L.nz);
            const double rn = cl.map_shared_rank(&s_new, 0)->pos[a], ro = s_A.r_class[a];
            const int lo = (int)floor(rn - p.R) - 2;  // as body_box
            G.ip[a] = (int)floor(rn);
            G.fn[a] = (float)(rn - (double)G.ip[a]);
            const int io = (int)floor(ro);
            G.fo[a] = (float)(ro - (double)io);
            int d = G.ip[a] - io;
            if (2 * d > n) d -= n;
            else if (2 * d <= -n) d += n;
            G.sh[a] = d;
            G.lrel[a] = lo - G.ip[a];
            G.w[a] = p.box_w[a];
            G.n3[a] = n;
            G.pos[a] = rn;
            G.old[a] = ro;
            s_lo[a] = lo;
            if (a == 0) {
                G.R = p.R;
                G.Rf = (float)p.R;
                G.R2f = (float)(p.R * p.R);
                G.band = band_of(G.Rf);
            }
        }
        __syncthreads();
        const ShellGeo& G = s_geo;
        const BodyState& s = s_cur;
        const int id = k + 1;
        // stencil entry b of this block's share (shared memory up to kStcBuf)
        auto entry = [&](long long b) -> uint32_t { return b - b0 < kStcBuf ? s_stc[b - b0] : __ldg(stc + b); };
        const int q = 1 - P;
        float mloc = FLT_MAX;
        double cacc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        long long lcount = 0;
        for (long long r0 = b0; r0 < b1; r0 += kFT) {
            const long long b = r0 + threadIdx.x;
            int uncover = 0, ox = 0, oy = 0, oz = 0;
            uint32_t emask = 0;
            float s32;
            if (b < b1) decode_off(entry(b), ox, oy, oz);
            if (b < b1 && geo_take(G, ox, oy, oz, s32)) {
                const bool now = geo_inside(G, s32, G.pos, ox, oy, oz);
                const bool was =
                    geo_inside(G, d2_off(ox + G.sh[0], oy + G.sh[1], oz + G.sh[2], G.fo), G.old, ox, oy, oz);
                mloc = fminf(mloc, fmaxf(fabsf(sqrtf(s32) - G.Rf) - 1e-3f, 0.0f));
                if (now != was) {
                    int x, y, z;
                    const int64_t n = geo_cell(L, G, ox, oy, oz, x, y, z);
                    // the owner, committed at once: nothing of this step reads it
                    L.own[n] = now ? id : 0;
                    L.own_prev[n] = now ? id : 0;
                    if (now) covered_momentum<true>(L, s, x, y, z, q, cacc);  // fluid -> solid: to the body
                    else uncover = 1;
                }
                if (!now) {
                    emask = geo_mask(G, ox, oy, oz);
                    lcount += __popc(emask);
                }
            }
            // each thread reads back only its own entries in phase B
            if (b - b0 < kStcBuf) s_emask[b - b0] = emask;
            // uncovered nodes of this round, refilled one per warp
            int nu;
            const int pos = block_scan<kFT>(uncover, &nu, s_scan);
            if (uncover) s_list[pos] = (int)(b - r0);
            __syncthreads();
            for (int u = warp; u < nu; u += kFT / 32) {
                int ux, uy, uz;
                decode_off(entry(r0 + s_list[u]), ux, uy, uz);
                geo_refill(L, G, s, ux, uy, uz, q, cacc);
            }
            __syncthreads();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mloc = fminf(mloc, __shfl_down_sync(0xffffffffu, mloc, o));
        if (lane == 0) s_min[warp] = mloc;
        const int had = cacc[0] != 0.0 || cacc[1] != 0.0 || cacc[2] != 0.0 || cacc[3] != 0.0 || cacc[4] != 0.0 ||
                        cacc[5] != 0.0;
        if (__syncthreads_or(had)) {
            block_sum_fixed<6, kFT>(cacc, sm, s_conv);
        } else if (threadIdx.x < 6) {
            s_conv[threadIdx.x] = 0.0;
        }
        lcount = block_sum_ll<kFT>(lcount, sml);
        if (threadIdx.x == 0) {
            s_count = lcount;
            float m = FLT_MAX;
            for (int r = 0; r < kFT / 32; ++r) m = fminf(m, s_min[r]);
            s_margin = m;
        }
        cl.sync();

        // ---- phase B: link list compaction, commit of the owners (as k_rebuild)
        // link counts and node margins of all blocks: lane r of warp 0 reads
        // block r's (integer sums and a minimum: any order gives the same)
        if (warp == 0) {
            const long long v = lane < KC ? *cl.map_shared_rank(&s_count, lane) : 0;
            float m = lane < KC ? *cl.map_shared_rank(&s_margin, lane) : FLT_MAX;
            long long all = v, bef = lane < rank ? v : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                all += __shfl_xor_sync(0xffffffffu, all, o);
                bef += __shfl_xor_sync(0xffffffffu, bef, o);
                m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            }
            if (lane == 0) {
                s_before = bef;
                if (rank == 0) {
                    if (all > p.link_cap) set_error(L.err, 8);
                    A.link_count = all < p.link_cap ? all : p.link_cap;
                    A.margin_bits = (unsigned long long)__double_as_longlong((double)m);
                }
            }
        }
        // conversion force: the blocks' partials, all fetched at once (sm is
        // free here), summed in rank order after the barrier
        if (rank == 0 && threadIdx.x >= 32 && threadIdx.x < 32 + 6 * KC) {
            const int t = threadIdx.x - 32;
            sm[t] = cl.map_shared_rank(s_conv, t / 6)[t % 6];
        }
        if (rank == 0 && threadIdx.x >= 192 && threadIdx.x < 195) {  // threads clear of the fetch
            const int a = threadIdx.x - 192;
            A.box_lo[a] = s_lo[a];
            A.r_class[a] = s.pos[a];
        }
        __syncthreads();
        if (rank == 0 && threadIdx.x >= 32 && threadIdx.x < 38) {
            const int c = threadIdx.x - 32;
            double t = 0.0;
            for (int r = 0; r < KC; ++r) t += sm[6 * r + c];
            // the update of this step consumed (zeroed) the previous booking
            if (c < 3) A.Fc[c] = t;
            else A.Tc[c - 3] = t;
        }
        const long long before = s_before;
        uint32_t* links = B.links + p.link_off;
        const long long cap = p.link_cap;
        long long base = before;
        for (long long r0 = b0; r0 < b1; r0 += kFT) {
            const long long b = r0 + threadIdx.x;
            uint32_t mask = 0;
            int64_t n = 0;
            if (b < b1) {
                int ox, oy, oz;
                decode_off(entry(b), ox, oy, oz);
                if (b - b0 < kStcBuf) {
                    mask = s_emask[b - b0];
                } else {  // beyond the buffer: as phase A computed it
                    float s32;
                    if (geo_take(G, ox, oy, oz, s32) && !geo_inside(G, s32, G.pos, ox, oy, oz))
                        mask = geo_mask(G, ox, oy, oz);
                }
                int x, y, z;
                if (mask) n = geo_cell(L, G, ox, oy, oz, x, y, z);
            }
            int tot;
            const int off = block_scan<kFT>(__popc(mask), &tot, s_scan);
            long long pos = base + off;
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                if (pos < cap) links[pos] = (uint32_t)(n * 32 + i);
                pos++;
            }
            base += tot;
        }
    }
    // no block leaves while another may still read its shared memory
    cl.sync();
    // tail != 0: this launch is the lattice's whole body step (one sphere and
    // nothing else, so the multi-kernel path never has work): the last
    // cluster to finish computes the near-body window of the coming sweeps,
    // as the rebuild kernel does otherwise.
    if (tail && B.win && rank == 0 && threadIdx.x == 0) {
        if (ncl == 1 && s_updated) {  // one cluster: the window from the state it holds
            sphere_window(s_L, s_p, s_new.pos, B.win);
            return;
        }
        __threadfence();
        if (atomicAdd(B.fused_done, 1) == ncl - 1) {
            *B.fused_done = 0;
            __threadfence();
            near_window<P>(B);
        }
    }
}

// ---------------------------------------------------------------- launchers

// which: 1 links, 2 classify, 3 convert, 4 rebuild, 5 tick.  The link kernel
// gets grid_links blocks over its static item list; the box kernels walk their
// device-built lists with grid_box blocks.
// ---------------------------------------------------------------- partially saturated cells
// (psm.cuh).  Per step, before the sweep of parity P: the previous step's
// solid fractions of each sphere are cleared (its box at the step's position,
// grown by two cells, covers where it was: a sphere moves under half a cell
// per step), the new ones written, then the force on each sphere summed from
// the pre-collision populations and the sphere advanced.  Items (body, block)
// as for the box kernels.

// Partially saturated cells (psm.cuh).  A step of parity P of a lattice
// whose spheres couple this way runs
//   k_psm_clear       the coverage the last step recorded, over each
//                     sphere's box grown by 2 (a sphere moves < 1/2 a step);
//   k_psm_cover<P>    each sphere's box at the state the step starts from,
//                     in chunks of kBB cells: the solid fraction and the
//                     covering sphere of every cell, and for each covered
//                     fluid cell the blended collision of the populations the
//                     step starts from (kept in psm_out) and its share of the
//                     force, torque and stresslet; the last block of a
//                     sphere sums the chunks' shares in chunk order and
//                     updates the sphere;
//   the sweep         every cell as usual, in place;
//   k_psm_scatter<P>  the covered fluid cells' results from psm_out into
//                     their write slots, over the sweep's.
// A covered cell's read and write slots belong to it alone within a sweep,
// so the sweep's own result for it is simply overwritten.
//
// Within a chunk the work is compacted, in cell order, so that warps run
// full: the cells to sample are taken one per warp (32 lanes share the 512
// sample points), and the covered fluid cells one per thread.

// Chunks of sphere p's box (kBB cells each) and the first one's index among
// all spheres' chunks.
__device__ __forceinline__ int psm_chunks(const BodyParams& p) {
    return (int)(((long long)p.box_w[0] * p.box_w[1] * p.box_w[2] + kBB - 1) / kBB);
}

// psm_out entry t of chunk q of sphere p, population i.
__device__ __forceinline__ int64_t psm_entry(const Bodies& B, const BodyParams& p, int q, int t, int i) {
    return (int64_t)i * B.psm_cap + p.psm_off + (int64_t)q * kBB + t;
}

// Write slot of population i of cell (x, y, z) in a sweep of parity q.
__device__ __forceinline__ int64_t write_slot(const Lattice& L, int i, int x, int y, int z, int q) {
    if (q == 0) return (int64_t)opp(i) * L.Np + cell_index(L, x, y, z);
    const int xs = wrapi(x + cx(i), L.nx), ys = wrapi(y + cy(i), L.ny), zs = wrapi(z + cz(i), L.nz);
    return (int64_t)i * L.Np + cell_index(L, xs, ys, zs);
}

// Ordered compaction within a block: the position of a kept thread among the
// kept threads of lower index, and (return) how many are kept.  sw: kBB / 32
// ints of shared memory.  Ends with the block synchronised.
__device__ __forceinline__ int block_compact(bool keep, int* sw, int* pos) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) sw[wid] = __popc(bal);
    __syncthreads();
    int off = 0, total = 0;
    for (int w = 0; w < kBB / 32; ++w) {
        off += w < wid ? sw[w] : 0;
        total += sw[w];
    }
    *pos = off + __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    return total;
}

// Fixed-order sum of G partials of K values each (any G), staged through
// shared memory kBB partials at a time: K x SEG threads each keep a running
// sum over their run of each pass, in pass order, then K threads add the SEG
// run sums.  sm: K * kBB + K * 8 doubles of shared memory.
template <int K>
__device__ __forceinline__ void ordered_sum_staged(const double* part, int G, double* sm, double* out) {
    constexpr int SEG = 8, LEN = kBB / SEG;
    double a = 0.0;  // thread t < K * SEG: component t / SEG, run t % SEG
    for (int base = 0; base < G; base += kBB) {
        const int n = G - base < kBB ? G - base : kBB;
        for (int t = threadIdx.x; t < n * K; t += blockDim.x) sm[t] = __ldcg(part + (size_t)base * K + t);
        __syncthreads();
        if ((int)threadIdx.x < K * SEG) {
            const int c = threadIdx.x / SEG, sg = threadIdx.x % SEG;
            for (int g = sg * LEN; g < (sg + 1) * LEN && g < n; ++g) a += sm[g * K + c];
        }
        __syncthreads();
    }
    double* sm2 = sm + K * kBB;
    if ((int)threadIdx.x < K * SEG) sm2[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < K) {
        double r = 0.0;
        for (int sg = 0; sg < SEG; ++sg) r += sm2[threadIdx.x * SEG + sg];
        out[threadIdx.x] = r;
    }
    __syncthreads();
}

// Step (4) of k_psm_cover for covered fluid cell t of chunk q at offset d
// (entry threadIdx.x of the chunk): the blended collision in V (FP64 for
// FP64 storage, FP32 for the others) of the deviations the step starts from,
// kept in psm_out, and the cell's force, torque and stresslet shares in acc.
template <class V, int P>
__device__ __forceinline__ void psm_cell_work(const Lattice& L, const Bodies& B, const BodyParams& p,
                                              const BodyState& s, int q, int t, const int lo[3], const int w[3],
                                              const V d[3], float eps, double acc[12]) {
    int x, y, z;
    box_cell(L, lo, w, (long long)q * kBB + t, x, y, z);
    V g[Q], out[Q], us[3], m[3] = {V(0), V(0), V(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int64_t slot = read_slot(L, i, x, y, z, P);
        if constexpr (sizeof(V) == 8) g[i] = ((const double*)L.F)[slot];
        else g[i] = load_dev(L, slot);
    }
    psm_surface_velocity<V>(p, s, d, us);
    const V Bw = psm_update<V>(g, (V)L.rho0, L.inc, (V)L.lambda_e, (V)L.lambda_o, us, (V)eps, out, m);
#pragma unroll
    for (int i = 0; i < Q; ++i) B.psm_out[psm_entry(B, p, q, threadIdx.x, i)] = (double)out[i];
    B.psm_cell[p.psm_off + (int64_t)q * kBB + threadIdx.x] = t;
    const V dF[3] = {-Bw * m[0], -Bw * m[1], -Bw * m[2]};
    const V tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) * V(1.0 / 3.0);
    const V a[12] = {dF[0], dF[1], dF[2],
                     d[1] * dF[2] - d[2] * dF[1], d[2] * dF[0] - d[0] * dF[2], d[0] * dF[1] - d[1] * dF[0],
                     -(d[0] * dF[0] - tr), -(d[1] * dF[1] - tr), -(d[2] * dF[2] - tr),
                     V(-0.5) * (d[0] * dF[1] + d[1] * dF[0]), V(-0.5) * (d[0] * dF[2] + d[2] * dF[0]),
                     V(-0.5) * (d[1] * dF[2] + d[2] * dF[1])};
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = (double)a[c];
}

__global__ void __launch_bounds__(kBB) k_psm_clear(const Bodies B, int P) {
    for (int it = blockIdx.x; it < B.n_psm_items; it += gridDim.x) {
        const int2 item = B.psm_items[it];
        const int k = item.x, q = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        int lo[3], w[3];
        body_box(L, p, B.state[P][k], lo, w);
        for (int a = 0; a < 3; ++a) {
            lo[a] -= 2;
            w[a] += 4;
        }
        long long b0, b1;
        box_range((long long)w[0] * w[1] * w[2], q, psm_chunks(p), b0, b1);
        const int32_t id = k + 1;
        for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
            int x, y, z;
            box_cell(L, lo, w, b, x, y, z);
            const int64_t c = cell_index(L, x, y, z);
            if (L.psm_id[c] == id) {
                L.psm_id[c] = 0;
                L.eps[c] = 0.0f;
            }
        }
    }
}

template <int P, class V>
__global__ void __launch_bounds__(kBB, 2) k_psm_cover(const Bodies B) {
    __shared__ double sm[12 * kBB + 12 * 8];
    __shared__ double s_tot[12];
    __shared__ int s_flag;
    __shared__ int s_w[kBB / 32];
    __shared__ int s_list[kBB];
    __shared__ float s_eps[kBB];
    __shared__ double s_d[3][kBB];  // each cell's offset from the centre
    __shared__ float s_df[3][kBB];  // the same in FP32
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < B.n_psm_items; it += gridDim.x) {
        const int2 item = B.psm_items[it];
        const int k = item.x, q = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        const BodyState& s = B.state[P][k];
        BodyAcc& A = B.acc[k];
        int lo[3], w[3];
        body_box(L, p, s, lo, w);
        const long long nbox = (long long)w[0] * w[1] * w[2];
        const int32_t id = k + 1;
        // (1) this thread's cell: its offset, the shortcut, the cells to sample
        const long long b = (long long)q * kBB + threadIdx.x;
        int x = 0, y = 0, z = 0, cls = 0;
        double d[3] = {0.0, 0.0, 0.0};
        if (b < nbox) {
            box_cell(L, lo, w, b, x, y, z);
            d[0] = min_image((double)x - s.pos[0], L.nx);
            d[1] = min_image((double)y - s.pos[1], L.ny);
            d[2] = min_image((double)z - s.pos[2], L.nz);
            cls = psm_class(d, p.R);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s_d[a][threadIdx.x] = d[a];
            s_df[a][threadIdx.x] = (float)d[a];
        }
        s_eps[threadIdx.x] = cls == 1 ? 1.0f : 0.0f;
        int pos;
        const int nsample = block_compact(cls == 2, s_w, &pos);
        if (cls == 2) s_list[pos] = threadIdx.x;
        __syncthreads();
        // (2) sampling, one cell per warp
        const float2 band = psm_screen(p.R);
        for (int j = wid; j < nsample; j += kBB / 32) {
            const int t = s_list[j];
            const double dt[3] = {s_d[0][t], s_d[1][t], s_d[2][t]};
            const float ft[3] = {s_df[0][t], s_df[1][t], s_df[2][t]};
            const int n = __reduce_add_sync(0xffffffffu, psm_lane_count(dt, ft, p.R, band, lane));
            if (lane == 0) s_eps[t] = n * (1.0f / 512.0f);
        }
        __syncthreads();
        // (3) record the coverage; the covered fluid cells
        const float e = s_eps[threadIdx.x];
        bool keep = false;
        if (e > 0.0f) {
            const int64_t c = cell_index(L, x, y, z);
            const int32_t old = atomicCAS(L.psm_id + c, 0, id);
            if (old != 0 && old != id) {
                set_error(L.err, 4);  // LB_ERR_OVERLAP: two spheres in one cell
            } else {
                L.eps[c] = e;
                keep = L.own[c] == 0;  // a wall cell stays a wall cell
            }
        }
        const int ncov = block_compact(keep, s_w, &pos);
        if (keep) s_list[pos] = threadIdx.x;
        __syncthreads();
        // (4) the covered fluid cells, one per thread, in cell order
        double acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = 0.0;
        if ((int)threadIdx.x < ncov) {
            const int t = s_list[threadIdx.x];
            V dv[3];
            if constexpr (sizeof(V) == 8) {
                for (int a = 0; a < 3; ++a) dv[a] = s_d[a][t];
            } else {
                for (int a = 0; a < 3; ++a) dv[a] = s_df[a][t];
            }
            psm_cell_work<V, P>(L, B, p, s, q, t, lo, w, dv, s_eps[t], acc);
        }
        const int64_t chunk = p.psm_off / kBB + q;
        if (threadIdx.x == 0) B.psm_count[chunk] = ncov;
        block_sum_fixed<12, kBB>(acc, sm, s_tot);
        if (threadIdx.x < 12) B.part_psm[chunk * 12 + threadIdx.x] = s_tot[threadIdx.x];
        if (!last_block(&A.counter_links, psm_chunks(p), &s_flag)) continue;
        ordered_sum_staged<12>(B.part_psm + (p.psm_off / kBB) * 12, psm_chunks(p), sm, s_tot);
        if (threadIdx.x < 32) update_body<P>(L, B, k, p, s, A, s_tot, &A, &B.state[1 - P][k]);
        __syncthreads();
    }
}

template <int P>
__global__ void __launch_bounds__(kBB) k_psm_scatter(const Bodies B) {
    for (int it = blockIdx.x; it < B.n_psm_items; it += gridDim.x) {
        const int2 item = B.psm_items[it];
        const int k = item.x, q = item.y;
        const BodyParams& p = B.par[k];
        const Lattice& L = B.lats[p.lat];
        const int n = B.psm_count[p.psm_off / kBB + q];
        if ((int)threadIdx.x >= n) continue;
        int lo[3], w[3];
        body_box(L, p, B.state[P][k], lo, w);  // the box k_psm_cover<P> covered
        const int t = B.psm_cell[p.psm_off + (int64_t)q * kBB + threadIdx.x];
        int x, y, z;
        box_cell(L, lo, w, (long long)q * kBB + t, x, y, z);
        if (L.storage == ST_F64) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                ((double*)L.F)[write_slot(L, i, x, y, z, P)] = B.psm_out[psm_entry(B, p, q, threadIdx.x, i)];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                store_dev(L, write_slot(L, i, x, y, z, P), (float)B.psm_out[psm_entry(B, p, q, threadIdx.x, i)]);
        }
    }
}

// Before the sweep of a step of parity P: clear and cover (two launches);
// f64: the lattice stores FP64 populations.
void launch_psm_cover(const Bodies& B, int parity, int grid, bool f64, cudaStream_t st) {
    k_psm_clear<<<grid, kBB, 0, st>>>(B, parity);
    if (f64) {
        if (parity == 0) k_psm_cover<0, double><<<grid, kBB, 0, st>>>(B);
        else k_psm_cover<1, double><<<grid, kBB, 0, st>>>(B);
    } else {
        if (parity == 0) k_psm_cover<0, float><<<grid, kBB, 0, st>>>(B);
        else k_psm_cover<1, float><<<grid, kBB, 0, st>>>(B);
    }
}

// After the sweep: the covered cells' results (one launch).
void launch_psm_scatter(const Bodies& B, int parity, int grid, cudaStream_t st) {
    if (parity == 0) k_psm_scatter<0><<<grid, kBB, 0, st>>>(B);
    else k_psm_scatter<1><<<grid, kBB, 0, st>>>(B);
}

void launch_body_kernel(int which, const Bodies& B, int parity, int grid_links, int grid_box, long long* step,
                        cudaStream_t st) {
    if (which == 1) {
        if (parity == 0) k_links<0><<<grid_links, kLB, 0, st>>>(B);
        else k_links<1><<<grid_links, kLB, 0, st>>>(B);
    } else if (which == 2) {
        if (parity == 0) k_classify<0><<<grid_box, kBB, 0, st>>>(B);
        else k_classify<1><<<grid_box, kBB, 0, st>>>(B);
    } else if (which == 3) {
        if (parity == 0) k_convert<0><<<grid_box, kBB, 0, st>>>(B);
        else k_convert<1><<<grid_box, kBB, 0, st>>>(B);
    } else if (which == 4) {
        if (parity == 0) k_rebuild<0><<<grid_box, kBB, 0, st>>>(B);
        else k_rebuild<1><<<grid_box, kBB, 0, st>>>(B);
    } else {
        k_tick<<<1, 1, 0, st>>>(B.n_box, B.n_rel, step);
    }
}

// Once per process and device, before the first launch of k_body_fused:
// allow clusters of 16 blocks (above the portable maximum of 8).
cudaError_t prepare_body_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_body_fused<0>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_body_fused<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Blocks per cluster of fused-kernel class c (see fused_class).
int fused_cluster(int c) { return c == 0 ? 16 : (c == 1 ? 8 : 4); }

// The fused body kernel over the spheres of class cls in B.fused_items:
// `clusters` clusters of fused_cluster(cls) blocks; tail: see k_body_fused.
// started: null, or an event (created with cudaEventDisableTiming) to fire
// once every block of the launch has begun (a launch-completion event): a
// stream that waits on it starts after the clusters are placed, not after
// the kernel ends.
void launch_body_fused(const Bodies& B, int parity, int cls, int clusters, cudaStream_t st, int tail,
                       cudaEvent_t started) {
    if (clusters <= 0) return;
    const int kc = fused_cluster(cls);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * kc);
    cfg.blockDim = dim3(kFT);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (started) {
        attr[cfg.numAttrs].id = cudaLaunchAttributeLaunchCompletionEvent;
        attr[cfg.numAttrs].val.launchCompletionEvent.event = started;
        attr[cfg.numAttrs].val.launchCompletionEvent.flags = 0;
        cfg.numAttrs++;
    }
    if (parity == 0) cudaLaunchKernelEx(&cfg, k_body_fused<0>, B, cls, tail);
    else cudaLaunchKernelEx(&cfg, k_body_fused<1>, B, cls, tail);
}

// A step's body kernels: links, classify, convert, rebuild (whose last block
// empties the work lists).
void launch_body_step(const Bodies& B, int parity, int grid_links, int grid_box, long long* step, cudaStream_t st) {
    for (int which = 1; which <= 4; ++which) launch_body_kernel(which, B, parity, grid_links, grid_box, step, st);
}

}  // namespace lbsq
