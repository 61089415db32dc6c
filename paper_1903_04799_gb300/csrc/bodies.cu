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
//                  "consforce", and the WCA force of Eq. "wca") and decides
//                  whether the body's cells must be re-classified;
//   k_classify<P>  new owner of every cell in the scan box of each body that
//                  moved far enough for a lattice node to cross its surface;
//   k_convert<P>   Aidun conversion of covered / uncovered cells, booking the
//                  conversion force; counts the new boundary links;
//   k_rebuild<P>   compacts the new link lists (block scan, canonical order
//                  within each body's scan box) and commits the new owners.
//
// Body state is double-buffered by step parity: the step of parity P reads
// state[P] and writes state[1-P], so a body's update never races with another
// body reading its position.  Every reduction is a fixed tree (warp shuffle,
// then shared memory, then per-block partials summed in block order), so the
// result does not depend on scheduling -- the same inputs give the same bits.
#include <cfloat>

#include "lbsq_internal.cuh"

namespace lbsq {

constexpr int kBlock = 256;

// ---------------------------------------------------------------- reductions

// Sum K doubles over the block; the result is valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
    __shared__ double sm[32 * K];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm[warp * K + k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v[k] = lane < nw ? sm[lane * K + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ long long block_sum_ll(long long v) {
    __shared__ long long sm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ double block_min(double v) {
    __shared__ double sm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sm[lane] : DBL_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

// Exclusive scan of one int per thread over the block; returns the thread's
// offset and writes the block total to *total.
__device__ __forceinline__ int block_scan(int v, int* total) {
    __shared__ int sm[33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? sm[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) sm[lane] = wi - w;  // exclusive warp offsets
        if (lane == nw - 1) sm[32] = wi;
    }
    __syncthreads();
    int res = sm[warp] + inc - v;
    *total = sm[32];
    __syncthreads();
    return res;
}

// Last-block election: every block calls this once after writing its
// partial; returns true in exactly one block (the last to arrive), which may
// then read all partials.  The counter resets itself for the next launch.
__device__ __forceinline__ bool last_block(int* counter, int nblocks) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int t = atomicAdd(counter, 1);
        is_last = (t == nblocks - 1);
        if (is_last) *counter = 0;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// In the elected last block: stage the G x K partials in shared memory with
// all threads (cache-global loads, so no stale L1 line is read), then thread 0
// sums them in block order -- the same fixed order as a serial loop.
constexpr int kMaxPart = 1536;
template <int K>
__device__ __forceinline__ void ordered_partial_sum(const double* part, int G, double (&tot)[K]) {
    __shared__ double sp[kMaxPart];
    for (int t = threadIdx.x; t < G * K; t += blockDim.x) sp[t] = __ldcg(part + t);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) tot[c] = 0.0;
    if (threadIdx.x == 0)
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int c = 0; c < K; ++c) tot[c] += sp[g * K + c];
}

// ---------------------------------------------------------------- geometry

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Wall velocity on the link from fluid node (x,y,z) along c_i, taken at the
// link midpoint: rigid motion (Eq. "vb") plus the squirmer slip (Eq.
// "squirmer"); d receives the midpoint's offset from the centre.
__device__ __forceinline__ void link_velocity(const Lattice& L, const BodyParams& p, const BodyState& s, int x,
                                              int y, int z, int i, double vb[3], double d[3]) {
    if (p.kind != BODY_SPHERE) {
        vb[0] = p.wall_vel[0];
        vb[1] = p.wall_vel[1];
        vb[2] = p.wall_vel[2];
        d[0] = d[1] = d[2] = 0.0;
        return;
    }
    d[0] = min_image(((double)x + 0.5 * cx(i)) - s.pos[0], L.nx);
    d[1] = min_image(((double)y + 0.5 * cy(i)) - s.pos[1], L.ny);
    d[2] = min_image(((double)z + 0.5 * cz(i)) - s.pos[2], L.nz);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double sl[3] = {0.0, 0.0, 0.0};
    if (r > 0.0) {
        double n[3] = {d[0] / r, d[1] / r, d[2] / r};
        double ct = s.e[0] * n[0] + s.e[1] * n[1] + s.e[2] * n[2];
        double a = p.B1 + p.B2 * ct;
        for (int k = 0; k < 3; ++k) sl[k] = a * (ct * n[k] - s.e[k]);
    }
    double w[3];
    cross3(s.omega, d, w);
    for (int k = 0; k < 3; ++k) vb[k] = s.vel[k] + w[k] + sl[k];
}

__device__ __forceinline__ double wca_force(double r, double sigma, double eps) {
    if (eps == 0.0 || r >= 1.122462048309373 * sigma) return 0.0;  // 2^(1/6)
    if (r < 0.05 * sigma) r = 0.05 * sigma;
    double sr = sigma / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
    return 24.0 * eps / r * (2.0 * sr6 * sr6 - sr6);
}

__device__ __forceinline__ void rotate_e(double* e, const double* w) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (th == 0.0) return;
    double k[3] = {w[0] / th, w[1] / th, w[2] / th};
    double sn, c;
    sincos(th, &sn, &c);
    double kxe[3];
    cross3(k, e, kxe);
    double ke = k[0] * e[0] + k[1] * e[1] + k[2] * e[2];
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = e[a] * c + kxe[a] * sn + k[a] * ke * (1.0 - c);
    double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) e[a] = r[a] / nr;
}

__device__ __forceinline__ int wrap_pos(int a, int n) { return ((a % n) + n) % n; }

__device__ __forceinline__ bool axis_overlap(int a, int wa, int b, int wb, int n) {
    if (wa >= n || wb >= n) return true;
    return wrap_pos(b - a, n) < wa || wrap_pos(a - b, n) < wb;
}

// ---------------------------------------------------------------- step kernels

template <int P>
__global__ void __launch_bounds__(kBlock) k_links(const Lattice L, const Bodies B) {
    const int k = blockIdx.y;
    const BodyParams& p = B.par[k];
    const int G = p.g_links;
    if ((int)blockIdx.x >= G) return;
    const BodyState& s = B.state[P][k];
    BodyAcc& A = B.acc[k];
    const long long cnt = A.link_count;
    const uint32_t* links = B.links + p.link_off;
    const int64_t Np = L.Np;
    double acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = 0.0;
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < cnt; l += (long long)G * blockDim.x) {
        const uint32_t code = links[l];
        const int64_t n = code >> 5;
        const int i = code & 31, ib = opp(i);
        int x, y, z;
        cell_coords(L, n, x, y, z);
        const int64_t ns = cell_index(L, wrapi(x + cx(i), L.nx), wrapi(y + cy(i), L.ny), wrapi(z + cz(i), L.nz));
        // where sweep P left f*_i of the fluid node, and where the next sweep reads
        // the reflected population f_ib of the fluid node
        const int64_t out_slot = P == 0 ? (int64_t)ib * Np + n : (int64_t)i * Np + ns;
        const int64_t in_slot = P == 0 ? (int64_t)i * Np + ns : (int64_t)ib * Np + n;
        const double fout = load_abs(L, out_slot, i);
        double vb[3], d[3];
        link_velocity(L, p, s, x, y, z, i, vb, d);
        const double cv = cx(i) * vb[0] + cy(i) * vb[1] + cz(i) * vb[2];
        const double fin = fout - 6.0 * wgt(i) * L.rho0 * cv;
        store_abs(L, in_slot, ib, fin);
        const double sf = fout + fin;
        const double dF[3] = {cx(i) * sf, cy(i) * sf, cz(i) * sf};
        double dT[3];
        cross3(d, dF, dT);
        const double tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) / 3.0;
        acc[0] += dF[0];
        acc[1] += dF[1];
        acc[2] += dF[2];
        acc[3] += dT[0];
        acc[4] += dT[1];
        acc[5] += dT[2];
        acc[6] -= d[0] * dF[0] - tr;
        acc[7] -= d[1] * dF[1] - tr;
        acc[8] -= d[2] * dF[2] - tr;
        acc[9] -= 0.5 * (d[0] * dF[1] + d[1] * dF[0]);
        acc[10] -= 0.5 * (d[0] * dF[2] + d[2] * dF[0]);
        acc[11] -= 0.5 * (d[1] * dF[2] + d[2] * dF[1]);
    }
    block_sum<12>(acc);
    double* part = B.part_links + ((size_t)k * B.G_links + blockIdx.x) * 12;
    if (threadIdx.x == 0)
        for (int c = 0; c < 12; ++c) part[c] = acc[c];
    if (!last_block(&A.counter_links, G)) return;

    // ---- final fixed-order sum of the partials
    double tot[12];
    ordered_partial_sum<12>(B.part_links + (size_t)k * B.G_links * 12, G, tot);
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        A.Fbb[a] = tot[a];
        A.Tbb[a] = tot[3 + a];
    }
    for (int a = 0; a < 6; ++a) A.Sbb[a] = tot[6 + a];

    // ---- symplectic Euler (velocity first, dt = 1)
    BodyState so = s;
    for (int a = 0; a < 3; ++a) {
        A.Fapp[a] = A.Fbb[a] + A.Fc[a];
        A.Tapp[a] = A.Tbb[a] + A.Tc[a];
        A.Fc[a] = 0.0;
        A.Tc[a] = 0.0;
    }
    int reclass = 0;
    if (p.kind == BODY_SPHERE && p.mobile) {
        double Fw[3] = {0.0, 0.0, 0.0};
        if (B.wca_eps != 0.0) {
            const int n3[3] = {L.nx, L.ny, L.nz};
            for (int j = 0; j < B.n; ++j) {
                if (j == k) continue;
                const BodyParams& q = B.par[j];
                const BodyState& t = B.state[P][j];
                if (q.kind == BODY_SPHERE) {
                    double dd[3];
                    for (int a = 0; a < 3; ++a) dd[a] = min_image(s.pos[a] - t.pos[a], n3[a]);
                    double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
                    double f = wca_force(dist - p.R - q.R, B.wca_sigma, B.wca_eps);
                    if (f != 0.0)
                        for (int a = 0; a < 3; ++a) Fw[a] += f * dd[a] / dist;
                } else {
                    const int ax = q.wall_axis;
                    double dd = min_image(s.pos[ax] - (double)q.wall_index, n3[ax]);
                    double f = wca_force(fabs(dd) - 0.5 - p.R, B.wca_sigma, B.wca_eps);
                    if (f != 0.0) Fw[ax] += dd > 0.0 ? f : -f;
                }
            }
        }
        const int n3[3] = {L.nx, L.ny, L.nz};
        for (int a = 0; a < 3; ++a) {
            so.vel[a] = s.vel[a] + (A.Fapp[a] + Fw[a]) / p.mass;
            so.omega[a] = s.omega[a] + A.Tapp[a] / p.inertia;
        }
        for (int a = 0; a < 3; ++a) {
            double q = s.pos[a] + so.vel[a];
            if (q >= (double)n3[a]) q -= (double)n3[a];
            else if (q < 0.0) q += (double)n3[a];
            so.pos[a] = q;
        }
        rotate_e(so.e, so.omega);
        double sp = so.vel[0] * so.vel[0] + so.vel[1] * so.vel[1] + so.vel[2] * so.vel[2];
        if (!(sp < 0.25)) set_error(B.err, 5);
        // Node crossing test: every node of the box kept its side of the surface
        // if the centre moved less than the distance of the nearest node to the
        // surface at the last classification (less a 1e-9 guard, far above the
        // FP64 error of the inside test).
        double dd[3];
        for (int a = 0; a < 3; ++a) dd[a] = min_image(so.pos[a] - A.r_class[a], n3[a]);
        double disp = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        double margin = __longlong_as_double((long long)A.margin_bits);
        reclass = !(disp < margin - 1e-9);
        if (reclass) A.margin_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
    }
    A.reclass = reclass;
    B.state[1 - P][k] = so;
}

// Box-partition helper: block g of G covers box cells [b0, b1).
__device__ __forceinline__ void box_range(long long total, int g, int G, long long& b0, long long& b1) {
    long long chunk = (total + G - 1) / G;
    b0 = (long long)g * chunk;
    b1 = b0 + chunk < total ? b0 + chunk : total;
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_classify(const Lattice L, const Bodies B, int32_t* own,
                                                       const int32_t* own_prev) {
    const int k = blockIdx.y;
    BodyAcc& A = B.acc[k];
    const BodyParams& p = B.par[k];
    const BodyState& s = B.state[1 - P][k];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // a body must rebuild its links when its own cells or those of an
        // intersecting box changed
        int rl = A.reclass;
        if (!rl) {
            int lo[3], w[3];
            body_box(L, p, s, lo, w);
            const int n3[3] = {L.nx, L.ny, L.nz};
            for (int j = 0; j < B.n && !rl; ++j) {
                if (!B.acc[j].reclass) continue;
                int loj[3], wj[3];
                body_box(L, B.par[j], B.state[1 - P][j], loj, wj);
                rl = axis_overlap(lo[0], w[0], loj[0], wj[0], n3[0]) && axis_overlap(lo[1], w[1], loj[1], wj[1], n3[1]) &&
                     axis_overlap(lo[2], w[2], loj[2], wj[2], n3[2]);
            }
        }
        A.relink = rl;
    }
    if (!A.reclass || (int)blockIdx.x >= p.g_box) return;
    int lo[3], w[3];
    body_box(L, p, s, lo, w);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            A.box_lo[a] = lo[a];
            A.r_class[a] = s.pos[a];
        }
    const int id = k + 1;
    long long b0, b1;
    box_range((long long)w[0] * w[1] * w[2], blockIdx.x, p.g_box, b0, b1);
    double mloc = DBL_MAX;
    for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        const int bx = (int)(b % w[0]), by = (int)((b / w[0]) % w[1]), bz = (int)(b / ((long long)w[0] * w[1]));
        const int x = wrapi(lo[0] + bx, L.nx), y = wrapi(lo[1] + by, L.ny), z = wrapi(lo[2] + bz, L.nz);
        const int64_t n = cell_index(L, x, y, z);
        const double dx = min_image((double)x - s.pos[0], L.nx);
        const double dy = min_image((double)y - s.pos[1], L.ny);
        const double dz = min_image((double)z - s.pos[2], L.nz);
        const bool in = inside_sphere(dx, dy, dz, p.R);
        const int old = own_prev[n];
        if (in) {
            if (old == 0) {
                int r = atomicCAS(&own[n], 0, id);
                if (r != 0 && r != id) set_error(B.err, 4);
            } else if (old != id) {
                set_error(B.err, 4);
            }
        } else if (old == id) {
            own[n] = 0;
        }
        // distance of the node to the surface, as a lower bound: FP32 square
        // root (relative error < 1e-6 on values below 1e3) minus 1e-4
        const float dist = sqrtf((float)(dx * dx + dy * dy + dz * dz));
        mloc = fmin(mloc, (double)fmaxf(fabsf(dist - (float)p.R) - 1e-4f, 0.0f));
    }
    mloc = block_min(mloc);
    if (threadIdx.x == 0) atomicMin(&A.margin_bits, (unsigned long long)__double_as_longlong(mloc));
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_convert(const Lattice L, const Bodies B, const int32_t* own,
                                                      const int32_t* own_prev) {
    const int k = blockIdx.y;
    BodyAcc& A = B.acc[k];
    const BodyParams& p = B.par[k];
    const int G = p.g_box;
    if (!A.relink || (int)blockIdx.x >= G) return;
    const BodyState& s = B.state[1 - P][k];
    const int q = 1 - P;  // parity of the next sweep
    const int id = k + 1;
    const bool conv = A.reclass != 0;
    int lo[3], w[3];
    body_box(L, p, s, lo, w);
    long long b0, b1;
    box_range((long long)w[0] * w[1] * w[2], blockIdx.x, G, b0, b1);
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    long long lcount = 0;
    for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        const int bx = (int)(b % w[0]), by = (int)((b / w[0]) % w[1]), bz = (int)(b / ((long long)w[0] * w[1]));
        const int x = wrapi(lo[0] + bx, L.nx), y = wrapi(lo[1] + by, L.ny), z = wrapi(lo[2] + bz, L.nz);
        const int64_t n = cell_index(L, x, y, z);
        const int now = own[n];
        if (conv) {
            const int was = own_prev[n];
            if ((was == 0 && now == id) || (was == id && now == 0)) {
                double d[3] = {min_image((double)x - s.pos[0], L.nx), min_image((double)y - s.pos[1], L.ny),
                               min_image((double)z - s.pos[2], L.nz)};
                double m[3] = {0.0, 0.0, 0.0};
                double sign;
                if (now == id) {
                    // fluid -> solid: the destroyed momentum goes to the body
                    for (int i = 0; i < Q; ++i) {
                        double fi = load_abs(L, read_slot(L, i, x, y, z, q), i);
                        m[0] += fi * cx(i);
                        m[1] += fi * cy(i);
                        m[2] += fi * cz(i);
                    }
                    sign = 1.0;
                } else {
                    // solid -> fluid: refill with the equilibrium of the mean density of
                    // the neighbours fluid now and before, moving with the body
                    double sum = 0.0;
                    int cnt = 0;
                    for (int i = 1; i < Q; ++i) {
                        const int xn = wrapi(x + cx(i), L.nx), yn = wrapi(y + cy(i), L.ny), zn = wrapi(z + cz(i), L.nz);
                        const int64_t nn = cell_index(L, xn, yn, zn);
                        if (own[nn] == 0 && own_prev[nn] == 0) {
                            double r = 0.0;
                            for (int j = 0; j < Q; ++j) r += load_abs(L, read_slot(L, j, xn, yn, zn, q), j);
                            sum += r;
                            cnt++;
                        }
                    }
                    const double rb = cnt > 0 ? sum / (double)cnt : L.rho0;
                    double wd[3];
                    cross3(s.omega, d, wd);
                    const double u[3] = {s.vel[0] + wd[0], s.vel[1] + wd[1], s.vel[2] + wd[2]};
                    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                    for (int i = 0; i < Q; ++i) {
                        const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
                        const double fi = wgt(i) * rb * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                        store_abs(L, read_slot(L, i, x, y, z, q), i, fi);
                        m[0] += fi * cx(i);
                        m[1] += fi * cy(i);
                        m[2] += fi * cz(i);
                    }
                    sign = -1.0;
                }
                double t[3];
                cross3(d, m, t);
                for (int a = 0; a < 3; ++a) {
                    acc[a] += sign * m[a];
                    acc[3 + a] += sign * t[a];
                }
            }
        }
        if (now == 0) {
            for (int i = 1; i < Q; ++i) {
                const int64_t nn =
                    cell_index(L, wrapi(x + cx(i), L.nx), wrapi(y + cy(i), L.ny), wrapi(z + cz(i), L.nz));
                lcount += own[nn] == id;
            }
        }
    }
    block_sum<6>(acc);
    lcount = block_sum_ll(lcount);
    if (threadIdx.x == 0) {
        double* part = B.part_conv + ((size_t)k * B.G_box + blockIdx.x) * 6;
        for (int c = 0; c < 6; ++c) part[c] = acc[c];
        B.part_count[(size_t)k * B.G_box + blockIdx.x] = (int)lcount;
    }
    if (!last_block(&A.counter_conv, G) || !conv) return;
    double tot[6];
    ordered_partial_sum<6>(B.part_conv + (size_t)k * B.G_box * 6, G, tot);
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        A.Fc[a] += tot[a];
        A.Tc[a] += tot[3 + a];
    }
}

template <int P>
__global__ void __launch_bounds__(kBlock) k_rebuild(const Lattice L, const Bodies B, const int32_t* own,
                                                      int32_t* own_prev) {
    const int k = blockIdx.y;
    BodyAcc& A = B.acc[k];
    const BodyParams& p = B.par[k];
    const int G = p.g_box;
    if (!A.relink || (int)blockIdx.x >= G) return;
    const BodyState& s = B.state[1 - P][k];
    const int id = k + 1;
    int lo[3], w[3];
    body_box(L, p, s, lo, w);
    // offset of this block's links: the counts of the blocks before it
    __shared__ long long s_base, s_total;
    {
        const int* pc = B.part_count + (size_t)k * B.G_box;
        long long before = 0, all = 0;
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            const long long v = __ldcg(pc + g);
            all += v;
            if (g < (int)blockIdx.x) before += v;
        }
        before = block_sum_ll(before);
        all = block_sum_ll(all);
        if (threadIdx.x == 0) {
            s_base = before;
            s_total = all;
            if (blockIdx.x == 0) {
                if (all > p.link_cap) set_error(B.err, 8);
                A.link_count = all < p.link_cap ? all : p.link_cap;
            }
        }
        __syncthreads();
    }
    long long base = s_base;
    uint32_t* links = B.links + p.link_off;
    long long b0, b1;
    box_range((long long)w[0] * w[1] * w[2], blockIdx.x, G, b0, b1);
    for (long long r0 = b0; r0 < b1; r0 += blockDim.x) {
        const long long b = r0 + threadIdx.x;
        uint32_t mask = 0;
        int64_t n = 0;
        if (b < b1) {
            const int bx = (int)(b % w[0]), by = (int)((b / w[0]) % w[1]), bz = (int)(b / ((long long)w[0] * w[1]));
            const int x = wrapi(lo[0] + bx, L.nx), y = wrapi(lo[1] + by, L.ny), z = wrapi(lo[2] + bz, L.nz);
            n = cell_index(L, x, y, z);
            if (own[n] == 0) {
                for (int i = 1; i < Q; ++i) {
                    const int64_t nn =
                        cell_index(L, wrapi(x + cx(i), L.nx), wrapi(y + cy(i), L.ny), wrapi(z + cz(i), L.nz));
                    if (own[nn] == id) mask |= 1u << i;
                }
            }
            if (A.reclass) own_prev[n] = own[n];
        }
        int tot;
        int off = block_scan(__popc(mask), &tot);
        long long pos = base + off;
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            if (pos < p.link_cap) links[pos] = (uint32_t)(n * 32 + i);
            pos++;
        }
        base += tot;
    }
}

// ---------------------------------------------------------------- launchers

void launch_body_step(const Lattice& L, const Bodies& B, int32_t* own, int32_t* own_prev, int parity,
                      cudaStream_t st) {
    dim3 gl(B.G_links, B.n), gb(B.G_box, B.n);
    if (parity == 0) {
        k_links<0><<<gl, kBlock, 0, st>>>(L, B);
        k_classify<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_convert<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_rebuild<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    } else {
        k_links<1><<<gl, kBlock, 0, st>>>(L, B);
        k_classify<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_convert<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_rebuild<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    }
}

// One body kernel of a step by kind (1 links, 2 classify, 3 convert, 4 rebuild),
// for the traced launch path.
void launch_body_kernel(int which, const Lattice& L, const Bodies& B, int32_t* own, int32_t* own_prev, int parity,
                        cudaStream_t st) {
    dim3 gl(B.G_links, B.n), gb(B.G_box, B.n);
    if (parity == 0) {
        if (which == 1) k_links<0><<<gl, kBlock, 0, st>>>(L, B);
        else if (which == 2) k_classify<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        else if (which == 3) k_convert<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        else k_rebuild<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    } else {
        if (which == 1) k_links<1><<<gl, kBlock, 0, st>>>(L, B);
        else if (which == 2) k_classify<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        else if (which == 3) k_convert<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        else k_rebuild<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    }
}

// Classification pass alone (used when a body is added).
void launch_classify_only(const Lattice& L, const Bodies& B, int32_t* own, const int32_t* own_prev, int parity,
                          cudaStream_t st) {
    dim3 gb(B.G_box, B.n);
    if (parity == 0) k_classify<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    else k_classify<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
}

// Rebuild the link lists of every body whose relink flag the host set, as if
// after a step of parity `parity` (the next sweep has parity 1 - parity).
void launch_relink(const Lattice& L, const Bodies& B, int32_t* own, int32_t* own_prev, int parity,
                   cudaStream_t st) {
    dim3 gb(B.G_box, B.n);
    if (parity == 0) {
        k_convert<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_rebuild<0><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    } else {
        k_convert<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
        k_rebuild<1><<<gb, kBlock, 0, st>>>(L, B, own, own_prev);
    }
}

}  // namespace lbsq
