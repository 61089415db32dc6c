// setup.cu -- kernels that initialise, inspect or export the lattice; none of
// them runs inside a time step.
#include <cfloat>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbsq_internal.cuh"

namespace lbsq {

constexpr int kB = 256;

__device__ __forceinline__ bool grid_cell(const Lattice& L, int64_t& n, int& x, int& y, int& z) {
    n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L.N) return false;
    cell_coords(L, n, x, y, z);
    return true;
}

static unsigned grid_for(int64_t N) { return (unsigned)((N + kB - 1) / kB); }

// Every population at rest equilibrium w_i rho0 (Sec. III).
__global__ void k_fill_rest(const Lattice L) {
    int64_t n;
    int x, y, z;
    if (!grid_cell(L, n, x, y, z)) return;
    for (int i = 0; i < Q; ++i) store_abs(L, (int64_t)i * L.Np + n, i, wgt(i) * L.rho0);
}

// Equilibrium of given fields, w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
// (incompressible: w_i (rho + rho0 (3 c.u + 9/2 (c.u)^2 - 3/2 u.u))), into
// the read slots of parity q.  rho[N], u[3][N] on the device.
__global__ void k_set_eq(const Lattice L, const double* rho, const double* u, int q) {
    int64_t n;
    int x, y, z;
    if (!grid_cell(L, n, x, y, z)) return;
    const double r = rho[n], ux = u[n], uy = u[L.N + n], uz = u[2 * L.N + n];
    const double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < Q; ++i) {
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const double fe = L.inc ? wgt(i) * (r + L.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu))
                                : wgt(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        store_abs(L, read_slot(L, i, x, y, z, q), i, fe);
    }
}

// f[19][N] (absolute values) <-> read slots of parity q.
__global__ void k_set_pop(const Lattice L, const double* f, int q) {
    int64_t n;
    int x, y, z;
    if (!grid_cell(L, n, x, y, z)) return;
    for (int i = 0; i < Q; ++i) store_abs(L, read_slot(L, i, x, y, z, q), i, f[(int64_t)i * L.N + n]);
}

__global__ void k_get_pop(const Lattice L, double* f, int q) {
    int64_t n;
    int x, y, z;
    if (!grid_cell(L, n, x, y, z)) return;
    for (int i = 0; i < Q; ++i) f[(int64_t)i * L.N + n] = load_abs(L, read_slot(L, i, x, y, z, q), i);
}

// rho = sum f_i and u = j / rho of fluid cells (Sec. III; incompressible
// equilibrium: u = j / rho0); 0 in solid cells.
__global__ void k_fields(const Lattice L, const int32_t* own, double* rho, double* u, int q) {
    int64_t n;
    int x, y, z;
    if (!grid_cell(L, n, x, y, z)) return;
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    if (own[n] == 0) {
        for (int i = 0; i < Q; ++i) {
            const double f = load_abs(L, read_slot(L, i, x, y, z, q), i);
            r += f;
            jx += f * cx(i);
            jy += f * cy(i);
            jz += f * cz(i);
        }
    }
    if (rho) rho[n] = r;
    if (u) {
        const double den = L.inc ? L.rho0 : r;
        u[n] = r != 0.0 ? jx / den : 0.0;
        u[L.N + n] = r != 0.0 ? jy / den : 0.0;
        u[2 * L.N + n] = r != 0.0 ? jz / den : 0.0;
    }
}

// Mass and momentum of the fluid: per-block partials, then a one-block pass
// that sums them in block order (a fixed order, hence reproducible bits).
__global__ void k_mass_partial(const Lattice L, const int32_t* own, double* part, int q) {
    int64_t n;
    int x, y, z;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (grid_cell(L, n, x, y, z) && own[n] == 0) {
        for (int i = 0; i < Q; ++i) {
            const double f = load_abs(L, read_slot(L, i, x, y, z, q), i);
            v[0] += f;
            v[1] += f * cx(i);
            v[2] += f * cy(i);
            v[3] += f * cz(i);
        }
    }
    __shared__ double sm[kB / 32][4];
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kB / 32; ++w)
            for (int k = 0; k < 4; ++k) t[k] += sm[w][k];
        for (int k = 0; k < 4; ++k) part[(size_t)blockIdx.x * 4 + k] = t[k];
    }
}

__global__ void k_mass_final(const double* part, int nblocks, double* out) {
    __shared__ double sm[kB][4];
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    // thread j sums blocks j, j + kB, ... ; then thread 0 sums the threads in order
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; ++k) t[k] += part[(size_t)b * 4 + k];
    for (int k = 0; k < 4; ++k) sm[threadIdx.x][k] = t[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < (int)blockDim.x; ++j)
            for (int k = 0; k < 4; ++k) s[k] += sm[j][k];
        for (int k = 0; k < 4; ++k) out[k] = s[k];
    }
}

// Count cells a new sphere would cover that are already solid.
__global__ void k_sphere_overlap(const Lattice L, const int32_t* own, double px, double py, double pz, double R,
                                 int W, int* count) {
    const long long total = (long long)W * W * W;
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= total) return;
    const int lx = (int)floor(px - R) - 2, ly = (int)floor(py - R) - 2, lz = (int)floor(pz - R) - 2;
    const int x = wrapi(lx + (int)(b % W), L.nx), y = wrapi(ly + (int)((b / W) % W), L.ny),
              z = wrapi(lz + (int)(b / ((long long)W * W)), L.nz);
    const double dx = min_image((double)x - px, L.nx), dy = min_image((double)y - py, L.ny),
                 dz = min_image((double)z - pz, L.nz);
    if (inside_sphere(dx, dy, dz, R) && own[cell_index(L, x, y, z)] != 0) atomicAdd(count, 1);
}

// Plane wall: count sphere-owned cells of the layer (kind[] maps id-1 -> kind),
// then claim the fluid cells of the layer (cells of other walls stay theirs).
__global__ void k_plane_overlap(const Lattice L, const int32_t* own, const int* kind, int axis, int index,
                                int* count) {
    int64_t n;
    int c[3];
    if (!grid_cell(L, n, c[0], c[1], c[2])) return;
    if (c[axis] != index) return;
    const int o = own[n];
    if (o != 0 && kind[o - 1] == BODY_SPHERE) atomicAdd(count, 1);
}

__global__ void k_plane_claim(const Lattice L, int32_t* own, int axis, int index, int id) {
    int64_t n;
    int c[3];
    if (!grid_cell(L, n, c[0], c[1], c[2])) return;
    if (c[axis] == index && own[n] == 0) own[n] = id;
}

// A round tube along z (BodyParams::tube): solid nodes already held by a
// sphere, counted; free solid nodes claimed for body `id`.
__global__ void k_tube_overlap(const Lattice L, const int32_t* own, const int* kind, const BodyParams q, int* count) {
    int64_t n;
    int c[3];
    if (!grid_cell(L, n, c[0], c[1], c[2])) return;
    if (!tube_solid(q, c[0], c[1])) return;
    const int o = own[n];
    if (o != 0 && kind[o - 1] == BODY_SPHERE) atomicAdd(count, 1);
}

__global__ void k_tube_claim(const Lattice L, int32_t* own, const BodyParams q, int id) {
    int64_t n;
    int c[3];
    if (!grid_cell(L, n, c[0], c[1], c[2])) return;
    if (tube_solid(q, c[0], c[1]) && own[n] == 0) own[n] = id;
}

// Work flag for set-up passes: body k (or all if k < 0) re-classifies (and
// its node margin restarts) or not.
__global__ void k_set_flags(BodyAcc* acc, int nb, int k, int reclass) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb || (k >= 0 && j != k)) return;
    acc[j].reclass = reclass;
    if (reclass) acc[j].margin_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
}

// ---------------------------------------------------------------- launchers

void launch_fill_rest(const Lattice& L, cudaStream_t st) { k_fill_rest<<<grid_for(L.N), kB, 0, st>>>(L); }
void launch_set_eq(const Lattice& L, const double* rho, const double* u, int q, cudaStream_t st) {
    k_set_eq<<<grid_for(L.N), kB, 0, st>>>(L, rho, u, q);
}
void launch_set_pop(const Lattice& L, const double* f, int q, cudaStream_t st) {
    k_set_pop<<<grid_for(L.N), kB, 0, st>>>(L, f, q);
}
void launch_get_pop(const Lattice& L, double* f, int q, cudaStream_t st) {
    k_get_pop<<<grid_for(L.N), kB, 0, st>>>(L, f, q);
}
void launch_fields(const Lattice& L, const int32_t* own, double* rho, double* u, int q, cudaStream_t st) {
    k_fields<<<grid_for(L.N), kB, 0, st>>>(L, own, rho, u, q);
}
int mass_partial_blocks(const Lattice& L) { return (int)grid_for(L.N); }
void launch_mass(const Lattice& L, const int32_t* own, double* part, double* out, int q, cudaStream_t st) {
    const int nb = (int)grid_for(L.N);
    k_mass_partial<<<nb, kB, 0, st>>>(L, own, part, q);
    k_mass_final<<<1, kB, 0, st>>>(part, nb, out);
}
void launch_sphere_overlap(const Lattice& L, const int32_t* own, const double* pos, double R, int W, int* count,
                           cudaStream_t st) {
    const long long total = (long long)W * W * W;
    k_sphere_overlap<<<(unsigned)((total + kB - 1) / kB), kB, 0, st>>>(L, own, pos[0], pos[1], pos[2], R, W, count);
}
void launch_plane_overlap(const Lattice& L, const int32_t* own, const int* kind, int axis, int index, int* count,
                          cudaStream_t st) {
    k_plane_overlap<<<grid_for(L.N), kB, 0, st>>>(L, own, kind, axis, index, count);
}
void launch_plane_claim(const Lattice& L, int32_t* own, int axis, int index, int id, cudaStream_t st) {
    k_plane_claim<<<grid_for(L.N), kB, 0, st>>>(L, own, axis, index, id);
}
void launch_tube_overlap(const Lattice& L, const int32_t* own, const int* kind, const BodyParams& q, int* count,
                         cudaStream_t st) {
    k_tube_overlap<<<grid_for(L.N), kB, 0, st>>>(L, own, kind, q, count);
}
void launch_tube_claim(const Lattice& L, int32_t* own, const BodyParams& q, int id, cudaStream_t st) {
    k_tube_claim<<<grid_for(L.N), kB, 0, st>>>(L, own, q, id);
}
void launch_set_flags(BodyAcc* acc, int nb, int k, int reclass, cudaStream_t st) {
    k_set_flags<<<(nb + kB - 1) / kB, kB, 0, st>>>(acc, nb, k, reclass);
}


// Shell stencil of a sphere of radius R for k_body_fused: the offsets o from
// the centre's node floor(r) for which some centre fraction f in [0,1]^3 puts
// |o - f|^2 inside the bounds of in_shell widened by 1, packed as
// (ox + 512) | (oy + 512) << 10 | (oz + 512) << 20, in (z, y, x) order.
// Requires R <= kStencilMaxR.
std::vector<uint32_t> shell_stencil(double R) {
    const double lo2 = R > 1.5 ? (R - 1.5) * (R - 1.5) - 0.25 : -1.0;
    const double hi2 = (R + 2.0) * (R + 2.0) + 0.25;
    const int m = (int)std::ceil(R + 4.0);
    std::vector<uint32_t> v;
    for (int oz = -m; oz <= m; ++oz)
        for (int oy = -m; oy <= m; ++oy)
            for (int ox = -m; ox <= m; ++ox) {
                const int o[3] = {ox, oy, oz};
                double dmin = 0.0, dmax = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double t = o[a];
                    const double nearest = t < 0.0 ? -t : (t > 1.0 ? t - 1.0 : 0.0);
                    const double farthest = std::max(std::fabs(t), std::fabs(t - 1.0));
                    dmin += nearest * nearest;
                    dmax += farthest * farthest;
                }
                if (dmin < hi2 + 1.0 && dmax > lo2 - 1.0)
                    v.push_back((uint32_t)(ox + 512) | (uint32_t)(oy + 512) << 10 | (uint32_t)(oz + 512) << 20);
            }
    return v;
}

}  // namespace lbsq
