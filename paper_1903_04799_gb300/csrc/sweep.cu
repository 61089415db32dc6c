// sweep.cu -- fused stream + collide over the whole lattice (Sec. III, Eq. "lb").
//
// One thread per cell, grid (x-blocks, ny, nz).  The update is the in-place
// AA pattern (see lbsq_internal.cuh): even steps read and write a cell's own
// 19 slots, odd steps read and write its 19 neighbour slots.  The kernel is
// geometry-free: solid cells are swept too (their slots are private to them,
// and every slot a fluid cell reads from a solid neighbour is rewritten by
// the link kernel after the sweep), so no flag field is read.
//
// Collision: TRT in pair form.  For the pair (i, ib) with c = c_i:
//   E = lambda_e (feq+ - f+),  O = lambda_o (feq- - f-),
//   f*_i = f_i + E + O,  f*_ib = f_ib + E - O,
// with feq+ = w (rho (1 - 3/2 u.u) + 9/2 rho (c.u)^2) and feq- = 3 w c.j.
// Reduced storages hold g_i = f_i - w_i rho0; the same algebra runs on g with
// rho = rho0 + sum g and feq+ - w rho0 = w (sum g - 3/2 rho u.u + 9/2 rho (c.u)^2),
// which keeps the small quantities small and so keeps FP32 accurate.
#include "lbsq_internal.cuh"

namespace lbsq {

struct SweepArgs {
    void* F;
    int nx, ny, nz;
    int64_t Np;
    double lambda_e, lambda_o, rho0;
    float scale, inv_scale;
};

template <class R, bool DEV>
__device__ __forceinline__ void collide_trt(R g[Q], R le, R lo, R rho0) {
    // pair sums and differences
    R s[10], d[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        s[p] = g[2 * p - 1] + g[2 * p];
        d[p] = g[2 * p - 1] - g[2 * p];
    }
    R sum = g[0];
#pragma unroll
    for (int p = 1; p <= 9; ++p) sum += s[p];
    R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        if (cx(2 * p - 1) == 1) jx += d[p];
        if (cx(2 * p - 1) == -1) jx -= d[p];
        if (cy(2 * p - 1) == 1) jy += d[p];
        if (cy(2 * p - 1) == -1) jy -= d[p];
        if (cz(2 * p - 1) == 1) jz += d[p];
        if (cz(2 * p - 1) == -1) jz -= d[p];
    }
    const R rho = DEV ? rho0 + sum : sum;
    const R inv = R(1) / rho;
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const R ju = jx * ux + jy * uy + jz * uz;  // rho u.u
    // base = (feq+ of the rest class) / w, minus rho0 for deviations
    const R base = (DEV ? sum : rho) - R(1.5) * ju;
    g[0] = g[0] + le * (R(1.0 / 3.0) * base - g[0]);
    const R hle = R(0.5) * le, hlo = R(0.5) * lo;
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const R w = (R)wgt(i);
        R cu = R(0), cj = R(0);
        if (cx(i) == 1) { cu += ux; cj += jx; }
        if (cx(i) == -1) { cu -= ux; cj -= jx; }
        if (cy(i) == 1) { cu += uy; cj += jy; }
        if (cy(i) == -1) { cu -= uy; cj -= jy; }
        if (cz(i) == 1) { cu += uz; cj += jz; }
        if (cz(i) == -1) { cu -= uz; cj -= jz; }
        const R ep = w * base + R(4.5) * w * (cu * cj);
        const R E = le * ep - hle * s[p];
        const R O = (R(3) * lo) * w * cj - hlo * d[p];
        g[i] = g[i] + (E + O);
        g[i + 1] = g[i + 1] + (E - O);
    }
}

template <int S, int P>
__global__ void __launch_bounds__(256) k_sweep(const SweepArgs a) {
    using ST = StoreT<S>;
    using T = typename ST::T;
    using R = typename ST::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    T* __restrict__ F = (T*)a.F;
    const int64_t Np = a.Np;
    const R isc = (R)a.inv_scale, sc = (R)a.scale;
    R g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int64_t off;
        if (P == 0) {
            off = (int64_t)i * Np + (x + (int64_t)nx * (y + (int64_t)ny * z));
        } else {
            const int ib = opp(i);
            off = (int64_t)ib * Np +
                  (xs[1 - cx(i)] + (int64_t)nx * (ys[1 - cy(i)] + (int64_t)ny * zs[1 - cz(i)]));
        }
        g[i] = ST::load(F + off, isc);
    }
    collide_trt<R, ST::dev>(g, (R)a.lambda_e, (R)a.lambda_o, (R)a.rho0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int64_t off;
        if (P == 0) {
            off = (int64_t)opp(i) * Np + (x + (int64_t)nx * (y + (int64_t)ny * z));
        } else {
            off = (int64_t)i * Np + (xs[1 + cx(i)] + (int64_t)nx * (ys[1 + cy(i)] + (int64_t)ny * zs[1 + cz(i)]));
        }
        ST::store(F + off, g[i], sc);
    }
}

template <int S>
static void launch_s(const SweepArgs& a, int parity, cudaStream_t st) {
    int bx = ((a.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    dim3 grid((a.nx + bx - 1) / bx, a.ny, a.nz);
    if (parity == 0) k_sweep<S, 0><<<grid, bx, 0, st>>>(a);
    else k_sweep<S, 1><<<grid, bx, 0, st>>>(a);
}

void launch_sweep(const Lattice& L, double lambda_e, double lambda_o, int parity, cudaStream_t st) {
    SweepArgs a;
    a.F = L.F;
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.Np = L.Np;
    a.lambda_e = lambda_e;
    a.lambda_o = lambda_o;
    a.rho0 = L.rho0;
    a.scale = L.scale;
    a.inv_scale = L.inv_scale;
    switch (L.storage) {
        case ST_F64: launch_s<ST_F64>(a, parity, st); break;
        case ST_F32: launch_s<ST_F32>(a, parity, st); break;
        case ST_F16: launch_s<ST_F16>(a, parity, st); break;
        default: launch_s<ST_BF16>(a, parity, st); break;
    }
}

}  // namespace lbsq
