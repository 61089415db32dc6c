// sweep_body.cuh -- the per-cell fused stream + collide of Sec. III, Eq. "lb",
// shared by the single-lattice sweep kernels (sweep.cu) and the multi-lattice
// tile sweep of the server (serve.cu), so that both run identical arithmetic.
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
#pragma once

#include "lbsq_internal.cuh"

namespace lbsq {

struct SweepArgs {
    void* F;
    int nx, ny, nz;
    int64_t Np;
    double lambda_e, lambda_o, rho0;
    float scale, inv_scale;
    // z-window split: mode 0 sweeps every plane; mode 1 ("far") the planes
    // outside the window win[0..1] = (z0, length); mode 2 ("near") the planes
    // inside it, blockIdx.z counting from z0
    int zmode;
    const int* win;
    // planes in descending order (blocks are dispatched roughly in blockIdx
    // order): sweeps alternate direction, so that a sweep first reads the
    // planes the previous sweep wrote last, which are still in L2.  Any plane
    // order gives the same result (each cell touches only its own slots).
    int reverse;
};

// Plane swept by this block, or -1 if none.
__device__ __forceinline__ int sweep_plane(const SweepArgs& a) {
    int bz = blockIdx.z;
    if (a.zmode == 0) return a.reverse ? a.nz - 1 - bz : bz;
    const int z0 = __ldg(a.win), len = __ldg(a.win + 1);
    if (a.zmode == 2) {
        if (bz >= len) return -1;
        const int z = z0 + (a.reverse ? len - 1 - bz : bz);
        return z >= a.nz ? z - a.nz : z;
    }
    if (a.reverse) bz = a.nz - 1 - bz;
    const int rel = bz - z0 < 0 ? bz - z0 + a.nz : bz - z0;
    return rel < len ? -1 : bz;
}

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

// One cell (x, y, z).
template <int S, int P>
__device__ __forceinline__ void sweep_one(const SweepArgs& a, int x, int y, int z) {
    using ST = StoreT<S>;
    using T = typename ST::T;
    using R = typename ST::R;
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

// Two-cell pair types: the stored element type T and its 2-vector.
template <class T> struct Pair;
template <> struct Pair<double> { using V = double2; __device__ static double lo(V v) { return v.x; } __device__ static double hi(V v) { return v.y; } __device__ static V make(double a, double b) { return make_double2(a, b); } };
template <> struct Pair<float> { using V = float2; __device__ static float lo(V v) { return v.x; } __device__ static float hi(V v) { return v.y; } __device__ static V make(float a, float b) { return make_float2(a, b); } };
template <> struct Pair<__half> { using V = __half2; __device__ static __half lo(V v) { return __low2half(v); } __device__ static __half hi(V v) { return __high2half(v); } __device__ static V make(__half a, __half b) { return __halves2half2(a, b); } };
template <> struct Pair<__nv_bfloat16> { using V = __nv_bfloat162; __device__ static __nv_bfloat16 lo(V v) { return __low2bfloat16(v); } __device__ static __nv_bfloat16 hi(V v) { return __high2bfloat16(v); } __device__ static V make(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); } };

// Decode / encode one stored element (same arithmetic as StoreT::load / store).
template <int S> __device__ __forceinline__ typename StoreT<S>::R dec(typename StoreT<S>::T v, float isc);
template <> __device__ __forceinline__ double dec<ST_F64>(double v, float) { return v; }
template <> __device__ __forceinline__ float dec<ST_F32>(float v, float) { return v; }
template <> __device__ __forceinline__ float dec<ST_F16>(__half v, float isc) { return __half2float(v) * isc; }
template <> __device__ __forceinline__ float dec<ST_BF16>(__nv_bfloat16 v, float isc) { return __bfloat162float(v) * isc; }
template <int S> __device__ __forceinline__ typename StoreT<S>::T enc(typename StoreT<S>::R v, float sc);
template <> __device__ __forceinline__ double enc<ST_F64>(double v, float) { return v; }
template <> __device__ __forceinline__ float enc<ST_F32>(float v, float) { return v; }
template <> __device__ __forceinline__ __half enc<ST_F16>(float v, float sc) { return __float2half_rn(v * sc); }
template <> __device__ __forceinline__ __nv_bfloat16 enc<ST_BF16>(float v, float sc) { return __float2bfloat16_rn(v * sc); }

// Two cells (x0, x0 + 1), x0 even; nx must be even.  Paired (vector)
// accesses wherever both cells' slots are adjacent and aligned: all
// directions on even steps, the directions with c_x = 0 on odd steps; scalar
// accesses for the x-shifted slots of odd steps.  Twice the bytes in flight per
// thread of the one-cell form, for the same arithmetic per cell.
template <int S, int P>
__device__ __forceinline__ void sweep_two(const SweepArgs& a, int x0, int y, int z) {
    using ST = StoreT<S>;
    using T = typename ST::T;
    using R = typename ST::R;
    using PV = Pair<T>;
    using V = typename PV::V;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    // x coordinates of cell k in {0,1} shifted by -1, 0, +1 (periodic)
    const int xm0 = x0 == 0 ? nx - 1 : x0 - 1;  // x0 - 1
    const int xp1 = x0 + 2 == nx ? 0 : x0 + 2;  // x0 + 2
    T* __restrict__ F = (T*)a.F;
    const int64_t Np = a.Np;
    const float isc = a.inv_scale, sc = a.scale;
    auto row = [&](int dy, int dz) -> int64_t { return (int64_t)nx * (ys[1 + dy] + (int64_t)ny * zs[1 + dz]); };
    R g0[Q], g1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (P == 0) {
            const V v = *reinterpret_cast<const V*>(F + (int64_t)i * Np + row(0, 0) + x0);
            g0[i] = dec<S>(PV::lo(v), isc);
            g1[i] = dec<S>(PV::hi(v), isc);
        } else {
            const T* base = F + (int64_t)opp(i) * Np + row(-cy(i), -cz(i));
            if (cx(i) == 0) {
                const V v = *reinterpret_cast<const V*>(base + x0);
                g0[i] = dec<S>(PV::lo(v), isc);
                g1[i] = dec<S>(PV::hi(v), isc);
            } else if (cx(i) == 1) {  // sources x0 - 1 and x0
                g0[i] = dec<S>(base[xm0], isc);
                g1[i] = dec<S>(base[x0], isc);
            } else {  // sources x0 + 1 and x0 + 2
                g0[i] = dec<S>(base[x0 + 1], isc);
                g1[i] = dec<S>(base[xp1], isc);
            }
        }
    }
    collide_trt<R, ST::dev>(g0, (R)a.lambda_e, (R)a.lambda_o, (R)a.rho0);
    collide_trt<R, ST::dev>(g1, (R)a.lambda_e, (R)a.lambda_o, (R)a.rho0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (P == 0) {
            *reinterpret_cast<V*>(F + (int64_t)opp(i) * Np + row(0, 0) + x0) =
                PV::make(enc<S>(g0[i], sc), enc<S>(g1[i], sc));
        } else {
            T* base = F + (int64_t)i * Np + row(cy(i), cz(i));
            if (cx(i) == 0) {
                *reinterpret_cast<V*>(base + x0) = PV::make(enc<S>(g0[i], sc), enc<S>(g1[i], sc));
            } else if (cx(i) == 1) {  // targets x0 + 1 and x0 + 2
                base[x0 + 1] = enc<S>(g0[i], sc);
                base[xp1] = enc<S>(g1[i], sc);
            } else {  // targets x0 - 1 and x0
                base[xm0] = enc<S>(g0[i], sc);
                base[x0] = enc<S>(g1[i], sc);
            }
        }
    }
}

// Arguments of a sweep of lattice L.
__host__ __device__ inline SweepArgs sweep_args(const Lattice& L, double lambda_e, double lambda_o) {
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
    a.zmode = 0;
    a.win = nullptr;
    a.reverse = 0;
    return a;
}

}  // namespace lbsq
