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

#include <type_traits>

#include "lbsq_internal.cuh"
#include "sweep_df.cuh"

namespace lbsq {

// Rate constants of the collision, computed once per sweep (FP64 and FP32):
// le, le / 3, 1 - le, -le / 2, -lo / 2, 3 lo / 18, 3 lo / 36, (1 - lo) / 2.
struct TrtK {
    double d[8];
    float f[8];
    int inc;  // 1: incompressible equilibrium, u = j / rho0 (the quadratic terms take 1/rho0)
    DfK df;   // the same constants (and rho0, 1/rho0) as double-float pairs, for FP64 storage
};
__host__ __device__ inline TrtK trt_constants(double le, double lo) {
    TrtK k;
    const double v[8] = {le,       le / 3.0,         1.0 - le,         -0.5 * le,
                         -0.5 * lo, 3.0 * lo / 18.0, 3.0 * lo / 36.0, 0.5 * (1.0 - lo)};
    for (int i = 0; i < 8; ++i) {
        k.d[i] = v[i];
        k.f[i] = (float)v[i];
    }
    k.inc = 0;
    return k;
}
struct SweepArgs {
    void* F;
    int nx, ny, nz;
    int64_t Np;
    double lambda_e, lambda_o, rho0;
    float scale, inv_scale;
    // rho0 in FP32 and in the 16-bit storages' scaled units (rho0 * scale),
    // converted once here rather than per thread (FP64 conversions issue at
    // the FP64 rate)
    float rho0f, rho0s;
    // near-body window split.  The window is the box of rows win[0..3] =
    // (z0, z length, y0, y length), periodic in both.  Mode 0 sweeps every
    // cell; mode 1 ("far") every cell outside the window; mode 2 ("near") the
    // cells inside it, blockIdx.z counting planes from z0 and the grid's rows
    // counting from y0
    TrtK K;  // collision constants (trt_constants)
    int zmode;
    const int* win;
    // planes in descending order (blocks are dispatched roughly in blockIdx
    // order): sweeps alternate direction, so that a sweep first reads the
    // planes the previous sweep wrote last, which are still in L2.  Any plane
    // order gives the same result (each cell touches only its own slots).
    int reverse;
    int* err;  // the lattice's device error word (bounded waits that run out)
    // stochastic rounding of BF16 stores (Lattice::sr): the step number comes
    // from the context's ping-pong counter (sr_ctr, advanced by the launch
    // with sr_writer set) or from the server's global step less start_step
    int sr, sr_writer;
    unsigned long long* sr_ctr;
    const long long* gstep;
    long long gstart;
    // two-cell form: the plane, this many planes ahead in sweep order, whose
    // sources each thread prefetches into L2 (0: none; see sweep_two)
    int pf;
};

// Plane of plane slot bz (grid z index, or a block's k-th plane in the
// multi-plane form), or -1 if none.  The far sweep leaves out a window plane
// only when the window spans every row.
__device__ __forceinline__ int sweep_plane_at(const SweepArgs& a, int bz) {
    if (a.zmode == 0) return a.reverse ? a.nz - 1 - bz : bz;
    const int z0 = __ldg(a.win), len = __ldg(a.win + 1);
    if (a.zmode == 2) {
        if (bz >= len) return -1;
        const int z = z0 + (a.reverse ? len - 1 - bz : bz);
        return z >= a.nz ? z - a.nz : z;
    }
    if (a.reverse) bz = a.nz - 1 - bz;
    const int rel = bz - z0 < 0 ? bz - z0 + a.nz : bz - z0;
    return rel < len && __ldg(a.win + 3) >= a.ny ? -1 : bz;
}

// Row swept by grid row ly on plane z (a plane sweep_plane_at returned), or
// -1 if none.
__device__ __forceinline__ int sweep_row(const SweepArgs& a, int ly, int z) {
    if (a.zmode == 0) return ly < a.ny ? ly : -1;
    const int y0 = __ldg(a.win + 2), ylen = __ldg(a.win + 3);
    if (a.zmode == 2) {
        if (ly >= ylen) return -1;
        const int y = y0 + ly;
        return y >= a.ny ? y - a.ny : y;
    }
    if (ly >= a.ny) return -1;
    const int z0 = __ldg(a.win), zlen = __ldg(a.win + 1);
    const int rz = z - z0 < 0 ? z - z0 + a.nz : z - z0;
    const int ry = ly - y0 < 0 ? ly - y0 + a.ny : ly - y0;
    return rz < zlen && ry < ylen ? -1 : ly;
}

// Plane swept by this block, or -1 if none.
__device__ __forceinline__ int sweep_plane(const SweepArgs& a) { return sweep_plane_at(a, blockIdx.z); }

// Arithmetic of the collision with every rounding spelled out (no contraction
// left to the compiler), so that every sweep form -- one, two or four cells
// per thread, the server's tiles -- gives a cell the same bits.
template <class V> struct Ar;
template <> struct Ar<double> {
    __device__ static double c(double x) { return x; }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    // 1/a by Newton-Raphson (r <- r + r (1 - a r)) from the FP32 reciprocal:
    // the seed's relative error (< 2^-23) squares at each step, so two steps
    // leave only the final rounding (within an ulp of the quotient), with 4
    // FP64 FMAs instead of a full division on this GPU's slow FP64 pipe.
    // For a in the normal FP32 range (here a = rho, about 1).
    __device__ static double rcp(double a) {
        double r = (double)__frcp_rn((float)a);
        double e = __fma_rn(-a, r, 1.0);
        r = __fma_rn(r, e, r);
        e = __fma_rn(-a, r, 1.0);
        return __fma_rn(r, e, r);
    }
};
template <> struct Ar<float> {
    __device__ static float c(double x) { return (float)x; }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static float rcp(float a) { return __fdiv_rn(1.0f, a); }
};
// Signed sum over the nine velocity pairs of the component c(2p - 1) of the
// pair's first member times d[p].  The first member of every pair has a
// leading +1, and the first pair with a nonzero component has it positive,
// so the sum starts from a term, never from zero, and needs no negation.
template <class V, int AX>
__device__ __forceinline__ V pair_moment(const V d[10]) {
    using A = Ar<V>;
    V acc{};
    bool first = true;
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const int c = AX == 0 ? cx(i) : (AX == 1 ? cy(i) : cz(i));
        if (c == 0) continue;
        if (first) acc = d[p];
        else acc = c > 0 ? A::add(acc, d[p]) : A::sub(acc, d[p]);
        first = false;
    }
    return acc;
}

// c_i . v for the first member i of a pair (leading component +1).
template <class V>
__device__ __forceinline__ V pair_dot(int i, V x, V y, V z) {
    using A = Ar<V>;
    const int a = cx(i), b = cy(i), c = cz(i);
    if (a != 0 && b != 0) return b > 0 ? A::add(x, y) : A::sub(x, y);
    if (a != 0 && c != 0) return c > 0 ? A::add(x, z) : A::sub(x, z);
    if (b != 0 && c != 0) return c > 0 ? A::add(y, z) : A::sub(y, z);
    return a != 0 ? x : (b != 0 ? y : z);
}

// TRT collision (Sec. III) of one cell (V = double or float), in pair form: with s = g_i + g_ib and d = g_i - g_ib for the nine pairs,
//   g_0 += le (f_0^eq - g_0),
//   g_i  += E + O,  g_ib += E - O,
//   E = le (w_i base + 9/2 w_i (c_i.u)(c_i.j)) - le/2 s,  O = 3 lo w_i c_i.j - lo/2 d,
// base = rho - 3/2 rho u.u (deviations: rho - rho0 - 3/2 rho u.u), u = j / rho.
// The incompressible equilibrium (K.inc) is the same with rho0 in place of
// rho in the quadratic terms: base = rho - 3/2 |j|^2 / rho0, u = j / rho0.
// DEV: g holds deviations f - w rho0 (rho = rho0 + sum g).
template <class V> __device__ __forceinline__ const V* trt_k(const TrtK& k);
template <> __device__ __forceinline__ const double* trt_k<double>(const TrtK& k) { return k.d; }
template <> __device__ __forceinline__ const float* trt_k<float>(const TrtK& k) { return k.f; }

template <class V, bool DEV>
__device__ __forceinline__ void collide_trt(V g[Q], const TrtK& K, V rho0) {
    using A = Ar<V>;
    const V* k = trt_k<V>(K);
    const V le = k[0];
    V s[10], d[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        s[p] = A::add(g[2 * p - 1], g[2 * p]);
        d[p] = A::sub(g[2 * p - 1], g[2 * p]);
    }
    V sum = g[0];
#pragma unroll
    for (int p = 1; p <= 9; ++p) sum = A::add(sum, s[p]);
    const V jx = pair_moment<V, 0>(d), jy = pair_moment<V, 1>(d), jz = pair_moment<V, 2>(d);
    const V rho = DEV ? A::add(rho0, sum) : sum;
    const V inv = A::rcp(K.inc ? rho0 : rho);
    // no velocity vector: rho u.u = |j|^2 / rho and (c.u)(c.j) = (c.j)^2 / rho
    const V ju = A::mul(A::fma(jz, jz, A::fma(jy, jy, A::mul(jx, jx))), inv);  // rho u.u
    const V base = A::fma(A::c(-1.5), ju, DEV ? sum : rho);
    const V q18 = A::mul(A::c(4.5 / 18.0), inv), q36 = A::mul(A::c(4.5 / 36.0), inv);
    const V lw18 = k[5], lw36 = k[6];
    const V wb18 = A::mul(A::c(1.0 / 18.0), base), wb36 = A::mul(A::c(1.0 / 36.0), base);
    if (k[2] == V(0)) {
        // le = 1 (every TRT and BGK configuration here): the even part relaxes
        // fully, so with h = (1 - lo)/2 d + 3 lo w (c.j) the pair update is
        //   g_i = ep + h,  g_ib = ep - h,  g_0 = base / 3,
        // the general form below with the s terms cancelled exactly.
        g[0] = A::mul(k[1], base);
        const V ch = k[7];
#pragma unroll
        for (int p = 1; p <= 9; ++p) {
            const int i = 2 * p - 1;
            const bool face = i < 7;
            const V cj = pair_dot<V>(i, jx, jy, jz);
            const V ep = A::fma(face ? q18 : q36, A::mul(cj, cj), face ? wb18 : wb36);
            const V h = A::fma(face ? lw18 : lw36, cj, A::mul(ch, d[p]));
            g[i] = A::add(ep, h);
            g[i + 1] = A::sub(ep, h);
        }
        return;
    }
    // g_0 + le (base / 3 - g_0) = (le / 3) base + (1 - le) g_0
    g[0] = A::fma(k[1], base, A::mul(k[2], g[0]));
    const V mhle = k[3], mhlo = k[4];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const bool face = i < 7;
        const V cj = pair_dot<V>(i, jx, jy, jz);
        const V ep = A::fma(face ? q18 : q36, A::mul(cj, cj), face ? wb18 : wb36);
        const V E = A::fma(le, ep, A::mul(mhle, s[p]));
        const V O = A::fma(face ? lw18 : lw36, cj, A::mul(mhlo, d[p]));
        g[i] = A::add(g[i], A::add(E, O));
        g[i + 1] = A::add(g[i + 1], A::sub(E, O));
    }
}

// 16-bit storages hold the deviations times a power of two s (FP16: 2^k,
// BF16: 1).  The collision is homogeneous of degree one in (g, rho0) -- u =
// j / rho does not change, every other term scales by s -- and scaling by a
// power of two commutes with every FP32 rounding (products, quotients, sums
// and FMAs alike, barring overflow and subnormals, far from these values).
// So the sweep collides the stored values as they are, with rho0 s for rho0,
// and gets the same bits as descaling, colliding and rescaling would, without
// a multiply per population.
template <int S> constexpr bool kScaled = S == ST_F16 || S == ST_BF16;

// ---- stochastic rounding of BF16 stores (SweepArgs::sr)
//
// The value's FP32 bits plus 16 random bits, truncated to the top 16 bits:
// rounds away from zero with probability equal to the dropped fraction of a
// BF16 unit, so the expected stored value is the value itself.  The random
// bits are a counter-based hash of (step, cell, population): a step key,
// then a cell key (both by the "lowbias32" integer hash of C. Wellons,
// 2018), then one multiply by an odd constant per population.  Every sweep
// form hashes the same (step, cell index, post-collision population), so the
// forms still agree bit for bit.
__device__ __forceinline__ uint32_t sr_mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// The random bits of a store come in pairs: one 32-bit word per pair of cells
// (2m, 2m + 1) (cell index n, pair n >> 1) and population i, its low half for
// the even cell and its high half for the odd one.  (Cells of a pair sit side
// by side in x when nx is even; for odd nx the pairing still gives every form
// the same bits.)
// The step number of this sweep, and (by the designated launch) the
// context's counter for the next.  Called by every thread of a sweep kernel
// before any early exit.
__device__ __forceinline__ uint32_t sr_step(const SweepArgs& a) {
    if (!a.sr) return 0u;
    if (a.gstep) return (uint32_t)(*a.gstep - a.gstart);
    const int q = a.reverse;  // the sweep's parity
    const unsigned long long t = a.sr_ctr[q];
    if (a.sr_writer && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0)
        a.sr_ctr[1 - q] = t + 1;
    return (uint32_t)t;
}
__device__ __forceinline__ uint32_t sr_step_key(const SweepArgs& a) { return sr_mix(sr_step(a) ^ 0x5bd1e995u); }
__device__ __forceinline__ uint32_t sr_pair_key(uint32_t step_key, uint32_t n) { return sr_mix((n >> 1) ^ step_key); }
// 32 random bits for post-collision population i of the pair with key k
__device__ __forceinline__ uint32_t sr_word(uint32_t k, int i) { return k * (0x9e3779b1u + 2u * (uint32_t)i * 0x61c88647u); }
// the 16 bits of a word for the even (low half) or odd (high half) cell
__device__ __forceinline__ uint32_t sr_half(uint32_t w, uint32_t n) { return (n & 1u) ? (w >> 16) : (w & 0xffffu); }
// The rounding itself is one conversion instruction per pair of values:
// cvt.rs.bf16x2.f32 (stochastic rounding, sm_100 family) converts (hi, lo)
// to a BF16 pair packed hi << 16 | lo, hi with the high 16 bits of rbits and
// lo with the low 16.  Checked on GB300 against the integer form
// (bits + r) >> 16 on a million random pairs: identical for every non-NaN
// value (subnormals, zeros and the carry into infinity included); a NaN comes
// out as the canonical NaN.
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
// BF16 bits of v (in the storage's units), rounded stochastically with the 16 bits r
__device__ __forceinline__ unsigned short bf16_sr(float v, uint32_t r) {
    return (unsigned short)cvt_rs_bf16x2(v, v, r);
}
// BF16 bits of (a, b), rounded stochastically with the halves of w, packed a | b << 16
__device__ __forceinline__ uint32_t bf16x2_sr(float a, float b, uint32_t w) { return cvt_rs_bf16x2(b, a, w); }

// One cell (x, y, z) with FP64 storage, collided in double-float arithmetic
// (sweep_df.cuh).  O32: element offsets in 32-bit arithmetic (the launch
// checks 19 Np < 2^32).
template <int P, bool O32 = false, bool LE1 = true>
__device__ __forceinline__ void sweep_one_df(const SweepArgs& a, int x, int y, int z) {
    using Off = typename std::conditional<O32, uint32_t, int64_t>::type;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    uint2* __restrict__ F = (uint2*)a.F;
    const Off Np = (Off)a.Np;
    auto cell = [&](int dx, int dy, int dz) -> Off {
        return (Off)xs[1 + dx] + (Off)nx * ((Off)ys[1 + dy] + (Off)ny * (Off)zs[1 + dz]);
    };
    // L2 prefetch of the sources a.pf planes ahead in sweep order (as in
    // sweep_two): their loads then wait on L2 rather than on HBM
    if (a.pf) {
        const int zp = z + (a.reverse ? -a.pf : a.pf);
        if (zp >= 0 && zp < nz) {
            const int zsp[3] = {zp == 0 ? nz - 1 : zp - 1, zp, zp == nz - 1 ? 0 : zp + 1};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const Off c = P == 0 ? (Off)x + (Off)nx * ((Off)y + (Off)ny * (Off)zp)
                                     : (Off)xs[1 - cx(i)] + (Off)nx * ((Off)ys[1 - cy(i)] + (Off)ny * (Off)zsp[1 - cz(i)]);
                const uint2* src = F + ((P == 0 ? (Off)i : (Off)opp(i)) * Np + c);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(src));
            }
        }
    }
    uint2 w[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
        w[i] = ld_stream(F + (P == 0 ? (Off)i * Np + cell(0, 0, 0) : (Off)opp(i) * Np + cell(-cx(i), -cy(i), -cz(i))));
    df g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = df_from_bits(w[i].x, w[i].y);
    const bool ok = collide_trt_df<LE1>(g, a.K.df, a.K.inc);
#pragma unroll
    for (int i = 0; i < Q; ++i) w[i] = df_to_bits(g[i]);
    if (!ok) {
#pragma unroll
        for (int i = 0; i < Q; ++i) w[i] = make_uint2(0u, 0x7ff80000u);  // NaN: keep a diverged cell visible
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
        st_stream(F + (P == 0 ? (Off)opp(i) * Np + cell(0, 0, 0) : (Off)i * Np + cell(cx(i), cy(i), cz(i))), w[i]);
}

// One cell (x, y, z).  FP64 storage collides in double-float arithmetic
// unless NATIVE (FP64 arithmetic, the measured reference form); O32 (caller
// checks 19 Np < 2^32) gives that form 32-bit element offsets.
template <int S, int P, bool NATIVE = false, bool O32 = false>
__device__ __forceinline__ void sweep_one(const SweepArgs& a, int x, int y, int z, uint32_t skey = 0u) {
    if constexpr (S == ST_F64 && !NATIVE) {
        if (a.K.df.le1) sweep_one_df<P, O32, true>(a, x, y, z);
        else sweep_one_df<P, O32, false>(a, x, y, z);
    } else {
    using ST = StoreT<S>;
    using T = typename ST::T;
    using R = typename ST::R;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    T* __restrict__ F = (T*)a.F;
    const int64_t Np = a.Np;
    // 16-bit storages collide in their scaled units (see kScaled)
    const R isc = kScaled<S> ? R(1) : (R)a.inv_scale, sc = kScaled<S> ? R(1) : (R)a.scale;
    const R rho0 = kScaled<S> ? (R)a.rho0s : (std::is_same<R, float>::value ? (R)a.rho0f : (R)a.rho0);
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
    collide_trt<R, ST::dev>(g, a.K, rho0);
    const uint32_t ncell = (uint32_t)(x + nx * (y + ny * z));
    const uint32_t ck = S == ST_BF16 && a.sr ? sr_pair_key(skey, ncell) : 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int64_t off;
        if (P == 0) {
            off = (int64_t)opp(i) * Np + (x + (int64_t)nx * (y + (int64_t)ny * z));
        } else {
            off = (int64_t)i * Np + (xs[1 + cx(i)] + (int64_t)nx * (ys[1 + cy(i)] + (int64_t)ny * zs[1 + cz(i)]));
        }
        if constexpr (S == ST_BF16) {
            if (a.sr) {
                st_stream(reinterpret_cast<unsigned short*>(F + off), bf16_sr((float)g[i], sr_half(sr_word(ck, i), ncell)));
                continue;
            }
        }
        ST::store(F + off, g[i], sc);
    }
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

// Encode two values into the storage's pair type (one packed conversion for
// the 16-bit storages; each half rounds as enc would).
template <int S> __device__ __forceinline__ typename Pair<typename StoreT<S>::T>::V enc2(float a, float b, float sc);
template <> __device__ __forceinline__ float2 enc2<ST_F32>(float a, float b, float) { return make_float2(a, b); }
template <> __device__ __forceinline__ __half2 enc2<ST_F16>(float a, float b, float sc) {
    return __floats2half2_rn(a * sc, b * sc);
}
template <> __device__ __forceinline__ __nv_bfloat162 enc2<ST_BF16>(float a, float b, float sc) {
    return __floats2bfloat162_rn(a * sc, b * sc);
}
template <> __device__ __forceinline__ double2 enc2<ST_F64>(float, float, float) { return make_double2(0.0, 0.0); }

// enc2 with the stochastic rounding of BF16 stores when sr is set (random
// bits w from sr_word)
template <int S>
__device__ __forceinline__ typename Pair<typename StoreT<S>::T>::V enc2_r(float a, float b, float sc, bool sr,
                                                                           uint32_t w) {
    if constexpr (S == ST_BF16) {
        if (sr) {
            const uint32_t p = bf16x2_sr(a, b, w);
            __nv_bfloat162 v;
            memcpy(&v, &p, 4);
            return v;
        }
    }
    return enc2<S>(a, b, sc);
}

// Two cells (x0, x0 + 1), x0 even; nx must be even.  Paired (vector)
// accesses wherever both cells' slots are adjacent and aligned: all
// directions on even steps, the directions with c_x = 0 on odd steps; scalar
// accesses for the x-shifted slots of odd steps.  Twice the bytes in flight per
// thread of the one-cell form, for the same arithmetic per cell.
// O32: element offsets in 32-bit arithmetic (the launch checks 19 Np < 2^32):
// three instructions an access instead of about seven.
template <int S, int P, bool O32, bool SR>
__device__ __forceinline__ void sweep_two_r(const SweepArgs& a, int x0, int y, int z, uint32_t skey) {
    using Off = typename std::conditional<O32, uint32_t, int64_t>::type;
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
    const Off Np = (Off)a.Np;
    const float isc = kScaled<S> ? 1.0f : a.inv_scale, sc = kScaled<S> ? 1.0f : a.scale;
    const R rho0 = kScaled<S> ? (R)a.rho0s : (std::is_same<R, float>::value ? (R)a.rho0f : (R)a.rho0);
    auto row = [&](int dy, int dz) -> Off { return (Off)nx * ((Off)ys[1 + dy] + (Off)ny * (Off)zs[1 + dz]); };
    // Prefetch into L2 what this thread's cells will read a.pf planes ahead in
    // sweep order: the block that sweeps that plane starts later, when the
    // blocks resident now (about a.pf - 2 planes of them) are done, and finds
    // its sources in L2.  A prefetch holds no register, so it adds to the bytes
    // in flight that the loads below are short of.
    if (a.pf) {
        const int zp = z + (a.reverse ? -a.pf : a.pf);
        if (zp >= 0 && zp < nz) {
            const int zsp[3] = {zp == 0 ? nz - 1 : zp - 1, zp, zp == nz - 1 ? 0 : zp + 1};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T* src = P == 0 ? F + ((Off)i * Np + (Off)nx * ((Off)y + (Off)ny * (Off)zp) + (Off)x0)
                                      : F + ((Off)opp(i) * Np +
                                             (Off)nx * ((Off)ys[1 - cy(i)] + (Off)ny * (Off)zsp[1 - cz(i)]) + (Off)x0);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(src));
            }
        }
    }
    R g0[Q], g1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (P == 0) {
            const V v = ld_stream(reinterpret_cast<const V*>(F + ((Off)i * Np + row(0, 0) + (Off)x0)));
            g0[i] = dec<S>(PV::lo(v), isc);
            g1[i] = dec<S>(PV::hi(v), isc);
        } else {
            const T* base = F + ((Off)opp(i) * Np + row(-cy(i), -cz(i)));
            if (cx(i) == 0) {
                const V v = ld_stream(reinterpret_cast<const V*>(base + x0));
                g0[i] = dec<S>(PV::lo(v), isc);
                g1[i] = dec<S>(PV::hi(v), isc);
            } else if (cx(i) == 1) {  // sources x0 - 1 and x0
                g0[i] = dec<S>(ld_stream(base + xm0), isc);
                g1[i] = dec<S>(ld_stream(base + x0), isc);
            } else {  // sources x0 + 1 and x0 + 2
                g0[i] = dec<S>(ld_stream(base + x0 + 1), isc);
                g1[i] = dec<S>(ld_stream(base + xp1), isc);
            }
        }
    }
    collide_trt<R, ST::dev>(g0, a.K, rho0);
    collide_trt<R, ST::dev>(g1, a.K, rho0);
    constexpr bool sr = SR;
    // cells x0 and x0 + 1 (x0 even, nx even) form one pair of the random bits
    const uint32_t kp = sr ? sr_pair_key(skey, (uint32_t)x0 + (uint32_t)nx * ((uint32_t)y + (uint32_t)ny * (uint32_t)z)) : 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint32_t w = sr ? sr_word(kp, i) : 0u;
        // both cells in one packed conversion, also where they are stored
        // apart (each half rounds as the scalar conversion would)
        const V e = enc2_r<S>(g0[i], g1[i], sc, sr, w);
        if (P == 0) {
            st_stream(reinterpret_cast<V*>(F + ((Off)opp(i) * Np + row(0, 0) + (Off)x0)), e);
        } else {
            T* base = F + ((Off)i * Np + row(cy(i), cz(i)));
            if (cx(i) == 0) {
                st_stream(reinterpret_cast<V*>(base + x0), e);
            } else if (cx(i) == 1) {  // targets x0 + 1 and x0 + 2
                st_stream(base + x0 + 1, Pair<T>::lo(e));
                st_stream(base + xp1, Pair<T>::hi(e));
            } else {  // targets x0 - 1 and x0
                st_stream(base + xm0, Pair<T>::lo(e));
                st_stream(base + x0, Pair<T>::hi(e));
            }
        }
    }
}

// The rounding mode is a compile-time branch of the two-cell body: one
// uniform branch per thread instead of a select between two conversions at
// every store.
template <int S, int P, bool O32 = false>
__device__ __forceinline__ void sweep_two(const SweepArgs& a, int x0, int y, int z, uint32_t skey = 0u) {
    if constexpr (S == ST_BF16) {
        if (a.sr) {
            sweep_two_r<S, P, O32, true>(a, x0, y, z, skey);
            return;
        }
    }
    sweep_two_r<S, P, O32, false>(a, x0, y, z, skey);
}

template <int S> __device__ __forceinline__ float dec16(unsigned int h, float isc);
template <> __device__ __forceinline__ float dec16<ST_F16>(unsigned int h, float isc) {
    return __half2float(__ushort_as_half((unsigned short)h)) * isc;
}
template <> __device__ __forceinline__ float dec16<ST_BF16>(unsigned int h, float isc) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)h)) * isc;
}
template <int S> __device__ __forceinline__ unsigned int enc16(float v, float sc);
template <> __device__ __forceinline__ unsigned int enc16<ST_F16>(float v, float sc) {
    return __half_as_ushort(__float2half_rn(v * sc));
}
template <> __device__ __forceinline__ unsigned int enc16<ST_BF16>(float v, float sc) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v * sc));
}

// Both values of a pair rounded to nearest, packed a | b << 16.
template <int S> __device__ __forceinline__ uint32_t enc16x2(float a, float b);
template <> __device__ __forceinline__ uint32_t enc16x2<ST_F16>(float a, float b) {
    const __half2 v = __floats2half2_rn(a, b);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}
template <> __device__ __forceinline__ uint32_t enc16x2<ST_BF16>(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// Collision of four cells x0 .. x0 + 3 of row (y, z) (x0 and nx multiples of
// 4) whose 16-bit populations g[i] hold two cells per 32-bit word (cell x0 in
// the low half of .x), in place: decode, TRT in FP32 in the storage's scaled
// units (see kScaled), encode (BF16 with stochastic rounding: the four cells
// are two pairs of the random bits).  Every four-cell form calls this, so they
// all give the same bits.
template <int S, bool SR>
__device__ __forceinline__ void collide_four_r(uint2 g[Q], const SweepArgs& a, uint32_t skey, int x0, int y, int z) {
    constexpr bool sr = SR;
    const float rho0 = a.rho0s;  // scaled units (see kScaled)
    const uint32_t n0 = (uint32_t)x0 + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
    const uint32_t k01 = sr ? sr_pair_key(skey, n0) : 0u, k23 = sr ? sr_pair_key(skey, n0 + 2u) : 0u;
    // the cells in pairs (x0, x0 + 1) and (x0 + 2, x0 + 3): a pair's word of
    // each population is decoded, both cells collide, and one packed
    // conversion writes the word back (each half rounds as the scalar
    // conversion would)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float ga[Q], gb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned int w = h == 0 ? g[i].x : g[i].y;
            ga[i] = dec16<S>(w & 0xffffu, 1.0f);
            gb[i] = dec16<S>(w >> 16, 1.0f);
        }
        collide_trt<float, true>(ga, a.K, rho0);
        collide_trt<float, true>(gb, a.K, rho0);
        const uint32_t kc = h == 0 ? k01 : k23;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t e = sr ? cvt_rs_bf16x2(gb[i], ga[i], sr_word(kc, i)) : enc16x2<S>(ga[i], gb[i]);
            (h == 0 ? g[i].x : g[i].y) = e;
        }
    }
}
template <int S>
__device__ __forceinline__ void collide_four(uint2 g[Q], const SweepArgs& a, uint32_t skey, int x0, int y, int z) {
    if constexpr (S == ST_BF16) {
        if (a.sr) {
            collide_four_r<S, true>(g, a, skey, x0, y, z);
            return;
        }
    }
    collide_four_r<S, false>(g, a, skey, x0, y, z);
}

// 16-bit storages, four cells per thread, blocks of whole rows: a row of nx
// cells is nx / 4 threads (nx % 4 == 0, nx <= 768), so the x-neighbours of
// every cell, the periodic wrap included, lie in the block.  Every global
// access is an aligned 8-byte chunk.  On odd steps the ten x-shifted
// directions go through a shared-memory copy of the rows: loads write the
// aligned source chunks there and read the shifted elements back; stores
// write the shifted results there and store the aligned chunks.  `buf` holds
// 10 x blockDim.y x nx elements.  All threads of the block take part in the
// barriers (`active`: the thread's row exists).
// O32: element offsets in 32-bit arithmetic (the launch checks 19 Np < 2^32).
template <int S, int P, bool O32 = false>
__device__ __forceinline__ void sweep_four_rows(const SweepArgs& a, int y, int z, bool active, unsigned short* buf,
                                                uint32_t skey = 0u) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = 4 * threadIdx.x;
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y >= ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    unsigned short* F = (unsigned short*)a.F;
    using Off = typename std::conditional<O32, uint32_t, int64_t>::type;
    const Off Np = (Off)a.Np;
    auto row = [&](int dy, int dz) -> Off { return (Off)nx * ((Off)ys[1 + dy] + (Off)ny * (Off)zs[1 + dz]); };
    unsigned short* rowbuf = buf + (int64_t)threadIdx.y * nx;  // + d * blockDim.y * nx for shifted direction d
    const int dstride = blockDim.y * nx;
    auto at = [&](int x) -> int { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    // even steps: L2 prefetch of the sources a.pf planes ahead (see sweep_two)
    if (P == 0 && a.pf && active) {
        const int zp = z + (a.reverse ? -a.pf : a.pf);
        if (zp >= 0 && zp < nz) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(F + ((Off)i * Np + (Off)nx * ((Off)y + (Off)ny * (Off)zp) +
                                                                   (Off)x0)));
        }
    }
    uint2 g[Q];
    int d = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (P == 0) {
            if (active) g[i] = ld_stream(reinterpret_cast<const uint2*>(F + ((Off)i * Np + row(0, 0) + (Off)x0)));
        } else {
            const unsigned short* base = F + ((Off)opp(i) * Np + row(-cy(i), -cz(i)));
            if (cx(i) == 0) {
                if (active) g[i] = ld_stream(reinterpret_cast<const uint2*>(base + x0));
            } else {
                if (active)
                    *reinterpret_cast<uint2*>(rowbuf + d * dstride + x0) = ld_stream(reinterpret_cast<const uint2*>(base + x0));
                ++d;
            }
        }
    }
    if (P == 1) {
        __syncthreads();
        d = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (cx(i) == 0) continue;
            const unsigned short* r = rowbuf + d * dstride;
            ++d;
            // sources x0 - 1 .. x0 + 2 (c_x = +1) or x0 + 1 .. x0 + 4 (c_x = -1)
            const int s0 = cx(i) == 1 ? x0 - 1 : x0 + 1;
            unsigned int e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = r[at(s0 + k)];
            g[i] = make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
        }
        __syncthreads();  // the buffer is reused for the stores
    }
    collide_four<S>(g, a, skey, x0, y, z);
    d = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint2 o = g[i];
        if (P == 0) {
            if (active) st_stream(reinterpret_cast<uint2*>(F + ((Off)opp(i) * Np + row(0, 0) + (Off)x0)), o);
        } else if (cx(i) == 0) {
            if (active) st_stream(reinterpret_cast<uint2*>(F + ((Off)i * Np + row(cy(i), cz(i)) + (Off)x0)), o);
        } else {
            // targets x0 + 1 .. x0 + 4 (c_x = +1) or x0 - 1 .. x0 + 2 (c_x = -1)
            unsigned short* r = rowbuf + d * dstride;
            ++d;
            const int t0 = cx(i) == 1 ? x0 + 1 : x0 - 1;
            r[at(t0)] = (unsigned short)(o.x & 0xffffu);
            r[at(t0 + 1)] = (unsigned short)(o.x >> 16);
            r[at(t0 + 2)] = (unsigned short)(o.y & 0xffffu);
            r[at(t0 + 3)] = (unsigned short)(o.y >> 16);
        }
    }
    if (P == 1) {
        __syncthreads();
        d = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (cx(i) == 0) continue;
            const unsigned short* r = rowbuf + d * dstride;
            ++d;
            if (active)
                st_stream(reinterpret_cast<uint2*>(F + ((Off)i * Np + row(cy(i), cz(i)) + (Off)x0)),
                          *reinterpret_cast<const uint2*>(r + x0));
        }
    }
}

// 16-bit storages, odd steps, four cells x0 .. x0 + 3 per thread (x0 and nx
// multiples of 4), no shared memory: each direction's four sources are the
// aligned 8-byte chunk at x0, shifted by one element with the element beyond
// its end (x0 - 1 for c_x = +1, x0 + 4 for c_x = -1, periodic) loaded on its
// own; the four results go out as one aligned 4-byte store of the middle two
// and 2-byte stores of the two ends.  Per shifted direction and four cells
// that is two loads and three stores, where two threads of the two-cell form
// issue four of each; the collision is the same (collide_four), so are the
// bits.
template <int S, bool O32 = false>
__device__ __forceinline__ void sweep_four_odd(const SweepArgs& a, int x0, int y, int z, uint32_t skey) {
    using Off = typename std::conditional<O32, uint32_t, int64_t>::type;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;   // x0 - 1
    const int xr = x0 + 4 == nx ? 0 : x0 + 4;   // x0 + 4
    unsigned short* __restrict__ F = (unsigned short*)a.F;
    const Off Np = (Off)a.Np;
    auto row = [&](int dy, int dz) -> Off { return (Off)nx * ((Off)ys[1 + dy] + (Off)ny * (Off)zs[1 + dz]); };
    // L2 prefetch of the sources a.pf planes ahead in sweep order (see sweep_two)
    if (a.pf) {
        const int zp = z + (a.reverse ? -a.pf : a.pf);
        if (zp >= 0 && zp < nz) {
            const int zsp[3] = {zp == 0 ? nz - 1 : zp - 1, zp, zp == nz - 1 ? 0 : zp + 1};
#pragma unroll
            for (int i = 0; i < Q; ++i)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(
                    F + ((Off)opp(i) * Np + (Off)nx * ((Off)ys[1 - cy(i)] + (Off)ny * (Off)zsp[1 - cz(i)]) + (Off)x0)));
        }
    }
    // g[i]: cells x0, x0 + 1 in .x, x0 + 2, x0 + 3 in .y (low half first)
    uint2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short* base = F + ((Off)opp(i) * Np + row(-cy(i), -cz(i)));
        const uint2 c = ld_stream(reinterpret_cast<const uint2*>(base + x0));
        if (cx(i) == 0) {
            g[i] = c;
        } else if (cx(i) == 1) {  // sources x0 - 1 .. x0 + 2
            const unsigned int e = ld_stream(base + xl);
            g[i] = make_uint2(__byte_perm(e, c.x, 0x5410), __byte_perm(c.x, c.y, 0x5432));
        } else {  // sources x0 + 1 .. x0 + 4
            const unsigned int e = ld_stream(base + xr);
            g[i] = make_uint2(__byte_perm(c.x, c.y, 0x5432), __byte_perm(c.y, e, 0x5432));
        }
    }
    collide_four<S>(g, a, skey, x0, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        unsigned short* base = F + ((Off)i * Np + row(cy(i), cz(i)));
        const uint2 o = g[i];
        const unsigned int mid = __byte_perm(o.x, o.y, 0x5432);  // cells x0 + 1, x0 + 2
        if (cx(i) == 0) {
            st_stream(reinterpret_cast<uint2*>(base + x0), o);
        } else if (cx(i) == 1) {  // targets x0 + 1 .. x0 + 4
            st_stream(base + x0 + 1, (unsigned short)(o.x & 0xffffu));
            st_stream(reinterpret_cast<unsigned int*>(base + x0 + 2), mid);
            st_stream(base + xr, (unsigned short)(o.y >> 16));
        } else {  // targets x0 - 1 .. x0 + 2
            st_stream(base + xl, (unsigned short)(o.x & 0xffffu));
            st_stream(reinterpret_cast<unsigned int*>(base + x0), mid);
            st_stream(base + x0 + 2, (unsigned short)(o.y >> 16));
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
    a.K = trt_constants(lambda_e, lambda_o);
    a.K.inc = L.inc;
    a.K.df = df_constants(lambda_e, lambda_o, L.rho0);
    a.rho0 = L.rho0;
    a.rho0f = (float)L.rho0;
    a.rho0s = (float)L.rho0 * L.scale;
    a.scale = L.scale;
    a.inv_scale = L.inv_scale;
    a.zmode = 0;
    a.win = nullptr;
    a.reverse = 0;
    a.err = L.err;
    a.pf = 0;
    a.sr = L.sr && L.storage == ST_BF16;
    a.sr_writer = 1;
    a.sr_ctr = L.sr_ctr;
    a.gstep = L.gstep;
    a.gstart = L.start_step;
    return a;
}

}  // namespace lbsq
