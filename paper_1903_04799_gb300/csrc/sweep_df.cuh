// sweep_df.cuh -- the TRT collision of Sec. III, Eq. "lb", for FP64 storage,
// computed in double-float arithmetic: every quantity is an unevaluated sum
// h + l of two FP32 numbers, carried by error-free transformations (Knuth's
// two-sum for additions, Dekker's product through FMA for multiplications).
//
// Why: GB300 issues FP64 arithmetic at about 2 lanes per SM and cycle against
// 128 for FP32.  A TRT update in FP64 is about 130 FP64 instructions per cell,
// which caps the FP64 sweep near a fifth of its HBM roofline.  The same update
// in double-float takes about 900 FP32 instructions, which the FP32 pipes
// retire in a third of the time the populations take to stream.
//
// Precision: FP64 storage holds the deviations g_i = f_i - w_i rho0, whose
// magnitude is that of the flow (|g| ~ 1e-3 here), not of f (~0.05 .. 1/3).
// The arithmetic carries about 47 significant bits of g, i.e. an absolute
// error near 2^-47 |g| per operation: below the rounding of f itself in FP64
// (ulp(1/3) / 2 = 2^-55), which is what the FP64 oracle carries.
//
// The conversions between an FP64 word and a pair run in integer arithmetic
// on the bit pattern (no FP64 instruction at all):
//   load:  h = the FP64 value truncated to 24 significant bits (exponent
//          rebiased 1023 -> 127), l = the remaining 29 mantissa bits, rounded
//          to 24 bits, with h's sign and exponent;
//   store: s = h + l rounded toward zero, e = (h + l) - s (same sign as s),
//          then the FP64 bits of s plus e counted in FP64 ulps of s.
// Magnitudes are clamped to [2^-126, 2^101) on load (deviations below 1e-38
// are zero for every purpose here); a cell whose density or momentum is not
// finite after that (NaN or Inf populations) stores NaN, so a diverged state
// stays visible to the mass sum and the body update.
#pragma once

#include <cstdint>

namespace lbsq {

// hi/lo parts of the collision's constants (DfK indices below), for DfK::h/l
enum DfIdx : int {
    DK_W18 = 0,  // 1/18
    DK_W3,       // 1/3
    DK_LW18,     // 3 lo / 18
    DK_LW36,     // 3 lo / 36
    DK_CH,       // (1 - lo) / 2
    DK_LE,       // le
    DK_LE3,      // le / 3
    DK_1MLE,     // 1 - le
    DK_MHLE,     // -le / 2
    DK_MHLO,     // -lo / 2
    DK_RHO0,     // rho0
    DK_IRHO0,    // 1 / rho0
    DK_N
};
struct DfK {
    float h[DK_N], l[DK_N];
    int le1;  // le == 1: the even part relaxes fully
};
__host__ __device__ inline void df_split(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}
__host__ __device__ inline DfK df_constants(double le, double lo, double rho0) {
    const double v[DK_N] = {1.0 / 18.0, 1.0 / 3.0, 3.0 * lo / 18.0, 3.0 * lo / 36.0, 0.5 * (1.0 - lo), le,
                            le / 3.0,   1.0 - le,  -0.5 * le,       -0.5 * lo,       rho0,             1.0 / rho0};
    DfK k;
    for (int i = 0; i < DK_N; ++i) df_split(v[i], k.h[i], k.l[i]);
    k.le1 = (1.0 - le) == 0.0;
    return k;
}

struct df {
    float h, l;
};

// ---- error-free transformations (every rounding explicit: no contraction)

// a + b = s + e exactly (Knuth), for any a, b
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// x + y: the exact sum of the high parts plus the low parts, left
// unnormalised (|l| grows by an ulp of the operands per addition)
__device__ __forceinline__ df dadd(df x, df y) {
    df s = two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return s;
}
__device__ __forceinline__ df dneg(df x) { return {-x.h, -x.l}; }
__device__ __forceinline__ df dsub(df x, df y) { return dadd(x, dneg(y)); }
// x * y: the exact product of the high parts (Dekker, through FMA) plus the
// cross terms.  The product of the low parts is left out: with |l| within a
// few ulps of |h| it is below 2^-46 of |x y|, the size of the rounding of the
// low parts themselves.
__device__ __forceinline__ df dmul(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return {p, e};
}
__device__ __forceinline__ df dsqr(df x) {
    const float p = __fmul_rn(x.h, x.h);
    const float t = __fadd_rn(x.h, x.h);
    float e = __fmaf_rn(x.h, x.h, -p);
    e = __fmaf_rn(t, x.l, e);
    return {p, e};
}
// x * c for an FP32 c
__device__ __forceinline__ df dmulf(df x, float c) {
    const float p = __fmul_rn(x.h, c);
    float e = __fmaf_rn(x.h, c, -p);
    e = __fmaf_rn(x.l, c, e);
    return {p, e};
}
// x * 2^k (exact)
__device__ __forceinline__ df dpow2(df x, float p2) { return {__fmul_rn(x.h, p2), __fmul_rn(x.l, p2)}; }
// |l| <= ulp(h) / 2 (Fast2Sum)
__device__ __forceinline__ df dnorm(df x) {
    const float s = __fadd_rn(x.h, x.l);
    return {s, __fsub_rn(x.l, __fsub_rn(s, x.h))};
}
// 1 / x for x near 1 (a density): FP32 estimate, one FP32 Newton step
// (relative error ~2^-24), then one step in double-float (error squared)
__device__ __forceinline__ df drcp(df x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x.h));
    r = __fmaf_rn(r, __fmaf_rn(-x.h, r, 1.0f), r);
    float e = __fmaf_rn(-x.h, r, 1.0f);  // 1 - x r, small: one rounding of itself
    e = __fmaf_rn(-x.l, r, e);
    return {r, __fmul_rn(r, e)};
}
__device__ __forceinline__ df dk(const DfK& K, int i) { return {K.h[i], K.l[i]}; }

// ---- FP64 word <-> double-float pair, in integer arithmetic

// (lo, hi) = the two 32-bit words of an FP64 value
__device__ __forceinline__ df df_from_bits(unsigned lo, unsigned hi) {
    const unsigned sign = hi & 0x80000000u;
    unsigned a = hi & 0x7fffffffu;
    a = umax(a, 897u << 20);                  // |g| >= 2^-126
    a = umin(a, (1124u << 20) - 1u);          // |g| < 2^101
    // exponent 1023 -> 127 and the top 23 mantissa bits: a truncated float
    const unsigned hb = __funnelshift_l(lo, a - (896u << 20), 3) | sign;
    // the remaining 29 bits weigh 2^(e - 52), e the unbiased exponent
    const float rem = __uint2float_rn(lo & 0x1fffffffu);
    const float pw = __uint_as_float(hb & 0xff800000u);  // +-2^e
    return {__uint_as_float(hb), __fmul_rn(__fmul_rn(rem, pw), 0x1p-52f)};
}
// FP64 bits of h + l (to ~2^-47 relative; |h + l| below 2^-75 may come out
// as any value of that size)
__device__ __forceinline__ uint2 df_to_bits(df x) {
    const float s = __fadd_rz(x.h, x.l);                  // |s| <= |h + l|
    const float e = __fsub_rn(x.l, __fsub_rn(s, x.h));    // (h + l) - s
    const unsigned sb = __float_as_uint(s), ab = sb & 0x7fffffffu;
    unsigned hi = ((ab >> 3) + (896u << 20)) | (sb & 0x80000000u);
    unsigned lo = sb << 29;
    // e in FP64 ulps of s, 2^(es - 127 - 52): fewer than 2^29 of them, so the
    // 52-bit mantissa cannot overflow.  For |s| < 2^-75 the scale's exponent
    // field wraps (or is Inf): the count is then garbage, an error below
    // 2^-75 in absolute value.
    const float pw = __uint_as_float((306u << 23) - (sb & 0x7f800000u));  // 2^(179 - es)
    const unsigned k = __float2uint_rn(__fmul_rn(fabsf(e), pw));
    asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(lo), "+r"(hi) : "r"(k));
    return make_uint2(lo, hi);
}

// Signed sum over the nine pairs of component AX of the pair's first member
// times d[p] (as pair_moment in sweep_body.cuh, in double-float).
template <int AX>
__device__ __forceinline__ df df_pair_moment(const df d[10]) {
    df acc{0.0f, 0.0f};
    bool first = true;
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const int c = AX == 0 ? cx(i) : (AX == 1 ? cy(i) : cz(i));
        if (c == 0) continue;
        if (first) acc = d[p];
        else acc = c > 0 ? dadd(acc, d[p]) : dsub(acc, d[p]);
        first = false;
    }
    return acc;
}
__device__ __forceinline__ df df_pair_dot(int i, df x, df y, df z) {
    const int a = cx(i), b = cy(i), c = cz(i);
    if (a != 0 && b != 0) return b > 0 ? dadd(x, y) : dsub(x, y);
    if (a != 0 && c != 0) return c > 0 ? dadd(x, z) : dsub(x, z);
    if (b != 0 && c != 0) return c > 0 ? dadd(y, z) : dsub(y, z);
    return a != 0 ? x : (b != 0 ? y : z);
}

// TRT collision (Sec. III) of one cell on deviations g_i = f_i - w_i rho0, in
// the pair form of collide_trt (sweep_body.cuh): with s = g_i + g_ib and
// d = g_i - g_ib for the nine pairs, sigma = sum g, rho = rho0 + sigma,
//   base = sigma - 3/2 |j|^2 / rho   (incompressible: / rho0),
//   ep   = w base + 9/2 w (c.j)^2 / rho,
//   le = 1:  g_0 = base / 3,  g_i = ep + h,  g_ib = ep - h,
//            h = 3 lo w c.j + (1 - lo)/2 d;
//   else:    g_0 += le (base / 3 - g_0),
//            E = le ep - le/2 s,  O = 3 lo w c.j - lo/2 d,
//            g_i += E + O,  g_ib += E - O.
// LE1: le == 1 (K.le1), the form taken.  Returns false when the cell's
// density or momentum is not finite.
template <bool LE1>
__device__ __forceinline__ bool collide_trt_df(df g[Q], const DfK& K, int inc) {
    df s[10], d[10];
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        s[p] = dadd(g[2 * p - 1], g[2 * p]);
        d[p] = dsub(g[2 * p - 1], g[2 * p]);
    }
    df sum = g[0];
#pragma unroll
    for (int p = 1; p <= 9; ++p) sum = dadd(sum, s[p]);
    sum = dnorm(sum);
    const df jx = dnorm(df_pair_moment<0>(d)), jy = dnorm(df_pair_moment<1>(d)), jz = dnorm(df_pair_moment<2>(d));
    const df j2 = dadd(dadd(dsqr(jx), dsqr(jy)), dsqr(jz));
    const bool ok = fabsf(sum.h) < 0x1p60f && j2.h < 0x1p100f;
    const df inv = inc ? dk(K, DK_IRHO0) : drcp(dnorm(dadd(dk(K, DK_RHO0), sum)));
    const df ju = dmul(j2, inv);                       // rho u.u
    const df base = dnorm(dsub(sum, dmulf(ju, 1.5f)));  // sigma - 3/2 rho u.u
    const df wb18 = dmul(base, dk(K, DK_W18)), wb36 = dpow2(wb18, 0.5f);
    const df lw18 = dk(K, DK_LW18), lw36 = dk(K, DK_LW36);
    if constexpr (LE1) {
        g[0] = dmul(base, dk(K, DK_W3));
        const df ch = dk(K, DK_CH);
#pragma unroll
        for (int p = 1; p <= 9; ++p) {
            const int i = 2 * p - 1;
            const bool face = i < 7;
            const df cj = df_pair_dot(i, jx, jy, jz);
            const df t = dmul(dsqr(cj), inv);  // (c.j)^2 / rho; 9/2 w = 1/4 (faces), 1/8 (edges)
            const df ep = dadd(dpow2(t, face ? 0.25f : 0.125f), face ? wb18 : wb36);
            const df h = dadd(dmul(face ? lw18 : lw36, cj), dmul(ch, d[p]));
            g[i] = dadd(ep, h);
            g[i + 1] = dsub(ep, h);
        }
        return ok;
    } else {
    g[0] = dadd(dmul(dk(K, DK_LE3), base), dmul(dk(K, DK_1MLE), g[0]));
    const df le = dk(K, DK_LE), mhle = dk(K, DK_MHLE), mhlo = dk(K, DK_MHLO);
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const bool face = i < 7;
        const df cj = df_pair_dot(i, jx, jy, jz);
        const df t = dmul(dsqr(cj), inv);
        const df ep = dadd(dpow2(t, face ? 0.25f : 0.125f), face ? wb18 : wb36);
        const df E = dadd(dmul(le, ep), dmul(mhle, s[p]));
        const df O = dadd(dmul(face ? lw18 : lw36, cj), dmul(mhlo, d[p]));
        g[i] = dadd(g[i], dadd(E, O));
        g[i + 1] = dadd(g[i + 1], dsub(E, O));
    }
    return ok;
    }
}

}  // namespace lbsq
