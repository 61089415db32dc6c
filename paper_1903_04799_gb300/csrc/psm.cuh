// psm.cuh -- partially saturated cells (Noble and Torczynski, 1998), the
// coupling Sec. IV A names as a remedy for the speed fluctuation of the
// link-coupled squirmer.  Used by the body kernels of bodies.cu.
//
// Every cell stays fluid.  A cell a sphere covers by the fraction eps of its
// volume collides with
//   f*_i = f_i + (1 - B) Omega_i + B Omega^s_i,
//   Omega^s_i = [f_ib - f_ib^eq(rho, u)] - [f_i - f_i^eq(rho, u_s)],
//   B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),  tau = 1 / lambda_e,
// Omega_i the TRT operator, (rho, u) the cell's moments, u_s the sphere's
// surface velocity at the node (rigid motion plus the squirmer slip, Eq. "vb"
// and Eq. "squirmer").  The fluid gains B sum_i Omega^s_i c_i; the sphere
// receives the opposite.  Arithmetic in FP64 for FP64 storage, in FP32 for
// the reduced storages (the force sums in FP64 for all).
#pragma once

#include "lbsq_internal.cuh"

namespace lbsq {

// Solid fraction of the unit cube about a node at offset d from the centre of
// a sphere of radius R: the share of its 8 x 8 x 8 points (k + 1/2)/8 - 1/2
// inside the sphere (a multiple of 1/512), each point decided by the exact
// FP64 inside test; 1 or 0 without sampling where the cube lies wholly inside
// or outside (its half-diagonal is below 0.87).  psm_class decides the
// shortcut: 1 (inside), 0 (outside) or 2 (sample).
__device__ __forceinline__ int psm_class(const double d[3], double R) {
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    const double lo = __dsub_rn(R, 0.87), hi = __dadd_rn(R, 0.87);
    if (lo > 0.0 && r2 < __dmul_rn(lo, lo)) return 1;
    if (r2 > __dmul_rn(hi, hi)) return 0;
    return 2;
}

// The inside count of the 16 sample points of lane l (0..31) of a sampled
// cell at offset d (df: d rounded to FP32): the columns (a, b) = (l / 8, l % 8)
// and (a + 4, b), all eight c of each; the 32 lanes together take the 512
// points once.
//
// The points are screened in FP32 first.  With M = R + 3 above every
// coordinate of a sampled point (|d| < R + 0.87 there), the FP32 value of
// (px^2 + py^2) + pz^2 -- d rounded to FP32, one rounding per add and
// product -- is within 1.3e-6 M^2 of the exact one, and R^2 in FP32 within
// 6e-8 R^2; the FP64 test's own error is below 1e-15 M^2.  A point whose FP32
// value lies more than m = 4e-6 M^2 from R^2 therefore takes the same side in
// both, and only points within m of the surface take the FP64 test.
// psm_screen gives (R^2 - m, R^2 + m) in FP32.
__device__ __forceinline__ float2 psm_screen(double R) {
    const double M = R + 3.0;
    const float m = (float)(4e-6 * M * M), R2 = (float)(R * R);
    return make_float2(R2 - m, R2 + m);
}

__device__ __forceinline__ int psm_lane_count(const double d[3], const float df[3], double R, float2 band, int l) {
    const int b = l & 7;
    const float ob = (b + 0.5f) * 0.125f - 0.5f;
    const float py = df[1] + ob;
    int count = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = (l >> 3) + 4 * h;
        const float oa = (a + 0.5f) * 0.125f - 0.5f;
        const float px = df[0] + oa;
        const float sab = px * px + py * py;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float oc = (c + 0.5f) * 0.125f - 0.5f;
            const float pz = df[2] + oc;
            const float s = sab + pz * pz;
            if (s < band.x) {
                ++count;
            } else if (s <= band.y) {
                count += inside_sphere(__dadd_rn(d[0], (double)oa), __dadd_rn(d[1], (double)ob),
                                       __dadd_rn(d[2], (double)oc), R);
            }
        }
    }
    return count;
}

// Surface velocity of sphere (p, s) at node offset d: v + w x d + slip, the
// slip by direction only (V = double or float).
template <class V>
__device__ __forceinline__ void psm_surface_velocity(const BodyParams& p, const BodyState& s, const V d[3], V us[3]) {
    const V e[3] = {(V)s.e[0], (V)s.e[1], (V)s.e[2]}, w[3] = {(V)s.omega[0], (V)s.omega[1], (V)s.omega[2]};
    const V r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    V sl[3] = {V(0), V(0), V(0)};
    if (r2 > V(0)) {
        const V ir = rsqrt(r2);
        const V n0 = d[0] * ir, n1 = d[1] * ir, n2 = d[2] * ir;
        const V ct = e[0] * n0 + e[1] * n1 + e[2] * n2;
        const V a = (V)p.B1 + (V)p.B2 * ct;
        sl[0] = a * (ct * n0 - e[0]);
        sl[1] = a * (ct * n1 - e[1]);
        sl[2] = a * (ct * n2 - e[2]);
    }
    us[0] = (V)s.vel[0] + (w[1] * d[2] - w[2] * d[1]) + sl[0];
    us[1] = (V)s.vel[1] + (w[2] * d[0] - w[0] * d[2]) + sl[1];
    us[2] = (V)s.vel[2] + (w[0] * d[1] - w[1] * d[0]) + sl[2];
}

// Whether component a of c is nonzero for some direction 2q - 1, q < p (the
// pairs before pair p).  Sums below start from their first nonzero term:
// 0 * x and 0 + x are not folded away in IEEE arithmetic.
__host__ __device__ constexpr bool psm_seen(int a, int p) {
    return p <= 1 ? false : (psm_seen(a, p - 1) || (a == 0 ? cx(2 * p - 3) : (a == 1 ? cy(2 * p - 3) : cz(2 * p - 3))) != 0);
}
__host__ __device__ constexpr int psm_c(int a, int i) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }

// c_i . v over the nonzero components of c_i.
template <class V>
__device__ __forceinline__ V psm_cdot(int i, const V v[3]) {
    V r = V(0);
    bool have = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c = psm_c(a, i);
        if (c != 0) {
            const V t = c > 0 ? v[a] : -v[a];
            r = have ? r + t : t;
            have = true;
        }
    }
    return r;
}

// One covered fluid cell with deviations g_i = f_i - w_i rho0: its
// post-collision deviations out (the blend above, with the TRT operator of
// rates le and lo) and the momentum sum m = sum_i Omega^s_i c_i.  Returns B.
// V = double (FP64 storage) or float (the reduced storages, whose stores
// carry FP32 precision at most).
//
// Pair form: for opposite directions i, ib the equilibrium at velocity u is
// w rho0 + E + O and w rho0 + E - O with the even part
// E = w (drho + rv (9/2 (c.u)^2 - 3/2 u.u)) and the odd part O = 3 w rv c.u,
// drho = rho - rho0 and rv = rho (rv = rho0 for the incompressible
// equilibrium, Sec. III); the same at u_s gives Es, Os.  With the
// non-equilibrium parts n_i = g_i - E - O, n_ib = g_ib - E + O:
//   Omega_i = -le (n_i + n_ib)/2 - lo (n_i - n_ib)/2,
//   Omega_ib = -le (n_i + n_ib)/2 + lo (n_i - n_ib)/2,
//   Omega^s_i = n_ib - (g_i - Es - Os),  Omega^s_ib = n_i - (g_ib - Es + Os).
template <class V>
__device__ __forceinline__ V psm_update(const V g[Q], V rho0, int inc, V le, V lo, const V us[3], V eps, V out[Q],
                                        V m[3]) {
    V dr = g[0], j[3] = {V(0), V(0), V(0)};
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1;
        const V sp = g[i] + g[opp(i)], dp = g[i] - g[opp(i)];
        dr += sp;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int c = psm_c(a, i);
            if (c != 0) {
                const V t = c > 0 ? dp : -dp;
                j[a] = psm_seen(a, p) ? j[a] + t : t;
            }
        }
    }
    const V rho = rho0 + dr;
    const V rv = inc ? rho0 : rho;  // the density of the velocity terms
    const V iden = V(1) / rv;
    const V u[3] = {j[0] * iden, j[1] * iden, j[2] * iden};
    const V uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], ss = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
    const V th = V(1) / le - V(0.5);
    const V B = eps * th / ((V(1) - eps) + th);
    const V hle = V(0.5) * le, hlo = V(0.5) * lo, cB = V(1) - B;
    {  // rest population: c = 0, no odd part
        const V E = V(wgt(0)) * (dr - V(1.5) * rv * uu), Es = V(wgt(0)) * (dr - V(1.5) * rv * ss);
        out[0] = g[0] + cB * (-le * (g[0] - E)) + B * (Es - E);
    }
    const V b18 = V(1.0 / 18.0) * (dr - V(1.5) * rv * uu), bs18 = V(1.0 / 18.0) * (dr - V(1.5) * rv * ss);
    const V b36 = V(1.0 / 36.0) * (dr - V(1.5) * rv * uu), bs36 = V(1.0 / 36.0) * (dr - V(1.5) * rv * ss);
    const V q18 = V(4.5 / 18.0) * rv, q36 = V(4.5 / 36.0) * rv, o18 = V(3.0 / 18.0) * rv, o36 = V(3.0 / 36.0) * rv;
#pragma unroll
    for (int p = 1; p <= 9; ++p) {
        const int i = 2 * p - 1, ib = opp(i);
        const bool face = i < 7;
        const V cu = psm_cdot(i, u), cs = psm_cdot(i, us);
        const V qw = face ? q18 : q36, ow = face ? o18 : o36;
        const V E = qw * cu * cu + (face ? b18 : b36), O = ow * cu;
        const V Es = qw * cs * cs + (face ? bs18 : bs36), Os = ow * cs;
        const V ni = g[i] - E - O, nb = g[ib] - E + O;
        const V ev = hle * (ni + nb), od = hlo * (ni - nb);
        const V si = nb - (g[i] - Es - Os), sb = ni - (g[ib] - Es + Os);
        out[i] = g[i] + cB * (-ev - od) + B * si;
        out[ib] = g[ib] + cB * (-ev + od) + B * sb;
        const V ds = si - sb;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int c = psm_c(a, i);
            if (c != 0) {
                const V t = c > 0 ? ds : -ds;
                m[a] = psm_seen(a, p) ? m[a] + t : t;
            }
        }
    }
    return B;
}

}  // namespace lbsq
