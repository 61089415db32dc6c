// psm.cuh -- partially saturated cells (Noble and Torczynski, 1998), the
// coupling Sec. IV A names as a remedy for the speed fluctuation of the
// link-coupled squirmer.  Shared by the body kernels (solid fractions and the
// force on each sphere, bodies.cu) and the sweep (the blended collision,
// sweep.cu), so that both evaluate the same solid operator.
//
// Every cell stays fluid.  A cell a sphere covers by the fraction eps of its
// volume collides with
//   f*_i = f_i + (1 - B) Omega_i + B Omega^s_i,
//   Omega^s_i = [f_ib - f_ib^eq(rho, u)] - [f_i - f_i^eq(rho, u_s)],
//   B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),  tau = 1 / lambda_e,
// Omega_i the TRT operator, (rho, u) the cell's moments, u_s the sphere's
// surface velocity at the node (rigid motion plus the squirmer slip, Eq. "vb"
// and Eq. "squirmer").  The fluid gains B sum_i Omega^s_i c_i; the sphere
// receives the opposite.  Arithmetic in FP64 for every storage.
#pragma once

#include "lbsq_internal.cuh"

namespace lbsq {

// Solid fraction of the unit cube about a node at offset d from the centre of
// a sphere of radius R: the share of its 8 x 8 x 8 points (k + 1/2)/8 - 1/2
// inside the sphere (a multiple of 1/512, decided by the exact inside test);
// 1 or 0 without sampling where the cube lies wholly inside or outside (its
// half-diagonal is below 0.87).
__device__ __forceinline__ double psm_fraction(const double d[3], double R) {
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    const double lo = __dsub_rn(R, 0.87), hi = __dadd_rn(R, 0.87);
    if (lo > 0.0 && r2 < __dmul_rn(lo, lo)) return 1.0;
    if (r2 > __dmul_rn(hi, hi)) return 0.0;
    int count = 0;
    for (int a = 0; a < 8; ++a) {
        const double px = __dadd_rn(d[0], (a + 0.5) / 8.0 - 0.5);
        for (int b = 0; b < 8; ++b) {
            const double py = __dadd_rn(d[1], (b + 0.5) / 8.0 - 0.5);
            for (int c = 0; c < 8; ++c)
                count += inside_sphere(px, py, __dadd_rn(d[2], (c + 0.5) / 8.0 - 0.5), R);
        }
    }
    return count / 512.0;
}

// Surface velocity of sphere (p, s) at node offset d: v + w x d + slip, the
// slip by direction only.
__device__ __forceinline__ void psm_surface_velocity(const BodyParams& p, const BodyState& s, const double d[3],
                                                     double us[3]) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double sl[3] = {0.0, 0.0, 0.0};
    if (r2 > 0.0) {
        const double r = sqrt(r2);
        const double n0 = d[0] / r, n1 = d[1] / r, n2 = d[2] / r;
        const double ct = s.e[0] * n0 + s.e[1] * n1 + s.e[2] * n2;
        const double a = p.B1 + p.B2 * ct;
        sl[0] = a * (ct * n0 - s.e[0]);
        sl[1] = a * (ct * n1 - s.e[1]);
        sl[2] = a * (ct * n2 - s.e[2]);
    }
    us[0] = s.vel[0] + (s.omega[1] * d[2] - s.omega[2] * d[1]) + sl[0];
    us[1] = s.vel[1] + (s.omega[2] * d[0] - s.omega[0] * d[2]) + sl[1];
    us[2] = s.vel[2] + (s.omega[0] * d[1] - s.omega[1] * d[0]) + sl[2];
}

// The solid operator Omega^s of a cell with (absolute) populations f, and
// its weight B.  inc: the incompressible equilibrium (u = j / rho0).
__device__ __forceinline__ double psm_solid(const double f[Q], double rho0, int inc, double le, const double us[3],
                                            double eps, double om[Q]) {
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        j[0] += f[i] * cx(i);
        j[1] += f[i] * cy(i);
        j[2] += f[i] * cz(i);
    }
    const double den = inc ? rho0 : rho;
    const double u[3] = {j[0] / den, j[1] / den, j[2] / den};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], ss = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
    double feq[Q], feqs[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
        const double cs = cx(i) * us[0] + cy(i) * us[1] + cz(i) * us[2];
        if (inc) {
            feq[i] = wgt(i) * (rho + rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
            feqs[i] = wgt(i) * (rho + rho0 * (3.0 * cs + 4.5 * cs * cs - 1.5 * ss));
        } else {
            feq[i] = wgt(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            feqs[i] = wgt(i) * rho * (1.0 + 3.0 * cs + 4.5 * cs * cs - 1.5 * ss);
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) om[i] = (f[opp(i)] - feq[opp(i)]) - (f[i] - feqs[i]);
    const double th = 1.0 / le - 0.5;
    return eps * th / ((1.0 - eps) + th);
}

// What the sweep needs of the bodies in PSM mode.
struct PsmArgs {
    const float* eps;        // solid fraction per cell (0: an ordinary fluid cell)
    const int32_t* psm_id;   // the covering sphere (body index + 1) per cell
    const int32_t* own;      // solid owner per cell: a covered wall cell stays a plain cell
    const BodyParams* par;
    const BodyState* state;  // the state the step starts from
};

}  // namespace lbsq
