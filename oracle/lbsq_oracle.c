/*
 * lbsq_oracle.c -- plain FP64 CPU restatement of the lattice Boltzmann
 * squirmer method of Kuron, Staerk, Burkard, de Graaf & Holm,
 * "A Lattice Boltzmann Model for Squirmers" (arXiv:1903.04799).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library
 * is checked against.  Only the tests, the smoke check and the CPU-baseline
 * leg of bench.py may load it.  It shares no code, header, table or helper
 * with the CUDA library; the D3Q19 tables below are typed out here on their
 * own.
 *
 * Design: two population arrays (push streaming), every loop written out in
 * the order of the method, FP64 everywhere, compiled with
 * -ffp-contract=off so that no multiply-add is fused.  The collide and
 * stream loops are split over z with OpenMP when available; each cell's
 * arithmetic is independent there, so the thread count does not change a
 * single bit.  Everything that sums over links or cells runs serially in
 * canonical order.
 *
 * One time step t -> t+1 (Sec. III; the paper does not print the order, the
 * reading used here is: collide, bounce, stream, integrate, remap):
 *   1. collide every fluid cell with the TRT operator (Eq. "lb");
 *   2. for every boundary link (fluid x, direction i, x+c_i solid), in
 *      canonical order (cell index, then i): reflect the post-collision
 *      population with the moving-wall shift (Sec. III, shifted bounce-back),
 *      where the wall velocity is the rigid-body velocity (Eq. "vb") plus the
 *      squirmer slip (Eq. "squirmer"), and add the exchanged momentum to the
 *      owner's force and torque (Eqs. "bbforce", "bbtorque");
 *   3. stream every other population to its fluid neighbour;
 *   4. symplectic Euler update of every mobile sphere from the momentum
 *      exchange, the conversion force of the previous remap (Eq. "consforce")
 *      and the optional WCA contact force (Eq. "wca");
 *   5. remap cells against the new positions: covered fluid cells lose their
 *      populations, uncovered cells are refilled with the equilibrium of the
 *      mean density of their fluid neighbours and the body's rigid velocity,
 *      and the created/destroyed momentum is booked as conversion force
 *      (Sec. III, last paragraph of the moving-boundary description).
 *
 * Readings of the paper where it is silent or garbled:
 *   - f_eq uses the standard second-order D3Q19 coefficients 9/2 and 3/2
 *     (the printed 1/6 cannot satisfy the second-moment identity);
 *   - "lambda_o lambda_e = 3/16" is the TRT magic parameter
 *     (1/lambda_e - 1/2)(1/lambda_o - 1/2) = 3/16;
 *   - u = j / rho (compressible form, consistent with f_eq ~ rho);
 *   - the shift uses rho0;
 *   - the wall velocity (Eq. "vb" plus the slip) and the lever arm of the
 *     torque are taken at the link midpoint x + c_i/2, where halfway
 *     bounce-back puts the wall.  The text names the boundary node; the
 *     midpoint is the reading that reproduces the speeds printed in Fig.
 *     "resolution" (R = 4, L = 10R: 0.974 printed; the node reading gives
 *     about 1.10, the midpoint reading 0.972);
 *   - conversion force: + on cover, - on uncover, with the angular analog,
 *     applied in the next update; the refill density is the mean over the
 *     D3Q19 neighbours that are fluid now and were fluid before the remap;
 *   - mass M = density * 4/3 pi R^3, I = 2/5 M R^2, dt = 1, velocity first;
 *   - WCA force is -dU/dr of the shifted LJ potential, r the surface gap.
 *
 * Parity unpinned in value (no pin but agreement with the CUDA library and
 * mirror symmetry, which a mirror-symmetric error passes):
 *   - the trajectories of a squirmer in a tube or near an obstacle (the
 *     boundary-element data the paper compares with are not in its text);
 *     the drag of a fixed sphere and the flow of the round tube are pinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* D3Q19 velocity set (Sec. III: rest, 6 face and 12 edge neighbours)  */
/* Order: rest, then opposite pairs next to each other.               */
/* ------------------------------------------------------------------ */
#define Q 19
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
/* Standard D3Q19 weights: 1/3 rest, 1/18 faces, 1/36 edges. */
static const double WT[Q] = {1.0 / 3.0,
                             1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* index of -c_i */
static int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

/* ------------------------------------------------------------------ */
/* Point functions (exported for the pin tests)                        */
/* ------------------------------------------------------------------ */

void oracle_velocities(int32_t* c /* [19][3] */) {
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
    }
}

void oracle_weights(double* w) {
    for (int i = 0; i < Q; ++i) w[i] = WT[i];
}

int32_t oracle_opposite(int32_t i) { return opposite(i); }

/* Equilibrium (Sec. III): f_i^eq = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u). */
void oracle_feq(double rho, const double* u, double* feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        feq[i] = WT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Incompressible equilibrium (He and Luo), the model in which Sec. III's
 * printed velocity u = sum f_i c_i holds as written (with rho0 = 1):
 * f_i^eq = w_i (rho + rho0 (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)), u = j / rho0. */
void oracle_feq_inc(double rho, double rho0, const double* u, double* feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        feq[i] = WT[i] * (rho + rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    }
}

/* Moments (Sec. III): rho = sum f_i, j = sum f_i c_i, u = j / rho. */
void oracle_moments(const double* f, double* rho, double* j) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        jx += f[i] * CX[i];
        jy += f[i] * CY[i];
        jz += f[i] * CZ[i];
    }
    *rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

/* TRT odd rate from the magic parameter (reading of "lambda_o lambda_e = 3/16"):
 * (1/lambda_e - 1/2)(1/lambda_o - 1/2) = magic. */
double oracle_lambda_odd(double lambda_e, double magic) {
    return 1.0 / (0.5 + magic / (1.0 / lambda_e - 0.5));
}

/* TRT collision of one cell (Eq. "lb", right-hand side). */
void oracle_collide(const double* f, double lambda_e, double lambda_o, double* fpost) {
    double rho, j[3], u[3], feq[Q];
    oracle_moments(f, &rho, j);
    u[0] = j[0] / rho;
    u[1] = j[1] / rho;
    u[2] = j[2] / rho;
    oracle_feq(rho, u, feq);
    for (int i = 0; i < Q; ++i) {
        int ib = opposite(i);
        double fp = 0.5 * (f[i] + f[ib]);
        double fm = 0.5 * (f[i] - f[ib]);
        double ep = 0.5 * (feq[i] + feq[ib]);
        double em = 0.5 * (feq[i] - feq[ib]);
        fpost[i] = f[i] - lambda_e * (fp - ep) - lambda_o * (fm - em);
    }
}

/* TRT collision of one cell towards the incompressible equilibrium, u = j / rho0. */
void oracle_collide_inc(const double* f, double lambda_e, double lambda_o, double rho0, double* fpost) {
    double rho, j[3], u[3], feq[Q];
    oracle_moments(f, &rho, j);
    u[0] = j[0] / rho0;
    u[1] = j[1] / rho0;
    u[2] = j[2] / rho0;
    oracle_feq_inc(rho, rho0, u, feq);
    for (int i = 0; i < Q; ++i) {
        int ib = opposite(i);
        double fp = 0.5 * (f[i] + f[ib]);
        double fm = 0.5 * (f[i] - f[ib]);
        double ep = 0.5 * (feq[i] + feq[ib]);
        double em = 0.5 * (feq[i] - feq[ib]);
        fpost[i] = f[i] - lambda_e * (fp - ep) - lambda_o * (fm - em);
    }
}

/* Squirmer surface slip (Eq. "squirmer"), d = position relative to the centre,
 * e = unit orientation: (B1 + B2 e.d/|d|)(e.d/|d| d/|d| - e). */
void oracle_slip(const double* d, const double* e, double B1, double B2, double* out) {
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r == 0.0) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    double n[3] = {d[0] / r, d[1] / r, d[2] / r};
    double ct = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
    double a = B1 + B2 * ct;
    for (int k = 0; k < 3; ++k) out[k] = a * (ct * n[k] - e[k]);
}

/* Inside test for a node at minimum-image offset d from a sphere of radius R:
 * (dx*dx + dy*dy) + dz*dz < R*R, evaluated in exactly this order. */
int32_t oracle_inside(const double* d, double R) {
    double s = d[0] * d[0] + d[1] * d[1];
    s = s + d[2] * d[2];
    return s < R * R;
}

/* Minimum image of a coordinate difference into (-n/2, n/2]. */
static double min_image(double d, int n) {
    double h = 0.5 * (double)n;
    if (d > h) d -= (double)n;
    else if (d <= -h) d += (double)n;
    return d;
}

double oracle_min_image(double d, int32_t n) { return min_image(d, n); }

/* ------------------------------------------------------------------ */
/* Simulation state                                                    */
/* ------------------------------------------------------------------ */

enum { OBJ_WALL = 0, OBJ_SPHERE = 1 };

typedef struct {
    int kind;
    int mobile;
    double R, B1, B2, mass, inertia;
    double pos[3], vel[3], omega[3], e[3];
    double wall_vel[3];        /* plane walls: velocity of the wall */
    int wall_axis, wall_index; /* plane walls; wall_axis -1: a round tube */
    double tube_c[2], tube_r;  /* round tube along z: axis (x, y) and radius */
    double Fbb[3], Tbb[3], Sbb[6];
    double Fc[3], Tc[3];             /* conversion force booked for the next update */
    double Fapplied[3], Tapplied[3]; /* hydrodynamic force/torque of the last update */
    double Fbb_last[3], Tbb_last[3]; /* F_bb, T_bb of the previous step (two-step average) */
} oobj;

typedef struct {
    int nx, ny, nz;
    long N;
    double lambda_e, lambda_o, rho0;
    double* f;     /* [19][N] current (post-stream) populations */
    double* fpost; /* [19][N] post-collision */
    double* fnew;  /* [19][N] next populations */
    int32_t* owner;
    int32_t* owner_prev;
    double g[3]; /* test-only body force, 0 on the method's path */
    double wca_sigma, wca_eps;
    int force_avg; /* 1: Ladd's two-step average of F_bb and T_bb */
    int inc;       /* 1: incompressible equilibrium (oracle_feq_inc) throughout */
    double link_at; /* where on a link v_b and the lever arm are taken: 0.5 (midpoint) or 1 (boundary node) */
    int conv;       /* conversion reading: 0 = the one used throughout, else an alternative (osim_set_conversion) */
    int local_rho;  /* 1: the bounce-back shift takes the density of the fluid node instead of rho0 */
    int psm;        /* 1: spheres couple by partially saturated cells (Noble-Torczynski), not links */
    double* eps;    /* PSM: solid fraction of each cell, [N] */
    int32_t* psm_id; /* PSM: the sphere (id) covering each cell, 0 = none, [N] */
    int nobj, capobj;
    oobj* obj; /* obj[k] has id k+1 */
    long step;
    int err;
} osim;

#define OERR_OK 0
#define OERR_INVALID 1
#define OERR_OVERLAP 4
#define OERR_DIVERGED 5

static long cidx(const osim* s, int x, int y, int z) {
    return (long)x + (long)s->nx * ((long)y + (long)s->ny * (long)z);
}

static void coords(const osim* s, long n, int* x, int* y, int* z) {
    *x = (int)(n % s->nx);
    long r = n / s->nx;
    *y = (int)(r % s->ny);
    *z = (int)(r / s->ny);
}

static int wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

/* periodic step of one along an axis */
static int step1(int a, int c, int n) {
    a += c;
    if (a < 0) a += n;
    else if (a >= n) a -= n;
    return a;
}

static long neighbour_xyz(const osim* s, int x, int y, int z, int i) {
    return cidx(s, step1(x, CX[i], s->nx), step1(y, CY[i], s->ny), step1(z, CZ[i], s->nz));
}

static long neighbour(const osim* s, long n, int i) {
    int x, y, z;
    coords(s, n, &x, &y, &z);
    return neighbour_xyz(s, x, y, z, i);
}

osim* osim_create(int32_t nx, int32_t ny, int32_t nz, double lambda_e, double lambda_o, double rho0) {
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    osim* s = (osim*)calloc(1, sizeof(osim));
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->lambda_e = lambda_e;
    s->lambda_o = lambda_o;
    s->rho0 = rho0;
    s->link_at = 0.5; /* link midpoint */
    s->f = (double*)malloc(sizeof(double) * Q * s->N);
    s->fpost = (double*)malloc(sizeof(double) * Q * s->N);
    s->fnew = (double*)malloc(sizeof(double) * Q * s->N);
    s->owner = (int32_t*)calloc(s->N, sizeof(int32_t));
    s->owner_prev = (int32_t*)calloc(s->N, sizeof(int32_t));
    for (int i = 0; i < Q; ++i)
        for (long n = 0; n < s->N; ++n) s->f[i * s->N + n] = WT[i] * rho0;
    s->capobj = 8;
    s->obj = (oobj*)calloc(s->capobj, sizeof(oobj));
    return s;
}

void osim_destroy(osim* s) {
    if (!s) return;
    free(s->f);
    free(s->fpost);
    free(s->fnew);
    free(s->owner);
    free(s->owner_prev);
    free(s->eps);
    free(s->psm_id);
    free(s->obj);
    free(s);
}

int32_t osim_error(const osim* s) { return s->err; }
int64_t osim_step_count(const osim* s) { return s->step; }

void osim_set_body_force(osim* s, const double* g) {
    s->g[0] = g[0];
    s->g[1] = g[1];
    s->g[2] = g[2];
}

void osim_set_contact(osim* s, double sigma, double eps) {
    s->wca_sigma = sigma;
    s->wca_eps = eps;
}

/* Ladd's coupling averages the momentum exchange over two consecutive steps;
 * Sec. III names the option and leaves it off.  on = 1: every update applies
 * (F_bb(t) + F_bb(t-1)) / 2 and the same for T_bb, with F_bb(t-1) = 0 before
 * an object's first step. */
void osim_set_force_average(osim* s, int on) { s->force_avg = on ? 1 : 0; }

/* Incompressible equilibrium (oracle_feq_inc) in the collision, the refill,
 * osim_set_equilibrium and the exported velocity u = j / rho0. */
void osim_set_incompressible(osim* s, int on) { s->inc = on ? 1 : 0; }

/* Where a link's wall velocity and lever arm are taken: at the midpoint
 * x + c_i/2 (at_node = 0, the reading used throughout) or at the boundary
 * node x + c_i that the text of Sec. III names (at_node = 1, kept to show
 * that this reading misses the speeds printed in Fig. "resolution"). */
void osim_set_link_at_node(osim* s, int at_node) { s->link_at = at_node ? 1.0 : 0.5; }

/* The density in the shift 6 w_i rho c_i.v_b of the moving-wall bounce-back
 * (Sec. III leaves it open): rho0 (on = 0, Ladd's original, the default) or
 * the density of the fluid node the link leaves (on = 1), the sum of its
 * post-collision populations. */
void osim_set_local_density(osim* s, int on) { s->local_rho = on ? 1 : 0; }

/* Alternative readings of the cell conversion of Sec. III (Eq. "consforce"),
 * kept to compare them with the speeds printed in Fig. "resolution":
 *   0: the reading used throughout (refill at the rigid velocity v + w x d,
 *      conversion momentum booked on the body);
 *   1: refill at the whole surface velocity, the squirmer slip included;
 *   2: conversion momentum not booked on the body (no F_c);
 *   3: refill at the density rho0 instead of the neighbours' mean. */
void osim_set_conversion(osim* s, int mode) { s->conv = mode; }

/* Populations to the equilibrium of the given fields (rho[N], u as SoA [3][N]). */
void osim_set_equilibrium(osim* s, const double* rho, const double* u) {
    for (long n = 0; n < s->N; ++n) {
        double uu[3] = {u[n], u[s->N + n], u[2 * s->N + n]};
        double feq[Q];
        if (s->inc) oracle_feq_inc(rho[n], s->rho0, uu, feq);
        else oracle_feq(rho[n], uu, feq);
        for (int i = 0; i < Q; ++i) s->f[i * s->N + n] = feq[i];
    }
}

void osim_set_populations(osim* s, const double* f) { memcpy(s->f, f, sizeof(double) * Q * s->N); }
void osim_get_populations(const osim* s, double* f) { memcpy(f, s->f, sizeof(double) * Q * s->N); }
void osim_get_owner(const osim* s, int32_t* owner) { memcpy(owner, s->owner, sizeof(int32_t) * s->N); }

static oobj* new_object(osim* s) {
    if (s->nobj == s->capobj) {
        s->capobj *= 2;
        s->obj = (oobj*)realloc(s->obj, sizeof(oobj) * s->capobj);
    }
    oobj* o = &s->obj[s->nobj];
    memset(o, 0, sizeof(oobj));
    return o;
}

/* node offset from the sphere centre, minimum image per axis */
static void sphere_offset(const osim* s, const oobj* o, int x, int y, int z, double* d) {
    d[0] = min_image((double)x - o->pos[0], s->nx);
    d[1] = min_image((double)y - o->pos[1], s->ny);
    d[2] = min_image((double)z - o->pos[2], s->nz);
}

/* Bounding box of lattice nodes that may lie within distance R + 2 of the centre:
 * per axis floor(p - R) - 2 ... floor(p - R) - 2 + W - 1, W = ceil(2R) + 6. */
static void sphere_box(const oobj* o, int* lo, int* W) {
    *W = (int)ceil(2.0 * o->R) + 6;
    for (int a = 0; a < 3; ++a) lo[a] = (int)floor(o->pos[a] - o->R) - 2;
}

/* Add a sphere.  Returns its id (>= 1) or -error. */
int32_t osim_add_sphere(osim* s, const double* pos, const double* e, double R, double B1, double beta,
                        int32_t mobile, double density) {
    double ne = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    int nmin = s->nx < s->ny ? (s->nx < s->nz ? s->nx : s->nz) : (s->ny < s->nz ? s->ny : s->nz);
    if (!(R > 0.0) || !(ne > 0.0) || !(2.0 * R + 6.0 < (double)nmin)) return -OERR_INVALID;
    oobj* o = new_object(s);
    o->kind = OBJ_SPHERE;
    o->mobile = mobile ? 1 : 0;
    o->R = R;
    o->B1 = B1;
    o->B2 = beta * B1;
    o->mass = density * (4.0 / 3.0) * M_PI * R * R * R;
    o->inertia = 0.4 * o->mass * R * R;
    o->pos[0] = pos[0] - floor(pos[0] / s->nx) * s->nx;
    o->pos[1] = pos[1] - floor(pos[1] / s->ny) * s->ny;
    o->pos[2] = pos[2] - floor(pos[2] / s->nz) * s->nz;
    for (int k = 0; k < 3; ++k) o->e[k] = e[k] / ne;
    int id = s->nobj + 1;
    if (s->psm) { /* partially saturated cells: the sphere claims no cell */
        s->nobj++;
        return id;
    }
    /* classify: the sphere's box */
    int lo[3], W;
    sphere_box(o, lo, &W);
    for (int bz = 0; bz < W; ++bz)
        for (int by = 0; by < W; ++by)
            for (int bx = 0; bx < W; ++bx) {
                int x = wrap(lo[0] + bx, s->nx), y = wrap(lo[1] + by, s->ny), z = wrap(lo[2] + bz, s->nz);
                double d[3];
                sphere_offset(s, o, x, y, z, d);
                if (oracle_inside(d, R) && s->owner[cidx(s, x, y, z)] != 0) return -OERR_OVERLAP;
            }
    for (int bz = 0; bz < W; ++bz)
        for (int by = 0; by < W; ++by)
            for (int bx = 0; bx < W; ++bx) {
                int x = wrap(lo[0] + bx, s->nx), y = wrap(lo[1] + by, s->ny), z = wrap(lo[2] + bz, s->nz);
                double d[3];
                sphere_offset(s, o, x, y, z, d);
                if (oracle_inside(d, R)) s->owner[cidx(s, x, y, z)] = id;
            }
    s->nobj++;
    return id;
}

/* Add a plane wall: one layer of solid cells at coordinate `index` along `axis`,
 * moving with velocity `vel` (zero for a no-slip wall).  Cells of the layer
 * that already belong to another wall stay with it (the corner columns of a
 * tube); a cell owned by a sphere is an overlap.  Returns id or -error. */
int32_t osim_add_plane_wall(osim* s, int32_t axis, int32_t index, const double* vel) {
    int n[3] = {s->nx, s->ny, s->nz};
    if (axis < 0 || axis > 2 || index < 0 || index >= n[axis]) return -OERR_INVALID;
    for (long c = 0; c < s->N; ++c) {
        int x[3];
        coords(s, c, &x[0], &x[1], &x[2]);
        if (x[axis] == index && s->owner[c] != 0 && s->obj[s->owner[c] - 1].kind == OBJ_SPHERE)
            return -OERR_OVERLAP;
    }
    oobj* o = new_object(s);
    o->kind = OBJ_WALL;
    o->wall_axis = axis;
    o->wall_index = index;
    for (int k = 0; k < 3; ++k) o->wall_vel[k] = vel ? vel[k] : 0.0;
    int id = s->nobj + 1;
    for (long c = 0; c < s->N; ++c) {
        int x[3];
        coords(s, c, &x[0], &x[1], &x[2]);
        if (x[axis] == index && s->owner[c] == 0) s->owner[c] = id;
    }
    s->nobj++;
    return id;
}

/* Whether node (x, y) lies in the solid of a round tube along z with axis
 * (cx, cy) and radius r: (x - cx)^2 + (y - cy)^2 >= r^2, evaluated in FP64 as
 * written (no contraction). */
static int tube_solid(int x, int y, double cx, double cy, double r) {
    const double dx = (double)x - cx, dy = (double)y - cy;
    return dx * dx + dy * dy >= r * r;
}

/* Round tube along z (the paper's tube flow, Sec. V): every node at distance
 * >= r from the axis (cx, cy) is a wall at rest, bounced back like a plane
 * wall.  Returns the object id, -OERR_OVERLAP if a sphere holds such a node. */
int32_t osim_add_tube(osim* s, double cx, double cy, double r) {
    if (!(r > 1.0) || !(cx >= 0.0) || !(cy >= 0.0) || !(cx <= s->nx - 1) || !(cy <= s->ny - 1)) return -OERR_INVALID;
    for (long c = 0; c < s->N; ++c) {
        int x, y, z;
        coords(s, c, &x, &y, &z);
        if (tube_solid(x, y, cx, cy, r) && s->owner[c] != 0 && s->obj[s->owner[c] - 1].kind == OBJ_SPHERE)
            return -OERR_OVERLAP;
    }
    oobj* o = new_object(s);
    o->kind = OBJ_WALL;
    o->wall_axis = -1;
    o->wall_index = 0;
    o->tube_c[0] = cx;
    o->tube_c[1] = cy;
    o->tube_r = r;
    for (int k = 0; k < 3; ++k) o->wall_vel[k] = 0.0;
    int id = s->nobj + 1;
    for (long c = 0; c < s->N; ++c) {
        int x, y, z;
        coords(s, c, &x, &y, &z);
        if (tube_solid(x, y, cx, cy, r) && s->owner[c] == 0) s->owner[c] = id;
    }
    s->nobj++;
    return id;
}

/* Boundary velocity of object o on the link from fluid node (x,y,z) along c_i,
 * taken at the link midpoint (x,y,z) + c_i/2: walls move rigidly; spheres:
 * v + omega x d (Eq. "vb") plus the squirmer slip (Eq. "squirmer"), with d the
 * minimum-image offset of the midpoint from the centre (returned as lever arm). */
static void boundary_velocity(const osim* s, const oobj* o, int x, int y, int z, int i, double* vb, double* d) {
    if (o->kind == OBJ_WALL) {
        for (int k = 0; k < 3; ++k) vb[k] = o->wall_vel[k];
        d[0] = d[1] = d[2] = 0.0;
        return;
    }
    d[0] = min_image(((double)x + s->link_at * CX[i]) - o->pos[0], s->nx);
    d[1] = min_image(((double)y + s->link_at * CY[i]) - o->pos[1], s->ny);
    d[2] = min_image(((double)z + s->link_at * CZ[i]) - o->pos[2], s->nz);
    double slip[3];
    oracle_slip(d, o->e, o->B1, o->B2, slip);
    vb[0] = o->vel[0] + (o->omega[1] * d[2] - o->omega[2] * d[1]) + slip[0];
    vb[1] = o->vel[1] + (o->omega[2] * d[0] - o->omega[0] * d[2]) + slip[1];
    vb[2] = o->vel[2] + (o->omega[0] * d[1] - o->omega[1] * d[0]) + slip[2];
}

static void cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* WCA (Eq. "wca", reading: -dU/dr of U = 4 eps((s/r)^12 - (s/r)^6) + eps):
 * magnitude of the repulsion at surface gap r, zero beyond 2^(1/6) sigma. */
double oracle_wca(double r, double sigma, double eps) {
    if (eps == 0.0 || r >= pow(2.0, 1.0 / 6.0) * sigma) return 0.0;
    if (r < 0.05 * sigma) r = 0.05 * sigma;
    double sr6 = pow(sigma / r, 6.0);
    return 24.0 * eps / r * (2.0 * sr6 * sr6 - sr6);
}

/* Contact force on mobile sphere a from every other sphere and every plane wall. */
static void contact_force(const osim* s, int a, double* F) {
    F[0] = F[1] = F[2] = 0.0;
    if (s->wca_eps == 0.0) return;
    const oobj* oa = &s->obj[a];
    int n[3] = {s->nx, s->ny, s->nz};
    for (int b = 0; b < s->nobj; ++b) {
        if (b == a) continue;
        const oobj* ob = &s->obj[b];
        if (ob->kind == OBJ_SPHERE) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = min_image(oa->pos[k] - ob->pos[k], n[k]);
            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double f = oracle_wca(dist - oa->R - ob->R, s->wca_sigma, s->wca_eps);
            if (f != 0.0)
                for (int k = 0; k < 3; ++k) F[k] += f * d[k] / dist;
        } else if (ob->wall_axis < 0) {
            /* round tube: its surface taken half a cell inside the first solid
             * radius, as for a plane wall; the force points to the axis */
            double dx = oa->pos[0] - ob->tube_c[0], dy = oa->pos[1] - ob->tube_c[1];
            double rho = sqrt(dx * dx + dy * dy);
            double gap = (ob->tube_r - 0.5) - rho - oa->R;
            double f = oracle_wca(gap, s->wca_sigma, s->wca_eps);
            if (f != 0.0 && rho > 0.0) {
                F[0] -= f * dx / rho;
                F[1] -= f * dy / rho;
            }
        } else {
            int ax = ob->wall_axis;
            double dd = min_image(oa->pos[ax] - (double)ob->wall_index, n[ax]);
            double gap = fabs(dd) - 0.5 - oa->R;
            double f = oracle_wca(gap, s->wca_sigma, s->wca_eps);
            if (f != 0.0) F[ax] += dd > 0.0 ? f : -f;
        }
    }
}

/* ---- step 1: collide ---------------------------------------------- */
static void collide_all(osim* s) {
    long N = s->N;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; ++n) {
        if (s->owner[n] != 0) continue;
        double f[Q], fp[Q];
        for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
        if (s->inc) oracle_collide_inc(f, s->lambda_e, s->lambda_o, s->rho0, fp);
        else oracle_collide(f, s->lambda_e, s->lambda_o, fp);
        if (s->g[0] != 0.0 || s->g[1] != 0.0 || s->g[2] != 0.0)
            for (int i = 0; i < Q; ++i) fp[i] += 3.0 * WT[i] * (CX[i] * s->g[0] + CY[i] * s->g[1] + CZ[i] * s->g[2]);
        for (int i = 0; i < Q; ++i) s->fpost[i * N + n] = fp[i];
    }
}

/* ---- step 2: boundary links in canonical order ---------------------- */
static void bounce_links(osim* s) {
    long N = s->N;
    for (int k = 0; k < s->nobj; ++k) {
        oobj* o = &s->obj[k];
        for (int a = 0; a < 3; ++a) o->Fbb[a] = o->Tbb[a] = 0.0;
        for (int a = 0; a < 6; ++a) o->Sbb[a] = 0.0;
    }
    for (int cz = 0; cz < s->nz; ++cz)
    for (int cy = 0; cy < s->ny; ++cy)
    for (int cx = 0; cx < s->nx; ++cx) {
        long n = cidx(s, cx, cy, cz);
        if (s->owner[n] != 0) continue;
        for (int i = 1; i < Q; ++i) {
            long m = neighbour_xyz(s, cx, cy, cz, i);
            int id = s->owner[m];
            if (id == 0) continue;
            oobj* o = &s->obj[id - 1];
            double vb[3], d[3];
            boundary_velocity(s, o, cx, cy, cz, i, vb, d);
            double fout = s->fpost[i * N + n];
            double cv = CX[i] * vb[0] + CY[i] * vb[1] + CZ[i] * vb[2];
            double rs = s->rho0;
            if (s->local_rho) {
                rs = 0.0;
                for (int j = 0; j < Q; ++j) rs += s->fpost[j * N + n];
            }
            double fin = fout - 6.0 * WT[i] * rs * cv;
            s->fnew[opposite(i) * N + n] = fin;
            /* momentum exchange: c_i (f_out + f_in) goes to the body */
            double dF[3] = {CX[i] * (fout + fin), CY[i] * (fout + fin), CZ[i] * (fout + fin)};
            double dT[3];
            cross(d, dF, dT);
            for (int a = 0; a < 3; ++a) {
                o->Fbb[a] += dF[a];
                o->Tbb[a] += dT[a];
            }
            /* force dipole the tractions exert on the fluid: minus the
             * symmetric traceless first moment of the force on the body (the
             * traction part of Batchelor's stresslet, sign flipped; for a
             * squirmer -(12 pi/5) eta R^2 B2 (e e - I/3)) */
            double tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) / 3.0;
            o->Sbb[0] -= d[0] * dF[0] - tr;
            o->Sbb[1] -= d[1] * dF[1] - tr;
            o->Sbb[2] -= d[2] * dF[2] - tr;
            o->Sbb[3] -= 0.5 * (d[0] * dF[1] + d[1] * dF[0]);
            o->Sbb[4] -= 0.5 * (d[0] * dF[2] + d[2] * dF[0]);
            o->Sbb[5] -= 0.5 * (d[1] * dF[2] + d[2] * dF[1]);
        }
    }
}

/* ---- step 3: stream ------------------------------------------------ */
static void stream_all(osim* s) {
    long N = s->N;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int cz = 0; cz < s->nz; ++cz)
    for (int cy = 0; cy < s->ny; ++cy)
    for (int cx = 0; cx < s->nx; ++cx) {
        long n = cidx(s, cx, cy, cz);
        if (s->owner[n] != 0) continue;
        s->fnew[n] = s->fpost[n]; /* rest population */
        for (int i = 1; i < Q; ++i) {
            long m = neighbour_xyz(s, cx, cy, cz, i);
            if (s->owner[m] == 0) s->fnew[i * N + m] = s->fpost[i * N + n];
        }
    }
    double* t = s->f;
    s->f = s->fnew;
    s->fnew = t;
}

/* ---- step 4: symplectic Euler ---------------------------------------- */
static void rotate(double* e, const double* w) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (th == 0.0) return;
    double k[3] = {w[0] / th, w[1] / th, w[2] / th};
    double c = cos(th), sn = sin(th);
    double kxe[3];
    cross(k, e, kxe);
    double ke = k[0] * e[0] + k[1] * e[1] + k[2] * e[2];
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = e[a] * c + kxe[a] * sn + k[a] * ke * (1.0 - c);
    double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) e[a] = r[a] / nr;
}

static void integrate(osim* s) {
    int n[3] = {s->nx, s->ny, s->nz};
    double (*Fw)[3] = (double (*)[3])calloc(s->nobj > 0 ? s->nobj : 1, sizeof(double[3]));
    for (int k = 0; k < s->nobj; ++k)
        if (s->obj[k].kind == OBJ_SPHERE && s->obj[k].mobile) contact_force(s, k, Fw[k]);
    for (int k = 0; k < s->nobj; ++k) {
        oobj* o = &s->obj[k];
        for (int a = 0; a < 3; ++a) {
            double Fh = o->Fbb[a], Th = o->Tbb[a];
            if (s->force_avg) {
                Fh = 0.5 * (o->Fbb[a] + o->Fbb_last[a]);
                Th = 0.5 * (o->Tbb[a] + o->Tbb_last[a]);
            }
            o->Fbb_last[a] = o->Fbb[a];
            o->Tbb_last[a] = o->Tbb[a];
            o->Fapplied[a] = Fh + o->Fc[a];
            o->Tapplied[a] = Th + o->Tc[a];
            o->Fc[a] = 0.0;
            o->Tc[a] = 0.0;
        }
        if (o->kind != OBJ_SPHERE || !o->mobile) continue;
        for (int a = 0; a < 3; ++a) {
            o->vel[a] += (o->Fapplied[a] + Fw[k][a]) / o->mass;
            o->omega[a] += o->Tapplied[a] / o->inertia;
        }
        for (int a = 0; a < 3; ++a) {
            double p = o->pos[a] + o->vel[a];
            if (p >= (double)n[a]) p -= (double)n[a];
            else if (p < 0.0) p += (double)n[a];
            o->pos[a] = p;
        }
        rotate(o->e, o->omega);
        double sp = o->vel[0] * o->vel[0] + o->vel[1] * o->vel[1] + o->vel[2] * o->vel[2];
        if (!(sp < 0.25)) s->err = OERR_DIVERGED;
    }
    free(Fw);
}

/* ---- step 5: remap cells of mobile spheres --------------------------- */
static double cell_density(const osim* s, long n) {
    double r = 0.0;
    for (int i = 0; i < Q; ++i) r += s->f[i * s->N + n];
    return r;
}

static void remap(osim* s) {
    long N = s->N;
    memcpy(s->owner_prev, s->owner, sizeof(int32_t) * N);
    /* new classification of every mobile sphere's box */
    for (int k = 0; k < s->nobj; ++k) {
        oobj* o = &s->obj[k];
        if (o->kind != OBJ_SPHERE || !o->mobile || s->psm) continue;
        int id = k + 1, lo[3], W;
        sphere_box(o, lo, &W);
        for (int bz = 0; bz < W; ++bz)
            for (int by = 0; by < W; ++by)
                for (int bx = 0; bx < W; ++bx) {
                    int x = wrap(lo[0] + bx, s->nx), y = wrap(lo[1] + by, s->ny), z = wrap(lo[2] + bz, s->nz);
                    long c = cidx(s, x, y, z);
                    double d[3];
                    sphere_offset(s, o, x, y, z, d);
                    int in = oracle_inside(d, o->R);
                    int old = s->owner_prev[c];
                    if (in) {
                        if (old != 0 && old != id) s->err = OERR_OVERLAP;
                        else s->owner[c] = id;
                    } else if (old == id) {
                        s->owner[c] = 0;
                    }
                }
    }
    /* conversion, in canonical cell order */
    for (long c = 0; c < N; ++c) {
        int was = s->owner_prev[c], now = s->owner[c];
        if (was == now) continue;
        int x, y, z;
        coords(s, c, &x, &y, &z);
        if (was == 0) {
            /* fluid -> solid: the destroyed momentum goes to the body */
            oobj* o = &s->obj[now - 1];
            double d[3], m[3] = {0.0, 0.0, 0.0}, t[3];
            sphere_offset(s, o, x, y, z, d);
            for (int i = 0; i < Q; ++i) {
                double fi = s->f[i * N + c];
                m[0] += fi * CX[i];
                m[1] += fi * CY[i];
                m[2] += fi * CZ[i];
                s->f[i * N + c] = 0.0;
            }
            cross(d, m, t);
            for (int a = 0; a < 3 && s->conv != 2; ++a) {
                o->Fc[a] += m[a];
                o->Tc[a] += t[a];
            }
        } else if (now == 0) {
            /* solid -> fluid: refill with the equilibrium of the mean density of
             * the neighbours that are fluid now and were fluid before, moving with
             * the body's rigid velocity; the created momentum is taken from it */
            oobj* o = &s->obj[was - 1];
            double sum = 0.0;
            int cnt = 0;
            for (int i = 1; i < Q; ++i) {
                long m = neighbour(s, c, i);
                if (s->owner[m] == 0 && s->owner_prev[m] == 0) {
                    sum += cell_density(s, m);
                    cnt++;
                }
            }
            double rb = cnt > 0 ? sum / (double)cnt : s->rho0;
            if (s->conv == 3) rb = s->rho0;
            double d[3], w[3], u[3];
            sphere_offset(s, o, x, y, z, d);
            cross(o->omega, d, w);
            for (int a = 0; a < 3; ++a) u[a] = o->vel[a] + w[a];
            if (s->conv == 1) {
                double sl[3];
                oracle_slip(d, o->e, o->B1, o->B2, sl);
                for (int a = 0; a < 3; ++a) u[a] += sl[a];
            }
            double feq[Q], m[3] = {0.0, 0.0, 0.0}, t[3];
            if (s->inc) oracle_feq_inc(rb, s->rho0, u, feq);
            else oracle_feq(rb, u, feq);
            for (int i = 0; i < Q; ++i) {
                s->f[i * N + c] = feq[i];
                m[0] += feq[i] * CX[i];
                m[1] += feq[i] * CY[i];
                m[2] += feq[i] * CZ[i];
            }
            cross(d, m, t);
            for (int a = 0; a < 3 && s->conv != 2; ++a) {
                o->Fc[a] -= m[a];
                o->Tc[a] -= t[a];
            }
        } else {
            s->err = OERR_OVERLAP; /* direct hand-over between two bodies */
        }
    }
}

/* ---- partially saturated cells (Noble and Torczynski, 1998) -----------
 * The remedy Sec. IV A names for the speed fluctuation: instead of link
 * bounce-back and cell conversion, every cell stays fluid and carries the
 * fraction eps of its volume (the unit cube about the node) that a sphere
 * covers.  Its collision blends the fluid operator with a solid one,
 *   f*_i = f_i + (1 - B) Omega_i + B Omega^s_i,
 *   Omega^s_i = [f_ib - f_ib^eq(rho, u)] - [f_i - f_i^eq(rho, u_s)],
 *   B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),  tau = 1 / lambda_e,
 * with Omega_i the TRT collision, (rho, u) the cell's moments and u_s the
 * sphere's surface velocity at the node (v + w x d + slip, Eq. "vb").  The
 * fluid gains B sum_i Omega^s_i c_i, which the sphere loses. */

/* Solid fraction of the cell at offset d from the centre of a sphere of
 * radius R: the share of the 8 x 8 x 8 points (k + 1/2)/8 - 1/2 of the unit
 * cube inside the sphere (exact multiples of 1/512); 1 or 0 without sampling
 * when the whole cube lies inside or outside (its half-diagonal is below 0.87). */
double oracle_psm_fraction(const double* d, double R) {
    double r2 = d[0] * d[0] + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    double lo = R - 0.87, hi = R + 0.87;
    if (lo > 0.0 && r2 < lo * lo) return 1.0;
    if (r2 > hi * hi) return 0.0;
    int count = 0;
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int c = 0; c < 8; ++c) {
                double p[3] = {d[0] + ((a + 0.5) / 8.0 - 0.5), d[1] + ((b + 0.5) / 8.0 - 0.5),
                               d[2] + ((c + 0.5) / 8.0 - 0.5)};
                count += oracle_inside(p, R);
            }
    return count / 512.0;
}

static void psm_fraction(osim* s) {
    long N = s->N;
    memset(s->eps, 0, sizeof(double) * N);
    memset(s->psm_id, 0, sizeof(int32_t) * N);
    for (int k = 0; k < s->nobj; ++k) {
        oobj* o = &s->obj[k];
        if (o->kind != OBJ_SPHERE) continue;
        int lo[3], W;
        sphere_box(o, lo, &W);
        for (int bz = 0; bz < W; ++bz)
            for (int by = 0; by < W; ++by)
                for (int bx = 0; bx < W; ++bx) {
                    int x = wrap(lo[0] + bx, s->nx), y = wrap(lo[1] + by, s->ny), z = wrap(lo[2] + bz, s->nz);
                    long c = cidx(s, x, y, z);
                    double d[3];
                    sphere_offset(s, o, x, y, z, d);
                    double e = oracle_psm_fraction(d, o->R);
                    if (e == 0.0) continue;
                    if (s->psm_id[c] != 0 && s->psm_id[c] != k + 1) s->err = OERR_OVERLAP;
                    s->eps[c] = e;
                    s->psm_id[c] = k + 1;
                }
    }
}

/* Surface velocity of sphere o at node offset d (the slip by direction only). */
static void psm_surface_velocity(const oobj* o, const double* d, double* us) {
    double slip[3];
    oracle_slip(d, o->e, o->B1, o->B2, slip);
    us[0] = o->vel[0] + (o->omega[1] * d[2] - o->omega[2] * d[1]) + slip[0];
    us[1] = o->vel[1] + (o->omega[2] * d[0] - o->omega[0] * d[2]) + slip[1];
    us[2] = o->vel[2] + (o->omega[0] * d[1] - o->omega[1] * d[0]) + slip[2];
}

/* The solid operator Omega^s of a cell with populations f, and its weight B. */
static double psm_solid_term(const osim* s, const double* f, const oobj* o, const double* d, double eps,
                             double* om) {
    double rho, j[3], u[3], us[3], feq[Q], feqs[Q];
    oracle_moments(f, &rho, j);
    double den = s->inc ? s->rho0 : rho;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / den;
    psm_surface_velocity(o, d, us);
    if (s->inc) {
        oracle_feq_inc(rho, s->rho0, u, feq);
        oracle_feq_inc(rho, s->rho0, us, feqs);
    } else {
        oracle_feq(rho, u, feq);
        oracle_feq(rho, us, feqs);
    }
    for (int i = 0; i < Q; ++i) {
        int ib = oracle_opposite(i);
        om[i] = (f[ib] - feq[ib]) - (f[i] - feqs[i]);
    }
    double th = 1.0 / s->lambda_e - 0.5;
    return eps * th / ((1.0 - eps) + th);
}

/* Post-collision populations of the cells a sphere covers in part (after
 * collide_all wrote the fluid operator's result for every cell). */
static void psm_collide(osim* s) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (s->psm_id[n] == 0 || s->owner[n] != 0) continue;
        const oobj* o = &s->obj[s->psm_id[n] - 1];
        int x, y, z;
        coords(s, n, &x, &y, &z);
        double d[3], f[Q], om[Q];
        sphere_offset(s, o, x, y, z, d);
        for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
        double B = psm_solid_term(s, f, o, d, s->eps[n], om);
        for (int i = 0; i < Q; ++i) {
            double fl = s->fpost[i * N + n] - f[i]; /* the fluid operator Omega_i */
            s->fpost[i * N + n] = f[i] + (1.0 - B) * fl + B * om[i];
        }
    }
}

/* Force, torque and stresslet on each sphere: minus the momentum the solid
 * operator gives the fluid, summed in cell order (after bounce_links, which
 * zeroes the sums). */
static void psm_forces(osim* s) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        if (s->psm_id[n] == 0 || s->owner[n] != 0) continue;
        oobj* o = &s->obj[s->psm_id[n] - 1];
        int x, y, z;
        coords(s, n, &x, &y, &z);
        double d[3], f[Q], om[Q];
        sphere_offset(s, o, x, y, z, d);
        for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
        double B = psm_solid_term(s, f, o, d, s->eps[n], om);
        double m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            m[0] += om[i] * CX[i];
            m[1] += om[i] * CY[i];
            m[2] += om[i] * CZ[i];
        }
        double dF[3] = {-B * m[0], -B * m[1], -B * m[2]}, dT[3];
        cross(d, dF, dT);
        for (int a = 0; a < 3; ++a) {
            o->Fbb[a] += dF[a];
            o->Tbb[a] += dT[a];
        }
        double tr = (d[0] * dF[0] + d[1] * dF[1] + d[2] * dF[2]) / 3.0;
        o->Sbb[0] -= d[0] * dF[0] - tr;
        o->Sbb[1] -= d[1] * dF[1] - tr;
        o->Sbb[2] -= d[2] * dF[2] - tr;
        o->Sbb[3] -= 0.5 * (d[0] * dF[1] + d[1] * dF[0]);
        o->Sbb[4] -= 0.5 * (d[0] * dF[2] + d[2] * dF[0]);
        o->Sbb[5] -= 0.5 * (d[1] * dF[2] + d[2] * dF[1]);
    }
}

/* Couple the spheres by partially saturated cells (on = 1) instead of link
 * bounce-back and conversion; walls keep their links.  Call before adding
 * spheres. */
void osim_set_psm(osim* s, int on) {
    s->psm = on ? 1 : 0;
    if (s->psm && !s->eps) {
        s->eps = (double*)calloc(s->N, sizeof(double));
        s->psm_id = (int32_t*)calloc(s->N, sizeof(int32_t));
    }
}

/* Solid fraction of every cell at the last step ([N], zero without PSM). */
void osim_get_eps(const osim* s, double* out) {
    for (long n = 0; n < s->N; ++n) out[n] = s->psm ? s->eps[n] : 0.0;
}

void osim_step(osim* s, int64_t nsteps) {
    for (int64_t t = 0; t < nsteps; ++t) {
        if (s->psm) psm_fraction(s);
        collide_all(s);
        if (s->psm) psm_collide(s);
        bounce_links(s);
        if (s->psm) psm_forces(s);
        stream_all(s);
        integrate(s);
        remap(s);
        s->step++;
    }
}

/* ---- outputs ---------------------------------------------------------- */

/* rho[N] and u as SoA [3][N]; solid cells report 0.  Either may be NULL. */
void osim_get_fields(const osim* s, double* rho, double* u) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        if (s->owner[n] == 0) {
            double f[Q];
            for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
            oracle_moments(f, &r, j);
        }
        if (rho) rho[n] = r;
        if (u) {
            const double den = s->inc ? s->rho0 : r; /* u = j / rho0 in the incompressible model */
            u[n] = r != 0.0 ? j[0] / den : 0.0;
            u[N + n] = r != 0.0 ? j[1] / den : 0.0;
            u[2 * N + n] = r != 0.0 ? j[2] / den : 0.0;
        }
    }
}

/* sum of rho over fluid cells, and total fluid momentum */
void osim_get_totals(const osim* s, double* mass, double* mom) {
    long N = s->N;
    double m = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (long n = 0; n < N; ++n) {
        if (s->owner[n] != 0) continue;
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * N + n];
            m += fi;
            j[0] += fi * CX[i];
            j[1] += fi * CY[i];
            j[2] += fi * CZ[i];
        }
    }
    *mass = m;
    if (mom) {
        mom[0] = j[0];
        mom[1] = j[1];
        mom[2] = j[2];
    }
}

static int valid_id(const osim* s, int32_t id) { return id >= 1 && id <= s->nobj; }

/* F, T: hydrodynamic force/torque of the last update (momentum exchange plus
 * conversion force); S: stresslet of the last step's links. */
int32_t osim_get_force_torque(const osim* s, int32_t id, double* F, double* T) {
    if (!valid_id(s, id)) return OERR_INVALID;
    const oobj* o = &s->obj[id - 1];
    for (int a = 0; a < 3; ++a) {
        F[a] = o->Fapplied[a];
        T[a] = o->Tapplied[a];
    }
    return OERR_OK;
}

int32_t osim_get_stresslet(const osim* s, int32_t id, double* S) {
    if (!valid_id(s, id)) return OERR_INVALID;
    for (int a = 0; a < 6; ++a) S[a] = s->obj[id - 1].Sbb[a];
    return OERR_OK;
}

int32_t osim_get_object_state(const osim* s, int32_t id, double* pos, double* vel, double* e, double* omega) {
    if (!valid_id(s, id)) return OERR_INVALID;
    const oobj* o = &s->obj[id - 1];
    for (int a = 0; a < 3; ++a) {
        if (pos) pos[a] = o->pos[a];
        if (vel) vel[a] = o->vel[a];
        if (e) e[a] = o->e[a];
        if (omega) omega[a] = o->omega[a];
    }
    return OERR_OK;
}

/* Boundary links of object id (or of all objects if id == 0), canonical order,
 * each written as cell_index * 32 + direction.  Returns the count (writes at
 * most cap entries). */
int64_t osim_get_links(const osim* s, int32_t id, int64_t* out, int64_t cap) {
    int64_t cnt = 0;
    for (long n = 0; n < s->N; ++n) {
        if (s->owner[n] != 0) continue;
        for (int i = 1; i < Q; ++i) {
            int o = s->owner[neighbour(s, n, i)];
            if (o == 0 || (id != 0 && o != id)) continue;
            if (cnt < cap) out[cnt] = (int64_t)n * 32 + i;
            cnt++;
        }
    }
    return cnt;
}

int32_t oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the collide and stream loops from now on (n >= 1); no effect
 * without OpenMP.  The results do not depend on it. */
void oracle_set_num_threads(int32_t n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Conversion force and torque booked by the last remap, to be applied in the
 * next update. */
int32_t osim_get_pending_conversion(const osim* s, int32_t id, double* Fc, double* Tc) {
    if (!valid_id(s, id)) return OERR_INVALID;
    for (int a = 0; a < 3; ++a) {
        Fc[a] = s->obj[id - 1].Fc[a];
        Tc[a] = s->obj[id - 1].Tc[a];
    }
    return OERR_OK;
}
