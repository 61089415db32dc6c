"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on the
same seeded inputs, element by element.

Tolerances:
  * FP64 storage: 1e-12 relative (max |gpu - oracle| / max |oracle| per field),
    the FP64 target; the two sides differ only in rounding order.
  * cell classification and boundary-link sets: bit-exact.
  * reduced storages: derived from the rounding of one stored value per
    population per step (FP32 2^-24, FP16 2^-11, BF16 2^-8 of the deviation
    f - w rho0) accumulated over the run; stated per test.
"""
import numpy as np
import pytest

from paper_1903_04799_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice, lbsq  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def make_pair(shape, collision="bgk", lambda_e=1.0, storage="f64"):
    g = Lattice(shape, collision=collision, lambda_e=lambda_e, storage=storage)
    o = OracleSim(*shape, lambda_e=lambda_e, collision=collision)
    return g, o


# ------------------------------------------------------------------ bulk fluid

@pytest.mark.parametrize("collision,lambda_e", [("bgk", 1.0), ("trt", 1.0), ("trt", 1.7), ("bgk", 0.6)])
@pytest.mark.parametrize("steps", [1, 2, 37])
def test_bulk_f64_parity(collision, lambda_e, steps):
    """Periodic box, smooth random fields, ragged sizes (not multiples of 32):
    FP64 populations within 1e-12 after even and odd step counts."""
    shape = (45, 19, 23)
    g, o = make_pair(shape, collision, lambda_e)
    rho, u = W.smooth_fields(shape, seed=7, drho=0.02, umax=0.05)
    g.set_fields(rho, u)
    o.set_equilibrium(rho, u)
    g.step(steps)
    o.step(steps)
    fg, fo = g.populations(), o.populations()
    assert rel(fg, fo) < 1e-12
    # deviations from rest: tighter view of the same comparison
    assert np.abs(fg - fo).max() < 1e-14


def test_bulk_random_populations_f64():
    """Far-from-equilibrium random populations (every relaxation mode excited)."""
    shape = (33, 17, 9)
    g, o = make_pair(shape, "trt", 1.3)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = W.random_populations(int(np.prod(shape)), seed=3, base=w, spread=0.2)
    g.set_populations(f)
    o.set_populations(f)
    g.step(11)
    o.step(11)
    assert np.abs(g.populations() - o.populations()).max() < 1e-14


def test_degenerate_lattices():
    """Lattices of one cell along an axis (self-periodic) and tiny boxes."""
    for shape in [(1, 16, 1), (7, 1, 5), (1, 1, 1), (2, 3, 64)]:
        g, o = make_pair(shape, "trt", 1.1)
        rho, u = W.smooth_fields(shape, seed=11)
        g.set_fields(rho, u)
        o.set_equilibrium(rho, u)
        g.step(5)
        o.step(5)
        assert np.abs(g.populations() - o.populations()).max() < 1e-14, shape


def test_lattice_size_limits():
    """lb_create admits fewer than 2^27 cells (boundary links are coded as
    cell << 5 | direction in 32 bits): 512^3 = 2^27 is refused before any
    allocation, 512 x 512 x 511 (FP16, 5 GB) is created and steps; a zero or
    negative extent is refused."""
    for shape in [(512, 512, 512), (0, 8, 8), (8, -1, 8)]:
        with pytest.raises(lbsq.LBError) as ex:
            Lattice(shape, collision="trt", storage="f16dev")
        assert ex.value.status == lbsq.LB_ERR_INVALID
    g = Lattice((512, 512, 511), collision="trt", storage="f16dev")
    g.step(2)
    _, P = g.mass()
    assert np.abs(P).max() < 1e-6
    g.close()


def test_mass_momentum_conserved_f64():
    shape = (40, 30, 20)
    g = Lattice(shape, collision="trt", storage="f64")
    rho, u = W.smooth_fields(shape, seed=5)
    g.set_fields(rho, u)
    m0, j0 = g.mass()
    g.step(200)
    m1, j1 = g.mass()
    assert abs(m1 - m0) < 1e-11 * m0
    assert np.abs(j1 - j0).max() < 1e-11


@pytest.mark.parametrize("collision,lambda_e", [("trt", 1.0), ("trt", 1.3), ("bgk", 0.8)])
def test_incompressible_bulk_f64_parity(collision, lambda_e):
    """The incompressible equilibrium (lb_params.equilibrium) against the
    oracle's, rho0 = 1.15 so that it differs from the compressible model:
    lb_set_fields, 1 and 26 steps of collision and streaming, and the
    exported u = j / rho0, within 1e-14."""
    shape, rho0 = (45, 19, 23), 1.15
    g = Lattice(shape, collision=collision, lambda_e=lambda_e, rho0=rho0, equilibrium="incompressible")
    o = OracleSim(*shape, lambda_e=lambda_e, collision=collision, rho0=rho0)
    o.set_incompressible(True)
    rho, u = W.smooth_fields(shape, seed=9, drho=0.03, umax=0.05)
    g.set_fields(rho0 * rho, u)
    o.set_equilibrium(rho0 * rho, u)
    for n in (1, 25):
        g.step(n)
        o.step(n)
        assert np.abs(g.populations() - o.populations()).max() < 1e-14
        rg, ug = g.fields()
        ro, uo = o.fields()
        assert np.abs(rg - ro).max() < 1e-14
        assert np.abs(ug - uo).max() < 1e-14


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16dev", 2e-2)])
def test_incompressible_free_swimmer(storage, tol):
    """A free squirmer crossing cells with the incompressible equilibrium
    (collision, refill of uncovered cells, export), rho0 = 1.2: FP64 within
    1e-12 of the oracle (fields, links, forces, states); reduced storages
    within the tolerances of the compressible runs."""
    shape, rho0 = (28, 26, 30), 1.2
    g = Lattice(shape, collision="trt", rho0=rho0, storage=storage, equilibrium="incompressible")
    o = OracleSim(*shape, lambda_e=1.0, collision="trt", rho0=rho0)
    o.set_incompressible(True)
    args = ((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0)
    gi = g.add_squirmer(*args, mobile=True, density=rho0)
    oi = o.add_sphere(*args, mobile=True, density=rho0)
    changed, prev = 0, o.owner()
    for _ in range(4):
        g.step(40)
        o.step(40)
        own = o.owner()
        changed += int((own != prev).sum())
        prev = own
        if storage == "f64":
            _compare_bodies(g, o, [gi], [oi])
    assert changed > 0
    if storage != "f64":
        _, ug = g.fields()
        _, uo = o.fields()
        both = (g.owner() == 0) & (o.owner() == 0)
        assert rel(ug[:, both], uo[:, both]) < tol
        vg, vo = g.state(gi)[1], o.state(oi)[1]
        assert np.abs(vg - vo).max() / np.abs(vo).max() < tol


# ------------------------------------------------------------------ classification

@pytest.mark.parametrize("pos,R", [((16.0, 16.0, 16.0), 4.0), ((0.0, 31.0, 0.5), 5.0),
                                   ((3.7, 12.2, 29.9), 6.3), ((15.5, 15.5, 15.5), 3.5)])
def test_classification_bit_exact(pos, R):
    shape = (32, 32, 32)
    g, o = make_pair(shape)
    gi = g.add_squirmer(pos, (0, 0, 1), R, 0.0, 0.0, mobile=False)
    oi = o.add_sphere(pos, (0, 0, 1), R, mobile=False)
    assert gi == oi
    assert (g.owner() == o.owner()).all()
    assert np.array_equal(np.sort(g.links()), np.sort(o.links()))


def test_overlap_rejected():
    from paper_1903_04799_gb300.lbsq import LBError, LB_ERR_OVERLAP
    g = Lattice((32, 32, 32))
    g.add_squirmer((10, 10, 10), (0, 0, 1), 4.0, 0.0, 0.0, mobile=False)
    before = g.owner()
    with pytest.raises(LBError) as ei:
        g.add_squirmer((16, 10, 10), (0, 0, 1), 4.0, 0.0, 0.0, mobile=False)
    assert ei.value.status == LB_ERR_OVERLAP
    assert (g.owner() == before).all()


# ------------------------------------------------------------------ bodies

W_I = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
C_NORM = np.array([0.0] + [1.0] * 6 + [np.sqrt(2.0)] * 12)


def gross_flux(o, oid, rho0=1.0):
    """Sum over the body's links of the magnitude of the exchanged momentum at
    rest, 2 w_i rho0 |c_i|: the scale of the terms whose sum is the force.
    The force is 10^2-10^4 times smaller than this sum of terms, so its FP64
    rounding error (either side's) is relative to this scale, not to |F|."""
    d = o.links(oid) % 32
    return float((2 * W_I[d] * rho0 * C_NORM[d]).sum())


def _compare_bodies(g, o, gids, oids, tol=1e-12, R=None):
    """FP64 parity: fields and body state within `tol` relative; per-body sums
    (F, T, S) within `tol` relative to the gross flux of their terms."""
    rg, ug = g.fields()
    ro, uo = o.fields()
    assert (g.owner() == o.owner()).all(), "classification differs"
    assert rel(ug, uo) < tol
    assert np.abs(rg - ro).max() < tol * g.params.rho0  # density relative to itself
    for gi, oi in zip(gids, oids):
        assert np.array_equal(np.sort(g.links(gi)), np.sort(o.links(oi)))
        flux = gross_flux(o, oi)
        Fg, Tg = g.force_torque(gi)
        Fo, To = o.force_torque(oi)
        lever = float(R) if R else 8.0  # |d| of the link midpoints, about R
        assert np.abs(Fg - Fo).max() < tol * max(flux, np.abs(Fo).max()), (Fg, Fo)
        assert np.abs(Tg - To).max() < tol * lever * max(flux, np.abs(Fo).max()), (Tg, To)
        Sg, So = g.stresslet(gi), o.stresslet(oi)
        assert np.abs(Sg - So).max() < tol * lever * max(flux, np.abs(Fo).max()), (Sg, So)
        sg, so = g.state(gi), o.state(oi)
        for a, b in zip(sg, so):
            assert np.abs(a - b).max() < 1e-12


def test_c1_fixed_squirmer_f64():
    """The 32^3 fixed-squirmer configuration, 500 BGK steps: u field, force,
    torque within 1e-12 of the oracle."""
    wl = W.c1_fixed_squirmer()
    g, o = make_pair(wl.shape, wl.collision, wl.lambda_e)
    b = wl.bodies[0]
    gi = g.add_squirmer(b.pos, b.e, b.R, b.B1, b.beta, mobile=b.mobile)
    oi = o.add_sphere(b.pos, b.e, b.R, b.B1, b.beta, mobile=b.mobile)
    g.step(wl.steps)
    o.step(wl.steps)
    _compare_bodies(g, o, [gi], [oi])


@pytest.mark.parametrize("beta", [0.0, -5.0, 5.0])
def test_free_swimmer_f64(beta):
    """A free squirmer crossing cells (conversion, refill, relinking, Newton-Euler)."""
    shape = (28, 26, 30)
    g, o = make_pair(shape, "trt", 1.0)
    args = ((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, beta)
    gi = g.add_squirmer(*args, mobile=True)
    oi = o.add_sphere(*args, mobile=True)
    changed = 0
    prev = o.owner()
    for _ in range(6):
        g.step(50)
        o.step(50)
        own = o.owner()
        changed += int((own != prev).sum())
        prev = own
        _compare_bodies(g, o, [gi], [oi])
    assert changed > 0


def test_walls_couette_and_tube():
    """A moving plane wall (Couette) and a square tube with a fixed obstacle."""
    shape = (6, 14, 5)
    g, o = make_pair(shape, "bgk", 0.9)
    g.add_plane_wall(1, 0)
    gw = g.add_plane_wall(1, 13, vel=(1e-3, 0, 2e-4))
    o.add_plane_wall(1, 0)
    ow = o.add_plane_wall(1, 13, vel=(1e-3, 0, 2e-4))
    g.step(301)
    o.step(301)
    _compare_bodies(g, o, [gw], [ow])

    shape = (18, 18, 40)
    g, o = make_pair(shape, "trt", 1.0)
    g.add_tube()
    for w in [(0, 0), (0, 17), (1, 0), (1, 17)]:
        o.add_plane_wall(*w)
    gs = g.add_squirmer((9.2, 8.9, 10.0), (0.1, 0.05, 1.0), 3.5, 0.02, 2.0, mobile=True)
    os_ = o.add_sphere((9.2, 8.9, 10.0), (0.1, 0.05, 1.0), 3.5, 0.02, 2.0, mobile=True)
    gob = g.add_obstacle((9.0, 9.0, 28.0), 3.0)
    oob = o.add_sphere((9.0, 9.0, 28.0), (0, 0, 1), 3.0, 0.0, 0.0, mobile=False)
    g.set_contact(1.0, 0.01)
    o.set_contact(1.0, 0.01)
    for _ in range(3):
        g.step(60)
        o.step(60)
        _compare_bodies(g, o, [gs, gob], [os_, oob])


@pytest.mark.parametrize("density_of_node,velocity_at_node", [(1, 0), (0, 1), (1, 1)])
def test_link_options_against_oracle(density_of_node, velocity_at_node):
    """The two open readings of the moving-wall bounce-back (lb_set_link_options
    against the oracle's switches): the shift with the fluid node's density,
    and the wall velocity and lever arm at the boundary node.  A free swimmer
    crossing cells (FP64, 1e-12 against the oracle; FP32 storage within the
    reduced-storage bound) and a Couette flow at density 1.05 (rho0 = 1)
    with a moving wall.  (The double-float FP64 sweep carries about 47 bits
    of the deviation f - w rho0: at a density 30 % off rho0 its rounding
    grows to a few times 1e-12 of u over these 301 steps.)"""
    shape = (28, 26, 30)
    args = ((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0)
    o = OracleSim(*shape, lambda_e=1.0, collision="trt")
    o.set_local_density(bool(density_of_node))
    o.set_link_at_node(bool(velocity_at_node))
    oi = o.add_sphere(*args, mobile=True)
    runs = {}
    for storage in ("f64", "f32"):
        g = Lattice(shape, collision="trt", storage=storage)
        g.set_link_options(density_of_node, velocity_at_node)
        runs[storage] = (g, g.add_squirmer(*args, mobile=True))
    for _ in range(3):
        o.step(40)
        for g, _ in runs.values():
            g.step(40)
        g, gi = runs["f64"]
        _compare_bodies(g, o, [gi], [oi], R=4.5)
    g, gi = runs["f32"]
    _, ug = g.fields()
    _, uo = o.fields()
    both = (g.owner() == 0) & (o.owner() == 0)
    assert rel(ug[:, both], uo[:, both]) < 2e-6
    for g, _ in runs.values():
        g.close()

    shape = (6, 14, 5)
    N = int(np.prod(shape))
    g, o = make_pair(shape, "bgk", 0.9)
    g.set_link_options(density_of_node, velocity_at_node)
    o.set_local_density(bool(density_of_node))
    o.set_link_at_node(bool(velocity_at_node))
    rho, u = np.full(N, 1.05), np.zeros((3, N))
    g.set_fields(rho, u)
    o.set_equilibrium(rho, u)
    g.add_plane_wall(1, 0)
    gw = g.add_plane_wall(1, 13, vel=(1e-3, 0, 2e-4))
    o.add_plane_wall(1, 0)
    ow = o.add_plane_wall(1, 13, vel=(1e-3, 0, 2e-4))
    g.step(301)
    o.step(301)
    _compare_bodies(g, o, [gw], [ow])


def test_classification_band_adversarial():
    """The fused body kernel decides "inside" in FP32 away from the sphere
    surface and in exact FP64 within an error band around it.  Here every
    sphere has R = 5, so R^2 = 25 is the squared distance of 30 lattice
    vectors ((5,0,0), (3,4,0), ...), and starts a random 1e-9 .. 1e-4 off an
    integer centre: at each re-classification of the first steps (the
    spheres move by about 1e-5 per step, and a sphere with a node on its
    surface re-classifies every step) dozens of nodes per sphere lie inside
    the band or at its edges.  Owners bit-exact with the oracle's exact FP64
    test at every step, and the fields and states within 1e-12."""
    shape = (64, 64, 64)
    rng = np.random.default_rng(77)
    g, o = make_pair(shape, "trt", 1.0)
    gids, oids = [], []
    for cx in (12, 32, 52):
        for cy in (12, 32, 52):
            for cz in (12, 42):
                off = rng.choice([-1.0, 1.0], 3) * 10.0 ** rng.uniform(-9, -4, 3)
                e = rng.standard_normal(3)
                args = ((cx + off[0], cy + off[1], cz + off[2]), tuple(e / np.linalg.norm(e)), 5.0, 0.02,
                        float(rng.uniform(-3, 3)))
                gids.append(g.add_squirmer(*args, mobile=True))
                oids.append(o.add_sphere(*args, mobile=True))
    for _ in range(12):
        g.step(1)
        o.step(1)
        assert (g.owner() == o.owner()).all()
    g.step(20)
    o.step(20)
    _compare_bodies(g, o, gids, oids, R=5.0)


def test_round_tube_swimmer_f64():
    """Sec. V tube flow: a squirmer swimming toward the wall of a round tube
    (lb_add_wall kind 3), with the contact force on (Eq. "wca"), which it
    reaches after about 100 steps.  Owners and link sets bit-exact; fields,
    body state, and the squirmer's and the tube's force, torque and stresslet
    within 1e-12 of the oracle."""
    shape = (24, 24, 28)
    g, o = make_pair(shape, "trt", 1.0)
    tg = g.add_round_tube(11.5, 11.5, 10.0)
    to = o.add_tube(11.5, 11.5, 10.0)
    args = ((16.4, 12.1, 13.7), (0.8, 0.3, 0.5), 3.0, 0.012, -2.0)
    gi = g.add_squirmer(*args, mobile=True)
    oi = o.add_sphere(*args, mobile=True)
    g.set_contact(1.0, 0.05)
    o.set_contact(1.0, 0.05)
    for _ in range(4):
        g.step(40)
        o.step(40)
        _compare_bodies(g, o, [gi, tg], [oi, to], R=10.0)


def test_two_swimmers_f64():
    shape = (40, 24, 24)
    g, o = make_pair(shape, "trt", 1.0)
    a = ((10.2, 12.1, 11.8), (1.0, 0.1, 0.0), 4.0, 0.03, -3.0)
    b = ((29.7, 11.6, 12.3), (-1.0, 0.05, 0.1), 4.0, 0.03, 3.0)
    gids = [g.add_squirmer(*a, mobile=True), g.add_squirmer(*b, mobile=True)]
    oids = [o.add_sphere(*a, mobile=True), o.add_sphere(*b, mobile=True)]
    for _ in range(4):
        g.step(40)
        o.step(40)
        _compare_bodies(g, o, gids, oids)


@pytest.mark.parametrize("setup", ["free", "split", "pair"])
def test_force_average_f64(setup):
    """Ladd's two-step force average (lb_set_force_average) against the
    oracle's: fields, links, forces and body states within 1e-12, on the
    single-sphere fused path, on split steps (a sphere in a large box, across
    the periodic faces) and on the multi-kernel path of two spheres near each
    other; checked after every block of steps."""
    if setup == "free":
        shape, bodies, blocks = (28, 26, 30), [((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0)], (7, 30)
    elif setup == "split":
        shape, bodies, blocks = (128, 96, 96), [((64.3, 2.7, 94.1), (0.3, 0.5, 1.0), 6.0, 0.05, -3.0)], (5, 16, 9)
    else:
        shape = (40, 24, 24)
        # 1.5 cells apart, swimming apart
        bodies = [((15.2, 12.1, 11.8), (-1.0, 0.1, 0.0), 4.0, 0.03, -3.0),
                  ((24.7, 11.6, 12.3), (1.0, 0.05, 0.1), 4.0, 0.03, 3.0)]
        blocks = (9, 20)
    g, o = make_pair(shape, "trt", 1.0)
    g.set_force_average(True)
    o.set_force_average(True)
    gids = [g.add_squirmer(*b, mobile=True) for b in bodies]
    oids = [o.add_sphere(*b, mobile=True) for b in bodies]
    for n in blocks:
        g.step(n)
        o.step(n)
        _compare_bodies(g, o, gids, oids, R=bodies[0][2])


def _random_spheres(rng, shape, count, R, min_dist):
    """`count` sphere centres by random sequential addition (minimum-image
    distance >= min_dist), random unit axes, beta ~ U[-4, 4]."""
    n = np.array(shape, dtype=float)
    pts, out = [], []
    while len(pts) < count:
        p = rng.uniform(0, n)
        if all(np.linalg.norm((p - q) - n * np.round((p - q) / n)) >= min_dist for q in pts):
            e = rng.standard_normal(3)
            pts.append(p)
            out.append((tuple(p), tuple(e / np.linalg.norm(e)), R, 0.03, float(rng.uniform(-4, 4))))
    return out


@pytest.mark.parametrize("count,shape,R", [(20, (48, 44, 40), 3.0), (80, (72, 64, 60), 2.6)])
def test_many_spheres_cluster_classes_f64(count, shape, R):
    """20 mobile squirmers (the fused kernel at 8 blocks per sphere) and 80 (4
    blocks), close enough that some grown scan boxes meet, so those spheres
    re-classify through the multi-kernel path while the rest stay fused:
    fields, classification, links, forces and states against the oracle."""
    rng = np.random.default_rng(1000 + count)
    bodies = _random_spheres(rng, shape, count, R, 2 * R + 2.5)
    g, o = make_pair(shape, "trt", 1.0)
    gids = [g.add_squirmer(*b, mobile=True) for b in bodies]
    oids = [o.add_sphere(*b, mobile=True) for b in bodies]
    for _ in range(3):
        g.step(20)
        o.step(20)
    _compare_bodies(g, o, gids, oids, R=R)


def test_c4_full_size_parity_f64():
    """The 256^3 suspension of 200 squirmers (R = 6) at full size, in the
    launch configuration bench.py times, 16 steps: classification, fields and
    every body's state against the oracle."""
    wl = W.c4_suspension()
    g = Lattice(wl.shape, collision="trt", storage="f64")
    o = OracleSim(*wl.shape, lambda_e=1.0, collision="trt")
    # B1 raised so that cells change within the run
    gids = [g.add_squirmer(b.pos, b.e, b.R, 0.05, b.beta, mobile=True) for b in wl.bodies]
    oids = [o.add_sphere(b.pos, b.e, b.R, 0.05, b.beta, mobile=True) for b in wl.bodies]
    g.step(16)
    o.step(16)
    assert (g.owner() == o.owner()).all()
    _, ug = g.fields()
    _, uo = o.fields()
    assert rel(ug, uo) < 1e-12
    for gi, oi in zip(gids, oids):
        for a, b in zip(g.state(gi), o.state(oi)):
            assert np.abs(a - b).max() < 1e-12


def test_determinism_bitwise():
    """The same run twice gives the same bits (fixed-order reductions)."""
    outs = []
    for _ in range(2):
        g = Lattice((28, 26, 30), collision="trt", storage="f64")
        gi = g.add_squirmer((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0, mobile=True)
        g.step(150)
        outs.append((g.populations(), g.force_torque(gi)[0], g.state(gi)[0]))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage,variant", [("f64", 0), ("f64", 1), ("f32", 0), ("f32", 1), ("f16dev", 0),
                                             ("f16dev", 1), ("f16dev", 3), ("bf16dev", 0), ("bf16dev", 3)])
def test_near_window_split_bitwise(storage, variant):
    """The split step -- the far sweep beside the body step, then the sweep of
    the near-body window, a box of rows bounded in z and y -- against
    whole-lattice sweeps (the traced mode never splits): the same bits for
    every population, owner and body state.  The swimmer sits across the
    periodic faces in y and z, so the window wraps on both axes, and crosses
    cells.  The run mixes eager units of both parities with graph replays,
    consecutive lb_step calls (the last step's body kernels left pending
    across them) and reads in between (which issue them)."""
    shape = (128, 96, 96)
    pos, e = (64.3, 2.7, 94.1), (0.3, 0.5, 1.0)
    runs = []
    for traced in (False, True):
        g = Lattice(shape, collision="trt", storage=storage)
        g.set_sweep_variant(variant)
        gi = g.add_squirmer(pos, e, 6.0, 0.05, -3.0, mobile=True)
        if traced:
            g.profile_begin()
        seen = []
        for n, read in ((5, False), (16, True), (3, False), (9, True), (1, True), (8, False), (8, False)):
            g.step(n)
            if read:
                seen.append(g.state(gi))
        if traced:
            g.profile_end()
        runs.append((g.populations(), g.owner(), g.state(gi), seen))
        g.close()
    (fa, oa, sa, ra), (fb, ob, sb, rb) = runs
    assert (oa == ob).all()
    assert np.array_equal(fa, fb)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    for u, v in zip(ra, rb):
        for x, y in zip(u, v):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("nx", [16, 36, 45, 50])
@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
def test_split_odd_steps_narrow_rows_bitwise(storage, nx):
    """The 16-bit odd steps of split sweeps (four cells per thread, each
    direction's sources an aligned chunk plus the element beyond its end)
    against whole-lattice sweeps, on rows of 4 and 9 four-cell groups: most
    threads of a warp hold no cells, and the groups at x = 0 and x = nx - 4
    take their end elements across the periodic x boundary, which the swimmer
    also crosses.  Ragged rows (nx = 45: one cell per thread; nx = 50: two
    cells per thread) take the other forms in both kinds of sweep."""
    shape = (nx, 40, 72)
    runs = []
    for traced in (False, True):
        g = Lattice(shape, collision="trt", storage=storage)
        gi = g.add_squirmer((0.6, 20.3, 30.2), (0.6, 0.2, 1.0), 3.0, 0.05, -2.0, mobile=True)
        if traced:
            g.profile_begin()
        g.step(3)
        g.step(40)
        if traced:
            g.profile_end()
        runs.append((g.populations(), g.owner(), g.state(gi)))
        g.close()
    (fa, oa, sa), (fb, ob, sb) = runs
    assert (oa == ob).all()
    assert np.array_equal(fa, fb)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


def _far_apart(g):
    # two isolated spheres 65 planes apart: the window spans the gap
    return [g.add_squirmer((48.3, 30.2, 40.1), (0.2, 0.1, 1.0), 5.0, 0.05, -3.0, mobile=True),
            g.add_squirmer((47.6, 70.4, 105.3), (-0.1, 0.2, -1.0), 5.0, 0.05, 4.0, mobile=True)]


def _close_pair(g):
    # two spheres 3.9 cells apart (the multi-kernel body path), swimming apart
    return [g.add_squirmer((48.3, 48.2, 60.1), (0.0, 0.1, -1.0), 5.0, 0.05, -3.0, mobile=True),
            g.add_squirmer((48.1, 48.4, 74.0), (0.1, 0.0, 1.0), 5.0, 0.05, 2.0, mobile=True)]


def _sphere_and_z_wall(g):
    # a z-normal wall at z = 0 and a sphere 60 planes away: the window spans
    # every row and the planes between them
    ids = [g.add_squirmer((48.3, 47.7, 62.2), (0.3, 0.2, 1.0), 5.0, 0.05, -2.0, mobile=True)]
    g.add_plane_wall(2, 0)
    return ids


@pytest.mark.parametrize("bodies", [_far_apart, _close_pair, _sphere_and_z_wall])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev"])
def test_near_window_split_several_bodies_bitwise(bodies, storage):
    """Split steps with more than one body, against whole-lattice sweeps: the
    window is one box around every body's range, so it also spans the gap
    between them and can be far longer than any one body's range.  The same
    bits for every population, owner and body state."""
    shape = (96, 96, 160)
    runs = []
    for traced in (False, True):
        g = Lattice(shape, collision="trt", storage=storage)
        ids = bodies(g)
        if traced:
            g.profile_begin()
        for n in (5, 16, 3, 9, 1, 8, 8):
            g.step(n)
        if traced:
            g.profile_end()
        runs.append((g.populations(), g.owner(), [g.state(i) for i in ids]))
        g.close()
    (fa, oa, sa), (fb, ob, sb) = runs
    assert (oa == ob).all()
    assert np.array_equal(fa, fb)
    for u, v in zip(sa, sb):
        for x, y in zip(u, v):
            assert np.array_equal(x, y)


# ------------------------------------------------------------------ reduced storage

@pytest.mark.parametrize("storage,tol", [("f32", 2e-6), ("f16dev", 2e-3), ("bf16dev", 1.5e-2)])
def test_reduced_storage_free_swimmer(storage, tol):
    """Reduced storages against the FP64 oracle: u field and body velocity after
    200 steps, the worst cell relative to max|u|.  The storage rounds each
    deviation g to 2^-24 (FP32), 2^-11 (FP16 at scale 2^14) or 2^-8 (BF16,
    stochastic) of itself every step.  |g| is about |u| / 6 here (3 w c.u),
    and the collision relaxes every non-conserved moment each step, so only
    the rounding of the conserved ones (rho, j) accumulates, as a random walk
    spread by diffusion: over 200 steps a few units of 2^-p |u|.  Measured on
    GB300: FP32 1.8e-7, FP16 1.5e-4, BF16 1.2e-3; the bounds are about ten
    times those."""
    shape = (28, 26, 30)
    g = Lattice(shape, collision="trt", storage=storage)
    o = OracleSim(*shape, lambda_e=1.0, collision="trt")
    args = ((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0)
    gi = g.add_squirmer(*args, mobile=True)
    oi = o.add_sphere(*args, mobile=True)
    g.step(200)
    o.step(200)
    _, ug = g.fields()
    _, uo = o.fields()
    both = (g.owner() == 0) & (o.owner() == 0)
    assert rel(ug[:, both], uo[:, both]) < tol
    vg, vo = g.state(gi)[1], o.state(oi)[1]
    assert np.abs(vg - vo).max() / np.abs(vo).max() < tol


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("nx,lambda_e", [(128, 1.0), (256, 1.0), (128, 1.3), (32, 1.0), (64, 1.0), (96, 1.0)])
def test_sweep_variants_bitwise_16bit(storage, nx, lambda_e):
    """Every sweep form gives the same bits as the one-cell form: the two-cell
    form and the whole-row four-cell form (odd-step x-shifts through shared
    memory; ny = 13: blocks with rows beyond the lattice; nx = 64 and 96:
    rows of 16 and 24 threads), alone and alternating by parity (the
    default); on both step parities, with a swimmer in the lattice and ragged
    ny, nz; with lambda_e = 1 (the collision's fully relaxed even part) and
    1.3 (the general form)."""
    shape = (nx, 13, 14)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = W.random_populations(int(np.prod(shape)), seed=11, base=w, spread=0.2)
    out = {}
    for variant in (0, 1, 2, 3):
        g = Lattice(shape, collision="trt", lambda_e=lambda_e, storage=storage)
        g.set_sweep_variant(variant)
        g.set_populations(f)
        gi = g.add_squirmer((nx / 2 + 0.3, 6.2, 6.9), (1.0, 0.2, 0.1), 3.0, 0.02, -1.0, mobile=True)
        g.step(7)
        out[variant] = (g.populations(), g.state(gi)[0])
    for v in (0, 2, 3):
        assert np.array_equal(out[v][0], out[1][0]), v
        assert np.array_equal(out[v][1], out[1][1]), v


def test_four_cell_f16_against_oracle():
    """FP16 storage on a 128-wide lattice (the four-cell sweep) against the
    FP64 oracle, with the tolerance of the two-cell FP16 test."""
    shape = (128, 16, 18)
    g = Lattice(shape, collision="trt", storage="f16dev")
    o = OracleSim(*shape, lambda_e=1.0, collision="trt")
    args = ((64.3, 7.8, 9.1), (1.0, 0.2, -0.1), 4.0, 0.03, 2.0)
    gi = g.add_squirmer(*args, mobile=True)
    oi = o.add_sphere(*args, mobile=True)
    g.step(120)
    o.step(120)
    _, ug = g.fields()
    _, uo = o.fields()
    both = (g.owner() == 0) & (o.owner() == 0)
    assert rel(ug[:, both], uo[:, both]) < 2e-2
    vg, vo = g.state(gi)[1], o.state(oi)[1]
    assert np.abs(vg - vo).max() / np.abs(vo).max() < 2e-2


# ------------------------------------------------------------------ full size

@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_c2_full_size_parity(storage, tol):
    """The 128^3 free-swimmer configuration at full size, in the launch
    configuration bench.py times: 24 steps against the oracle, whole fields
    (the oracle finishes 24 steps of 2.1 M cells in seconds)."""
    wl = W.c2_free_swimmer(beta=-5.0)
    b = wl.bodies[0]
    g = Lattice(wl.shape, collision="trt", storage=storage)
    o = OracleSim(*wl.shape, lambda_e=1.0, collision="trt")
    # an off-node start and a tilted axis so that cells change
    pos, e = (64.3, 63.8, 64.1), (0.2, 0.1, 1.0)
    gi = g.add_squirmer(pos, e, b.R, 0.05, b.beta, mobile=True)
    oi = o.add_sphere(pos, e, b.R, 0.05, b.beta, mobile=True)
    g.step(24)
    o.step(24)
    assert (g.owner() == o.owner()).all()
    _, ug = g.fields()
    _, uo = o.fields()
    assert rel(ug, uo) < tol
    assert np.abs(g.state(gi)[1] - o.state(oi)[1]).max() < tol * np.abs(o.state(oi)[1]).max()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16dev", 2e-2)])
def test_c3_full_size_parity(storage, tol):
    """The 256^3 pusher (R = 16, beta = -3) at full size, in the launch
    configuration bench.py times for each storage (split near/far steps; for
    FP16 the alternating four-cell and two-cell sweeps): 12 steps against the
    oracle, whole fields.  Reduced-storage tolerances as in the small free
    swimmer test; the body velocity is compared relative to its own size."""
    wl = W.c3_pusher()
    b = wl.bodies[0]
    g = Lattice(wl.shape, collision="trt", storage=storage)
    o = OracleSim(*wl.shape, lambda_e=1.0, collision="trt")
    # off-node start, tilted axis and a larger B1 so that cells change
    pos, e = (128.4, 127.7, 128.2), (0.1, -0.2, 1.0)
    gi = g.add_squirmer(pos, e, b.R, 0.05, b.beta, mobile=True)
    oi = o.add_sphere(pos, e, b.R, 0.05, b.beta, mobile=True)
    g.step(12)
    o.step(12)
    og, oo = g.owner(), o.owner()
    if storage != "f16dev":
        assert (og == oo).all()
    else:
        # the FP16 body drifts from the oracle's by about 1e-4 in 12 steps:
        # owners must agree wherever a node is farther than the drift from
        # the sphere surface at both positions (at the last classification)
        pg, po = g.state(gi)[0], o.state(oi)[0]
        drift = np.abs(pg - po).max() + np.abs(g.state(gi)[1]).max()
        nx, ny, nz = wl.shape
        lo = np.floor(pg - b.R - 2).astype(int)
        ax = [np.arange(lo[a], lo[a] + int(2 * b.R) + 6) for a in range(3)]
        zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(float)
        idx = (xx % nx) + nx * ((yy % ny) + ny * (zz % nz))
        near_box = np.zeros(pts.shape[0], bool)
        for c in (pg, po):
            d = pts - c
            d -= np.array(wl.shape) * np.round(d / np.array(wl.shape))
            near_box |= np.abs(np.linalg.norm(d, axis=1) - b.R) < 2 * drift + 1e-9
        near = np.zeros(og.size, bool)
        near[idx.ravel()[near_box]] = True
        assert near.sum() < 0.2 * (og != 0).sum()
        assert (og[~near] == oo[~near]).all()
    _, ug = g.fields()
    _, uo = o.fields()
    both = (og == 0) & (oo == 0)
    assert rel(ug[:, both], uo[:, both]) < tol
    vg, vo = g.state(gi)[1], o.state(oi)[1]
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
