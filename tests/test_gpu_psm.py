"""Partially saturated cells (Noble and Torczynski), the coupling Sec. IV A
names as a remedy for the fluctuating swim speed of the link-coupled
squirmer, on the GPU against the FP64 oracle (OracleSim.set_psm).

FP64 storage: solid fractions identical (exact multiples of 1/512 on both
sides), fields, states and forces within 1e-12 -- the blended collision is
FP64 arithmetic on both sides and ordinary cells differ only by the
double-float collision's rounding.  Reduced storages: bounded by their own
rounding, with the tolerances of the link-coupled parity tests."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice, lbsq  # noqa: E402


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# two mobile squirmers, off-node centres and tilted axes; the first reaches
# into the plane wall at z = 0, so some covered cells are wall cells
SHAPE = (48, 44, 40)
SPHERES = [((14.3, 20.6, 5.3), (0.3, -0.2, 1.0), 5.0, 0.01, -3.0),
           ((33.7, 22.1, 24.4), (-0.5, 0.4, -0.6), 6.0, 0.008, 2.0)]


def _setup(storage="f64", wall=True, spheres=SPHERES, shape=SHAPE):
    g = Lattice(shape, collision="trt", storage=storage)
    g.set_coupling("psm")
    o = OracleSim(*shape, lambda_e=1.0, collision="trt")
    o.set_psm(True)
    if wall:
        g.add_plane_wall(2, 0)
        o.add_plane_wall(2, 0)
    gi, oi = [], []
    for pos, e, R, B1, beta in spheres:
        gi.append(g.add_squirmer(pos, e, R, B1, beta, mobile=True))
        oi.append(o.add_sphere(pos, e, R, B1, beta, mobile=True))
    return g, o, gi, oi


def test_psm_fp64_matches_oracle():
    """96 steps in chunks of 1, 7, 8, 16 and 64 (single steps and the 8-step
    graphs): after each chunk the solid fractions and the owners identical,
    the fields within 1e-12 of max|u|, each squirmer's state within 1e-12,
    its force and torque within 1e-12 of the size of their cell terms.  At
    the start nine covered cells are wall cells; they stay wall cells."""
    g, o, gi, oi = _setup()
    for n in (1, 7, 8, 16, 64):
        g.step(n)
        o.step(n)
        eg, eo = g.solid_fraction(), o.eps()
        assert (eg == eo).all()
        own = o.owner()
        assert (g.owner() == own).all()
        if n == 1:  # covered wall cells (the first squirmer then swims off the wall)
            assert ((eo > 0) & (own != 0)).sum() == 9
        assert eo.max() == 1.0 and ((eo > 0) & (eo < 1)).any()
        rg, ug = g.fields()
        ro, uo = o.fields()
        assert _rel(ug, uo) < 1e-12
        assert np.abs(rg - ro).max() < 1e-12
        for a, b, sp in zip(gi, oi, SPHERES):
            for x, y in zip(g.state(a), o.state(b)):
                assert np.abs(x - y).max() < 1e-12, (x, y)
            Fg, Tg = g.force_torque(a)
            Fo, To = o.force_torque(b)
            # force and torque are residuals of cell terms whose sum of sizes
            # is about rho0 |u_s| times the surface, 4 pi R^2 B1 (torque: R
            # times that): their rounding scales with that sum, not with the
            # residual
            R, B1 = sp[2], sp[3]
            sF = 4 * math.pi * R ** 2 * B1
            assert np.abs(Fg - Fo).max() < 1e-12 * sF
            assert np.abs(Tg - To).max() < 1e-12 * R * sF
    # the populations of the fluid cells (a wall cell's are never read)
    fl = o.owner() == 0
    assert np.abs(g.populations()[:, fl] - o.populations()[:, fl]).max() < 1e-13
    g.close()


def test_psm_sphere_across_the_periodic_faces():
    """A squirmer straddling the periodic faces in x and y: its box, its
    solid fractions and its force sums wrap.  FP64 against the oracle, 24
    steps in chunks of 1, 7 and 16: solid fractions identical, fields and
    state within 1e-12, force and torque within 1e-12 of their cell terms."""
    shape = (40, 36, 32)
    pos, e, R, B1, beta = (0.8, 35.4, 16.3), (0.5, -0.3, 1.0), 5.0, 0.01, -2.0
    g = Lattice(shape, collision="trt")
    g.set_coupling("psm")
    o = OracleSim(*shape, lambda_e=1.0, collision="trt")
    o.set_psm(True)
    gi = g.add_squirmer(pos, e, R, B1, beta, mobile=True)
    oi = o.add_sphere(pos, e, R, B1, beta, mobile=True)
    sF = 4 * math.pi * R ** 2 * B1
    for n in (1, 7, 16):
        g.step(n)
        o.step(n)
        eo = o.eps()
        assert (g.solid_fraction() == eo).all()
        e3 = eo.reshape(shape[2], shape[1], shape[0])  # x fastest
        assert e3[:, :, 0].max() > 0 and e3[:, :, -1].max() > 0  # covered on both sides of x = 0
        _, ug = g.fields()
        _, uo = o.fields()
        assert _rel(ug, uo) < 1e-12
        for x, y in zip(g.state(gi), o.state(oi)):
            assert np.abs(x - y).max() < 1e-12, (x, y)
        Fg, Tg = g.force_torque(gi)
        Fo, To = o.force_torque(oi)
        assert np.abs(Fg - Fo).max() < 1e-12 * sF
        assert np.abs(Tg - To).max() < 1e-12 * R * sF
    g.close()


@pytest.mark.parametrize("storage,tol", [("f32", 2e-5), ("f16dev", 5e-3), ("bf16dev", 3e-2)])
def test_psm_reduced_storage_against_oracle(storage, tol):
    """The same configuration, 64 steps, reduced storages: the velocity field
    within tol of max|u| and each squirmer's velocity within tol of its
    speed.  The solid fractions depend on the positions alone: they agree but
    where a sample point lies within the position error of the surface (under
    1 % of the covered cells, by at most 8/512)."""
    g, o, gi, oi = _setup(storage)
    g.step(64)
    o.step(64)
    _, ug = g.fields()
    _, uo = o.fields()
    assert _rel(ug, uo) < tol
    for a, b in zip(gi, oi):
        vg, vo = g.state(a)[1], o.state(b)[1]
        assert np.abs(vg - vo).max() < tol * np.linalg.norm(vo), (vg, vo)
    eg, eo = g.solid_fraction(), o.eps()
    assert np.abs(eg - eo).max() <= 8 / 512
    assert (eg != eo).sum() < 0.01 * (eo > 0).sum()
    g.close()


@pytest.mark.parametrize("option", ["incompressible", "force_average", "bgk_1.3"])
def test_psm_options_against_oracle(option):
    """The coupling under the method's options, FP64 against the oracle's
    same switches, 48 steps of the two-squirmer set-up: the incompressible
    equilibrium (in both operators of the blend), Ladd's two-step force
    average, and BGK at lambda_e = 1.3 (B depends on tau = 1 / lambda_e).
    Fields within 1e-12 of max|u|, states within 1e-12."""
    le = 1.3 if option == "bgk_1.3" else 1.0
    coll = "bgk" if option == "bgk_1.3" else "trt"
    eq = "incompressible" if option == "incompressible" else "compressible"
    g = Lattice(SHAPE, collision=coll, lambda_e=le, equilibrium=eq)
    g.set_coupling("psm")
    o = OracleSim(*SHAPE, lambda_e=le, collision=coll)
    o.set_psm(True)
    if option == "incompressible":
        o.set_incompressible(True)
    if option == "force_average":
        g.set_force_average(True)
        o.set_force_average(True)
    gi = [g.add_squirmer(pos, e, R, B1, beta, mobile=True) for pos, e, R, B1, beta in SPHERES]
    oi = [o.add_sphere(pos, e, R, B1, beta, mobile=True) for pos, e, R, B1, beta in SPHERES]
    for n in (8, 40):
        g.step(n)
        o.step(n)
        _, ug = g.fields()
        _, uo = o.fields()
        assert _rel(ug, uo) < 1e-12
        for a, b in zip(gi, oi):
            for x, y in zip(g.state(a), o.state(b)):
                assert np.abs(x - y).max() < 1e-12, (x, y)
    assert (g.solid_fraction() == o.eps()).all()
    g.close()


def test_psm_momentum_balance_at_96_cubed():
    """A free pusher (R = 8) in a 96^3 periodic box, 200 FP64 steps: every
    cell stays fluid, and fluid momentum plus M v stays zero to roundoff --
    the sphere takes exactly the momentum the solid operator gives the fluid
    (a property of the method at any size, checked beyond the oracle's
    sizes)."""
    R, L = 8.0, 96
    g = Lattice((L, L, L), collision="trt")
    g.set_coupling("psm")
    oid = g.add_squirmer((L / 2 + 0.3, L / 2 - 0.2, L / 2 + 0.1), (0.2, 0.1, 1.0), R, 0.01, -1.0)
    M = 4 / 3 * math.pi * R ** 3
    for _ in range(10):
        g.step(20)
        _, P = g.mass()
        v = g.state(oid)[1]
        assert np.abs(P + M * v).max() < 1e-11, (P, M * v)
    assert (g.owner() == 0).all()
    eps = g.solid_fraction()
    assert abs(eps.sum() / M - 1) < 2e-3
    assert np.linalg.norm(v) > 0.3 * (2 * 0.01 / 3)  # it swims
    g.close()


def test_psm_overlap_sets_the_error():
    """Two spheres whose cells meet: the first step reports LB_ERR_OVERLAP
    (an error status; the context then refuses further steps)."""
    g = Lattice((40, 40, 40), collision="trt")
    g.set_coupling("psm")
    g.add_squirmer((15.0, 20.0, 20.0), (0, 0, 1), 5.0, 0.0, 0.0)
    g.add_squirmer((24.9, 20.0, 20.0), (0, 0, 1), 5.0, 0.0, 0.0)  # overlap by 0.1: cells shared
    g.step(1)
    with pytest.raises(lbsq.LBError) as ex:
        g.sync()
    assert ex.value.status == lbsq.LB_ERR_OVERLAP
    with pytest.raises(lbsq.LBError):
        g.step(1)
    g.close()


def test_psm_coupling_rules_and_tracing():
    """The coupling is set before the first sphere; an obstacle (lb_add_wall
    kind 2) is a sphere too.  The traced step launches the solid-fraction and
    force kernels under kind 1 and the sweep under kind 0, with the same
    result as the graph path."""
    g = Lattice((32, 32, 32), collision="trt")
    g.add_squirmer((16, 16, 16), (0, 0, 1), 4.0, 0.01, 0.0)
    with pytest.raises(lbsq.LBError) as ex:
        g.set_coupling("psm")
    assert ex.value.status == lbsq.LB_ERR_INVALID
    g.close()
    runs = []
    for traced in (False, True):
        g = Lattice((32, 32, 32), collision="trt")
        g.set_coupling("psm")
        g.add_obstacle((8.2, 8.4, 8.1), 3.0)
        gi = g.add_squirmer((20.3, 19.7, 16.2), (0.1, 0, 1), 4.0, 0.01, -1.0)
        if traced:
            g.profile_begin()
            g.step(16)
            prof = g.profile_end()
            kinds = list(prof)
            assert prof[kinds[0]][1] == 16 and prof[kinds[1]][1] >= 16, prof
        else:
            g.step(16)
        runs.append((g.populations(), g.state(gi)))
        g.close()
    assert (runs[0][0] == runs[1][0]).all()
    for a, b in zip(runs[0][1], runs[1][1]):
        assert (a == b).all()
