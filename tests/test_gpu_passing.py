"""Two squirmers passing each other (Sec. "Interaction between Two Squirmers",
Fig. "ishikawa"): two pullers (beta = 5, R = 9) in a 250^3 periodic box, 12R
apart along their axes and offset laterally, through the C ABI.

The comparison data of the figure (boundary-element trajectories) are not in
the paper's text.  What is checked instead:
  * parity with the FP64 oracle at full size for the first steps;
  * the half-turn symmetry of the set-up: the rotation by pi about the x axis
    through the box centre maps the lattice, the velocity set and each sphere
    onto the other, so the run must stay symmetric up to rounding.
"""
import numpy as np
import pytest

from paper_1903_04799_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def half_turn_cells(n):
    """Cell index map of the half turn about the x axis through (n/2, n/2):
    (x, y, z) -> (x, -y mod n, -z mod n), cells x-fastest."""
    i = np.arange(n)
    m = (-i) % n
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return (x + n * (m[y] + n * m[z])).ravel()


def test_passing_full_size_parity_f64():
    """The 250^3 pair at full size against the oracle: 6 steps with B1 raised
    so that cells change; owners bit-exact, u and both bodies' states within
    1e-12."""
    wl = W.two_squirmers_passing()
    g = Lattice(wl.shape, collision="trt", storage="f64")
    o = OracleSim(*wl.shape, lambda_e=1.0, collision="trt")
    ids = []
    for b in wl.bodies:
        ids.append((g.add_squirmer(b.pos, b.e, b.R, 0.05, b.beta, mobile=True),
                    o.add_sphere(b.pos, b.e, b.R, 0.05, b.beta, mobile=True)))
    g.step(6)
    o.step(6)
    assert (g.owner() == o.owner()).all()
    _, ug = g.fields()
    _, uo = o.fields()
    assert rel(ug, uo) < 1e-12
    for gi, oi in ids:
        for a, b in zip(g.state(gi), o.state(oi)):
            assert np.abs(a - b).max() < 1e-12


@pytest.mark.parametrize("storage,steps,tol", [("f64", 300, 1e-10), ("f32", 300, 1e-3)])
def test_passing_half_turn_symmetry(storage, steps, tol):
    """Under the half turn R: (x, y, z) -> (x, -y, -z) about the box centre the
    second sphere is the image of the first.  After `steps` steps the state of
    sphere 2 equals R applied to the state of sphere 1, the owner field maps
    onto itself with the two ids exchanged, and u(R x) = R u(x).  The two
    sides round in different orders (each sphere sums its own links, each cell
    its own populations), so the match is to rounding, grown over the run:
    1e-10 of the largest value in FP64, 1e-3 in FP32 (FP32 rounding of
    populations near 1 leaves about 1e-7 in u, against |u| of order 1e-2)."""
    wl = W.two_squirmers_passing()
    n = wl.shape[0]
    g = Lattice(wl.shape, collision="trt", storage=storage)
    a, b = (g.add_squirmer(s.pos, s.e, s.R, s.B1, s.beta, mobile=True) for s in wl.bodies)
    g.step(steps)
    flip = np.array([1.0, -1.0, -1.0])
    pa, va, ea, wa = g.state(a)
    pb, vb, eb, wb = g.state(b)
    centre = np.array([0.0, n / 2, n / 2])
    image = centre + flip * (pa - centre)
    image = np.where(flip < 0, (image + n) % n, image)
    assert np.abs(pb - image).max() < tol * n
    vmax = max(np.abs(va).max(), np.abs(vb).max())
    assert np.abs(vb - flip * va).max() < tol * vmax
    assert np.abs(eb - flip * ea).max() < tol
    assert np.abs(wb - flip * wa).max() < tol * max(np.abs(wa).max(), 1e-30) + 1e-14
    # the spheres moved: the check is not of a state at rest
    assert np.linalg.norm(pa - np.array(wl.bodies[0].pos)) > 0.1
    perm = half_turn_cells(n)
    own = g.owner()
    swap = own.copy()
    swap[own == a], swap[own == b] = b, a
    assert np.array_equal(own[perm], swap)
    _, u = g.fields()
    assert rel(u[:, perm], flip[:, None] * u) < tol
