"""Sec. V tube flow: a neutral squirmer (R = 9) in a round tube of diameter
D = 20R/3 and length 3 pi R, periodic along the axis (workloads.tube_oscillation).

The boundary-element trajectories the paper compares with are not in its
text, so the run is checked by parity with the FP64 oracle over its first
steps, at full size, and by the mirror symmetry of a start on the axis."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice  # noqa: E402
from paper_1903_04799_gb300 import workloads as W  # noqa: E402


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _gpu(t, storage="f64"):
    b = t.body
    g = Lattice(t.shape, collision="trt", storage=storage)
    tube = g.add_round_tube(t.axis[0], t.axis[1], t.radius)
    gi = g.add_squirmer(b.pos, b.e, b.R, b.B1, b.beta, mobile=True)
    g.set_contact(*t.contact)
    return g, gi, tube


def test_tube_run_first_steps_match_oracle():
    """The paper's configuration at full size (64 x 64 x 85), started at
    y0 = -R: 120 steps in FP64 against the oracle.  Owners bit-exact; fields
    and the squirmer's state within 1e-12."""
    t = W.tube_oscillation(y0_over_R=-1.0)
    b = t.body
    g, gi, _ = _gpu(t)
    o = OracleSim(*t.shape, lambda_e=1.0, collision="trt")
    o.add_tube(t.axis[0], t.axis[1], t.radius)
    oi = o.add_sphere(b.pos, b.e, b.R, b.B1, b.beta, mobile=True)
    o.set_contact(*t.contact)
    for _ in range(3):
        g.step(40)
        o.step(40)
        assert (g.owner() == o.owner()).all()
        _, ug = g.fields()
        _, uo = o.fields()
        assert _rel(ug, uo) < 1e-12
        for a, c in zip(g.state(gi), o.state(oi)):
            assert np.abs(a - c).max() < 1e-12
    g.close()


def test_tube_centred_start_stays_on_the_axis():
    """A squirmer started on the axis, parallel to it: the lattice, the tube
    and the sphere are mirror-symmetric about the planes x = c and y = c
    (c = 31.5, between two nodes), so it must swim along the axis without
    drifting or turning, and its flow must keep the symmetry: after 3000
    FP64 steps the centre stays within 1e-10 of the axis, e within 1e-12 of
    +z, and u_x, u_y odd under the mirror to 1e-12 of max|u|."""
    t = W.tube_oscillation(y0_over_R=0.0)
    g, gi, _ = _gpu(t)
    g.step(3000)
    p, v, e, w = g.state(gi)
    c = np.array(t.axis)
    assert np.abs(p[:2] - c).max() < 1e-10, p
    assert np.abs(e - np.array([0.0, 0.0, 1.0])).max() < 1e-12, e
    assert v[2] > 0.5 * (2 * t.body.B1 / 3)  # it does swim
    _, u = g.fields()
    nx, ny, nz = t.shape
    ux, uy = u[0].reshape(nz, ny, nx), u[1].reshape(nz, ny, nx)
    scale = np.abs(u).max()
    assert np.abs(ux + ux[:, :, ::-1]).max() < 1e-12 * scale
    assert np.abs(uy + uy[:, ::-1, :]).max() < 1e-12 * scale
    assert np.abs(ux - ux[:, ::-1, :]).max() < 1e-12 * scale
    g.close()
