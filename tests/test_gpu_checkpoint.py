"""Checkpoint and resume through the C ABI: a context restored from a
checkpoint, stepped on, gives the same bits as the context that wrote it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_04799_gb300 import Lattice  # noqa: E402
from paper_1903_04799_gb300.lbsq import LBError  # noqa: E402


def _free_swimmer(storage):
    g = Lattice((28, 26, 30), collision="trt", storage=storage)
    ids = [g.add_squirmer((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0, mobile=True)]
    return g, ids


def _split_swimmer(storage):
    # one sphere in a large box: split steps, a pending body step, four window
    # slots; the window wraps in y and z
    g = Lattice((128, 96, 96), collision="trt", storage=storage)
    ids = [g.add_squirmer((64.3, 2.7, 94.1), (0.3, 0.5, 1.0), 6.0, 0.05, -3.0, mobile=True)]
    return g, ids


def _two_swimmers_and_wall(storage):
    # spheres that come near each other take the multi-kernel body path; the
    # wall is a still body whose bounce-back is a plain copy
    g = Lattice((48, 44, 40), collision="trt", storage=storage)
    ids = [g.add_squirmer((20.2, 21.7, 18.3), (1.0, 0.2, 0.1), 4.0, 0.02, 2.0, mobile=True),
           g.add_squirmer((31.6, 22.4, 19.1), (-1.0, 0.1, 0.0), 4.0, 0.02, -2.0, mobile=True)]
    g.add_plane_wall(2, 2)
    return g, ids


def _psm_swimmers(storage):
    # partially saturated cells: solid fractions found afresh each step, from
    # positions the restore replaces (the restore clears the recorded ones)
    g = Lattice((44, 40, 40), collision="trt", storage=storage)
    g.set_coupling("psm")
    g.add_plane_wall(2, 0)
    ids = [g.add_squirmer((14.3, 20.6, 6.3), (0.3, -0.2, 1.0), 5.0, 0.02, -3.0, mobile=True),
           g.add_squirmer((30.7, 21.1, 24.4), (-0.5, 0.4, -0.6), 5.5, 0.015, 2.0, mobile=True)]
    return g, ids


def _snapshot(g, ids):
    out = [g.populations(), g.owner(), np.int64(g.steps)]
    for i in ids:
        out += list(g.state(i)) + list(g.force_torque(i)) + [g.stresslet(i), g.links(i)]
    return out


@pytest.mark.parametrize("setup,storage,before,after", [
    (_free_swimmer, "f64", 37, 29),
    (_free_swimmer, "bf16dev", 40, 24),
    (_split_swimmer, "f32", 21, 19),
    (_split_swimmer, "f16dev", 13, 16),
    (_two_swimmers_and_wall, "f16dev", 30, 25),
    (_two_swimmers_and_wall, "f64", 26, 21),
    (_psm_swimmers, "f64", 19, 22),
    (_psm_swimmers, "bf16dev", 24, 17),
])
def test_resume_is_bitwise(setup, storage, before, after):
    """Run `before` steps, checkpoint, run `after` more; a second context set
    up the same way, restored from the checkpoint and run `after` steps, ends
    with the same populations, owners, step count, body states, forces,
    stresslets, link lists and solid fractions, bit for bit.  Step counts cover eager steps,
    graph replays and a checkpoint taken with body kernels pending."""
    a, ids = setup(storage)
    a.step(before)
    blob = a.checkpoint()
    a.step(after)
    want = _snapshot(a, ids)
    want_eps = a.solid_fraction()
    a.close()
    b, ids_b = setup(storage)
    b.step(3)  # anything done before the restore is replaced
    b.restore(blob)
    b.step(after)
    got = _snapshot(b, ids_b) + [b.solid_fraction()]
    want = want + [want_eps]
    b.close()
    assert len(got) == len(want)
    for k, (x, y) in enumerate(zip(got, want)):
        assert np.array_equal(np.asarray(x), np.asarray(y)), k


def test_restore_rejects_other_setups():
    """A checkpoint restores only into the same lattice with the same bodies;
    anything else is refused with LB_ERR_INVALID and the context is left as
    it was."""
    a, _ = _free_swimmer("f32")
    a.step(5)
    blob = a.checkpoint()
    a.close()
    other_shape = Lattice((28, 26, 32), collision="trt", storage="f32")
    other_shape.add_squirmer((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0, mobile=True)
    other_storage, _ = _free_swimmer("f64")
    other_model = Lattice((28, 26, 30), collision="trt", storage="f32", equilibrium="incompressible")
    other_model.add_squirmer((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.5, 0.03, -2.0, mobile=True)
    other_body = Lattice((28, 26, 30), collision="trt", storage="f32")
    other_body.add_squirmer((13.3, 12.7, 14.1), (0.3, -0.4, 1.0), 4.0, 0.03, -2.0, mobile=True)
    same, ids = _free_swimmer("f32")
    same.step(2)
    before = _snapshot(same, ids)
    for g, b in ((other_shape, blob), (other_storage, blob), (other_model, blob), (other_body, blob),
                 (same, blob[:-8]),
                 (same, b"not a checkpoint" * 8)):
        with pytest.raises(LBError) as err:
            g.restore(b)
        assert err.value.status == 1  # LB_ERR_INVALID
    after = _snapshot(same, ids)
    for x, y in zip(after, before):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    for g in (other_shape, other_storage, other_model, other_body, same):
        g.close()
