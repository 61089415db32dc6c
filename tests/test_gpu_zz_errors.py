"""Failure detection on the GPU without a GPU fault: a state the scheme cannot
carry (NaN populations, injected from the host) is caught by the body update
on the device, reported at the next synchronising call as LB_ERR_DIVERGED,
and the context then refuses to step (LB_ERR_STATE).  The diverged body is
held in place, so no kernel indexes from a runaway position."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_04799_gb300 import Lattice  # noqa: E402
from paper_1903_04799_gb300.lbsq import LB_ERR_DIVERGED, LB_ERR_STATE, LBError  # noqa: E402


@pytest.mark.parametrize("shape,pos,R", [((28, 26, 30), (13.3, 12.7, 14.1), 4.5),
                                         ((128, 96, 96), (64.3, 40.7, 50.1), 6.0)])
def test_nan_state_is_reported_as_divergence(shape, pos, R):
    """The second lattice splits its steps (near window, pending body step)."""
    g = Lattice(shape, collision="trt", storage="f64")
    gi = g.add_squirmer(pos, (0.3, -0.4, 1.0), R, 0.03, -2.0, mobile=True)
    g.step(5)
    f = g.populations()
    f[:] = np.nan
    g.set_populations(f)
    g.step(3)
    with pytest.raises(LBError) as ei:
        g.state(gi)
    assert ei.value.status == LB_ERR_DIVERGED
    with pytest.raises(LBError) as ei:
        g.step(1)
    assert ei.value.status == LB_ERR_STATE
    g.close()
