"""The bulk flow field of Sec. "Squirmers in Bulk" (Fig. "bulk") on the CUDA
path, at the paper's resolution R = 8 in a periodic box of 10R: the flow
around a free squirmer against Eq. "squirmerflow" summed over a sphere of
periodic images.

The paper reports a mean deviation of about 8 % at R = 8 once the regions at
45 degrees from e are left out.  The deviation here is
sum |u - u_an| / sum |u_an| over the fluid nodes with R + 1.5 < r < 2R outside
the cones 30-60 and 120-150 degrees from e, averaged over three snapshots 200
steps apart.  The FP64 oracle gives 4 % (beta = 0), 10 % (beta = 5) and 11 %
(beta = -5) on this set-up: in a 10R box the puller swims at 0.91 v0 and the
pusher at 1.12 v0, and the analytic field assumes v0.  The bound is 13 %.
"""
import numpy as np
import pytest

from squirmer_flow import periodic_squirmer_flow

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_04799_gb300 import Lattice  # noqa: E402


@pytest.mark.parametrize("beta", [-5.0, 0.0, 5.0])
def test_bulk_flow_field_R8(beta):
    R, L, B1 = 8.0, 80, 0.01
    g = Lattice((L, L, L), collision="trt", storage="f32")
    sid = g.add_squirmer((L / 2, L / 2, L / 2), (0.0, 0.0, 1.0), R, B1, beta, mobile=True)
    idx = np.arange(L ** 3)
    x = np.stack([idx % L, (idx // L) % L, idx // (L * L)]).astype(float)
    lo, hi = np.cos(np.radians(60)), np.cos(np.radians(30))
    g.step(2000)
    devs = []
    for _ in range(3):
        p, _, e, _ = g.state(sid)
        _, u = g.fields()
        d = x - p[:, None]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=0)
        cos = np.abs(e @ d) / np.maximum(r, 1e-12)
        m = (g.owner() == 0) & (r > R + 1.5) & (r < 2 * R) & ~((cos > lo) & (cos < hi))
        ua = periodic_squirmer_flow(d[:, m], e, R, B1, beta, L)
        devs.append(np.linalg.norm(u[:, m] - ua, axis=0).sum() / np.linalg.norm(ua, axis=0).sum())
        g.step(200)
    g.close()
    assert np.mean(devs) < 0.13, devs
