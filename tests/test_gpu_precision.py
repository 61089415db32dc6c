"""Reduced-precision storage against the FP64 oracle: the swim speed of
Eq. "squirmer-speed" within 1e-3 relative, and the stochastic rounding of BF16
stores.

The workloads are the free-swimmer and pusher configurations at R = 8 in a
64^3 periodic box (L = 8R), long enough for the flow near the sphere to settle
(R^2 / nu = 384 steps): the swim speed is the mean of v.e over steps 600 ..
1200.  The oracle runs the same configuration in FP64 on the host.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice  # noqa: E402

WGT = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
STEPS, FROM = 1200, 600


def _speed_series(sim, oid, steps):
    v = []
    for _ in range(steps):
        sim.step(1)
        _, vel, e, _ = sim.state(oid)
        v.append(vel @ e)
    return np.array(v)


@pytest.mark.parametrize("B1,beta", [(0.005, 0.0), (0.002, -3.0)])
def test_swim_speed_of_every_storage_within_1e_3_of_the_oracle(B1, beta):
    """Free swimmer (B1 = 0.005, beta = 0, as the 128^3 configuration) and
    pusher (B1 = 0.002, beta = -3, as the 256^3 one) at R = 8, L = 64: the
    mean swim speed of FP32, FP16- and BF16-deviation storage within 1e-3
    relative of the FP64 oracle's, and FP64 storage within 1e-11."""
    L, R = 64, 8.0
    pos, e = (L / 2 + 0.1, L / 2 + 0.2, L / 2), (0.0, 0.0, 1.0)
    o = OracleSim(L, L, L, lambda_e=1.0, collision="trt")
    oi = o.add_sphere(pos, e, R, B1, beta, mobile=True)
    Uo = _speed_series(o, oi, STEPS)[FROM:].mean()
    assert 0.9 < Uo / (2 * B1 / 3) < 1.05
    tol = {"f64": 1e-11, "f32": 1e-3, "f16dev": 1e-3, "bf16dev": 1e-3}
    for st, t in tol.items():
        g = Lattice((L, L, L), collision="trt", storage=st)
        gi = g.add_squirmer(pos, e, R, B1, beta, mobile=True)
        U = _speed_series(g, gi, STEPS)[FROM:].mean()
        g.close()
        assert abs(U - Uo) / abs(Uo) < t, (st, U, Uo)


def _bf16_round(x):
    """Round-to-nearest-even of FP32 values to BF16 (the top 16 bits)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("rounding", ["stochastic", "nearest"])
def test_bf16_rounding_of_a_uniform_state(rounding):
    """Every cell starts from the same populations, BF16 numbers off
    equilibrium, so every cell's collision gives the same FP32 values x_i.
    An FP32-storage lattice, which collides with the same FP32 arithmetic,
    stores x_i itself.  Round to nearest stores one BF16 number per
    population everywhere, the nearest to x_i.  Stochastic rounding stores
    the two BF16 numbers around x_i, the upper one in a fraction of the cells
    equal to where x_i lies between them (within five standard errors), so
    the mean stored value is x_i."""
    shape = (64, 32, 32)
    N = int(np.prod(shape))
    g_in = _bf16_round(WGT * 1.2345e-3 * (1.0 + 0.3 * np.sin(np.arange(19.0))))
    f = np.repeat((WGT + g_in)[:, None], N, axis=1)
    ref = Lattice(shape, collision="trt", storage="f32")
    ref.set_populations(f)
    ref.step(1)
    x = ref.populations()[:, 0] - WGT  # x_i, FP32 values
    ref.close()
    g = Lattice(shape, collision="trt", storage="bf16dev", rounding=rounding)
    g.set_populations(f)
    g.step(1)
    out = g.populations() - WGT[:, None]
    g.close()
    two = 0
    for i in range(19):
        vals = np.unique(out[i])
        if rounding == "nearest":
            assert vals.size == 1 and vals[0] == _bf16_round(x[i]), (i, vals, x[i])
            continue
        if vals.size == 1:  # x_i is a BF16 number
            assert vals[0] == x[i], (i, vals, x[i])
            continue
        assert vals.size == 2, (i, vals)
        two += 1
        lo, hi = vals
        assert lo < x[i] < hi
        p = (x[i] - lo) / (hi - lo)
        frac = np.mean(out[i] == hi)
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / N) + 1e-3, (i, frac, p)
    if rounding == "stochastic":
        assert two >= 10
