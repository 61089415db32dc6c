"""The allocation-free entry point lb_fluid_totals_static.

Some callers cannot allocate device memory: a host framework that owns all of
it through its own pool, a latency-critical loop where cudaMalloc would
synchronise the device, a monitoring hook that must not change the footprint
of the program it watches.  lb_fluid_totals_static serves them: it sums the
fluid mass and momentum of buffers the caller owns, with its scratch in a
fixed file-scope device array.  This test calls it through the C ABI and
checks it against the library's own allocating sum, lb_get_mass, and against
an exactly rounded host sum (math.fsum) of the same populations, on two calls
in a row: the shared array keeps the previous call's partials, and the
second call (a smaller lattice) must not see them.  A call after the first
one on a device must leave the device's free memory and torch's allocation
count unchanged.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_04799_gb300 import Lattice, lbsq  # noqa: E402
from paper_1903_04799_gb300 import workloads as W  # noqa: E402

WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _case(shape, seed):
    g = Lattice(shape, collision="trt", storage="f64")
    c = [s / 2 for s in shape]
    g.add_squirmer((c[0] + 0.3, c[1] - 0.2, c[2] + 0.1), (0.2, 0.1, 1.0), 4.2, 0.01, -2.0, mobile=True)
    f = W.random_populations(g.N, seed=seed, base=WEIGHTS, spread=0.1)
    g.set_populations(f)
    g.step(3)
    mass, mom = g.mass()  # the library's own (allocating) reduction
    f_host, own_host = g.populations(), g.owner()
    f_dev = torch.tensor(f_host, dtype=torch.float64, device="cuda").contiguous()
    own_dev = torch.tensor(own_host, dtype=torch.int32, device="cuda").contiguous()
    g.close()
    # exactly rounded sums over the fluid cells, on the host
    ff = f_host[:, own_host == 0]
    c = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                  [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                  [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], dtype=np.float64)
    exact = np.array([math.fsum(ff.ravel())] + [math.fsum((c[a][:, None] * ff).ravel()) for a in range(3)])
    return f_dev, own_dev, mass, mom, exact


def test_static_totals_match_allocating_sum_twice():
    results = []
    for k, (shape, seed) in enumerate((((45, 19, 23), 1), ((20, 17, 22), 2))):
        f_dev, own_dev, mass, mom, exact = _case(shape, seed)
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        lbsq.lb_fluid_totals_static(f_dev.data_ptr(), own_dev.data_ptr(), own_dev.numel(), out.data_ptr(),
                                    stream.cuda_stream)
        torch.cuda.synchronize()
        if k > 0:  # the first call on the device may load the module; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == used0
        got = out.cpu().numpy()
        # FP64 sums in different orders: within 1e-12 of the mass (the gross scale)
        assert abs(got[0] - mass) < 1e-12 * mass
        assert np.abs(got[1:] - mom).max() < 1e-12 * mass
        # and against the exactly rounded host sums: N additions of FP64 terms
        assert np.abs(got - exact).max() < 1e-13 * exact[0]
        results.append(got)
    assert not np.allclose(results[0], results[1])


def test_static_totals_reject_bad_sizes():
    with pytest.raises(lbsq.LBError) as ei:
        lbsq.lb_fluid_totals_static(1, 0, 0, 1, 0)
    assert ei.value.status == lbsq.LB_ERR_INVALID
    with pytest.raises(lbsq.LBError) as ei:
        lbsq.lb_fluid_totals_static(1, 0, (1 << 27) + 1, 1, 0)
    assert ei.value.status == lbsq.LB_ERR_INVALID
