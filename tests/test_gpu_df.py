"""The FP64-storage collision in double-float arithmetic (pairs of FP32
numbers) against the same collision in FP64 arithmetic (sweep form 1), on the
GPU.  Both collide the stored deviations g = f - w rho0; the double-float form
carries about 47 significant bits, so one step differs from the FP64 form by
about 2^-46 of the cell's largest deviation.  The FP64 parity tests against
the oracle (test_gpu_parity.py) run the double-float form, the default."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_04799_gb300 import Lattice  # noqa: E402
from paper_1903_04799_gb300 import workloads as W  # noqa: E402

WGT = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
VEL = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
       (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def _run(f, shape, variant, steps, collision="trt", lambda_e=1.0, body=False, equilibrium=None):
    kw = {} if equilibrium is None else {"equilibrium": equilibrium}
    g = Lattice(shape, collision=collision, lambda_e=lambda_e, storage="f64", **kw)
    g.set_sweep_variant(variant)
    g.set_populations(f)
    gi = None
    if body:
        gi = g.add_squirmer((shape[0] / 2 + 0.3, 6.2, 6.9), (1.0, 0.2, 0.1), 3.0, 0.02, -1.0, mobile=True)
    g.step(steps)
    out = g.populations(), (g.state(gi) if body else None)
    g.close()
    return out


@pytest.mark.parametrize("collision,lambda_e", [("trt", 1.0), ("trt", 1.3), ("bgk", 1.0), ("bgk", 1.7)])
@pytest.mark.parametrize("spread", [0.01, 0.5])
@pytest.mark.parametrize("steps", [1, 2, 9])
def test_double_float_matches_fp64_arithmetic(collision, lambda_e, spread, steps):
    """Random populations w (1 + spread U[-1, 1]) on a ragged periodic lattice:
    after 1, 2 and 9 steps (both parities) every population of the
    double-float sweep is within 2^-44 * steps of the largest deviation of
    the FP64 sweep's."""
    shape = (37, 13, 11)
    f = W.random_populations(int(np.prod(shape)), seed=5, base=WGT, spread=spread)
    a, _ = _run(f, shape, 0, steps, collision, lambda_e)
    b, _ = _run(f, shape, 1, steps, collision, lambda_e)
    scale = np.abs(b - WGT[:, None]).max()
    assert np.abs(a - b).max() <= 2.0 ** -44 * steps * scale


def test_double_float_incompressible_and_body():
    """The incompressible equilibrium and a moving squirmer (links, conversion
    and refill on FP64 deviations in both runs): 40 steps, populations and the
    body state within 1e-12 of the FP64 sweep's."""
    shape = (40, 13, 14)
    f = W.random_populations(int(np.prod(shape)), seed=8, base=WGT, spread=0.02)
    for eq in ("compressible", "incompressible"):
        a, sa = _run(f, shape, 0, 40, body=True, equilibrium=eq)
        b, sb = _run(f, shape, 1, 40, body=True, equilibrium=eq)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b - WGT[:, None]).max()
        for x, y in zip(sa, sb):
            assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)


def _source_cells(shape):
    """src[i, n]: the cell whose post-collision population i cell n holds after
    one step (the neighbour n - c_i, periodic)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    src = np.empty((19, x.size), np.int64)
    for i, (cx, cy, cz) in enumerate(VEL):
        src[i] = ((x - cx) % nx) + nx * (((y - cy) % ny) + ny * ((z - cz) % nz))
    return src


def test_double_float_wide_range_and_special_values():
    """Deviations of magnitudes 1e-30 .. 1e-1 with random signs, cells at rest
    (zero deviation) and one cell of NaN populations, one step.  Every
    population that a cell with a finite state sends out is within 2^-45 of
    that cell's largest input deviation (plus 1e-30, plus an ulp of w_i rho0)
    of the FP64 sweep's; what
    a cell at rest sends out stays at rest to 1e-30; what the NaN cell sends
    out is NaN, and nothing else is."""
    shape = (32, 9, 10)
    N = int(np.prod(shape))
    rng = np.random.default_rng(3)
    g = np.sign(rng.uniform(-1, 1, (19, N))) * 10.0 ** rng.uniform(-30, -1, (19, N))
    rest = rng.choice(N, 40, replace=False)
    g[:, rest] = 0.0
    f = WGT[:, None] + g
    nan_cell = 77
    f[:, nan_cell] = np.nan
    a, _ = _run(f, shape, 0, 1)
    b, _ = _run(f, shape, 1, 1)
    src = _source_cells(shape)
    from_nan = src == nan_cell
    assert np.isnan(a[from_nan]).all()
    assert np.isfinite(a[~from_nan]).all()
    scale = np.abs(g).max(axis=0)[src]
    err = np.abs(a - b)
    ok = ~from_nan
    # plus one ulp of w_i rho0: the populations are read back as w_i rho0 + g
    tol = 2.0 ** -45 * scale + 1e-30 + np.spacing(WGT)[:, None]
    assert (err[ok] <= tol[ok]).all(), (err[ok] / tol[ok]).max()
    from_rest = np.isin(src, rest)
    assert np.abs(a - WGT[:, None])[from_rest].max() <= 1e-30
