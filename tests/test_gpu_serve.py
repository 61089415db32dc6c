"""The request server: continuous batching of independent simulations.

* Each request's result is bitwise the same alone and in a mix with other
  requests (of other sizes, storages and geometries) that arrive while it
  runs: kernels never mix two lattices' data and every per-body reduction has
  a fixed order.
* A request stops exactly at its own step count, in the middle of a round.
* A served FP64 request matches the single-lattice path and the FP64 oracle
  within the FP64 tolerance (1e-12).
* Admission respects the HBM budget: requests wait until memory frees up.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import OracleSim  # noqa: E402
from paper_1903_04799_gb300 import Lattice, lbsq  # noqa: E402
from paper_1903_04799_gb300.lbsq import Server, make_request  # noqa: E402


def requests():
    return [
        make_request(0, (30, 26, 28), "f64", pos=(14.2, 12.7, 13.1), e=(0.3, -0.4, 1.0), R=4.5, B1=0.03,
                     beta=-2.0, steps=150),
        make_request(1, (18, 18, 40), "f32", pos=(9.1, 8.8, 20.0), e=(0.1, 0.05, 1.0), R=3.5, B1=0.02,
                     beta=2.0, wca=(1.0, 0.01), steps=121),
        make_request(2, (40, 40, 40), "f16dev", pos=(20.0, 20.0, 9.0), e=(0.05, 0.0, 1.0), R=4.0, B1=0.02,
                     beta=0.0, obstacle=(20.0, 20.0, 22.0, 4.0), wca=(1.0, 0.01), steps=170),
        make_request(0, (36, 32, 34), "bf16dev", pos=(17.5, 15.5, 16.5), e=(1.0, 0.2, 0.0), R=5.0, B1=0.02,
                     beta=4.0, steps=96),
    ]


def run_server(reqs, arrive_at_round, budget=1 << 30, max_resident=8, round_steps=16, tile_units=700):
    srv = Server(budget_bytes=budget, max_resident=max_resident, round_steps=round_steps, tile_units=tile_units)
    tickets = {}
    results = {}
    rnd = 0
    while len(results) < len(reqs):
        for i, r in enumerate(reqs):
            if i not in tickets and arrive_at_round[i] <= rnd:
                tickets[i] = srv.submit(r)
        srv.advance()
        rnd += 1
        for i, t in tickets.items():
            if i in results:
                continue
            res = srv.poll(t)
            if res.state in (lbsq.LB_REQ_DONE, lbsq.LB_REQ_FAILED):
                results[i] = res
        assert rnd < 200
    srv.close()
    return results


def as_array(res):
    return np.array(list(res.pos) + list(res.vel) + list(res.e) + list(res.omega) + list(res.F) + list(res.T)
                    + [res.mean_speed] + list(res.mean_vel))


def test_alone_equals_mix_bitwise():
    reqs = requests()
    mix = run_server(reqs, arrive_at_round=[0, 1, 1, 4])
    for i, r in enumerate(reqs):
        alone = run_server([r], arrive_at_round=[0])[0]
        assert alone.state == lbsq.LB_REQ_DONE and mix[i].state == lbsq.LB_REQ_DONE
        assert alone.steps_done == r.steps == mix[i].steps_done
        assert np.array_equal(as_array(alone), as_array(mix[i])), i


def test_served_request_matches_context_and_oracle():
    """FP64 request with an odd step count: the server stops it mid-round; its
    final state matches the single-lattice context and the FP64 oracle."""
    r = requests()[0]
    r.steps = 137
    res = run_server([r], arrive_at_round=[0])[0]
    g = Lattice((r.nx, r.ny, r.nz), collision="trt", storage="f64")
    gid = g.add_squirmer(tuple(r.pos), tuple(r.e), r.R, r.B1, r.beta, mobile=True)
    g.step(r.steps)
    o = OracleSim(r.nx, r.ny, r.nz, lambda_e=1.0, collision="trt")
    oid = o.add_sphere(tuple(r.pos), tuple(r.e), r.R, r.B1, r.beta, mobile=True)
    o.step(r.steps)
    pg, vg, eg, _ = g.state(gid)
    po, vo, eo, _ = o.state(oid)
    for a, b, c in ((res.pos, pg, po), (res.vel, vg, vo), (res.e, eg, eo)):
        a = np.array(list(a))
        assert np.abs(a - b).max() < 1e-12
        assert np.abs(a - c).max() < 1e-12


def test_admission_waits_for_memory():
    """A budget that holds one 40^3 FP16 request at a time: the others queue and
    start as memory frees up; all finish with their own results."""
    reqs = [make_request(0, (40, 40, 40), "f16dev", pos=(20.2, 19.9, 20.1), e=(0, 0, 1), R=4.0, B1=0.02,
                         beta=b, steps=40) for b in (-3.0, 0.0, 3.0)]
    srv = Server(budget_bytes=int(5.5e6), max_resident=4, round_steps=16, tile_units=1024)
    tickets = [srv.submit(r) for r in reqs]
    running, queued = srv.advance()
    assert running == 1 and queued == 2
    done = {}
    for _ in range(60):
        srv.advance()
        for t in tickets:
            if t not in done:
                res = srv.poll(t)
                if res.state == lbsq.LB_REQ_DONE:
                    done[t] = res
        if len(done) == 3:
            break
    assert len(done) == 3
    speeds = [done[t].mean_speed for t in tickets]
    assert all(s > 0 for s in speeds)
    srv.close()


def test_failed_request_reports_overlap():
    """A squirmer placed inside the obstacle fails with LB_ERR_OVERLAP and does
    not disturb the other request."""
    bad = make_request(2, (40, 40, 40), "f32", pos=(20.0, 20.0, 22.0), R=4.0, B1=0.02,
                       obstacle=(20.0, 20.0, 22.0, 4.0), steps=32)
    good = requests()[0]
    res = run_server([bad, good], arrive_at_round=[0, 0])
    assert res[0].state == lbsq.LB_REQ_FAILED and res[0].status == lbsq.LB_ERR_OVERLAP
    alone = run_server([good], arrive_at_round=[0])[0]
    assert np.array_equal(as_array(alone), as_array(res[1]))


def test_autotuned_tiles_give_the_same_bits():
    """A server that picks its tile shape by timing candidates at creation
    (tile_units = 0; the autotuner sweeps two synthetic 96^3 lattices) serves
    the mix with the same bits as fixed 700-unit tiles: every cell's update is
    independent of the tiling."""
    reqs = requests()
    fixed = run_server(reqs, [0] * len(reqs))
    tuned = run_server(reqs, [0] * len(reqs), tile_units=0)
    for i in range(len(reqs)):
        assert tuned[i].state == lbsq.LB_REQ_DONE
        assert np.array_equal(as_array(fixed[i]), as_array(tuned[i])), i
