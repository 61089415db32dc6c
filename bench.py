"""Benchmark of the lattice Boltzmann squirmer hot path on GB300.

One step = one whole time step of the method on the device: fused TRT
stream-collide of every cell, shifted bounce-back on every boundary link with
the squirmer surface velocity, FP64 momentum-exchange force/torque reduction,
symplectic Euler update, and (when a lattice node crosses the surface) cell
conversion and link rebuild.

Headline: the 256^3 pusher (R = 16, beta = -3, B1 = 0.002, TRT magic 3/16)
with FP64 population storage (the deviations f - w rho0, collided in
double-float arithmetic), in MLUPS (million lattice-cell updates per second,
all cells counted).  The populations (2.55 GB) are far larger than L2; L2 is
also flushed (512 MiB write) before every timed iteration of up to 64 steps,
outside the timed events.  The same workload in FP32, FP16- and
BF16-deviation storage, the precision sweep of the four storages and the
serving mix are reported in the same line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--storage f64|f32|f16dev|bf16dev] [--skip-...]

Prints ONE JSON line (rank 0).  Under torchrun every rank advances its own
lattice (independent replicas, weak scaling); time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, mixed-prec vs FP64 (≤1e-3 U err); p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0
BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
ARITH = {"f64": "f64", "f32": "f32", "f16dev": "f32", "bf16dev": "f32"}
ARITH_NOTE = {"f64": "double-float collision (pairs of f32, ~47 significant bits) of f64-stored deviations; "
                     "bodies, forces and Newton-Euler in f64",
              "f32": "f32 collision of f32-stored deviations; bodies in f64",
              "f16dev": "f32 collision of f16-stored deviations (scale 2^14); bodies in f64",
              "bf16dev": "f32 collision of bf16-stored deviations; bodies in f64"}
KERNEL = {"f64": "k_sweep_df (one cell per thread)", "f32": "k_sweep2 (two cells per thread)",
          "f16dev": "k_sweep4r (even steps) / k_sweep2 (odd steps)",
          "bf16dev": "k_sweep4r (even steps) / k_sweep2 (odd steps)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def sweep_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("sweep.cu", "sweep_body.cuh", "sweep_df.cuh", "lbsq_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1903_04799_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(key: str):
    """DRAM bytes per launch of the sweep from a committed ncu summary, or None
    when there is none or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(key)
    if not d or d.get("source_sha") != sweep_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        load = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm

def build_lattice(storage, shape, bodies, collision="trt", lambda_e=1.0, device=0, coupling="links"):
    from paper_1903_04799_gb300 import Lattice
    g = Lattice(shape, collision=collision, lambda_e=lambda_e, storage=storage, device=device)
    if coupling != "links":
        g.set_coupling(coupling)
    ids = [g.add_squirmer(b.pos, b.e, b.R, b.B1, b.beta, mobile=b.mobile) for b in bodies]
    return g, ids


L2_BYTES = 129e6


def chunk_for(g, storage):
    """Steps per timed iteration: 64 (eight replays of the library's 8-step
    graph) when the populations are larger than L2, else 1 (L2 flushed before
    every step, so a lattice that fits in L2 is still read from HBM).  Each
    iteration starts after a flush, so its first steps run with a cold L2;
    64 steps make that start a small part of the iteration, as in a long run."""
    return 64 if g.N * 19 * BYTES[storage] > L2_BYTES else 1


def timed_steps(g, steps, flush, torch, chunk):
    """The production path: steps launched through lb_step in iterations of
    `chunk` steps, each iteration between CUDA events on the lattice's stream,
    L2 flushed before each iteration (outside the events).  Returns the
    per-step times and the number of library kernel launches in the region."""
    s = torch.cuda.ExternalStream(g._stream.cuda_stream)
    chunks = [chunk] * (steps // chunk) + ([steps % chunk] if steps % chunk else [])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    launches0 = g.launches
    with torch.cuda.stream(s):
        for k, c in enumerate(chunks):
            flush.zero_()
            ev[k][0].record(s)
            g.step(c)
            ev[k][1].record(s)
    torch.cuda.synchronize()
    step_ms = []
    for (a, b), c in zip(ev, chunks):
        step_ms += [a.elapsed_time(b) / c] * c
    return step_ms, g.launches - launches0


def traced_steps(g, steps, flush, torch):
    """Per-kernel device times: the same steps launched kernel by kernel with a
    CUDA event before and after each kernel (lb_profile_begin/end), on the
    lattice's stream, L2 flushed before each step (outside the events)."""
    s = torch.cuda.ExternalStream(g._stream.cuda_stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    g.profile_begin()
    with torch.cuda.stream(s):
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(s)
            g.step(1)
            ev[k][1].record(s)
    prof = g.profile_end()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], prof


def run_variant(storage, wl, steps, warmup, flush, torch, device=0, form=0, coupling="links"):
    g, ids = build_lattice(storage, wl.shape, wl.bodies, wl.collision, wl.lambda_e, device, coupling)
    if form:
        g.set_sweep_variant(form)
    g.step(warmup)
    g.sync()
    chunk = chunk_for(g, storage)
    step_ms, launches = timed_steps(g, steps, flush, torch, chunk)
    _, prof = traced_steps(g, min(steps, 200), flush, torch)
    g.close()
    total = sum(step_ms)
    cells = wl.cells
    sweep_ms = prof["sweep"][0] / max(prof["sweep"][1], 1)
    return {"ms_per_step": total / steps, "mlups": cells * steps / (total * 1e-3) / 1e6,
            "sweep_ms": sweep_ms, "sweep_bytes": cells * 2 * 19 * BYTES[storage],
            "kernels_ms": {k: v[0] / max(min(steps, 200), 1) for k, v in prof.items()},
            "launches": launches, "steps_per_timed_iteration": chunk}


def swim_speed(storage, wl, torch, device=0, chunk=200):
    g, ids = build_lattice(storage, wl.shape, wl.bodies, wl.collision, wl.lambda_e, device)
    v = []
    steps = wl.steps
    for k in range(0, steps, chunk):
        g.step(chunk)
        if k >= steps // 2:
            _, vel, e, _ = g.state(ids[0])
            v.append(float(vel @ e))
    g.close()
    return float(np.mean(v))


def psm_run(flush, torch, hbm, device=0):
    """Partially saturated cells (lb_set_coupling), the coupling Sec. IV A
    names against the speed fluctuation of the link-coupled squirmer:
    (1) the 256^3 pusher stepped with it in each storage, beside the link
    coupling; (2) the swim speed of the Fig. "resolution" squirmer (R = 4,
    L = 10R, B1 = 0.001, FP64) with both couplings: mean and spread of v.e /
    v0 over steps 1500..3000."""
    from paper_1903_04799_gb300 import Lattice
    from paper_1903_04799_gb300 import workloads as W
    wl = W.c3_pusher()
    out = {"workload": wl.name, "steps": 64}
    for st in ("f64", "f32", "bf16dev"):
        r = run_variant(st, wl, 64, 8, flush, torch, device, coupling="psm")
        out[st] = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"],
                   "sweep_frac": r["sweep_bytes"] / (r["sweep_ms"] * 1e-3) / 1e9 / hbm,
                   "kernels_ms_per_step": r["kernels_ms"]}
    R, L, B1 = 4.0, 40, 0.001
    v0 = 2 * B1 / 3
    spread = {}
    for coupling in ("links", "psm"):
        g = Lattice((L, L, L), collision="trt", device=device)
        if coupling == "psm":
            g.set_coupling("psm")
        oid = g.add_squirmer((L / 2 + 0.1, L / 2 + 0.2, L / 2), (0.0, 0.0, 1.0), R, B1, 0.0)
        g.step(1500)
        v = []
        for _ in range(1500):
            g.step(1)
            _, vel, e, _ = g.state(oid)
            v.append(float(vel @ e) / v0)
        g.close()
        spread[coupling] = {"U_over_v0": float(np.mean(v)), "spread_over_v0": float(np.std(v))}
    out["speed_fig_resolution_R4"] = {**spread, "window": "steps 1500..3000, FP64",
                                      "printed_link_spread": 0.081}
    return out


def e2e_run(wl, storage, steps, device, torch):
    """The public API end to end from pinned host buffers.  Set-up (lb_create,
    lb_add_squirmer) comes first, outside the timed region, as loading a model
    does.  Timed: the initial density and velocity fields uploaded
    (lb_set_fields), then every step lb_step(1) followed by a read of the
    squirmer's state (lb_get_object_state, which synchronises), and at the end
    the density and velocity fields read back (lb_get_fields)."""
    from paper_1903_04799_gb300 import workloads as W
    from paper_1903_04799_gb300 import lbsq
    N = wl.cells
    rho0, u0 = W.smooth_fields(wl.shape, seed=1, drho=0.0, umax=0.0)
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()  # noqa: E731
    rho_in, u_in, rho_out, u_out = pin(N), pin(3 * N), pin(N), pin(3 * N)
    rho_in[:] = rho0
    u_in[:] = u0.reshape(-1)
    g, ids = build_lattice(storage, wl.shape, wl.bodies, wl.collision, wl.lambda_e, device)
    g.sync()
    torch.cuda.synchronize()
    lib = lbsq.load()
    dp = lambda a: a.ctypes.data_as(lbsq._DP)  # noqa: E731
    st = [np.empty(3) for _ in range(4)]
    t0 = time.perf_counter()
    lbsq._check(g.ctx, lib.lb_set_fields(g.ctx, dp(rho_in), dp(u_in)), "lb_set_fields")
    for _ in range(steps):
        lbsq._check(g.ctx, lib.lb_step(g.ctx, 1), "lb_step")
        lbsq._check(g.ctx, lib.lb_get_object_state(g.ctx, ids[0], *[dp(a) for a in st]), "lb_get_object_state")
    lbsq._check(g.ctx, lib.lb_get_fields(g.ctx, dp(rho_out), dp(u_out)), "lb_get_fields")
    t = time.perf_counter() - t0
    g.close()
    return {"value": N * steps / t / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": int(4 * N * 8 / steps),
            "d2h_bytes_per_step": int(12 * 8 + 4 * N * 8 / steps),
            "steps": steps, "wall_s": t,
            "note": ("timed: lb_set_fields from pinned host buffers, then per step lb_step(1) + "
                     "lb_get_object_state (96 B), then lb_get_fields into pinned host buffers; "
                     "lb_create / lb_add_squirmer before the timed region")}


def serve_run(torch, device=0, n=256, budget=24 << 30, load=0.8):
    """The serving mix (256 Poisson arrivals; periodic box / square tube /
    obstacle geometries; R ~ U[3, 12]; steps ~ U[2000, 20000]; FP16-deviation
    or FP32 storage) through lb_server: requests are submitted when their
    arrival time has passed (host wall clock) and admitted as slots and HBM
    budget free up.  The arrival rate is set to `load` times a capacity
    measured first on the leading requests of the mix.  Latency = finish
    (end of the round in which the request completed, host clock) - arrival."""
    from paper_1903_04799_gb300 import lbsq
    from paper_1903_04799_gb300 import workloads as W

    def req_of(m):
        return lbsq.make_request(m.geometry, m.shape, m.storage, pos=m.pos, e=m.e, R=m.R, B1=m.B1, beta=m.beta,
                                 obstacle=m.obstacle, wca=m.wca, steps=m.steps)

    srv = lbsq.Server(budget_bytes=budget, max_resident=64, round_steps=64, device=device)
    info0 = srv.info()
    # capacity: the first 24 requests all resident, 6 rounds
    probe = W.serving_mix(n=24, rate=1.0)
    for m in probe:
        srv.submit(req_of(m))
    srv.advance()
    c0, t0 = srv.info()["cell_updates"], time.perf_counter()
    for _ in range(6):
        srv.advance()
    cap = (srv.info()["cell_updates"] - c0) / (time.perf_counter() - t0)
    srv.close()
    mix = W.serving_mix(n=n, rate=1.0)
    work = np.mean([m.cells * m.steps for m in mix])
    rate = load * cap / work
    mix = W.serving_mix(n=n, rate=rate)
    srv = lbsq.Server(budget_bytes=budget, max_resident=64, round_steps=64, tile_units=info0["tile_units"],
                      device=device)
    tickets, finish, pending = {}, {}, list(range(n))
    t_start = time.perf_counter()
    max_res = 0
    while len(finish) < n:
        now = time.perf_counter() - t_start
        while pending and mix[pending[0]].arrival <= now:
            i = pending.pop(0)
            tickets[i] = srv.submit(req_of(mix[i]))
        running, queued = srv.advance()
        max_res = max(max_res, running)
        now = time.perf_counter() - t_start
        for i, t in tickets.items():
            if i in finish:
                continue
            res = srv.poll(t)
            if res.state in (lbsq.LB_REQ_DONE, lbsq.LB_REQ_FAILED):
                finish[i] = (now, res.state)
        if running == 0 and queued == 0 and pending:
            time.sleep(max(0.0, mix[pending[0]].arrival - (time.perf_counter() - t_start)))
    info = srv.info()
    srv.close()
    lat = np.array([finish[i][0] - mix[i].arrival for i in range(n)])
    span = max(f[0] for f in finish.values()) - mix[0].arrival
    failed = sum(1 for f in finish.values() if f[1] != lbsq.LB_REQ_DONE)
    # algorithmic population traffic of the mix, 2 * 19 * bytes per cell update
    sbytes = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
    traffic = sum(m.cells * m.steps * 2 * 19 * sbytes[m.storage] for m in mix)
    hbm, _ = peaks()
    return {"requests": n, "failed": failed, "p50_s": float(np.percentile(lat, 50)),
            "hbm_gbs_achieved": traffic / span / 1e9, "hbm_frac": traffic / span / 1e9 / hbm,
            "hbm_note": "sum over requests of cells x steps x 2 x 19 x bytes per population, over the busy span",
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "aggregate_mlups": info["cell_updates"] / span / 1e6, "busy_span_s": span,
            "offered_load": load, "capacity_mlups_probe": cap / 1e6, "arrival_rate_per_s": rate,
            "max_resident": max_res, "tile_units": info["tile_units"], "blocks_per_sm": info["blocks_per_sm"],
            "round_steps": 64, "hbm_budget_gb": budget / 2**30}


def host_cpu() -> str:
    """The host CPU's model as the kernel reports it, with the core count."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and not model:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return f"{platform.machine()} {model} x{os.cpu_count()}".replace("  ", " ")


def fluid_fraction(wl) -> float:
    """Fraction of the workload's cells that are fluid at the start: nodes
    strictly inside a sphere, (dx^2 + dy^2) + dz^2 < R^2 with minimum-image
    offsets, are solid.  A pure host count (the same rule the library and the
    oracle classify by)."""
    n3 = np.array(wl.shape)
    solid = 0
    for b in wl.bodies:
        lo = [int(np.floor(b.pos[a] - b.R)) for a in range(3)]
        hi = [int(np.ceil(b.pos[a] + b.R)) for a in range(3)]
        axes = [np.arange(lo[a], hi[a] + 1) for a in range(3)]
        d = [((ax - b.pos[a]) + n3[a] / 2) % n3[a] - n3[a] / 2 for a, ax in enumerate(axes)]
        dx, dy, dz = np.meshgrid(d[0], d[1], d[2], indexing="ij")
        solid += int(((dx * dx + dy * dy) + dz * dz < b.R * b.R).sum())
    return 1.0 - solid / wl.cells


def cpu_baseline(wl, budget_s=15.0, single_budget_s=8.0):
    """The oracle as it stands, on the host cores, a bounded sample of the
    workload; then the same on one core."""
    from oracle import oracle as O
    s = O.OracleSim(*wl.shape, lambda_e=wl.lambda_e, collision=wl.collision)
    for b in wl.bodies:
        s.add_sphere(b.pos, b.e, b.R, b.B1, b.beta, b.mobile)
    s.step(1)

    def timed(budget):
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget and n < 10000:
            s.step(1)
            n += 1
        return n, time.perf_counter() - t0

    cores = O.num_threads()
    n, t = timed(budget_s)
    O.set_num_threads(1)
    try:
        n1, t1 = timed(single_budget_s)
    finally:
        O.set_num_threads(cores)
    return {"value": wl.cells * n / t / 1e6, "unit": "MLUPS", "cores": cores,
            "kind": "oracle", "sample": f"{n} full time steps of {wl.name} after 1 warm-up step",
            "single_core": {"value": wl.cells * n1 / t1 / 1e6, "unit": "MLUPS",
                            "sample": f"{n1} more full time steps of {wl.name} on 1 thread"},
            "host": host_cpu()}


def precision_sweep(torch, device=0, steps=None):
    """The 256^3 pusher (R = 16, beta = -3, B1 = 0.002) run 10 000 steps with
    populations stored as FP64, FP32, FP16 and BF16 deviations (FP32 collision
    for the last three).  Errors against the FP64 run: velocity field
    ||u - u64|| / ||u64|| over cells fluid in both runs (final step);
    stresslet ||S - S64||_F / ||S64||_F and swim speed |U - U64| / |U64|, both
    averaged over the second half of the run.  The FP64 run stands in for the
    FP64 oracle at this size: the two agree within 1e-12 on the parity tests."""
    from paper_1903_04799_gb300 import workloads as W
    wl = W.c3_pusher(steps=steps or 10000)
    out, ref = {}, None
    for st in ("f64", "f32", "f16dev", "bf16dev"):
        g, ids = build_lattice(st, wl.shape, wl.bodies, wl.collision, wl.lambda_e, device)
        S_acc, U_acc, n = np.zeros(6), 0.0, 0
        chunk = 100
        t0 = time.perf_counter()
        for k in range(0, wl.steps, chunk):
            g.step(chunk)
            if k + chunk > wl.steps // 2:
                S_acc += g.stresslet(ids[0])
                _, v, e, _ = g.state(ids[0])
                U_acc += float(v @ e)
                n += 1
        wall = time.perf_counter() - t0
        _, u = g.fields()
        own = g.owner()
        g.close()
        S, U = S_acc / n, U_acc / n
        if st == "f64":
            ref = (u, own, S, U)
            out[st] = {"U_over_v0": U / (2 * 0.002 / 3), "S_zz": S[2], "wall_s": wall}
            continue
        both = (own == 0) & (ref[1] == 0)
        du = u[:, both] - ref[0][:, both]
        out[st] = {"u_l2_err": float(np.sqrt((du ** 2).sum() / (ref[0][:, both] ** 2).sum())),
                   "stresslet_err": float(np.linalg.norm(S - ref[2]) / np.linalg.norm(ref[2])),
                   "swim_speed_err": abs(U - ref[3]) / abs(ref[3]),
                   "U_over_v0": U / (2 * 0.002 / 3), "wall_s": wall}
    v0 = 2 * 0.002 / 3
    eta = 1 / 6
    # traction force dipole of a squirmer: -(12 pi / 5) eta R^2 B2 (e e - I/3)
    S_closed = -(12 * np.pi / 5) * eta * 16 ** 2 * (-3 * 0.002) * 2 / 3
    return {"workload": wl.name, "steps": wl.steps, "reference": "FP64 storage run (GPU)",
            "stresslet_zz_closed_form": S_closed, "v0": v0, "storages": out}


def oscillation_of(y, z, L):
    """Amplitude and period of an oscillating lateral displacement y(t): the
    mean |y| at the turning points (local extrema that alternate in sign) and
    the mean spacing of every other turning point, in steps and in distance
    travelled along the periodic axis of length L (z unwrapped).  None with
    fewer than three turning points."""
    y = np.asarray(y, float)
    dz = np.diff(np.asarray(z, float))
    dz[dz < -L / 2] += L
    dz[dz > L / 2] -= L
    zu = np.concatenate([[0.0], np.cumsum(dz)])
    ext = []
    for k in range(1, len(y) - 1):
        if (y[k] - y[k - 1]) * (y[k + 1] - y[k]) < 0 and (not ext or np.sign(y[k]) != np.sign(y[ext[-1]])):
            ext.append(k)
    if len(ext) < 3:
        return None
    ext = np.array(ext)
    return {"amplitude": float(np.abs(y[ext]).mean()), "period_samples": float((ext[2:] - ext[:-2]).mean()),
            "period_travel": float(np.mean(zu[ext[2:]] - zu[ext[:-2]])), "turning_points": int(len(ext))}


def tube_run(torch, device=0, storage="f32", sample=200):
    """Sec. V tube flow: the neutral squirmer (R = 9) in the round tube
    D = 20R/3, L = 3 pi R, started parallel to the axis at y0 = -R; its
    lateral displacement sampled every `sample` steps; amplitude and period
    of the oscillation (both in units of R)."""
    from paper_1903_04799_gb300 import workloads as W
    t = W.tube_oscillation()
    b = t.body
    g = build_lattice(storage, t.shape, [], "trt", 1.0, device)[0]
    g.add_round_tube(t.axis[0], t.axis[1], t.radius)
    gi = g.add_squirmer(b.pos, b.e, b.R, b.B1, b.beta, mobile=True)
    g.set_contact(*t.contact)
    ys, zs, t0 = [], [], time.perf_counter()
    for _ in range(0, t.steps, sample):
        g.step(sample)
        p = g.state(gi)[0]
        ys.append(float(p[1] - t.axis[1]))  # the squirmer stays in the plane x = axis (mirror symmetry)
        zs.append(float(p[2]))
    wall = time.perf_counter() - t0
    g.close()
    osc = oscillation_of(ys, zs, t.shape[2])
    out = {"workload": t.name, "storage": storage, "steps": t.steps, "B1": b.B1, "wall_s": wall,
           "mlups": t.cells * t.steps / wall / 1e6, "y_over_R_first_last": [ys[0] / b.R, ys[-1] / b.R],
           "closest_wall_gap_over_R": float((t.radius - 0.5 - b.R - np.max(np.abs(ys))) / b.R)}
    if osc:
        out.update({"amplitude_over_R": osc["amplitude"] / b.R, "period_steps": osc["period_samples"] * sample,
                    "wavelength_over_R": osc["period_travel"] / b.R, "turning_points": osc["turning_points"]})
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """x maximised over all ranks (a replica job takes as long as its slowest
    rank); x itself without a process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells_per_rank: int, steps: int, ranks: int, total_ms: float) -> float:
    """Whole-job throughput of `ranks` replicas that each advanced
    cells_per_rank cells by `steps` steps in total_ms (max over ranks)."""
    return ranks * cells_per_rank * steps / (total_ms * 1e-3) / 1e6


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, ws, local, dist


def ours(args):
    import torch
    from paper_1903_04799_gb300 import lbsq
    from paper_1903_04799_gb300 import workloads as W
    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    lbsq.load()
    hbm, peak_kind = peaks()
    wl = W.c3_pusher()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    head = args.storage

    # ---- headline timed region
    g, ids = build_lattice(head, wl.shape, wl.bodies, wl.collision, wl.lambda_e, local)
    g.step(args.warmup)
    g.sync()
    clocks = ClockSampler(local) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    chunk = chunk_for(g, head)
    step_ms, launches = timed_steps(g, args.steps, flush, torch, chunk)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    # per-kernel attribution: traced pass of the same lattice right after
    n_traced = min(args.steps, 200)
    traced_ms, prof = traced_steps(g, n_traced, flush, torch)
    g.close()
    total_ms = max_over_ranks(sum(step_ms), dist, f"cuda:{local}")
    cells = wl.cells
    value = job_mlups(cells, args.steps, ws, total_ms)
    sweep_ms = prof["sweep"][0] / max(prof["sweep"][1], 1)
    sweep_bytes = cells * 2 * 19 * BYTES[head]
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    b = wl.bodies[0]
    res = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": ARITH[head],
        "data": "synthetic",
        "config": {"workload": wl.name, "shape": list(wl.shape), "R": b.R, "B1": b.B1, "beta": b.beta,
                   "collision": "trt(lambda_e=1, magic=3/16)", "storage": head, "arith": ARITH_NOTE[head],
                   "step": "sweep + links/force/Newton-Euler + classify + convert + rebuild",
                   "l2": (f"populations {cells * 19 * BYTES[head] / 1e6:.0f} MB vs L2 129 MB; "
                          f"L2 flushed (512 MiB write, outside the events) before every timed iteration "
                          f"of {chunk} step(s)"),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": ncu_traffic(f"sweep_{head}_{wl.name}"),
                     "kernel": KERNEL[head], "bytes_per_launch": sweep_bytes,
                     "per_unit": f"2*19*{BYTES[head]} B per cell update", "peak_kind": peak_kind,
                     "sweep_ms": sweep_ms},
        "fluid_mlups": round(value * fluid_fraction(wl), 1),
        "kernels_ms_per_step": {k: v[0] / max(v[1], 1) * (v[1] / n_traced) for k, v in prof.items()},
        "kernels_note": ("links = k_body_fused (bounce-back, force, Newton-Euler, re-classification, "
                         "conversions and link rebuild of each isolated sphere, one thread-block cluster "
                         "per sphere) plus k_links (walls); classify / convert / rebuild = the multi-kernel "
                         "path for spheres near another body (launched empty otherwise; not launched at all "
                         "for a lattice with a single sphere outside the traced pass)"),
        "traced": {"steps": n_traced, "ms_per_step": sum(traced_ms) / n_traced,
                   "note": "kernel-by-kernel launches with CUDA events between kernels, right after the "
                           "timed region; source of the per-kernel times and of the roofline's sweep time"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if ws == 1:
        # the same workload in every storage (and FP64 with FP64 arithmetic)
        variants = {head: {"mlups": value, "sweep_frac": achieved / hbm, "steps": args.steps}}
        if not args.skip_variants:
            for st, form in (("f64", 0), ("f64", 1), ("f32", 0), ("f16dev", 0), ("bf16dev", 0)):
                key = st if form == 0 else f"{st}_fp64_arith"
                if key == head:
                    continue
                r = run_variant(st, wl, 64, 8, flush, torch, local, form)
                variants[key] = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"], "steps": 64,
                                 "sweep_frac": r["sweep_bytes"] / (r["sweep_ms"] * 1e-3) / 1e9 / hbm,
                                 "kernels_ms_per_step": r["kernels_ms"], "kernel": KERNEL[st] if form == 0
                                 else "k_sweep (one cell per thread, FP64 arithmetic)"}
            if "f64" in variants:
                res["mixed_vs_f64"] = {k: variants[k]["mlups"] / variants["f64"]["mlups"]
                                       for k in ("f32", "f16dev", "bf16dev", "f64_fp64_arith") if k in variants}
        res["variants"] = variants
        if not args.skip_precision:
            res["precision_c3"] = precision_sweep(torch, local)
        if not args.skip_accuracy:
            acc = {}
            wl2 = W.c2_free_swimmer(beta=0.0)
            v0 = 2 * 0.005 / 3
            ref = None
            for st in ("f64", "f32", "f16dev", "bf16dev"):
                U = swim_speed(st, wl2, torch, local)
                ref = U if st == "f64" else ref
                acc[st] = {"U_over_v0": U / v0, "rel_err_vs_f64": abs(U - ref) / abs(ref)}
            res["swim_speed_c2"] = {"workload": wl2.name, "steps": wl2.steps,
                                    "window": "mean of v.e over the last half", **acc}
        if not args.skip_extra:
            extra = {}
            for wlx, sts in ((W.c2_free_swimmer(beta=0.0), ("f32", "f64")), (W.c4_suspension(), ("f32",))):
                for st in sts:
                    r = run_variant(st, wlx, 64, 8, flush, torch, local)
                    extra[f"{wlx.name}_{st}"] = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"],
                                                 "sweep_frac": r["sweep_bytes"] / (r["sweep_ms"] * 1e-3) / 1e9 / hbm,
                                                 "kernels_ms_per_step": r["kernels_ms"],
                                                 "steps_per_timed_iteration": r["steps_per_timed_iteration"]}
            res["extra"] = extra
        if not args.skip_tube:
            res["tube_oscillation"] = tube_run(torch, local)
        if not args.skip_psm:
            res["psm"] = psm_run(flush, torch, hbm, local)
        if not args.skip_serve:
            res["serving_c5"] = serve_run(torch, local)
        res["e2e"] = e2e_run(wl, head, args.steps, local, torch)
        if not args.skip_cpu:
            res["cpu_baseline"] = cpu_baseline(wl)
    else:
        res["e2e"] = None
    print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm

def reference(args):
    """The oracle timed as it stands on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1903_04799_gb300 import workloads as W
    wl = W.c3_pusher()
    s = O.OracleSim(*wl.shape, lambda_e=wl.lambda_e, collision=wl.collision)
    for b in wl.bodies:
        s.add_sphere(b.pos, b.e, b.R, b.B1, b.beta, b.mobile)
    for _ in range(args.warmup):
        s.step(1)
    budget, n, t0 = 150.0, 0, time.perf_counter()
    while n < args.steps and time.perf_counter() - t0 < budget:
        s.step(1)
        n += 1
    t = time.perf_counter() - t0
    v = wl.cells * n / t / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": 0,
        "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(n, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "shape": list(wl.shape), "storage": "f64 (oracle)"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{n} of the requested {args.steps} full time steps of {wl.name} "
                                   f"(bounded to {budget:.0f} s)", "host": host_cpu()},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_sweep(spec: str):
    """A bare periodic lattice (no bodies), stepped a few times: only the
    sweep kernels run.  spec = STORAGE:N:STEPS[:FORM] (FORM as
    lb_set_sweep_variant).  For ncu captures of one sweep kernel on a lattice
    of N^3 cells; prints nothing but a one-line confirmation."""
    import torch
    from paper_1903_04799_gb300 import Lattice
    parts = spec.split(":")
    st, n, steps = parts[0], int(parts[1]), int(parts[2])
    form = int(parts[3]) if len(parts) > 3 else 0
    g = Lattice((n, n, n), collision="trt", storage=st)
    if form:
        g.set_sweep_variant(form)
    g.step(steps)
    g.sync()
    torch.cuda.synchronize()
    g.close()
    print(f"profile-sweep {st} {n}^3 {steps} steps form {form}: ok", flush=True)


def profile_psm(spec: str):
    """The pusher of the 256^3 workload (R = 16, beta = -3) at the centre of
    an N^3 box, coupled by partially saturated cells, stepped STEPS times one
    step per call (no graphs): for ncu captures of k_psm_clear, k_psm_cover and
    k_psm_scatter (their work depends on the sphere, not on N).
    spec = STORAGE:N:STEPS."""
    import torch
    from paper_1903_04799_gb300 import workloads as W
    st, n, steps = spec.split(":")
    n, steps = int(n), int(steps)
    wl = W.c3_pusher(n)
    b = wl.bodies[0]
    g, _ = build_lattice(st, wl.shape, [], wl.collision, wl.lambda_e, 0, coupling="psm")
    g.add_squirmer(b.pos, b.e, b.R, b.B1, b.beta, mobile=True)
    for _ in range(steps):
        g.step(1)
    g.sync()
    torch.cuda.synchronize()
    g.close()
    print(f"profile-psm {st} {n}^3 {steps} steps: ok", flush=True)


def profile_bodies(spec: str):
    """The 200-squirmer suspension (256^3, R = 6), stepped STEPS times one
    step per call (no graphs): for ncu captures of the fused body kernel with
    many spheres (4-block clusters).  spec = STORAGE:STEPS."""
    import torch
    from paper_1903_04799_gb300 import workloads as W
    st, steps = spec.split(":")
    wl = W.c4_suspension()
    g, _ = build_lattice(st, wl.shape, wl.bodies, wl.collision, wl.lambda_e, 0)
    for _ in range(int(steps)):
        g.step(1)
    g.sync()
    torch.cuda.synchronize()
    g.close()
    print(f"profile-bodies {st} {steps} steps: ok", flush=True)


def profile_serve(spec: str):
    """The server with the first 24 requests of the serving mix resident
    (FP32 and FP16-deviation lattices of 32^3 .. 160^3), advanced ROUNDS
    rounds of 64 steps: for ncu launch lists and captures of the tile sweep
    and the body kernels.  spec = ROUNDS."""
    from paper_1903_04799_gb300 import lbsq
    from paper_1903_04799_gb300 import workloads as W
    srv = lbsq.Server(budget_bytes=4 << 30, max_resident=64, round_steps=64)  # the 24 requests need 1.7 GB
    for m in W.serving_mix(n=24, rate=1.0):
        srv.submit(lbsq.make_request(m.geometry, m.shape, m.storage, pos=m.pos, e=m.e, R=m.R, B1=m.B1,
                                     beta=m.beta, obstacle=m.obstacle, wca=m.wca, steps=m.steps))
    for _ in range(int(spec)):
        srv.advance()
    info = srv.info()
    srv.close()
    print(f"profile-serve {spec} rounds: ok ({info['cell_updates']} cell updates)", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f64", choices=list(BYTES))
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-precision", action="store_true")
    ap.add_argument("--skip-tube", action="store_true")
    ap.add_argument("--skip-psm", action="store_true")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="run the 256^3 storage precision sweep (about 2 minutes) instead of the benchmark")
    ap.add_argument("--profile-sweep", metavar="STORAGE:N:STEPS[:FORM]",
                    help="step a bare N^3 lattice (sweep kernels only), for ncu captures, instead of the benchmark")
    ap.add_argument("--profile-psm", metavar="STORAGE:N:STEPS",
                    help="step the pusher under partially saturated cells, for ncu captures, instead of the benchmark")
    ap.add_argument("--profile-bodies", metavar="STORAGE:STEPS",
                    help="step the 200-squirmer suspension one step per call, for ncu captures, instead of the benchmark")
    ap.add_argument("--profile-serve", metavar="ROUNDS",
                    help="advance the server with 24 resident requests, for ncu captures, instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_sweep:
        profile_sweep(args.profile_sweep)
    elif args.profile_psm:
        profile_psm(args.profile_psm)
    elif args.profile_bodies:
        profile_bodies(args.profile_bodies)
    elif args.profile_serve:
        profile_serve(args.profile_serve)
    elif args.impl == "reference":
        reference(args)
    elif args.precision_sweep:
        import torch
        print(json.dumps({"precision_sweep": precision_sweep(torch)}), flush=True)
    else:
        ours(args)


if __name__ == "__main__":
    main()
