"""Benchmark: finest-level zones/s to 1e-10 relative residual.

Workload: 3D, base 64^3 on [-1,1]^3 plus 3 nested 64^3 levels (ratio 2,
centred), compact polynomial sphere rho = (1 - r^2/R^2)^3, R = 0.3, centred at
(0.05, 0.03, 0.02), G = 1, closed-form Dirichlet outer boundary, V(2,2)
cycles to 1e-10 relative residual per level, forces by Eq. 2.  Zones are the
cells whose potential and force are returned: 4 * 64^3 per solve.

One step = set the density of every level (device to device), solve all
levels coarse to fine, compute potential and forces of every level.  Steps
are timed one by one with CUDA events on the solver's stream; a 256 MiB
buffer (larger than the 129 MB L2) is written between steps, outside the
timed events.  Forms: plain FP64, and FP32 V-cycles inside FP64 defect
correction ("mixed").  `value` is the fastest form whose results stay within
1e-2 of the discretisation error of the FP64 result.

Beside the headline: the finest multigrid level's FP32 smoothing timed as
the solve graph launches it (mg_time_smoothing) against the measured HBM
copy bandwidth, with its algorithmic bytes, and the whole step's algorithmic
bytes over its time -- for this workload (L2-resident) and for the
DRAM-resident one of 4 nested 256^3 levels with 8 compact spheres, whose
zones/s are measured in the same run (--no-scale leaves it out).

--impl reference times the CPU FP64 oracle, as it stands, on every host
core: one full solve of the workload per core per step, in parallel
processes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2001_02327_gb300 import inputs as I  # noqa: E402

METRIC = "finest-level zones/s to 1e-10 rel. residual: plain FP64 vs mixed/learned"
UNIT = "zones/s"
WORKLOAD = "3D nested 4x64^3, offset compact sphere (m=3, R=0.3), V(2,2) to 1e-10 rel. residual, Eq. 2 forces"
NU = (2, 2)
TOL = 1e-10


def make_workload():
    H = I.config_3d_offset_sphere(64, 4)
    return H, I.level_inputs(H)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_id), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Runner:
    """One hierarchy resident on the GPU plus its inputs and outputs."""

    def __init__(self, mg, torch, H, inp, stream, precision, tune_cache=None, unet=None, autotune=True, inner_max=0,
                 inner_cycles=3, forces_call=False):
        self.mg, self.torch, self.H = mg, torch, H
        self.stream = stream
        guess = mg.MG_GUESS_LEARNED if unet is not None else mg.MG_GUESS_INTERP
        self.opt = mg.options(nu_pre=NU[0], nu_post=NU[1], max_cycles=60, rel_tol=TOL, precision=precision,
                              inner_cycles=inner_cycles, inner_max=inner_max, guess=guess, stream=stream)
        self.h = mg.mg_create_hierarchy([mg.desc_from(H)], self.opt)
        if unet is not None:
            from paper_2001_02327_gb300 import unet as U
            U.mg_set_unet(self.h, unet)
        # launch plan of the FP32 V-cycle chosen by measurement (setup, untimed);
        # without it the library's default plan
        if autotune:
            mg.mg_autotune(self.h, tune_cache)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.d_in = [{k: dev(v) for k, v in d.items()} for d in inp]
        self.d_phi = [torch.zeros((n,) * 3, dtype=torch.float64, device="cuda") for n in H.n]
        self.d_F = [torch.zeros((3,) + (n,) * 3, dtype=torch.float64, device="cuda") for n in H.n]
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        self.h_in = [{k: pin(v) for k, v in d.items()} for d in inp]
        self.h_phi = [torch.zeros((n,) * 3, dtype=torch.float64).pin_memory().numpy() for n in H.n]
        self.h_F = [torch.zeros((3,) + (n,) * 3, dtype=torch.float64).pin_memory().numpy() for n in H.n]
        self.stats = None
        self.forces_call = forces_call
        self.out_host = False
        if not forces_call:
            self.outputs(False)

    def outputs(self, host):
        """Where mg_solve writes each level's potential and forces: the device
        arrays or the page-locked host arrays (a change rebuilds the solve
        graph once, at the next solve)."""
        phi, F = (self.h_phi, self.h_F) if host else (self.d_phi, self.d_F)
        for l in range(self.H.num_levels):
            self.mg.mg_set_outputs(self.h, 0, l, phi[l], F[l])
        self.out_host = host

    def step(self, host=False):
        """One step: the inputs into the hierarchy, the solve, which also
        writes every level's potential and forces (Eq. 2) to the outputs."""
        mg = self.mg
        if host != self.out_host and not self.forces_call:
            self.outputs(host)
        src = self.h_in if host else self.d_in
        for l in range(self.H.num_levels):
            if l == 0:
                mg.mg_set_density(self.h, 0, 0, src[0]["rho"], src[0]["bc_rho"], src[0]["bc_phi"])
            else:
                mg.mg_set_density(self.h, 0, l, src[l]["rho"])
        _, self.stats = mg.mg_solve(self.h, 1)
        if self.forces_call:       # the same results through one mg_forces call per level
            phi, F = (self.h_phi, self.h_F) if host else (self.d_phi, self.d_F)
            for l in range(self.H.num_levels):
                mg.mg_forces(self.h, 0, l, phi[l], F[l])

    def io_bytes(self):
        h2d = sum(a.nbytes for d in self.h_in for a in d.values())
        d2h = sum(a.nbytes for a in self.h_phi) + sum(a.nbytes for a in self.h_F)
        return h2d, d2h

    def results(self):
        self.torch.cuda.synchronize()
        return [(p.cpu().numpy(), F.cpu().numpy()) for p, F in zip(self.d_phi, self.d_F)]

    def close(self):
        self.mg.mg_destroy(self.h)


def gpu_ident(torch, local):
    """nvidia-smi -i argument for the torch device: its UUID when known."""
    u = getattr(torch.cuda.get_device_properties(local), "uuid", None)
    if u is None:
        return local
    u = str(u)
    return u if u.startswith("GPU-") else "GPU-" + u


def time_device(runner, torch, steps, warmup, flush):
    s = runner.stream
    for _ in range(warmup):
        runner.step()
    torch.cuda.synchronize()
    times = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(s):
            flush.zero_()
        ev[k][0].record(s)
        runner.step()
        ev[k][1].record(s)
    torch.cuda.synchronize()
    for a, b in ev:
        times.append(a.elapsed_time(b))
    return times


def time_e2e(runner, torch, steps):
    runner.step(host=True)          # untimed: switches the outputs to the host arrays
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        runner.step(host=True)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3 / steps


def profile_pass(runner, torch, steps):
    mg = runner.mg
    mg.mg_profile(runner.h, 1)
    for _ in range(steps):
        runner.step()
    prof = mg.mg_profile_read(runner.h)
    mg.mg_profile(runner.h, 0)
    return prof


def max_over_ranks(x, device="cpu"):
    """The largest x over all ranks of the process group (the job takes as
    long as its slowest rank); x itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ms, world_size):
    """Whole-job units per second: every rank processes units_per_rank
    (replicas, weak scaling) in ms milliseconds of the slowest rank."""
    return world_size * units_per_rank / (ms * 1e-3)


def measured_peaks(key="hbm_gbs"):
    """A measured peak (HBM copy GB/s or dense bf16 TFLOP/s) and its source."""
    fallback = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}[key]
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if key in d:
            return d[key], "measured"
    return fallback, "fallback"


def kernel_traffic(key):
    """DRAM bytes per launch of the kernel `key` from the committed ncu
    summary (profiles/ncu_traffic.json), if it was taken on the current
    kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(key)
    if not ent or ent.get("csrc_sha256") != kernel_source_sha():
        return None
    return ent.get("dram_bytes_per_launch")


SMOOTH_SOURCES = ("mg_box.cu", "mg_internal.h", "mg_kernels.cu", "mg_wave.cu")


def kernel_source_sha():
    """sha256 over the CUDA sources that define the smoothing kernels
    (k_smooth_colour, k_wave, kx_smooth32 and their headers), in this order."""
    hs = hashlib.sha256()
    for f in SMOOTH_SOURCES:
        hs.update(open(os.path.join(ROOT, "paper_2001_02327_gb300", "csrc", f), "rb").read())
    return hs.hexdigest()


def _oracle_solve(args):
    """One oracle solve of the benchmark workload (a worker of the all-core
    baseline; builds its own inputs, returns its wall time)."""
    from oracle import oracle as O
    H, inp = make_workload()
    t0 = time.perf_counter()
    O.solve_hierarchy(H, inp, NU[0], NU[1], 60, TOL)
    return time.perf_counter() - t0


def oracle_all_cores(procs):
    """Throughput of the oracle on every host core: `procs` independent solves
    of the workload at once, one per process (spawned, so that no process
    inherits a CUDA context).  Returns (zones/s, wall seconds)."""
    import multiprocessing as mp
    H, _ = make_workload()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_solve, range(procs))           # warm-up: imports, library load
        t0 = time.perf_counter()
        pool.map(_oracle_solve, range(procs))
        wall = time.perf_counter() - t0
    return procs * H.zones() / wall, wall


def cpu_baseline(H, inp):
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    O.solve_hierarchy(H, inp, NU[0], NU[1], 60, TOL)
    dt = time.perf_counter() - t0
    procs = os.cpu_count() or 1
    v_all, wall = oracle_all_cores(procs)
    return {"value": H.zones() / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full solve of the workload (all 4 levels, forces included), {dt:.2f} s, single thread",
            "all_cores": {"value": v_all, "unit": UNIT, "cores": procs,
                          "sample": f"{procs} independent full solves at once, one process per core, {wall:.2f} s"}}


# ---------------------------------------------------------------------------
# measured rooflines: the finest multigrid level's smoothing, timed as the
# solve graph launches it, and the whole solve's algorithmic bytes
# ---------------------------------------------------------------------------
SMOOTH_KINDS = ("smooth_colour_finest", "smooth_wave_finest")


def kernel_roofline(mg, h, level, prof_per_step, ms_per_step, workload, traffic_key, sustained):
    """Roofline of the finest multigrid level's FP32 smoothing of refinement
    level `level`: per-launch time from mg_time_smoothing (launches captured
    back to back in one CUDA graph with programmatic dependent launch, as the
    solve runs them), algorithmic bytes from the library (1.5 words per
    active cell per one-colour launch, 3 per plane-marching launch), the
    launches per step from the host-loop profile of the same plan."""
    us, by = mg.mg_time_smoothing(h, 0, level, 0, 20)
    kind = next((k for k in SMOOTH_KINDS if k in prof_per_step), None)
    per_step = prof_per_step[kind][0] if kind else 0.0
    peak, src = measured_peaks()
    achieved = by / (us * 1e-6) / 1e9
    code = mg.mg_tuning(h, 0, level)[0][0]
    plan = ("colour-split storage, one colour per launch (kx_smooth32)" if code == 65536 else
            "plane-marching sweeps (k_wave)" if code < 0 else "temporally blocked legs" if code > 0 else
            "plain storage, one colour per launch (k_smooth_colour)")
    key = f"{traffic_key}/{kind}" + ("/split" if code == 65536 else "")
    traffic = kernel_traffic(key) if kind else None
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_over_algorithmic": round(traffic / by, 3) if traffic else None,
            "kernel": kind or "smooth", "plan": plan, "workload": workload, "launch_us": round(us, 3),
            "bytes_per_launch": by,
            "byte_model": "active cells x 4 B x (1.5 per one-colour launch: Phi read, half of f read, half of Phi "
                          "written; 3 per plane-marching launch of nu sweeps: Phi and f read once, Phi written once)",
            "timing": "mg_time_smoothing: 20 launches in one CUDA graph with programmatic dependent launch, "
                      "CUDA events around 5 replays on the solver's stream",
            "launches_per_step": per_step, "kernel_ms_per_step": round(per_step * us * 1e-3, 4),
            "ms_per_step": round(ms_per_step, 4),
            "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)" + ("; timed alone" if not sustained else "")}


def solve_bytes(H, stats, precision):
    """Algorithmic DRAM bytes of one step (set_density + solve + potential and
    forces out): per refinement level, 7.1 words per active cell per V-cycle
    (Phi and f read and Phi written going down and coming up, a quarter word
    of transfer, 8/7 for the coarse multigrid levels), 40 B per cell per FP64
    defect-correction step of the mixed form (residual and accumulation), and
    64 B per cell of the level for the density in and the outputs."""
    w = 4 if precision == "mixed" else 8
    total = 0.0
    for l in range(H.num_levels):
        M3 = float(H.n[l] + 2) ** H.dim
        st = stats[0][l]
        total += 7.1 * w * M3 * st["cycles"] + 64.0 * float(H.n[l]) ** H.dim
        if precision == "mixed":
            total += 40.0 * M3 * st["outer_steps"]
    return total


def whole_solve_roofline(H, stats, precision, ms):
    by = solve_bytes(H, stats, precision)
    peak, src = measured_peaks()
    achieved = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "bytes_per_step": by, "ms_per_step": round(ms, 4),
            "byte_model": "per level: 7.1 words x active cells x V-cycles (FP32 words in the mixed form) + 40 B x "
                          "active cells x defect-correction steps (mixed) + 64 B x cells of Omega (density in, "
                          "potential and forces out)", "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)"}


def scale_case(mg, torch, stream, flush, steps, warmup, tune_cache, inner_cycles, inner_max):
    """The DRAM-resident workload: 4 nested 256^3 levels, 8 compact spheres;
    mixed form (the reported one) and FP64, set_density + solve (potential
    and forces written by mg_solve), CUDA events, L2 flushed between steps."""
    H = I.config_3d_spheres(256, 4, 8)
    inp = I.level_inputs(H)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_in = [{k: dev(v) for k, v in d.items()} for d in inp]
    F = [torch.empty((3,) + (m,) * 3, dtype=torch.float64, device="cuda") for m in H.n]
    P = [torch.empty((m,) * 3, dtype=torch.float64, device="cuda") for m in H.n]
    out = {}
    for name, prec in (("mixed", mg.MG_MIXED), ("fp64", mg.MG_FP64)):
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=NU[0], nu_post=NU[1], max_cycles=60,
                                                                 rel_tol=TOL, precision=prec,
                                                                 inner_cycles=inner_cycles,
                                                                 inner_max=inner_max, stream=stream))
        try:
            if prec == mg.MG_MIXED:
                mg.mg_autotune(h, tune_cache)
            for l in range(H.num_levels):
                mg.mg_set_outputs(h, 0, l, P[l], F[l])

            def step():
                mg.mg_set_density(h, 0, 0, d_in[0]["rho"], d_in[0]["bc_rho"], d_in[0]["bc_phi"])
                for l in range(1, H.num_levels):
                    mg.mg_set_density(h, 0, l, d_in[l]["rho"])
                return mg.mg_solve(h, 1)[1]

            for _ in range(warmup):
                st = step()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                with torch.cuda.stream(stream):
                    flush.zero_()
                a.record(stream)
                st = step()
                b.record(stream)
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            t = statistics.median(ms)
            ep = ef = 0.0
            for l in range(H.num_levels):
                X = H.centres(l, 0)
                pa, fa = H.potential(X), H.force(X)
                ep = max(ep, float(np.max(np.abs(P[l].cpu().numpy() - pa)) / np.max(np.abs(pa))))
                ef = max(ef, float(np.max(np.abs(np.moveaxis(F[l].cpu().numpy(), 0, -1) - fa)) / np.max(np.abs(fa))))
            res = {"zones_per_s": H.zones() / (t * 1e-3), "ms_per_step": t, "ms_min": min(ms),
                   "cycles_per_level": [st[0][l]["cycles"] for l in range(H.num_levels)],
                   "outer_steps_per_level": [st[0][l]["outer_steps"] for l in range(H.num_levels)],
                   "max_rel_res": max(st[0][l]["rel_res"] for l in range(H.num_levels)),
                   "max_rel_err_phi_vs_closed_form": ep, "max_rel_err_F_vs_closed_form": ef,
                   "whole_solve_roofline": whole_solve_roofline(H, st, name, t)}
            if prec == mg.MG_MIXED:
                res["plan_finest"] = mg.mg_tuning(h, 0, 0)[0][:8]
                mg.mg_profile(h, 1)
                step()
                prof = mg.mg_profile_read(h)
                mg.mg_profile(h, 0)
                res["kernel_roofline"] = kernel_roofline(mg, h, 0, prof, t, "4 nested 256^3 levels (finest "
                                                         "multigrid level 258^3, 69 MB per FP32 array)",
                                                         "scale_4x256cubed", sustained=True)
            out[name] = res
        finally:
            mg.mg_destroy(h)
    out["workload"] = ("3D, 4 nested 256^3 levels on [-1,1]^3, 8 compact spheres (m=3) with centres in the finest "
                       "box, radii U[0.02,0.1]x2, masses U[0.5,2]; V(2,2) to 1e-10; Eq. 2 forces")
    out["zones_per_solve"] = H.zones()
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg

    H, inp = make_workload()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    forms = {}
    results = {}
    plans = [("fp64", mg.MG_FP64, None), ("mixed", mg.MG_MIXED, None)]
    net = None
    if not args.no_learned:
        net = train_guess_network(torch)
        plans.append(("mixed_learned", mg.MG_MIXED, net))
    kroof = None
    for name, prec, unet in plans:
        r = Runner(mg, torch, H, inp, stream, prec, args.tune_cache, unet, not args.no_autotune, args.inner_max,
                   args.inner_cycles, args.forces_call)
        try:
            # the first solve of each form carries an NVTX range, so that a
            # profiler can select exactly one solve's launches
            torch.cuda.nvtx.range_push(f"{name}_solve")
            r.step()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            results[name] = r.results()
            cyc = [r.stats[0][l]["cycles"] for l in range(H.num_levels)]
            stats = r.stats
            if ws > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            sampler = ClockSampler(gpu_ident(torch, local))
            sampler.start()
            times = time_device(r, torch, args.steps, args.warmup, flush)
            clocks = sampler.stop()
            total = max_over_ranks(sum(times), device="cuda")
            ms = total / args.steps
            e2e_ms = max_over_ranks(time_e2e(r, torch, max(3, args.steps // 2)), device="cuda")
            h2d, d2h = r.io_bytes()
            nprof = max(3, min(args.steps, 10))
            prof = profile_pass(r, torch, nprof)
            per_step = {k: (v[0] / nprof, v[1] / nprof, v[2] / nprof) for k, v in prof.items()}
            forms[name] = {"value": job_throughput(H.zones(), ms, ws), "ms_per_step": ms,
                           "ms_min": min(times), "cycles": cyc, "e2e_ms": e2e_ms, "h2d": h2d, "d2h": d2h,
                           "prof": per_step, "clocks": clocks,
                           "whole_solve": whole_solve_roofline(H, stats, "fp64" if prec == mg.MG_FP64 else "mixed",
                                                               ms)}
            if name == "mixed":
                kroof = kernel_roofline(mg, r.h, 0, per_step, ms, "4 nested 64^3 levels (finest multigrid level "
                                        "66^3, 1.1 MB per FP32 array: L2-resident, launch-latency bound)",
                                        "bench_4x64cubed", sustained=True)
        finally:
            r.close()

    # accuracy of every other form against FP64 (budget: 1e-2 of the discretisation error)
    errors = {}
    for name in forms:
        if name == "fp64":
            continue
        worst = 0.0
        for l in range(H.num_levels):
            X = H.centres(l, 0)
            p64, F64 = results["fp64"][l]
            pm, Fm = results[name][l]
            disc = np.max(np.abs(p64 - H.potential(X)))
            discF = np.max(np.abs(np.moveaxis(F64, 0, -1) - H.force(X)))
            worst = max(worst, np.max(np.abs(pm - p64)) / disc, np.max(np.abs(Fm - F64)) / discF)
        errors[name] = float(worst)
    best = max((k for k in forms if k == "fp64" or errors[k] < 1e-2), key=lambda k: forms[k]["value"])
    worst = errors["mixed"]
    if net is not None:
        from paper_2001_02327_gb300 import unet as U
        U.mg_unet_destroy(net)
    fb = forms[best]

    # the DRAM-resident workload, where a fraction of the HBM roofline means something
    scale = None if args.no_scale else scale_case(mg, torch, stream, flush, max(3, min(args.steps, 10)), 2,
                                                    args.tune_cache, args.inner_cycles, args.inner_max)

    launches = int(round(sum(v[0] for v in fb["prof"].values()))) * args.steps
    out = {
        "metric": METRIC, "value": fb["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": fb["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64"}.get(best, "f32+f64+bf16"),
        "data": "synthetic (closed-form density and boundary potential)",
        "config": {"workload": WORKLOAD, "zones_per_solve": H.zones(), "levels": H.num_levels, "n": 64,
                   "nu": list(NU), "rel_tol": TOL, "form": best, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}",
                   "launch_plan": "default" if args.no_autotune else "mg_autotune (timed at setup)",
                   "mixed_inner_cycles": f"{args.inner_cycles}, then chosen per step up to {args.inner_max}"
                   if args.inner_max else f"{args.inner_cycles} per step"},
        "forms": {k: {"zones_per_s": v["value"], "ms_per_step": v["ms_per_step"], "cycles_per_level": v["cycles"],
                      "whole_solve_roofline": v["whole_solve"],
                      "kernels_host_loop_profile": {kk: {"launches": round(vv[0], 1), "ms": round(vv[1], 4)}
                                                    for kk, vv in v["prof"].items()}}
                  for k, v in forms.items()},
        "mixed_error_vs_fp64_over_discretisation": worst,
        "form_error_vs_fp64_over_discretisation": errors,
        "e2e": {"value": job_throughput(H.zones(), fb["e2e_ms"], ws), "unit": UNIT, "h2d_bytes_per_step": fb["h2d"],
                "d2h_bytes_per_step": fb["d2h"]},
        "gpu_launches": launches,
        "roofline": kroof,
        "clocks": fb["clocks"],
    }
    if scale is not None:
        out["scale_4x256cubed"] = scale
        out["roofline_dram_resident"] = scale["mixed"].get("kernel_roofline")
    if not args.no_batch:
        # the uneven batch of 512 hierarchies, and 512 small ones (the persistent launch's case)
        out["batch_512"] = batch_case(mg, torch, 512, I.EDGES, 2, 2, args.inner_cycles, args.inner_max)
        out["batch_512_small"] = batch_case(mg, torch, 512, (16, 24, 32), 3, 2, args.inner_cycles, args.inner_max)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(H, inp)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, as it stands
# ---------------------------------------------------------------------------
def train_guess_network(torch):
    """The learned initial guess's network, trained before the timed runs on
    samples the solver generates (hierarchies of 64^3 levels with random
    compact spheres, none of them the benchmark workload): small and quick,
    enough to time the solve with a network in it."""
    from paper_2001_02327_gb300 import learned as LR
    from paper_2001_02327_gb300 import unet as U
    data = LR.make_samples(torch, 48, n=64, seed0=I.BASE_SEED + 4000, levels=3)
    net = U.mg_unet_create(64, 4, seed=1)
    LR.train(torch, net, data, steps=300, batch=4, lr=1e-3)
    torch.cuda.synchronize()
    return net


def run_reference(args):
    """The CPU FP64 oracle, as it stands, on every host core: each step is
    one full solve of the workload per core, in parallel processes
    (independent solves; the oracle itself is single-threaded)."""
    import multiprocessing as mp
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    H, _ = make_workload()
    procs = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_solve, range(procs))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_solve, range(procs))
        dt = (time.perf_counter() - t0) / args.steps
    v = procs * H.zones() / dt
    sample = (f"{procs} independent full solves of the workload per step (all 4 levels, forces included), one "
              f"single-threaded process per host core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (closed-form density and boundary potential)",
        "config": {"workload": WORKLOAD, "zones_per_solve": H.zones(), "levels": H.num_levels, "n": 64,
                   "nu": list(NU), "rel_tol": TOL, "form": "oracle", "solves_per_step": procs},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_level_case(args):
    """One 3D level of n=254 (arrays of 258^3 doubles, 137 MB each: larger
    than L2) with seeded random density and boundary, a fixed number of
    V-cycles.  Used for profiler captures of the kernels on DRAM-resident
    data; prints one line of timing, not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    n = args.level_n
    rng = np.random.default_rng(I.BASE_SEED + 254)
    H = I.Hierarchy(3, [n], [(0.0, 0.0, 0.0)], 1.0 / n, 1.0, [], f"level{n}")
    dev = lambda a: torch.from_numpy(a).cuda()
    rho, bcr, bcp = (dev(rng.standard_normal((k,) * 3)) for k in (n, n + 2, n + 4))
    prec = mg.MG_MIXED if args.precision == "mixed" else mg.MG_FP64
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(max_cycles=args.cycles, rel_tol=0.0, precision=prec,
                                                             inner_cycles=1))
    try:
        for rep in range(2):
            mg.mg_set_density(h, 0, 0, rho, bcr, bcp)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = mg.mg_solve(h, 1, allow_noconv=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        print(json.dumps({"case": f"level n={n}", "precision": args.precision, "cycles": st[0][0]["cycles"],
                          "ms": dt * 1e3, "rel_res": st[0][0]["rel_res"]}))
    finally:
        mg.mg_destroy(h)


def run_smoothing_case(args):
    """The finest multigrid level's FP32 smoothing of one 3D level of n cells
    per edge (mixed precision, the library's default plan unless MG_WAVE /
    MG_WAVE_PLAN choose the plane-marching sweeps), timed by mg_time_smoothing
    with `--launches` launches.  For profiler captures (under MG_SOLVE_GRAPH=0
    the launches run without a graph, where a profiler sees them); prints one
    line, not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    n = args.level_n
    H = I.Hierarchy(3, [n], [(0.0, 0.0, 0.0)], 1.0 / n, 1.0, [], f"level{n}")
    h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=NU[0], nu_post=NU[1], precision=mg.MG_MIXED))
    try:
        us, by = mg.mg_time_smoothing(h, 0, 0, 0, args.launches)
        print(json.dumps({"case": f"smoothing, finest multigrid level of a {n}^3 level", "plan": mg.mg_tuning(h, 0, 0)[0][0],
                          "us_per_launch": us, "bytes_per_launch": by, "GB_per_s": by / us / 1e3}))
    finally:
        mg.mg_destroy(h)


def batch_case(mg, torch, nb, edges, steps, warmup, inner_cycles, inner_max, autotune=False, forces_call=False):
    """Uneven batch: nb seeded hierarchies (2-4 levels, edges drawn from
    `edges`, 1-4 compact spheres each), mixed precision, V(2,2) to 1e-10,
    solved together in one graph launch (graph branches or the persistent
    launch, as the library's cost model picks), every level's forces written
    by mg_solve; CUDA events around set_density + mg_solve, mean of `steps`."""
    Hs = [I.random_hierarchy(I.BASE_SEED + b, edges=edges) for b in range(nb)]
    zones = sum(H.zones() for H in Hs)
    opt = mg.options(nu_pre=NU[0], nu_post=NU[1], max_cycles=60, rel_tol=TOL, precision=mg.MG_MIXED,
                     inner_cycles=inner_cycles, inner_max=inner_max)
    h = mg.mg_create_hierarchy([mg.desc_from(H) for H in Hs], opt)
    try:
        if autotune:
            mg.mg_autotune(h, None)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        ins = []
        for H in Hs:
            inp = I.level_inputs(H)
            ins.append([{k: dev(v) for k, v in d.items()} for d in inp])
        Fs = [[torch.empty((3,) + (n,) * 3, dtype=torch.float64, device="cuda") for n in H.n] for H in Hs]
        for b, H in enumerate(Hs):
            for l in range(H.num_levels):
                if not forces_call:
                    mg.mg_set_outputs(h, b, l, None, Fs[b][l])
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def step():
            for b, H in enumerate(Hs):
                d = ins[b]
                mg.mg_set_density(h, b, 0, d[0]["rho"], d[0]["bc_rho"], d[0]["bc_phi"])
                for l in range(1, H.num_levels):
                    mg.mg_set_density(h, b, l, d[l]["rho"])
            st = mg.mg_solve(h, len(Hs))[1]
            if forces_call:
                for b, H in enumerate(Hs):
                    for l in range(H.num_levels):
                        mg.mg_forces(h, b, l, None, Fs[b][l])
            return st

        for _ in range(warmup):
            st = step()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            ev0.record()
            st = step()
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        dt = sum(ms) / len(ms) * 1e-3
        worst = max(st[b][l]["rel_res"] for b, H in enumerate(Hs) for l in range(H.num_levels))
        cyc = sum(st[b][l]["cycles"] for b, H in enumerate(Hs) for l in range(H.num_levels))
        npers = mg.mg_persistent_count(h)
        return {"case": f"batch of {len(Hs)} uneven hierarchies, edges {list(edges)}", "zones": zones,
                "ms_per_solve": dt * 1e3, "zones_per_s": zones / dt, "worst_rel_res": worst,
                "fp32_cycles_total": cyc, "autotune": bool(autotune),
                "batched_kernels": os.environ.get("MG_BATCHED", "0") == "1",
                "solve_plan": "persistent launch" if npers == len(Hs) else
                              ("graph branches" if npers == 0 else f"persistent launch for {npers}, graph branches"),
                "timing": f"CUDA events around set_density + mg_solve (writing every level's forces), mean of {steps}"}
    finally:
        mg.mg_destroy(h)


def run_batch_case(args):
    """Uneven batch of `--batch` hierarchies (edges from {32,48,64,96,128}
    or `--batch-edges`); prints one line of timing, not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    edges = tuple(int(e) for e in args.batch_edges.split(",")) if args.batch_edges else I.EDGES
    print(json.dumps(batch_case(mg, torch, args.batch, edges, args.steps, args.warmup, args.inner_cycles,
                                args.inner_max, args.autotune, args.forces_call)))


def run_scale_case(args):
    """4 nested 256^3 levels on [-1,1]^3, 8 compact spheres (m = 3) with centres
    in the finest box, radii U[0.02,0.1] x 2, masses U[0.5,2]; V(2,2) to 1e-10,
    FP64 and mixed.  Prints one line per form (zones/s of set_density + solve +
    forces, CUDA events; max errors of potential and force against the closed
    form), not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    H = I.config_3d_spheres(args.level_n if args.level_n != 254 else 256, args.scale_levels, 8)
    inp = I.level_inputs(H)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_in = [{k: dev(v) for k, v in d.items()} for d in inp]
    n = H.n[0]
    F = [torch.empty((3,) + (m,) * 3, dtype=torch.float64, device="cuda") for m in H.n]
    P = [torch.empty((m,) * 3, dtype=torch.float64, device="cuda") for m in H.n]
    forms = [f for f in (("fp64", mg.MG_FP64), ("mixed", mg.MG_MIXED)) if f[0] in args.forms.split(",")]
    for name, prec in forms:
        h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=NU[0], nu_post=NU[1], max_cycles=60,
                                                                 rel_tol=TOL, precision=prec,
                                                                 inner_cycles=args.inner_cycles,
                                                                 inner_max=args.inner_max))
        try:
            if prec == mg.MG_MIXED:
                mg.mg_autotune(h, args.tune_cache)

            for l in range(H.num_levels):
                mg.mg_set_outputs(h, 0, l, P[l], F[l])

            def step():
                mg.mg_set_density(h, 0, 0, d_in[0]["rho"], d_in[0]["bc_rho"], d_in[0]["bc_phi"])
                for l in range(1, H.num_levels):
                    mg.mg_set_density(h, 0, l, d_in[l]["rho"])
                return mg.mg_solve(h, 1)[1]

            for _ in range(args.warmup):
                st = step()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                ev0.record()
                st = step()
                ev1.record()
                torch.cuda.synchronize()
                ms.append(ev0.elapsed_time(ev1))
            ep = ef = 0.0
            for l in range(H.num_levels):
                X = H.centres(l, 0)
                pa, fa = H.potential(X), H.force(X)
                ep = max(ep, float(np.max(np.abs(P[l].cpu().numpy() - pa)) / np.max(np.abs(pa))))
                ef = max(ef, float(np.max(np.abs(np.moveaxis(F[l].cpu().numpy(), 0, -1) - fa)) / np.max(np.abs(fa))))
            t = statistics.median(ms)
            print(json.dumps({"case": f"{H.num_levels} nested {n}^3 levels, 8 spheres", "form": name, "zones": H.zones(),
                              "ms_per_solve": t, "zones_per_s": H.zones() / (t * 1e-3),
                              "cycles_per_level": [st[0][l]["cycles"] for l in range(H.num_levels)],
                              "max_rel_res": max(st[0][l]["rel_res"] for l in range(H.num_levels)),
                              "max_rel_err_phi": ep, "max_rel_err_F": ef,
                              "timing": "CUDA events around set_density + mg_solve (writing potential and forces), "
                                        "median"}), flush=True)
        finally:
            mg.mg_destroy(h)


def run_box_case(args):
    """Box (non-cubic) patches: 3 nested patches of 512 x 256 x 256 cells (each
    halving the box [-1,1] x [-0.5,0.5]^2 about its centre) around the offset
    compact sphere; V(2,2) to 1e-10, FP64 and mixed, through include/mg_box.h.
    One line per form (zones/s of set_density + solve + forces, CUDA events;
    max errors against the closed form; cycles), then the finest multigrid
    level's colour pass timed back to back (DRAM-resident: 514 x 258 x 258
    cells per array) against the measured HBM bandwidth."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    n = tuple(int(v) for v in args.box_n.split("x"))
    H = I.box_3d_sphere(n=n, levels=3)
    inp = I.level_inputs(H)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_in = [{k: dev(v) for k, v in d.items()} for d in inp]
    shape = tuple(reversed(n))
    F = [torch.empty((3,) + shape, dtype=torch.float64, device="cuda") for _ in range(H.num_levels)]
    P = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(H.num_levels)]
    peak, peak_src = measured_peaks("hbm_gbs")
    for name, prec in (("fp64", mg.MG_FP64), ("mixed", mg.MG_MIXED)):
        b = mg.mg_box_create(mg.box_desc_from(H), mg.options(nu_pre=NU[0], nu_post=NU[1], max_cycles=60,
                                                             rel_tol=TOL, precision=prec,
                                                             inner_cycles=args.inner_cycles,
                                                             inner_max=args.inner_max))
        try:
            def step():
                mg.mg_box_set_density(b, 0, d_in[0]["rho"], d_in[0]["bc_rho"], d_in[0]["bc_phi"])
                for l in range(1, H.num_levels):
                    mg.mg_box_set_density(b, l, d_in[l]["rho"])
                st = mg.mg_box_solve(b, H.num_levels)[1]
                for l in range(H.num_levels):
                    mg.mg_box_forces(b, l, P[l], F[l])
                return st

            for _ in range(args.warmup):
                st = step()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                ev0.record()
                st = step()
                ev1.record()
                torch.cuda.synchronize()
                ms.append(ev0.elapsed_time(ev1))
            ep = ef = 0.0
            for l in range(H.num_levels):
                X = H.centres(l, 0)
                pa, fa = H.potential(X), H.force(X)
                ep = max(ep, float(np.max(np.abs(P[l].cpu().numpy() - pa)) / np.max(np.abs(pa))))
                ef = max(ef, float(np.max(np.abs(np.moveaxis(F[l].cpu().numpy(), 0, -1) - fa)) / np.max(np.abs(fa))))
            t = statistics.median(ms)
            us, by = mg.mg_box_time_smoothing(b, 0, 0, args.launches)
            print(json.dumps({"case": f"3 nested box patches of {'x'.join(map(str, n))} cells, offset sphere",
                              "form": name, "zones": H.zones(), "ms_per_solve": t,
                              "zones_per_s": H.zones() / (t * 1e-3),
                              "cycles_per_patch": [s["cycles"] for s in st],
                              "outer_steps_per_patch": [s["outer_steps"] for s in st],
                              "max_rel_res": max(s["rel_res"] for s in st),
                              "max_rel_err_phi": ep, "max_rel_err_F": ef,
                              "timing": "CUDA events around set_density + mg_box_solve + mg_box_forces, median",
                              "finest_colour_pass": {"us": us, "bytes": by, "GBps": by / (us * 1e-6) / 1e9,
                                                     "frac": by / (us * 1e-6) / 1e9 / peak,
                                                     "peak_GBps": peak, "peak_source": peak_src,
                                                     "byte_model": "1.5 words per cell (Phi read once, its "
                                                                   "colour written, f of the colour read)",
                                                     "timing": f"{args.launches} back-to-back launches, "
                                                               "CUDA events"}}), flush=True)
        finally:
            mg.mg_box_destroy(b)


def run_box_smoothing_case(args):
    """The finest multigrid level's FP32 colour pass of a box patch
    (--box-n cells; mixed-precision storage) timed alone, `--launches`
    back-to-back launches: a short command for profiler captures."""
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    n = tuple(int(v) for v in args.box_n.split("x"))
    H = I.box_3d_sphere(n=n, levels=1)
    b = mg.mg_box_create(mg.box_desc_from(H), mg.options(precision=mg.MG_MIXED))
    try:
        us, by = mg.mg_box_time_smoothing(b, 0, 0, args.launches)
        peak, src = measured_peaks("hbm_gbs")
        print(json.dumps({"case": f"box patch {args.box_n}, finest FP32 colour pass", "us": us, "bytes": by,
                          "GBps": by / (us * 1e-6) / 1e9, "frac": by / (us * 1e-6) / 1e9 / peak,
                          "peak_source": src, "launches": args.launches}), flush=True)
    finally:
        mg.mg_box_destroy(b)


def run_unet_case(args):
    """The learned guess's 3D U-Net on a batch of 4 samples of 64^3: one
    forward pass and one training step (forward, backward, AdamW) timed with
    CUDA events; FLOPs counted from the architecture (2 x 27 x C_in x C_out
    per output voxel of every 3x3x3 convolution; the backward pass counts
    twice that: data and weight gradients).  Prints one line, not the
    benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import unet as U
    n, B = 64, 4
    # (C_in, C_out, resolution divisor) of the nine convolutions
    convs = [(3, 16, 1), (16, 16, 1), (16, 32, 2), (32, 32, 2), (32, 64, 4), (64, 64, 8), (128, 32, 4), (64, 16, 2),
             (32, 16, 1)]
    fwd = sum(2.0 * 27 * ci * co * B * (n // dv) ** 3 for ci, co, dv in convs)
    rng = np.random.default_rng(I.BASE_SEED + 64)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rho, phi, res, tru = (dev(rng.standard_normal((B, n, n, n))) for _ in range(4))
    frho = np.full(B, 1e-3)
    u = U.mg_unet_create(n, B, seed=3)
    try:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = {}
        for name, fn, flops in (("forward", lambda: U.mg_unet_forward(u, B, n, rho, phi, res, frho), fwd),
                                ("train_step", lambda: U.mg_unet_train_step(u, B, n, rho, phi, res, tru, frho,
                                                                           lr=1e-4), 3 * fwd)):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                ev0.record()
                fn()
                ev1.record()
                torch.cuda.synchronize()
                ms.append(ev0.elapsed_time(ev1))
            t = statistics.median(ms)
            out[name] = {"ms": t, "tflops": flops / (t * 1e-3) / 1e12}
        peak, src = measured_peaks(key="bf16_tflops")
        print(json.dumps({"case": f"U-Net, batch {B} x {n}^3", "conv_flops_forward": fwd, **out,
                          "bf16_peak_tflops": peak, "peak_source": src,
                          "note": "times include host<->device copies of y / loss made by these calls"}))
    finally:
        U.mg_unet_destroy(u)


def run_2d_case(args):
    """2D workloads: 3 nested 64^2 levels (density (1 - r^2/0.25)^4, closed-form
    outer boundary, V(2,2)) and the model of Sec. 3.1 at N = 1024 (4 levels,
    V(2,1)); FP64 and mixed, solved to 1e-10 with forces.  Prints one line per
    workload and form (zones/s of set_density + solve + forces, CUDA events,
    median), not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import mg
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for H, nu in ((I.config_2d_disk(64, 3), (2, 2)), (I.paper_2d(1024), (2, 1))):
        inp = I.level_inputs(H)
        d = [{k: dev(v) for k, v in x.items()} for x in inp]
        F = [torch.empty((2, n, n), dtype=torch.float64, device="cuda") for n in H.n]
        for name, prec in (("fp64", mg.MG_FP64), ("mixed", mg.MG_MIXED)):
            h = mg.mg_create_hierarchy([mg.desc_from(H)], mg.options(nu_pre=nu[0], nu_post=nu[1], max_cycles=60,
                                                                     rel_tol=TOL, precision=prec,
                                                                     inner_cycles=args.inner_cycles,
                                                                     inner_max=args.inner_max))
            try:
                if prec == mg.MG_MIXED:
                    mg.mg_autotune(h, args.tune_cache)

                for l in range(H.num_levels):
                    mg.mg_set_outputs(h, 0, l, None, F[l])

                def step():
                    mg.mg_set_density(h, 0, 0, d[0]["rho"], d[0]["bc_rho"], d[0]["bc_phi"])
                    for l in range(1, H.num_levels):
                        mg.mg_set_density(h, 0, l, d[l]["rho"])
                    return mg.mg_solve(h, 1)[1]

                for _ in range(args.warmup):
                    st = step()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ms = []
                for _ in range(args.steps):
                    torch.cuda.synchronize()
                    ev0.record()
                    st = step()
                    ev1.record()
                    torch.cuda.synchronize()
                    ms.append(ev0.elapsed_time(ev1))
                t = statistics.median(ms)
                print(json.dumps({"case": H.name, "form": name, "zones": H.zones(), "ms_per_solve": t,
                                  "zones_per_s": H.zones() / (t * 1e-3),
                                  "cycles_per_level": [st[0][l]["cycles"] for l in range(H.num_levels)],
                                  "max_rel_res": max(st[0][l]["rel_res"] for l in range(H.num_levels))}), flush=True)
            finally:
                mg.mg_destroy(h)


def run_learned_case(args):
    """The learned initial guess end to end: training samples generated by the
    solver (hierarchies of 64^3 levels with 1-8 random compact spheres), the
    network trained on them, then V-cycles, wall time and difference from the
    zero-guess solution with the zero, interpolated and learned guesses on
    held-out hierarchies of 3 levels of 64^3 and of 128^3.  Prints one line,
    not the benchmark record."""
    import torch
    from paper_2001_02327_gb300 import build
    build.build()
    from paper_2001_02327_gb300 import learned as LR
    from paper_2001_02327_gb300 import unet as U
    t0 = time.perf_counter()
    train = LR.make_samples(torch, args.samples, n=64, seed0=1000)
    val = LR.make_samples(torch, 32, n=64, seed0=90000)
    t_gen = time.perf_counter() - t0
    net = U.mg_unet_create(64, 4, seed=1)
    nets = []
    try:
        v0 = LR.validation_loss(torch, net, val)
        t0 = time.perf_counter()
        losses = LR.train(torch, net, train, steps=args.train_steps, batch=4, lr=1e-3)
        t_train = time.perf_counter() - t0
        v1 = LR.validation_loss(torch, net, val)
        p = U.mg_unet_get_params(net)
        out = {"case": "learned initial guess", "samples": args.samples, "train_steps": args.train_steps,
               "gen_s": t_gen, "train_s": t_train, "val_loss_before": v0, "val_loss_after": v1,
               "train_loss_last50": float(np.mean(losses[-50:]))}
        for n, count, seed in ((64, 4, 200000), (128, 2, 300000)):
            e = U.mg_unet_create(n, 1, seed=0)
            nets.append(e)
            U.mg_unet_set_params(e, p)
            out[f"eval_{n}"] = LR.evaluate(torch, e, [LR.random_nested(seed + k, n, 3) for k in range(count)])
        print(json.dumps(out), flush=True)
    finally:
        for e in [net] + nets:
            U.mg_unet_destroy(e)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="leave out the mixed + learned-guess form")
    ap.add_argument("--no-scale", action="store_true", help="leave out the 4x256^3 DRAM-resident workload")
    ap.add_argument("--no-batch", action="store_true", help="leave out the 512-hierarchy batches")
    ap.add_argument("--inner-cycles", type=int, default=3,
                    help="mixed forms: FP32 V-cycles of the first defect-correction step (of every step "
                         "with --inner-max 0)")
    ap.add_argument("--inner-max", type=int, default=8,
                    help="mixed forms: cap of the FP32 V-cycles each defect-correction step after the first "
                         "may choose (0: three in every step)")
    ap.add_argument("--forces-call", action="store_true",
                    help="results through one mg_forces call per level after mg_solve instead of the outputs "
                         "mg_solve fills itself (mg_set_outputs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch plan (a fixed plan for profiler captures)")
    ap.add_argument("--samples", type=int, default=256, help="learned case: training samples")
    ap.add_argument("--train-steps", type=int, default=1500, help="learned case: training steps")
    ap.add_argument("--launches", type=int, default=4, help="smoothing case: launches per timing")
    ap.add_argument("--case", default="bench",
                    choices=["bench", "level", "smoothing", "batch", "scale", "unet", "learned", "2d", "box",
                             "box_smoothing"],
                    help="level: one DRAM-resident 3D level for profiler captures; batch: uneven hierarchies")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--box-n", default="512x256x256", help="box case: cells per axis of each patch")
    ap.add_argument("--batch-edges", default="", help="batch case: cells per edge to draw from, e.g. 16,24,32")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--level-n", type=int, default=254)
    ap.add_argument("--forms", default="fp64,mixed", help="scale case: the forms to run, from fp64,mixed")
    ap.add_argument("--scale-levels", type=int, default=4, help="scale case: nested levels (4: the workload)")
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--tune-cache", default=None,
                    help="file for the mixed form's launch plan: read if present, written after tuning")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.case == "level":
        run_level_case(args)
    elif args.case == "smoothing":
        run_smoothing_case(args)
    elif args.case == "batch":
        run_batch_case(args)
    elif args.case == "scale":
        run_scale_case(args)
    elif args.case == "unet":
        run_unet_case(args)
    elif args.case == "learned":
        run_learned_case(args)
    elif args.case == "2d":
        run_2d_case(args)
    elif args.case == "box":
        run_box_case(args)
    elif args.case == "box_smoothing":
        run_box_smoothing_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
