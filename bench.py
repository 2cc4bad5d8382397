"""Benchmark: batched 3D E,T,pH-REMD C(pH,E)MD steps on one GB300.

Workload (one "step" = one step of the full schedule for every walker: Born
radii, GB + Coulomb + LJ pair pass, chain rule + bonded terms, Langevin; MC
sweeps every 10 steps, one exchange attempt every 100): 8 E x 6 T x 8 pH = 384
replicas over three seeded synthetic systems of 500, 2000 and 8000 atoms
(128 replicas each), FP32 pair arithmetic with int64 fixed-point accumulation.

Metric: aggregate replica-steps/s (and unordered GB pair-evaluations/s through
all three pair passes), batched launch; the same steps issued as per-replica
launches are timed beside it, over the same step indices.  The timed window
is placed on the schedule so that it holds an exchange step (and MC steps in
their proportion): whole 100-step periods when K is a multiple of 100, else
the K steps around step 100; the line reports which events it held.  Smaller
legs: the 160-atom single replica (FP64), 8 x 160 E-REMD and 64 x 2400
E,pH-REMD workloads, each through the C ABI from host buffers.  One JSON line
on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the ranks share the one 384-replica grid: each
advances a load-balanced part of its walkers on its own GPU, and at every
exchange step the 40-byte per-walker exchange rows are all-gathered over NCCL
and every rank runs the same exchange attempt (paper_1809_07726_gb300/shard.py).
The value is the grid's replica-steps over the max-over-ranks time (strong
scaling: the total work is fixed).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aggregate replica-steps/s & GB pair evals/s, batched vs per-replica launches"
WORKLOAD = "3D E,T,pH-REMD: 8 E x 6 T x 8 pH = 384 replicas over 500/2000/8000-atom systems"
# Algorithmic cost of one unordered pair in each pass, counted from the forms
# the method evaluates for a far pair (r >= r_far: the HCT series; over 99 % of
# the pairs here): FP32 lane operations (an FMA counts once) and MUFU
# operations (rsqrt, rcp, ex2).  born: distance 6, 1/r^4 from 1/r^2 (one rcp) 1,
# two series terms (y, P, s^3) 14, r^-4-weighted fused sums 2; gb: distance 6, GB kernel and dE/dR 18, LJ 9, Coulomb 2,
# force and partner force 6 (minus fused products), 3 MUFU; chain: distance 6,
# powers 2 (1/r^2 from one rcp), two dH/dr series 12, weights 5, forces 6.
PASS_COST = {"born": (23, 1), "gb": (40, 3), "chain": (31, 1)}
# A GB pair with D = r^2 / (4 R_i R_j) >= 18 needs no exponential and no second
# square root (1/f = 1/r and e^-D to FP32 precision): distance 6, D 2, LJ 9,
# charges and eps 2, combined GB + Coulomb force factor ((q_i q_j / r) / eps_out
# + LJ) / r^2 2, forces 6, 1 MUFU.
GB_FAR_COST = (27, 1)
GB_FAR_D = 18.0
# GB-energy backward (Born radii recomputed): born 23/1 + GB adjoint (energy,
# dE/dR, dE/dq, direct dE/dx) 32/2 + chain adjoint (dH/dr and dH/ds both ways,
# dH/drt = 0 far, r^-4-weighted fused s sums) 45/1
BACKWARD_COST = (100, 4)
# the same with the GB adjoint in its far form (1/f = 1/r: no exponential, no
# dE/dR term; 22 FP32 lane operations and 1 MUFU) for a pair with D >= 18
BACKWARD_FAR_COST = (90, 3)
N_SM = 152
# DRAM bytes (read + write) per launch of a pass's pair kernel, from one
# one-kernel ncu capture of each current kernel on this workload
PASS_DRAM_BYTES = {"born": 32.95e6 + 0.0, "gb": 89.23e6 + 6.39e6, "chain": 59.84e6 + 0.06e6}
FP32_LANES = 128   # FP32 lane operations per clock per SM
MUFU_LANES = 16    # MUFU operations per clock per SM


def clk_per_pair_per_sm(fp32, mufu):
    """The FP32 (FMA) pipe and the MUFU pipe work in parallel; packed f32x2
    instructions keep issue slots off the critical path, so a pass needs
    max(fp32 / 128, mufu / 16) SM clocks per pair."""
    return max(fp32 / FP32_LANES, mufu / MUFU_LANES)


def pairs_per_clk_per_sm(fp32, mufu):
    return 1.0 / clk_per_pair_per_sm(fp32, mufu)


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, and the
    clocks-event reasons bit mask) for one device, found by PCI bus id when
    torch reports it, else by index.  Unavailable -> ok is False."""
    SM = 1  # NVML_CLOCK_SM
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, pci, idx):
        import ctypes
        self.c = ctypes
        self.ok = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            rc = lib.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(h)) if pci else 1
            if rc != 0 and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) != 0:
                return
            try:
                self.reasons_fn = lib.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:
                self.reasons_fn = lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.lib, self.h, self.ok = lib, h, True
        except (OSError, AttributeError):
            self.ok = False

    def max_sm(self):
        v = self.c.c_uint()
        return float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, self.c.byref(v)) == 0 else None

    def sample(self):
        v, r = self.c.c_uint(), self.c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.c.byref(v)) != 0:
            return None
        bits = r.value if self.reasons_fn(self.h, self.c.byref(r)) == 0 else 0
        return float(v.value), {nm for b, nm in self.BITS.items() if bits & b}


def _pci_bus_id(dev):
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:  # older torch without the PCI fields, or no GPU
        return None


class ClockSampler:
    """Clocks and throttle reasons sampled during the timed region: nvidia-smi
    every 100 ms (the recipe's query) and NVML every 10 ms in a thread, so a
    window of a few hundred ms still holds tens of samples.  The median SM
    clock is taken over the NVML samples when there are any."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NVML_PERIOD_S = 0.010

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.pci = _pci_bus_id(gpu_index)
        self.proc = None
        self.lines = []
        self.nv_sm, self.nv_reasons, self.nv_max = [], set(), None
        self.stop = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        self.nvml = _Nvml(self.pci, self.idx)
        if self.nvml.ok:
            self.nv_max = self.nvml.max_sm()
            self.tn = threading.Thread(target=self._poll, daemon=True)
            self.tn.start()
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def _poll(self):
        while not self.stop.wait(self.NVML_PERIOD_S):
            s = self.nvml.sample()
            if s:
                self.nv_sm.append(s[0])
                self.nv_reasons |= s[1]

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml.ok:
            self.tn.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set(self.nv_reasons)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        src = self.nv_sm or sm
        if not src:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(src), "sm_max_mhz": mx or self.nv_max, "reasons": sorted(reasons),
                "samples": len(src), "sampler": "nvml 10 ms" if self.nv_sm else "nvidia-smi 100 ms",
                "nvidia_smi_samples": len(sm),
                "nvidia_smi_sm_mhz": statistics.median(sm) if sm else None}


def workload():
    from paper_1809_07726_gb300 import synth
    return synth.config_c4()


def gb_far_fraction(eng, systems, grid, samples=200000, seed=0, walkers=None):
    """Fraction of the workload's unordered pairs with D >= GB_FAR_D, from the
    engine's current positions and Born radii (one walker per system, random
    pairs), weighted by each system's pair count over the grid (or over the
    given walkers, the ones this engine advances)."""
    rng = np.random.default_rng(seed)
    x_all, r_all = eng.positions(), eng.born_radii()
    sos = np.asarray(grid.system_of_slot)
    if walkers is not None:
        keep = np.zeros(len(sos), bool)
        keep[np.asarray(walkers)] = True
        sos = np.where(keep, sos, -1)
    num = den = 0.0
    for s in np.unique(sos[sos >= 0]):
        w = int(np.nonzero(sos == s)[0][0])  # the first walker of system s
        sl = eng.walker_slice(w)
        x, R = x_all[sl], r_all[sl]
        n = len(R)
        if n < 2:
            continue
        i = rng.integers(0, n, samples)
        j = rng.integers(0, n, samples)
        keep = i != j
        i, j = i[keep], j[keep]
        D = ((x[i] - x[j]) ** 2).sum(1) / (4.0 * R[i] * R[j])
        pairs = n * (n - 1) / 2 * np.count_nonzero(sos == s)
        num += pairs * float((D >= GB_FAR_D).mean())
        den += pairs
    return num / den if den else 0.0


def pass_clk(name, gb_far=0.0):
    """SM clocks per unordered pair of a pass at its algorithmic cost; the GB
    pass mixes the far form (fraction gb_far of the pairs) with the full one."""
    if name == "gb":
        return gb_far * clk_per_pair_per_sm(*GB_FAR_COST) + (1.0 - gb_far) * clk_per_pair_per_sm(*PASS_COST["gb"])
    return clk_per_pair_per_sm(*PASS_COST[name])


def pair_count(systems, grid):
    n = [systems[s].n for s in grid.system_of_slot]
    return sum(k * (k - 1) // 2 for k in n)


def aggregate_max(t_local, world, device=None):
    """Max over ranks of a per-rank time (all ranks call it)."""
    if world == 1:
        return t_local
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = "cpu"
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(grid_walkers, steps, t_max):
    """Replica-steps of the whole grid (every rank's share of it) over the
    slowest rank's time."""
    return grid_walkers * steps / t_max


def schedule_launches(t, mc_ph=10, mc_redox=10, ex_every=100):
    """Kernels one batched FP32 step t launches through a one-step cph_run:
    position staging + Born-radii pair kernel + finish, GB staging + pair
    kernel + finish, chain pair kernel + bonded terms + force finish,
    observables, Langevin, the step-counter tick; each MC sweep kind adds the
    staging of its charges and radii and its per-site and per-walker kernels,
    an exchange step its row and attempt kernels."""
    n = 3 + 3 + 3 + 1 + 1 + 1
    if t > 0:
        n += 3 * (int(t % mc_ph == 0) + int(t % mc_redox == 0)) + 2 * int(t % ex_every == 0)
    return n


def window_start(steps, warmup, period=100):
    """First step of the timed window: whole schedule periods (from step
    period + 1, after the warm-up steps) when K is a multiple of the exchange
    period, else the K steps around the first exchange step, so the window
    holds an exchange attempt and MC steps in their proportion."""
    if steps % period == 0:
        return period * (1 + warmup // period) + 1
    return max(warmup + 1, period - steps // 2 + 1)


def schedule_events(first, steps, mc_ph=10, mc_redox=10, ex_every=100):
    """MC and exchange events of steps first .. first + steps - 1."""
    ts = range(first, first + steps)
    return {"first_step": first, "last_step": first + steps - 1,
            "mc_ph_steps": sum(1 for t in ts if t > 0 and t % mc_ph == 0),
            "mc_redox_steps": sum(1 for t in ts if t > 0 and t % mc_redox == 0),
            "exchange_steps": sum(1 for t in ts if t > 0 and t % ex_every == 0)}


# ----------------------------------------------------------------- oracle arm

def oracle_sample(systems, grid, walkers, n_steps, seed, threads=1, t0=1):
    """Time the FP64 oracle (as it stands) on ``walkers`` for n_steps of the
    schedule from step t0, its walkers spread over ``threads`` host threads
    (the oracle's C routines release the interpreter lock); returns (seconds,
    unordered pairs processed)."""
    import oracle
    W = oracle.Walkers(systems, grid, seed=seed)
    W.t = t0
    W.threads = threads
    t = time.perf_counter()
    oracle.run_schedule(W, n_steps, walkers=walkers)
    dt = time.perf_counter() - t
    pairs = sum(systems[grid.system_of_slot[w]].n * (systems[grid.system_of_slot[w]].n - 1) // 2
                for w in walkers) * n_steps
    return dt, pairs


def c4_oracle_walkers(grid, per_system):
    """``per_system`` walkers of each system of the 3D workload, largest
    system first (the workload holds equally many walkers of each system, so
    the sample has the workload's mix)."""
    sos = np.asarray(grid.system_of_slot)
    out = []
    for s in sorted(np.unique(sos), reverse=True):
        out += [int(w) for w in np.nonzero(sos == s)[0][:per_system]]
    return out


def host_cores():
    return os.cpu_count() or 1


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores.  Each step is a
    bounded sample of the 3D workload: one schedule step (step 1, an MD step)
    of k walkers of each of the three systems, k = the host's core count, on
    that many threads; the sample has the workload's mix, so its
    replica-steps per second are the workload's at this core count."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    systems, grid = workload()
    ncores = host_cores()
    k = min(ncores, 128)
    sample = c4_oracle_walkers(grid, k)
    for _ in range(args.warmup):
        oracle_sample(systems, grid, sample, 1, seed=4, threads=ncores)
    secs = 0.0
    pairs = 0
    for _ in range(args.steps):
        dt, p = oracle_sample(systems, grid, sample, 1, seed=4, threads=ncores)
        secs += dt
        pairs += p
    value = len(sample) * args.steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "replica-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "replicas_per_step": len(sample),
                       "parallelism": f"cpu oracle, {ncores} threads"},
            "pair_evals_per_s": pairs / secs,
            "cpu_baseline": {"value": value, "unit": "replica-steps/s", "cores": ncores, "kind": "oracle",
                             "sample": f"per step: one MD step (step 1) of {k} walkers of each of the "
                                       f"500/2000/8000-atom systems ({len(sample)} walkers, the "
                                       "workload's mix) on all host cores; measured, not scaled"},
            "e2e": {"value": value, "unit": "replica-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU arm

def backward_leg(dev, stream, barrier, sm_mhz, n_eval=5):
    """a9: GB-energy backward w.r.t. x, q, rho for 128 replicas of an 8000-atom
    system (Born radii recomputed), CUDA events on the launching stream."""
    import torch

    from paper_1809_07726_gb300 import cphremd, synth
    s5, x5, q5, rho5 = synth.config_c5()
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    xt, qt, rt, st5 = f32(x5), f32(q5), f32(rho5), f32(s5.screen)
    ws = cphremd._workspace(q5.shape[0], q5.shape[1], dev)
    up = torch.ones(q5.shape[0], dtype=torch.float64, device=dev)
    for _ in range(2):
        cphremd.gb_energy_backward(xt, qt, rt, st5, up, workspace=ws)
    barrier()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(n_eval):
        cphremd.gb_energy_backward(xt, qt, rt, st5, up, workspace=ws)
    b1.record(stream)
    barrier()
    bw_ms = b0.elapsed_time(b1) / n_eval
    bw_pairs = q5.shape[0] * q5.shape[1] * (q5.shape[1] - 1) // 2
    bw_achieved = bw_pairs / (bw_ms / 1e3) / 1e9
    # far-form share of the pairs, from the engine's Born radii of replica 0
    import copy
    s0 = copy.deepcopy(s5)
    s0.x = np.ascontiguousarray(x5[0], dtype=np.float64).reshape(-1, 3)
    s0.rho = np.asarray(rho5[0], dtype=np.float64)
    s0.q = np.asarray(q5[0], dtype=np.float64)
    g0 = synth.Grid(np.array([0.0]), np.array([7.0]), np.array([300.0]), np.zeros(1, np.int32))
    e0 = cphremd.init_system([s0], g0, seed=1)
    e0.evaluate()
    far = gb_far_fraction(e0, [s0], g0)
    clk = far * clk_per_pair_per_sm(*BACKWARD_FAR_COST) + (1.0 - far) * clk_per_pair_per_sm(*BACKWARD_COST)
    bw_peak = N_SM * (sm_mhz or 2070.0) * 1e6 / clk / 1e9
    return {"workload": "GB energy backward w.r.t. x, q, rho: 128 replicas x 8000 atoms",
            "ms_per_eval": bw_ms, "evals_per_s": q5.shape[0] / (bw_ms / 1e3),
            "pair_evals_per_s": bw_pairs / (bw_ms / 1e3),
            "roofline": {"bound": "alu", "achieved": bw_achieved, "peak": bw_peak,
                         "unit": "Gpair/s", "frac": bw_achieved / bw_peak,
                         "algorithmic_cost": {"full": list(BACKWARD_COST), "gb_far": list(BACKWARD_FAR_COST),
                                              "gb_far_fraction": far}}}


def timed_window(eng, stream, flush, first, steps, warmup):
    """Run eng to step first - warmup, then warmup steps, then time ``steps``
    steps one cph_run(1) each with CUDA events on the launching stream and an
    L2 flush write before every timed step.  Returns the per-step ms list."""
    import torch
    t = eng.get_step()
    if t < first - warmup:
        eng.run(first - warmup - t)
    eng.run(warmup)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        eng.run(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def config_leg(name, cfg, precision, n_steps, dev, stream, sm_mhz, oracle_plan=None):
    """One of the smaller workloads through the public API: device time of
    n_steps of cph_run (CUDA events) after a few warm-up steps, and end to end
    from host buffers (init_system uploads the systems, run, then the final
    positions and energies are read back) in wall time.  oracle_plan = a list
    of (walkers, steps, threads) samples of the FP64 oracle to time."""
    import torch

    from paper_1809_07726_gb300 import cphremd
    systems, grid = cfg()
    W = grid.n_slots
    pairs_step = pair_count(systems, grid)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    eng = cphremd.init_system(systems, grid, seed=7, precision=precision)
    eng.autotune()
    eng.run(n_steps)
    x = eng.positions()
    e = eng.energies()
    e2e_s = time.perf_counter() - w0
    h2d = sum(s.n * (3 * 8 + 7 * 8) for s in systems) + sum(systems[s].n * 3 * 8 for s in grid.system_of_slot)
    d2h = x.nbytes + e.nbytes
    # device time of n_steps on an engine warmed by a few schedule periods
    # (graphs captured, caches warm)
    eng2 = cphremd.init_system(systems, grid, seed=7, precision=precision)
    chunk = eng2.autotune()
    shapes = ["symmetric" if v == cphremd.SHAPE_SYMMETRIC else "warp per atom" for v in eng2.tile_shapes()]
    eng2.run(min(n_steps, 201))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = eng2.get_step()
    a.record(stream)
    eng2.run(n_steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    eng2.status()
    out = {"workload": name, "replicas": W, "atoms": [s.n for s in systems],
           "precision": "FP64" if precision == cphremd.PREC_FP64 else "FP32 pair math, int64 fixed point",
           "autotuned_chunk_jtiles": chunk, "tile_shapes": shapes,
           "steps": n_steps, "steps_timed_from": c0, "ms_per_step": ms / n_steps,
           "value": W * n_steps / (ms / 1e3), "unit": "replica-steps/s",
           "pair_evals_per_s": pairs_step * n_steps / (ms / 1e3),
           "e2e": {"value": W * n_steps / e2e_s, "unit": "replica-steps/s", "seconds": e2e_s,
                   "h2d_bytes": h2d, "d2h_bytes": d2h,
                   "includes": "init_system from host buffers, autotune, run, read back positions "
                               "and energies"}}
    if precision == cphremd.PREC_FP32:
        far = gb_far_fraction(eng2, systems, grid)
        step_peak = N_SM * (sm_mhz or 2070.0) * 1e6 / sum(pass_clk(n, far) for n in ("born", "gb", "chain"))
        pass_ms = eng2.time_passes(reps=3)
        out["pass_ms"] = [float(v) for v in pass_ms]
        out["roofline"] = {"bound": "alu", "unit": "Gpair/s",
                           "achieved": pairs_step / (sum(pass_ms) / 1e3) / 1e9,
                           "peak": step_peak / 1e9,
                           "frac": (pairs_step / (sum(pass_ms) / 1e3)) / step_peak,
                           "basis": "three pair passes against the step roofline (FP32 lanes, MUFU)"}
    else:
        out["roofline"] = {"bound": "latency",
                           "note": "FP64 mode, one small system: a step is ~10 dependent launches "
                                   "of a few microseconds each"}
    del eng, eng2
    if oracle_plan is not None:
        # plans: (walkers, steps, threads); the first is the leg's cpu_baseline,
        # the others are the same workload at another core count
        runs = []
        for ws, n, threads in oracle_plan:
            secs, pairs = oracle_sample(systems, grid, ws, n, seed=7, threads=threads, t0=1)
            ev = schedule_events(1, n)
            runs.append({"value": len(ws) * n / secs, "unit": "replica-steps/s", "cores": threads,
                         "kind": "oracle", "seconds": secs,
                         "sample": f"{n} schedule steps (steps 1-{n}, {ev['mc_ph_steps']} of them with MC "
                                   f"sweeps) of {len(ws)} walker(s) on {threads} thread(s); measured"})
        out["cpu_baseline"] = runs[0]
        if len(runs) > 1:
            out["cpu_baseline"]["other_core_counts"] = runs[1:]
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1809_07726_gb300 import build, cphremd, shard, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # NCCL between GPUs; CPH_BENCH_DIST_BACKEND=gloo runs the same sharded
        # path with host collectives (several ranks may then share a device)
        dist.init_process_group(os.environ.get("CPH_BENCH_DIST_BACKEND", "nccl"))
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    systems, grid = workload()
    total_pairs = pair_count(systems, grid)
    W = grid.n_slots
    seed = 4
    sharded = world > 1
    parts = shard.partition([s.n for s in systems], grid.system_of_slot, world)
    mine = parts[rank]
    local_pairs = sum(systems[grid.system_of_slot[w]].n * (systems[grid.system_of_slot[w]].n - 1) // 2
                      for w in mine)

    def make_engine():
        e = cphremd.init_system(systems, grid, seed=seed)
        if not sharded:
            return e, e.run
        e.set_local_walkers(mine)
        drv = shard.ShardedRun(e, shard.torch_allgather(), 10, 10, 100)
        return e, drv.run

    eng, advance = make_engine()
    # L2 flush buffer (256 MB > 129 MB L2), written before every timed step
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    chunk = eng.autotune()  # tile shapes for this workload (outside the timed region)
    shapes = ["symmetric" if v == cphremd.SHAPE_SYMMETRIC else "warp per atom" for v in eng.tile_shapes()]
    first = window_start(args.steps, args.warmup)
    events = schedule_events(first, args.steps)
    advance(1)  # step 0
    advance(first - args.warmup - 1)  # to the warm-up steps (window_start leaves room)
    ck = eng.get_state()  # the per-replica runs restart from here: same steps, same work
    advance(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    t_first = eng.get_step()
    assert t_first == first
    with ClockSampler(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            advance(1)
            ends[k].record(stream)
            launches += schedule_launches(t_first + k)
        barrier()
        wall = time.perf_counter() - wall0
    eng.status()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(ms) / 1e3
    t_max = aggregate_max(t_local, world, dev)
    value = whole_job_value(W, args.steps, t_max)
    clocks = clk.summary()
    ms_step = 1e3 * t_max / args.steps

    # graph replay of whole schedule periods (no flush between steps); a
    # sharded engine leaves its exchange steps to the host driver
    period = 100
    graph_ms = None
    if not sharded:
        while eng.get_step() % period != 1:
            eng.run(1)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        eng.run(period)
        g1.record(stream)
        barrier()
        graph_ms = g0.elapsed_time(g1) / period

    # dominant pair pass: CUDA events around each pass on the launching stream
    pass_ms = eng.time_passes(reps=3)
    # per-SM pipe rates behind the roofline, measured on this GPU at its current clock
    fp32_rate, mufu_rate = cphremd.probe_pipe_rates()
    names = ["born", "gb", "chain"]
    dom = int(np.argmax(pass_ms))
    f_mhz = clocks["sm_mhz"] or 2070.0
    gb_far = gb_far_fraction(eng, systems, grid, walkers=mine)
    peak = N_SM * f_mhz * 1e6 / pass_clk(names[dom], gb_far) / 1e9
    achieved = local_pairs / (pass_ms[dom] / 1e3) / 1e9
    step_peak = N_SM * f_mhz * 1e6 / sum(pass_clk(n, gb_far) for n in names) / 1e9

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": value, "ms_per_step": ms_step,
                              "window": events, "pass_ms": [float(x) for x in pass_ms],
                              "clocks": clocks}), flush=True)
        return
    # the same steps as per-replica launches: restart from the checkpoint, same window
    pr_ms = pr8_ms = None
    pr_pass_ms = []
    if not sharded:
        eng.set_launch_mode(cphremd.LAUNCH_PER_REPLICA)
        eng.autotune()
        eng.set_state(ck)
        barrier()
        pr_ms = sum(timed_window(eng, stream, flush, first, args.steps, args.warmup)) / args.steps
        pr_pass_ms = eng.time_passes(reps=1)
        # and spread over 8 streams (as 8 processes per GPU would overlap)
        eng.set_replica_streams(8)
        eng.set_state(ck)
        barrier()
        pr8_ms = sum(timed_window(eng, stream, flush, first, args.steps, args.warmup)) / args.steps
    del eng

    # end to end through the public API from host buffers: init (H2D of the
    # systems) + per-step run and D2H of energies and the condition map
    barrier()
    e2e0 = time.perf_counter()
    e2, adv2 = make_engine()
    h2d = sum(s.n * (3 * 8 + 7 * 8) for s in systems) + sum(
        systems[s].n * 3 * 8 for s in grid.system_of_slot)
    n_e2e = args.steps
    d2h = 0
    for _ in range(n_e2e):
        adv2(1)
        e2.energies()
        e2.condition_map()
        d2h += W * 6 * 8 + W * 4
    barrier()
    e2e_s = aggregate_max(time.perf_counter() - e2e0, world, dev)
    e2e_value = W * n_e2e / e2e_s
    del e2

    backward = backward_leg(dev, stream, barrier if not sharded else torch.cuda.synchronize,
                            clocks["sm_mhz"]) if rank == 0 else None

    # the smaller workloads, each through the C ABI from host buffers
    ncores = host_cores()
    legs = {}
    if not args.no_legs:
        on_cpu = world == 1 and rank == 0
        # oracle samples: C1 whole (one walker: the oracle spreads walkers, not
        # atoms, over threads, so one core is all it uses); C2 on one core and
        # on one thread per walker; C3 on every core and one walker on one core
        legs["c1"] = config_leg("C(pH,E)MD, 1 replica of 160 atoms, FP64, 1000 steps", synth.config_c1,
                                cphremd.PREC_FP64, 1000, dev, stream, clocks["sm_mhz"],
                                [([0], 1000, 1)] if on_cpu else None)
        legs["c2"] = config_leg("1D E-REMD, 8 replicas of 160 atoms, FP32, 20000 steps", synth.config_c2,
                                cphremd.PREC_FP32, 20000, dev, stream, clocks["sm_mhz"],
                                [(list(range(8)), 200, 1), (list(range(8)), 200, min(8, ncores))]
                                if on_cpu else None)
        legs["c3"] = config_leg("2D E,pH-REMD, 64 replicas of 2400 atoms, FP32, 2000 steps", synth.config_c3,
                                cphremd.PREC_FP32, 2000, dev, stream, clocks["sm_mhz"],
                                [(list(range(min(ncores, 64))), 10, ncores), ([0], 2, 1)]
                                if on_cpu else None)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1:
        import oracle
        oracle.build()
        k = min(ncores, 128)
        sample = c4_oracle_walkers(grid, k)
        secs_all, pairs_all = oracle_sample(systems, grid, sample, 1, seed=seed, threads=ncores)
        one = c4_oracle_walkers(grid, 1)
        secs1, _ = oracle_sample(systems, grid, one, 1, seed=seed, threads=1)
        cpu = {"value": len(sample) / secs_all, "unit": "replica-steps/s", "cores": ncores, "kind": "oracle",
               "sample": f"one MD step (step 1) of {k} walkers of each of the 500/2000/8000-atom "
                         f"systems ({len(sample)} walkers, the workload's mix) on {ncores} threads, "
                         f"{secs_all:.1f} s; measured, not scaled",
               "one_core": {"value": len(one) / secs1, "cores": 1,
                            "sample": f"one MD step of one walker of each system, {secs1:.1f} s "
                                      "single-threaded"}}

    line = {
        "metric": METRIC, "value": value, "unit": "replica-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "replicas": W, "atoms": [s.n for s in systems],
                   "precision": "FP32 pair math, int64 fixed-point accumulation",
                   "schedule": "MC (pH then redox) every 10 steps, exchange every 100 (E,pH,T)",
                   "l2": "256 MB buffer written before every timed step",
                   "autotuned_chunk_jtiles": chunk, "autotuned_tile_shapes": shapes,
                   "parallelism": ("replicas batched per launch" if not sharded else
                                   f"one grid sharded by walker over {world} GPUs (rank 0: {len(mine)} "
                                   "walkers); exchange rows all-gathered over "
                                   f"{os.environ.get('CPH_BENCH_DIST_BACKEND', 'nccl')} at exchange steps")},
        "window": events,
        "pair_evals_per_s": total_pairs * args.steps / t_max,
        "per_replica": None if sharded else {
            "value": W / (pr_ms / 1e3), "unit": "replica-steps/s", "ms_per_step": pr_ms,
            "same_window": True, "pass_ms": [float(x) for x in pr_pass_ms],
            "speedup_batched": pr_ms / ms_step,
            "streams_8": {"value": W / (pr8_ms / 1e3), "ms_per_step": pr8_ms,
                          "speedup_batched": pr8_ms / ms_step}},
        "graph_replay": None if sharded else {"value": W / (graph_ms / 1e3), "unit": "replica-steps/s",
                                              "ms_per_step": graph_ms, "steps": period},
        "pass_ms": {n: float(x) for n, x in zip(names, pass_ms)},
        "roofline": {"bound": "alu", "kernel": f"k_{names[dom]}_sym", "achieved": achieved,
                     "peak": peak, "unit": "Gpair/s", "frac": achieved / peak, "traffic": PASS_DRAM_BYTES.get(names[dom]),
                     "traffic_basis": "DRAM read + write bytes per launch of the pass's pair kernel (ncu)",
                     "peak_basis": f"{N_SM} SM x {f_mhz:.0f} MHz (median sampled) / "
                                   f"{pass_clk(names[dom], gb_far):.4f} SM clocks per pair, a pair's form "
                                   "costing max(fp32/128, mufu/16) clocks (FP32 lanes, MUFU)",
                     "algorithmic_cost": {n: list(PASS_COST[n]) for n in names} | {
                         "gb_far": list(GB_FAR_COST), "gb_far_fraction": gb_far,
                         "gb_far_rule": f"D = r^2/(4 R_i R_j) >= {GB_FAR_D:g}"},
                     "step_frac": (total_pairs / (sum(pass_ms) / 1e3) / 1e9) / step_peak},
        "e2e": {"value": e2e_value, "unit": "replica-steps/s",
                "h2d_bytes_per_step": h2d / n_e2e, "d2h_bytes_per_step": d2h / n_e2e},
        "backward": backward,
        "configs": legs,
        "pipe_rates": {"fp32_lane_ops_per_clk_per_sm": fp32_rate / (N_SM * f_mhz * 1e6),
                       "mufu_ops_per_clk_per_sm": mufu_rate / (N_SM * f_mhz * 1e6),
                       "assumed": [FP32_LANES, MUFU_LANES],
                       "probe": "packed f32x2 FMA loop and rsqrt.approx loop, best of 3"},
        "gpu_launches": launches,
        "clocks": clocks | {"ms_x_mhz": ms_step * (clocks["sm_mhz"] or float("nan"))},
        "wall_s": wall,
    }
    if cpu:
        line["cpu_baseline"] = cpu
        # the differentiation workload's oracle: energy and analytic gradient of
        # one replica of the 8000-atom system, single-threaded, measured
        s5, x5, q5, rho5 = synth.config_c5(n_rep=1)
        t0 = time.perf_counter()
        oracle.gb_grad(x5[0], q5[0], rho5[0], s5.screen)
        secs5 = time.perf_counter() - t0
        if backward is not None:
            backward["cpu_baseline"] = {"value": 1.0 / secs5, "unit": "replica evaluations/s", "cores": 1,
                                        "kind": "oracle", "seconds": secs5,
                                        "sample": "E_GB and its x, q, rho gradient of one 8000-atom "
                                                  "replica, single-threaded; measured"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--leg", default="all", choices=["all", "backward"],
                    help="backward: time only the GB-energy backward leg (128 x 8000)")
    ap.add_argument("--quick", action="store_true",
                    help="batched timing only (no per-replica, e2e or CPU legs); for profiling")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the 160-atom and 2400-atom workload legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.leg == "backward":
        import torch
        torch.cuda.set_device(0)
        from paper_1809_07726_gb300 import build
        build.build()
        dev = torch.device("cuda", 0)
        print(json.dumps({"leg": "backward", **backward_leg(dev, torch.cuda.current_stream(dev),
                                                             torch.cuda.synchronize, None)}),
              flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
