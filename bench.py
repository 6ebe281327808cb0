#!/usr/bin/env python
"""Throughput of the noisy-QAOA MPDO hot path on GB300 through libmpdo's C ABI.

Workload ("chain100"): N = 100 three-level atoms, QAOA p = 3 on the TFIM (J = h = 1),
chi = 256, K = 16, Rydberg decay 0.005 and dephasing 0.005 per block, crosstalk phase
0.01 rad, post-promotion 0.01 rad, seeded angles (seed 3).  One step = one full circuit:
reset to |+>^N, the 3 layers (297 two-site updates: Gram contractions, Jacobi
eigensolves, split, Kraus truncation with PPT) and the TFIM energy / success probability.
One step runs a batch of such circuits (--batch, default 32, seeded angle draws)
concurrently through the library's batch executor (one CUDA stream and host thread per
circuit in flight); the single-circuit latency is reported beside it.

value  = two-site updates per second, whole job (all ranks), device-resident inputs.
e2e    = the same metric through the host-buffer API (mpdo_batch_run_host: every step
         each worker converts its circuit's ops, copies them from pinned host memory and
         runs them; energies read back), wall clock.
Also reported: QAOA energy evaluations per second, the roofline of the dominant kernel
class, the CPU oracle on a bounded sample (cpu_baseline), SM clocks during the timed
region, and the kernel launch count.

Multi-GPU: one circuit does not shard (the bond sweep is sequential), so --gpus N runs N
independent replicas (weak scaling), launched with torchrun.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The batch executor runs one stream per circuit in flight; with the default 8 hardware
# work queues, streams share queues and wait on each other's launches.  Read when the
# CUDA context is created, so it is set before torch initialises CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import synth  # noqa: E402

METRIC = "MPDO site-updates/s and QAOA energy evals/s at chi=256, vs FP64 plain at ≤1e-6"
STEP_SCALARS_BYTES = 64
DEV_STATS_BYTES = 48


WORKLOAD = "chain100"
GATE_MODEL = "g0"      # g0: ideal CZ + closed-form noise per block; g1: Gaussian-pulse CZ
PULSE_STEPS = 2000     # integration steps of the G1 pulse channel


def workload():
    return synth.chain40() if WORKLOAD == "chain40" else synth.chain100()


_CZ_CACHE = {}


def lib_layers(lib, c):
    """The library-built op lists of every layer of circuit c in the selected gate model."""
    if GATE_MODEL == "g0":
        return lib.circuit_layers(c)
    key = ("lib", c.gamma_diss, c.gamma_deph, c.b0, c.b1)
    if key not in _CZ_CACHE:
        _CZ_CACHE[key] = lib.build_cz_pulse(c.gamma_diss, c.gamma_deph, c.b0, c.b1,
                                            n_steps=PULSE_STEPS)[0]
    return [lib.build_qaoa_layer_cz(c.n_sites, k, c.alpha[k], c.beta[k], _CZ_CACHE[key], c.J,
                                    c.bz, c.xtalk_phase) for k in range(c.p)]


def oracle_layer_ops(c, k):
    """The oracle's ops of layer k in the selected gate model (its own pulse integration)."""
    from oracle import qaoa as oqaoa
    if GATE_MODEL == "g0":
        return oqaoa.layer_ops(c, k)
    from oracle import pulse as opulse
    key = ("oracle", c.gamma_diss, c.gamma_deph, c.b0, c.b1, c.bd)
    if key not in _CZ_CACHE:
        _CZ_CACHE[key] = opulse.cz_superop(c.gamma_diss, c.gamma_deph, c.b0, c.b1, c.bd,
                                           PULSE_STEPS)[0]
    return oqaoa.layer_ops_cz(c, k, _CZ_CACHE[key])


PREC_DESC = {
    "mixed": "mixed: complex64 site tensors and large contractions (FP32), Gram matrices with "
             "FP64 products and sums, FP32 Jacobi sweeps with FP64 refinement, FP64 cuts, PPT "
             "and observables",
    "c64": "complex64 throughout (FP32 Grams and Jacobi), FP64 scalars and observables",
    "fp64": "complex128 throughout",
}


def workload_desc(c, prec, sv):
    return {"workload": f"{WORKLOAD}: N={c.n_sites} atoms (d=3), QAOA p={c.p}, chi={c.chi_max}, "
                        f"K={c.k_max}, decay {c.gamma_diss}, dephasing {c.gamma_deph}, "
                        f"crosstalk {c.xtalk_phase} rad, "
                        + (f"post-promotion {c.delta_pp} rad, " if GATE_MODEL == "g0" else "")
                        + f"TFIM J={c.J} h={c.hx}, seed {c.seed}",
            "updates_per_circuit": c.p * (c.n_sites - 1),
            "precision": PREC_DESC[prec], "bond_cut": f"s > {sv:g} s_max" if sv else "numerical floor",
            "parallelism": "replicas",
            "gate_model": ("G0 (gate level)" if GATE_MODEL == "g0" else
                           f"G1 (Gaussian-pulse CZ of Fig. 1, rates per pulse, {PULSE_STEPS} "
                           f"integration steps)"),
            "l2": "flushed between timed steps (256 MiB write)"}


# --------------------------------------------------------------------- CPU oracle
def bond_cut(args):
    """The bond cut of the timed configuration (s > cut * s_max; 0 = numerical floor)."""
    if args.sv_cutoff is not None:
        return args.sv_cutoff
    return 0.0 if args.prec == "c64" else 1e-4


def oracle_sample(c, budget_s: float, n_steps: int = 0, sv: float = 0.0):
    """Time the oracle on the workload: layers 1..p-1 in full, then layer-p updates (the
    expensive ones) up to budget_s (or n_steps of them); extrapolate one full circuit."""
    from oracle import mpdo as ompdo, qaoa as oqaoa
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max,
                   sv_cutoff=sv if sv > 0 else 1e-14)
    layer_t = []
    for k in range(c.p - 1):
        t0 = time.perf_counter()
        for i, kr in oracle_layer_ops(c, k):
            m.apply_two_site(i, kr)
        layer_t.append(time.perf_counter() - t0)
    last = oracle_layer_ops(c, c.p - 1)
    per = []
    t_start = time.perf_counter()
    for i, kr in last:
        t0 = time.perf_counter()
        m.apply_two_site(i, kr)
        per.append(time.perf_counter() - t0)
        if n_steps and len(per) >= n_steps:
            break
        if not n_steps and time.perf_counter() - t_start > budget_s:
            break
    return layer_t, per, len(last)


def oracle_rate(layer_t, per, n_last):
    t_circ = sum(layer_t) + n_last * statistics.mean(per)
    return t_circ


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    c = workload()
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import mpdo as ompdo, qaoa as oqaoa
    sv = bond_cut(args)
    t0 = time.perf_counter()
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max,
                   sv_cutoff=sv if sv > 0 else 1e-14)
    layer_t = []
    for k in range(c.p - 1):
        t1 = time.perf_counter()
        for i, kr in oracle_layer_ops(c, k):
            m.apply_two_site(i, kr)
        layer_t.append(time.perf_counter() - t1)
    last = oracle_layer_ops(c, c.p - 1)
    per = []
    for s, (i, kr) in enumerate(last[: args.warmup + args.steps]):
        t1 = time.perf_counter()
        m.apply_two_site(i, kr)
        if s >= args.warmup:
            per.append(time.perf_counter() - t1)
    t_circ = oracle_rate(layer_t, per, len(last))
    ups = c.p * (c.n_sites - 1) / t_circ
    sample = (f"layers 1..{c.p - 1} in full ({sum(layer_t):.1f} s), then {args.warmup} untimed + "
              f"{len(per)} timed layer-{c.p} updates (mean {statistics.mean(per):.2f} s); one "
              f"circuit extrapolated as layers + {len(last)} x mean")
    line = {"impl": "reference", "metric": METRIC, "value": ups, "unit": "site-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(per), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(c, args.prec, sv),
            "oracle": "complex128 NumPy oracle on the host cores, same bond cut",
            "energy_evals_per_s": 1.0 / t_circ,
            "cpu_baseline": {"value": ups, "unit": "site-updates/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": ups, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------- GPU arm
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def alu_peak_tflops(prec: str, sm_max_mhz: float) -> float:
    """CUDA-core FMA peak from unit counts: 152 SMs x lanes/clk x 2 flops x max clock.
    FP32: 128 FMA lanes per SM; FP64: 2 FMA per SM per clock on GB300."""
    lanes = 2 if prec == "fp64" else 128
    return 152 * lanes * 2 * sm_max_mhz * 1e6 / 1e12


def layer_bytes(layers, elt):
    tot = 0
    for layer in layers:
        for _, k in layer:
            tot += (2 * k.shape[0] * 81 + 2 * 729) * elt
    return tot


def max_over_ranks(ms: float, dist=None, device: str = "cuda") -> float:
    """The job's time: the slowest rank's (all-reduce MAX over the process group); the
    value itself on one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, units_per_step: float, total_ms: float) -> float:
    """Whole-job units per second under weak scaling: every rank processes units_per_step
    per step, and the job takes the slowest rank's time."""
    return world * steps * units_per_step / (total_ms / 1e3)


def batch_circuits(c, batch):
    """The batch of one step: `batch` copies of the workload with seeded angle draws."""
    out = []
    for j in range(batch):
        if j == 0:
            out.append(c)
            continue
        a, b = synth._angles(synth.rng_for(c.seed * 1000 + j), c.p)
        d = synth.scaled(c)
        d.alpha, d.beta, d.seed = a, b, c.seed * 1000 + j
        out.append(d)
    return out


def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    c = workload()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        layer_t, per, n_last = oracle_sample(c, args.cpu_budget, sv=bond_cut(args))
        t_circ = oracle_rate(layer_t, per, n_last)
        ups = c.p * (c.n_sites - 1) / t_circ
        cpu = {"value": ups, "unit": "site-updates/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": (f"{WORKLOAD} oracle: layers 1..{c.p - 1} in full ({sum(layer_t):.1f} s) "
                          f"+ {len(per)} layer-{c.p} updates (mean {statistics.mean(per):.2f} s); "
                          f"circuit time extrapolated as layers + {n_last} x mean = {t_circ:.0f} s")}

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2309_08572_gb300 as lib

    prec = args.prec
    sv = bond_cut(args)
    circs = batch_circuits(c, args.batch)
    host_layers = [lib_layers(lib, ci) for ci in circs]
    m_max = max(k.shape[0] for L in host_layers for layer in L for _, k in layer)
    lprec = "fp64" if prec == "fp64" else "c64"
    pool = [lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec=lprec, own_stream=True,
                     gram_fp64=(prec == "mixed"), sv_cutoff=sv)
            for _ in range(args.batch)]
    dls = [[pool[0].upload_layer(layer) for layer in L] for L in host_layers]
    descs = [dict(n_sites=ci.n_sites, chi_max=ci.chi_max, k_max=ci.k_max, layers=d, J=ci.J,
                  hx=ci.hx, b=ci.bz) for ci, d in zip(circs, dls)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    updates = c.p * (c.n_sites - 1)
    # GEMM tile shapes picked by the library's autotuner (untimed)
    tuned = [lib.autotune_gemm(pr, reps=3) for pr in (0, 1)] if args.autotune else None

    def step():
        return lib.batch_run(pool, descs)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    # single-circuit latency and kernel-class breakdown (one profiled circuit, untimed)
    g = pool[0]
    g.profile(7)
    t0 = time.perf_counter()
    single = lib.batch_run([g], descs[:1])
    single_ms = 1e3 * (time.perf_counter() - t0)
    prof = [g.profile_read(k) for k in range(3)]
    g.profile(0)
    dom = max(range(3), key=lambda k: prof[k]["ms"])
    names = {0: "complex GEMM (cgemm_kernel)",
             1: "eigensolver (jacobi_smem_kernel sweeps; mixed mode: FP32 sweeps + FP64 "
                "refinement products)",
             2: "other kernels"}

    # timed region: K steps (each a batch of circuits run concurrently), events around
    # each step on the current stream after a device-wide synchronisation; L2 flushed
    # between steps outside the events
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    for m in pool:
        m.profile(1 << dom)
    launches0 = lib.kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        res = step()
        torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = lib.kernel_launches() - launches0
    dprofs = [m.profile_read(dom) for m in pool]
    for m in pool:
        m.profile(0)
    dprof = {k: sum(d[k] for d in dprofs) for k in ("ms", "launches", "flops")}
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(times), dist)
    value = job_throughput(world, args.steps, args.batch * updates, total_ms)

    # end to end through the host-buffer API: every step uploads each circuit's ops from
    # host memory, runs the batch and reads the energies back
    h2d = sum(layer_bytes(L, 16 if prec == "fp64" else 8) for L in host_layers)
    if prec == "mixed":   # the channel partial traces travel in FP64
        h2d = sum(sum((2 * k.shape[0] * 81 * 8 + 2 * 729 * 16) for _, k in layer)
                  for L in host_layers for layer in L)
    d2h = args.batch * (4 * 8 + updates * 2 * STEP_SCALARS_BYTES + c.p * DEV_STATS_BYTES)
    # the circuits' ops in host memory, in the C ABI's layout (marshalled once, untimed)
    hosts = [lib.HostCircuit(ci.n_sites, ci.chi_max, ci.k_max, L, J=ci.J, hx=ci.hx, b=ci.bz)
             for ci, L in zip(circs, host_layers)]
    torch.cuda.synchronize()
    te = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lib.batch_run_host(pool, hosts)
        te.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(1e3 * sum(te), dist)
    e2e_value = job_throughput(world, len(te), args.batch * updates, e2e_ms)

    # roofline of the dominant class
    pk = peaks()
    smax = (ck or {}).get("sm_max_mhz") or pk.get("sm_max_mhz", 2070.0)
    roof = {"kernel": names[dom],
            "share_of_single_circuit": prof[dom]["ms"] / max(1e-9, sum(p["ms"] for p in prof)),
            "launches_per_step": dprof["launches"] / max(1, args.steps),
            "avg_launch_us": 1e3 * dprof["ms"] / max(1, dprof["launches"])}
    if dom in (0, 1) and dprof["flops"] > 0:
        achieved = dprof["flops"] / (dprof["ms"] / 1e3) / 1e12
        peak = alu_peak_tflops(prec, smax)
        roof.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "traffic_note": "not a per-launch constant of this class (sizes vary); one "
                                     "ncu capture of a level solve (n=24) read 36.6 KB and "
                                     "wrote 0 B of DRAM: the solves live in shared memory",
                     "flops_per_launch": dprof["flops"] / max(1, dprof["launches"]),
                     "peak_note": f"CUDA-core {'FP64' if prec == 'fp64' else 'FP32'} FMA peak from "
                                  f"unit counts (152 SMs x {'2' if prec == 'fp64' else '128'} FMA/clk "
                                  f"x 2) at {smax:.0f} MHz; achieved = flops per launch / mean "
                                  f"launch duration (concurrent circuits); flops = "
                                  + ("8 m n k per complex GEMM" if dom == 0 else
                                     "multiply-adds executed by the Jacobi rotations")})
    else:
        roof.update({"bound": "latency", "achieved": None, "peak": None, "unit": None,
                     "frac": None, "traffic": None})

    # the plain FP64 single-circuit form on the same circuit and cut: its time, and the
    # error of this run's circuit 0 against it, per observable
    fp64 = None
    if not args.no_fp64_compare and prec != "fp64" and rank == 0 and world == 1:
        g64 = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec="fp64", own_stream=True,
                       sv_cutoff=sv)
        dl64 = [g64.upload_layer(layer) for layer in host_layers[0]]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = lib.batch_run([g64], [dict(descs[0], layers=dl64)])
        t64 = time.perf_counter() - t0
        ups64 = updates / t64
        fp64 = {"ms_per_circuit": 1e3 * t64, "site_updates_per_s": ups64,
                "factor_batched_vs_fp64_single": value / ups64,
                "factor_single_vs_fp64_single": (1e3 * t64) / single_ms,
                "rel_err": {k: abs(res[0][j] - r64[0][j]) / abs(r64[0][j])
                            for j, k in enumerate(("e_raw", "e_succ", "p_succ", "trace"))},
                "bond_cut": f"s > {sv:g} s_max" if sv else "numerical floor"}
        for dl in dl64:
            g64.free_uploaded(dl)
        g64.close()

    if rank == 0:
        cfg = workload_desc(c, prec, sv)
        cfg["gemm_tiles"] = (f"autotuned ({tuned[0]} FP64 and {tuned[1]} FP32 buckets)"
                             if tuned else "built-in size rules")
        cfg["batch"] = f"{args.batch} circuits per step, run concurrently (one stream each); " \
                       f"circuit 0 uses seed {c.seed}, circuit j seeded angles {c.seed}*1000+j"
        line = {"metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "c64": "f32", "mixed": "f32+f64"}[prec],
                "data": "synthetic",
                "config": cfg,
                "energy_evals_per_s": world * args.steps * args.batch / (total_ms / 1e3),
                "single_circuit": {"ms": single_ms, "site_updates_per_s": updates / (single_ms / 1e3),
                                   "result": dict(zip(("e_raw", "e_succ", "p_succ", "trace"),
                                                      single[0].tolist()))},
                "roofline": roof,
                "kernel_profile_single_circuit_ms": {names[k]: prof[k]["ms"] for k in range(3)},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": ck, "fp64_plain": fp64}
        print(json.dumps(line), flush=True)
    for d in dls:
        for dl in d:
            pool[0].free_uploaded(dl)
    for m in pool:
        m.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch512(args):
    """The batched workload: 512 circuits (N ~ U{20..100}, chi in {32,64,128}, K = 8,
    p in {1,2}, log-uniform rates, seed 4) per step through the executor, mixed precision
    at the same bond cut; value = site-updates/s over all of them."""
    import torch
    import paper_2309_08572_gb300 as lib
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sv = bond_cut(args)
    circs = synth.batch512()
    host_layers = [lib_layers(lib, ci) for ci in circs]
    m_max = max(k.shape[0] for L in host_layers for layer in L for _, k in layer)
    n_cap = max(ci.n_sites for ci in circs)
    chi_cap = max(ci.chi_max for ci in circs)
    k_cap = max(ci.k_max for ci in circs)
    lprec = "fp64" if args.prec == "fp64" else "c64"
    pool = [lib.Mpdo(n_cap, chi_cap, k_cap, m_max=m_max, prec=lprec, own_stream=True,
                     gram_fp64=(args.prec == "mixed"), sv_cutoff=sv)
            for _ in range(args.batch)]
    dls = [[pool[0].upload_layer(layer) for layer in L] for L in host_layers]
    descs = [dict(n_sites=ci.n_sites, chi_max=ci.chi_max, k_max=ci.k_max, layers=d, J=ci.J,
                  hx=ci.hx, b=ci.bz) for ci, d in zip(circs, dls)]
    updates = sum(ci.p * (ci.n_sites - 1) for ci in circs)
    tuned = [lib.autotune_gemm(pr, reps=3) for pr in (0, 1)] if args.autotune else None
    for _ in range(args.warmup):
        lib.batch_run(pool, descs)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times = []
    launches0 = lib.kernel_launches()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = lib.batch_run(pool, descs)
        torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = lib.kernel_launches() - launches0
    ck = clocks.stop()
    total_ms = sum(times)
    # end to end: the circuits' ops from host memory through the host-layer executor
    hosts = [lib.HostCircuit(ci.n_sites, ci.chi_max, ci.k_max, L, J=ci.J, hx=ci.hx, b=ci.bz)
             for ci, L in zip(circs, host_layers)]
    te = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lib.batch_run_host(pool, hosts)
        te.append(time.perf_counter() - t0)
    h2d = sum(sum((2 * k.shape[0] * 81 * (16 if args.prec == "fp64" else 8) + 2 * 729 * 16)
                  for _, k in layer) for L in host_layers for layer in L)
    line = {"metric": METRIC, "value": args.steps * updates / (total_ms / 1e3),
            "unit": "site-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "c64": "f32", "mixed": "f32+f64"}[args.prec],
            "data": "synthetic",
            "config": {"workload": "batch512: 512 circuits, N ~ U{20..100}, chi in {32,64,128}, "
                                   "K=8, p in {1,2}, decay/dephasing log-U[1e-4,1e-2], seed 4",
                       "updates_per_step": updates, "precision": PREC_DESC[args.prec],
                       "bond_cut": f"s > {sv:g} s_max" if sv else "numerical floor",
                       "pool": f"{args.batch} handles (one stream each) sized N=100, chi=128, K=8",
                       "gemm_tiles": (f"autotuned ({tuned[0]} FP64 and {tuned[1]} FP32 buckets)"
                                      if tuned else "built-in size rules"),
                       "l2": "inputs far larger than L2 across the step"},
            "energy_evals_per_s": args.steps * len(circs) / (total_ms / 1e3),
            "e2e": {"value": len(te) * updates / sum(te), "unit": "site-updates/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": len(circs) * 4 * 8 + updates * 2 * STEP_SCALARS_BYTES
                    + sum(ci.p for ci in circs) * DEV_STATS_BYTES},
            "gpu_launches": launches,
            "finite": bool(np.all(np.isfinite(out))), "clocks": ck}
    print(json.dumps(line), flush=True)
    for d in dls:
        for dl in d:
            pool[0].free_uploaded(dl)
    for m in pool:
        m.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["mixed", "c64", "fp64"], default="mixed",
                    help="mixed: FP32 tensors with FP64 Grams and small matrices (default)")
    ap.add_argument("--sv-cutoff", type=float, default=None,
                    help="bond cut s > cutoff * s_max (default 1e-4; c64: its numerical floor)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 single-circuit comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--autotune", action="store_true",
                    help="pick GEMM tile shapes with the library's autotuner before timing "
                         "(default: the built-in size rules, faster under concurrency)")
    ap.add_argument("--gate-model", choices=["g0", "g1"], default="g0",
                    help="g0: ideal CZ with closed-form noise per block; g1: the Gaussian-pulse "
                         "CZ channel integrated from the Lindbladian (chain workloads)")
    ap.add_argument("--batch", type=int, default=32,
                    help="circuits per step, run concurrently by the batch executor")
    ap.add_argument("--workload", choices=["chain100", "chain40", "batch512"], default="chain100",
                    help="chain40 (N=40, p=2, chi=64, K=8) is the small profiling case")
    args = ap.parse_args()
    global WORKLOAD, GATE_MODEL
    WORKLOAD = args.workload
    GATE_MODEL = args.gate_model
    if GATE_MODEL == "g1" and WORKLOAD == "batch512":
        # every circuit there has its own rates, i.e. its own pulse integration
        ap.error("--gate-model g1 runs the chain workloads only")
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch512(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
