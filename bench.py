#!/usr/bin/env python
"""Throughput of the noisy-QAOA MPDO hot path on GB300 through libmpdo's C ABI.

Workload ("chain100"): N = 100 three-level atoms, QAOA p = 3 on the TFIM (J = h = 1),
chi = 256, K = 16, Rydberg decay 0.005 and dephasing 0.005 per block, crosstalk phase
0.01 rad, post-promotion 0.01 rad, seeded angles (seed 3).  One circuit = reset to |+>^N,
the 3 layers (297 two-site updates: Gram contractions, eigensolves, split, Kraus truncation
with PPT) and the TFIM energy / success probability.  The bond cut is reading A4's for the
reduced-precision modes, s > 1e-7 s_max, applied at each mode's numerical floor (mixed forms:
lambda = s^2 > 1e-13 lambda_max, i.e. s > 3.2e-7 s_max); at that cut three layers take the bond
dimension to D = 33, which the line reports (chi_used_max, mean D).  "chain100deep" runs the
same chain with p = 8 layers, where D reaches chi = 256.
One step runs a batch of circuits (--batch, default 32, seeded angle draws) concurrently
through the library's batch executor (one CUDA stream and host thread per circuit in flight).

value  = two-site updates per second, whole job (all ranks), device-resident inputs.
e2e    = the same metric through the host-buffer API (mpdo_batch_run_host: every step each
         worker converts its circuit's ops, copies them from pinned host memory and runs
         them; energies read back), wall clock.
Also reported: QAOA energy evaluations per second; the plain FP64 form on the same circuits
(single circuit and batched) and the error of every energy and probability against the
CPU oracle; the GPU-wide roofline of the dominant kernel class against peaks measured on this
GPU; the oracle on a bounded sample (cpu_baseline); SM clocks during the timed region; the
kernel launch counts.

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
    return {"chain40": synth.chain40, "chain100": synth.chain100,
            "chain100deep": synth.chain100deep}[WORKLOAD]()


# Product engines and Gram precision of each --prec form: (library precision, FP64 Grams).
FORMS = {"mixed": ("c64", True), "mixed-tc": ("tf32x3", True), "c64": ("c64", False),
         "tf32x3": ("tf32x3", False), "bf16x3": ("bf16x3", False), "fp64": ("fp64", False)}
# Relative rounding of one Gram entry of each form (the library's numerical floor of the
# cuts is lambda > 10 eps lambda_max).
FORM_EPS = {"mixed": 1e-14, "mixed-tc": 1e-14, "c64": 6e-8, "tf32x3": 2.4e-7, "bf16x3": 1.5e-5,
            "fp64": 1e-16}


def effective_cut(prec: str, sv: float) -> float:
    """The bond cut the library applies for a requested s > sv s_max: lambda = s^2 above
    max(sv^2, 10 eps) lambda_max, i.e. s > max(sv, sqrt(10 eps)) s_max."""
    return max(sv, float(np.sqrt(10.0 * FORM_EPS[prec])))


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
             "FP64 products and sums, FP32 Jacobi sweeps with FP64 refinement, FP64 cuts, PPT, "
             "trace and observables",
    "mixed-tc": "mixed-tc: complex64 site tensors; the FP32 contractions (new centre, inner "
                "isometry) on the tensor cores in TF32x3 split precision (tcgen05, FP32 "
                "accumulation); the Grams and other FP64 products as exact BF16 slice products "
                "on the tensor cores summed in FP64; FP32 Jacobi sweeps with FP64 refinement; "
                "FP64 cuts, PPT, trace and observables",
    "c64": "complex64 throughout (FP32 Grams and Jacobi), FP64 scalars and observables",
    "tf32x3": "complex64 with every large product (Grams included) on the tensor cores in "
              "TF32x3 split precision (tcgen05, FP32 accumulation), FP32 Jacobi",
    "bf16x3": "complex64 with every large product on the tensor cores in BF16x3 split "
              "precision (tcgen05, FP32 accumulation), FP32 Jacobi",
    "fp64": "complex128 throughout",
}


def workload_desc(c, prec, sv):
    eff = effective_cut(prec, sv)
    return {"workload": f"{WORKLOAD}: N={c.n_sites} atoms (d=3), QAOA p={c.p}, chi={c.chi_max}, "
                        f"K={c.k_max}, decay {c.gamma_diss}, dephasing {c.gamma_deph}, "
                        f"crosstalk {c.xtalk_phase} rad, "
                        + (f"post-promotion {c.delta_pp} rad, " if GATE_MODEL == "g0" else "")
                        + f"TFIM J={c.J} h={c.hx}, seed {c.seed}; bond cut s > {eff:.2g} s_max "
                        f"(reading A4: {sv:g} requested, the form's floor sqrt(10 eps) applied)",
            "updates_per_circuit": c.p * (c.n_sites - 1),
            "precision": PREC_DESC[prec],
            "bond_cut": f"s > {eff:.3g} s_max (requested {sv:g}; floor of the form "
                        f"{np.sqrt(10 * FORM_EPS[prec]):.2g})",
            "parallelism": "replicas",
            "gate_model": ("G0 (gate level)" if GATE_MODEL == "g0" else
                           f"G1 (Gaussian-pulse CZ of Fig. 1, rates per pulse, {PULSE_STEPS} "
                           f"integration steps)"),
            "l2": "flushed between timed steps (256 MiB write)"}


# --------------------------------------------------------------------- CPU oracle
def bond_cut(args):
    """The requested bond cut s > cut * s_max: reading A4 (1e-7 for the reduced-precision
    forms, 1e-14 for FP64) unless --sv-cutoff is given."""
    if args.sv_cutoff is not None:
        return args.sv_cutoff
    return 1e-14 if args.prec == "fp64" else 1e-7


def oracle_sample(c, budget_s: float, n_steps: int = 0, sv: float = 0.0):
    """Time the oracle on the workload: layers 1..p-1 in full, then layer-p updates (the
    expensive ones) up to budget_s (or n_steps of them); extrapolate one full circuit."""
    from oracle import mpdo as ompdo, qaoa as oqaoa
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max, sv_cutoff=sv)
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
    eff = effective_cut(args.prec, sv)
    t0 = time.perf_counter()
    m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max, sv_cutoff=eff)
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
            "oracle": f"complex128 NumPy oracle on the host cores, same bond cut (s > {eff:.3g} "
                      f"s_max)",
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


def measure_peaks(torch):
    """Dense GEMM throughput of this GPU per arithmetic, as roofline denominators (cuBLAS
    through torch.matmul, CUDA events, best of 5 after 2 warm-ups): FP64 (4096^3), FP32 on
    the CUDA cores (TF32 off, 8192^3) and TF32 (8192^3); 2 n^3 flops each."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, tf32, n in (("fp64", torch.float64, False, 4096),
                                  ("fp32", torch.float32, False, 8192),
                                  ("tf32", torch.float32, True, 8192)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            for _ in range(2):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def oracle_results(circs, sv, n_max):
    """The CPU oracle's observables for the first n_max circuits at bond cut sv."""
    from oracle import mpdo as ompdo, observables as oobs, qaoa as oqaoa
    out = []
    for c in circs[:n_max]:
        m = ompdo.MPDO(c.n_sites, oqaoa.plus_state(), c.chi_max, c.k_max, sv_cutoff=sv)
        for k in range(c.p):
            for i, kr in oracle_layer_ops(c, k):
                m.apply_two_site(i, kr)
        out.append(oobs.expect_energy(m, c.J, c.hx, c.bz))
    return out


KEYS = ("e_raw", "e_succ", "p_succ", "trace")


def rel_errors(res_rows, refs):
    """max over circuits of |gpu - oracle| / |oracle|, per observable."""
    errs = {}
    for j, key in enumerate(KEYS):
        errs[key] = max(abs(row[j] - r[key]) / abs(r[key]) for row, r in zip(res_rows, refs))
    return errs


def single_circuit(lib, g, dls, circ):
    """One circuit on handle g, layer by layer (untimed detail): truncation statistics,
    the bond dimensions reached and the result."""
    import torch
    g.reconfigure(circ.n_sites, circ.chi_max, circ.k_max)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chi_max = k_max = 0
    for dl in dls:
        st = g.apply_uploaded(dl)
        chi_max = max(chi_max, st["chi_used_max"])
        k_max = max(k_max, st["k_used_max"])
    e = g.expect_energy(circ.J, circ.hx, circ.bz)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    b, kd, _ = g.dims()
    return {"ms": ms, "chi_used_max": int(chi_max), "k_used_max": int(k_max),
            "mean_bond_dim_final": float(np.mean(b)), "max_bond_dim_final": int(np.max(b)),
            "result": {k: float(e[k]) for k in KEYS}}


def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    c = workload()
    prec = args.prec
    sv = bond_cut(args)
    eff = effective_cut(prec, sv)
    circs = batch_circuits(c, args.batch)
    cpu = None
    refs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        layer_t, per, n_last = oracle_sample(c, args.cpu_budget, sv=eff)
        t_circ = oracle_rate(layer_t, per, n_last)
        ups = c.p * (c.n_sites - 1) / t_circ
        cpu = {"value": ups, "unit": "site-updates/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": (f"{WORKLOAD} oracle at the same cut (s > {eff:.3g} s_max): layers "
                          f"1..{c.p - 1} in full ({sum(layer_t):.1f} s) + {len(per)} layer-{c.p} "
                          f"updates (mean {statistics.mean(per):.2f} s); circuit time "
                          f"extrapolated as layers + {n_last} x mean = {t_circ:.0f} s")}
    if rank == 0 and world == 1 and args.oracle_check > 0:
        # the oracle's observables of the first circuits, for the error of every output
        refs = oracle_results(circs, eff, args.oracle_check)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2309_08572_gb300 as lib

    lprec, gram = FORMS[prec]
    host_layers = [lib_layers(lib, ci) for ci in circs]
    m_max = max(k.shape[0] for L in host_layers for layer in L for _, k in layer)
    pool = [lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec=lprec, own_stream=True,
                     gram_fp64=gram, sv_cutoff=sv)
            for _ in range(args.batch)]
    dls = [[pool[0].upload_layer(layer) for layer in L] for L in host_layers]
    descs = [dict(n_sites=ci.n_sites, chi_max=ci.chi_max, k_max=ci.k_max, layers=d, J=ci.J,
                  hx=ci.hx, b=ci.bz) for ci, d in zip(circs, dls)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    updates = c.p * (c.n_sites - 1)
    tuned = [lib.autotune_gemm(pr, reps=3) for pr in (0, 1)] if args.autotune else None

    def step():
        return lib.batch_run(pool, descs)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    # single-circuit latency, bond dimensions reached and kernel-class breakdown (untimed)
    g = pool[0]
    g.profile(7)
    single = single_circuit(lib, g, dls[0], circs[0]) if not args.no_single else None
    prof = [g.profile_read(k) for k in range(3)]
    g.profile(0)
    names = {0: "complex GEMMs (cgemm_kernel, cgemm_small_kernel, FP64-product cgemm_wide; "
                "tc_gemm_kernel for the tensor-core forms)",
             1: "eigensolvers (pchol_kernel, osj_kernel, jacobi_smem_kernel / jacobi_coop_kernel "
                "FP32 sweeps, FP64 refinement sg_refine_kernel, level_out_kernel)",
             2: "other kernels (selection, PPT, phi, layout)"}

    # timed region: K steps (each a batch of circuits run concurrently); events around each
    # step on the current stream after a device-wide synchronisation; L2 flushed between steps
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    for m in pool:
        m.profile(3)
    launches0 = lib.kernel_launches()
    tc0 = lib.tc_gemm_launches()
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
    tc_launches = lib.tc_gemm_launches() - tc0
    cls = [{k: sum(m.profile_read(q)[k] for m in pool) for k in ("ms", "launches", "flops")}
           for q in (0, 1)]
    for m in pool:
        m.profile(0)
    ck = clocks.stop()
    total_ms = max_over_ranks(sum(times), dist)
    ms_step = total_ms / args.steps
    value = job_throughput(world, args.steps, args.batch * updates, total_ms)

    # end to end through the host-buffer API: every step uploads each circuit's ops from
    # host memory, runs the batch and reads the energies back
    elt = 16 if prec == "fp64" else 8
    gelt = 16 if (prec == "fp64" or gram) else 8   # channel partial traces: Gram precision
    h2d = sum(sum((2 * k.shape[0] * 81 * elt + 2 * 729 * gelt) for _, k in layer)
              for L in host_layers for layer in L)
    d2h = args.batch * (4 * 8 + updates * 2 * STEP_SCALARS_BYTES + c.p * DEV_STATS_BYTES)
    hosts = [lib.HostCircuit(ci.n_sites, ci.chi_max, ci.k_max, L, J=ci.J, hx=ci.hx, b=ci.bz)
             for ci, L in zip(circs, host_layers)]
    torch.cuda.synchronize()
    te = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lib.batch_run_host(pool, hosts)
        te.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(1e3 * sum(te), dist) if te else None
    e2e_value = job_throughput(world, len(te), args.batch * updates, e2e_ms) if te else None

    # peaks of this GPU and the GPU-wide roofline of the dominant class: its flops per step
    # (8 m n k per complex product at the actual dims; the eigensolvers' executed rotations
    # and FP64 refinement products) over the step time
    pk = peaks()
    mp = measure_peaks(torch) if rank == 0 and not args.no_peaks else {}
    dom = 0 if cls[0]["ms"] >= cls[1]["ms"] else 1
    fl_step = cls[dom]["flops"] / args.steps
    roof = {"kernel": names[dom], "scope": "GPU-wide: class flops per step / ms_per_step",
            "class_ms_per_step_summed_over_streams": cls[dom]["ms"] / args.steps,
            "launches_per_step": cls[dom]["launches"] / args.steps,
            "share_of_single_circuit": (prof[dom]["ms"] / max(1e-9, sum(q["ms"] for q in prof))
                                        if single else None)}
    if fl_step > 0 and mp:
        achieved = fl_step / (ms_step / 1e3) / 1e12
        if dom == 0 and prec in ("tf32x3", "bf16x3"):
            peak, pname = mp["tf32"] if prec == "tf32x3" else pk.get("bf16_tflops_sustained", 0), \
                "TF32 cuBLAS, measured here" if prec == "tf32x3" else "BF16 cuBLAS, sustained"
            bound = "tensor"
        elif prec == "fp64":
            peak, pname, bound = mp["fp64"], "FP64 DGEMM (cuBLAS), measured here", "alu"
        else:
            peak, pname, bound = mp["fp32"], "FP32 SGEMM on the CUDA cores (cuBLAS, TF32 off), " \
                                             "measured here", "alu"
        roof.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "peak_source": pname,
                     "traffic_note": "not a per-launch constant of this class (hundreds of shapes "
                                     "per circuit); the ncu summaries in profiles/ give DRAM bytes "
                                     "of the individual kernels"})
    else:
        roof.update({"bound": "latency", "achieved": None, "peak": None, "unit": None,
                     "frac": None, "traffic": None})

    # the plain FP64 form on the same circuits and cut: one circuit alone, and the batch run
    # concurrently (handles capped at chi = 64: the cut keeps D below that, checked)
    fp64 = None
    if not args.no_fp64_compare and prec != "fp64" and rank == 0 and world == 1 and single:
        g64 = lib.Mpdo(c.n_sites, c.chi_max, c.k_max, m_max=m_max, prec="fp64", own_stream=True,
                       sv_cutoff=eff)
        dl64 = [g64.upload_layer(layer) for layer in host_layers[0]]
        s64 = single_circuit(lib, g64, dl64, circs[0])
        for dl in dl64:
            g64.free_uploaded(dl)
        g64.close()
        fp64 = {"single_circuit": s64,
                "site_updates_per_s_single": updates / (s64["ms"] / 1e3),
                "factor_single_vs_fp64_single": s64["ms"] / single["ms"]}
        if not args.no_fp64_batch and single["chi_used_max"] < 64 and s64["chi_used_max"] < 64:
            pool64 = [lib.Mpdo(c.n_sites, 64, c.k_max, m_max=m_max, prec="fp64", own_stream=True,
                               sv_cutoff=eff) for _ in range(args.batch)]
            dlb = [[pool64[0].upload_layer(layer) for layer in L] for L in host_layers]
            d64 = [dict(dd, chi_max=64, layers=d) for dd, d in zip(descs, dlb)]
            lib.batch_run(pool64, d64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r64 = lib.batch_run(pool64, d64)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            fp64.update({"batched_ms_per_step": 1e3 * tb,
                         "site_updates_per_s_batched": args.batch * updates / tb,
                         "factor_batched_vs_fp64_batched": value / (args.batch * updates / tb),
                         "batched_pool": f"{args.batch} FP64 handles with chi cap 64 (the cut "
                                         f"keeps D <= {s64['chi_used_max']})"})
            for d in dlb:
                for dl in d:
                    pool64[0].free_uploaded(dl)
            for m in pool64:
                m.close()
        fp64["factor_batched_vs_fp64_single"] = value / fp64["site_updates_per_s_single"]
        fp64["bond_cut"] = f"s > {eff:.3g} s_max (same as the timed form)"

    if rank == 0:
        cfg = workload_desc(c, prec, sv)
        cfg["gemm_tiles"] = (f"autotuned ({tuned[0]} FP64 and {tuned[1]} FP32 buckets)"
                             if tuned else "built-in size rules")
        cfg["batch"] = f"{args.batch} circuits per step, run concurrently (one stream each); " \
                       f"circuit 0 uses seed {c.seed}, circuit j seeded angles {c.seed}*1000+j"
        if single is None:
            # the timed circuits' reached dimensions, from the pool handles' final state
            bd, kd, _ = pool[0].dims()
            single_dims = {"chi_used_max": int(max(bd)), "k_used_max": int(max(kd)),
                           "mean_bond_dim_final": float(np.mean(bd))}
        else:
            single_dims = single
        cfg["chi_used_max"] = single_dims["chi_used_max"]
        cfg["k_used_max"] = single_dims["k_used_max"]
        cfg["mean_bond_dim"] = single_dims["mean_bond_dim_final"]
        errs = None
        if refs:
            errs = {"vs": f"CPU oracle (complex128) at the same cut, circuits 0..{len(refs) - 1} "
                          f"of the batch, max relative error",
                    "batched": rel_errors(np.asarray(res)[:len(refs)], refs)}
        line = {"metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "c64": "f32", "mixed": "f32+f64", "mixed-tc": "tf32x3+f64",
                          "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[prec],
                "data": "synthetic",
                "config": cfg,
                "energy_evals_per_s": world * args.steps * args.batch / (total_ms / 1e3),
                "single_circuit": (dict(single, site_updates_per_s=updates / (single["ms"] / 1e3))
                                   if single else None),
                "error_vs_oracle": errs,
                "roofline": roof,
                "peaks_measured_tflops": mp,
                "kernel_profile_single_circuit_ms": ({names[k]: prof[k]["ms"] for k in range(3)}
                                                     if single else None),
                "kernel_class_ms_per_step_summed_over_streams": {
                    names[q]: cls[q]["ms"] / args.steps for q in (0, 1)},
                "cpu_baseline": cpu,
                "e2e": ({"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h} if te else None),
                "gpu_launches": launches, "tc_gemm_launches": tc_launches, "clocks": ck,
                "fp64_plain": fp64}
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
    lprec, gram = FORMS[args.prec]
    pool = [lib.Mpdo(n_cap, chi_cap, k_cap, m_max=m_max, prec=lprec, own_stream=True,
                     gram_fp64=gram, sv_cutoff=sv)
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
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "c64": "f32", "mixed": "f32+f64", "mixed-tc": "tf32x3+f64",
                      "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[args.prec],
            "data": "synthetic",
            "config": {"workload": "batch512: 512 circuits, N ~ U{20..100}, chi in {32,64,128}, "
                                   "K=8, p in {1,2}, decay/dephasing log-U[1e-4,1e-2], seed 4",
                       "updates_per_step": updates, "precision": PREC_DESC[args.prec],
                       "bond_cut": f"s > {effective_cut(args.prec, sv):.3g} s_max (requested "
                                   f"{sv:g})",
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


def run_compare(args):
    """Fig. 7's comparison on this GPU: the collision probability (anticoncentration) of the
    8-site random circuit with gamma_diss = 0.1 (depth 40, i.e. 20 two-layer periods, Haar
    one-qubit gates and noisy CZ brickwork, seed 5), for the vectorized MPO with naive and
    with purity-preserving truncation on the bond and for the MPDO, against the update time
    per two-layer period.  Errors are the mean over the last 5 periods of |Z - Z_ref| / Z_ref,
    Z_ref from the MPDO at (chi 64, K 16), whose points converge fastest; the MPDO at
    (chi 32, K 8) is reported beside it as a check of the reference.  Points: FP64, bond cut
    s > 1e-7 s_max, except the vMPO at chi = 128 (tensor-core form, s > 1e-5 s_max).  One
    line of JSON with every point and its collision probabilities."""
    import torch
    import paper_2309_08572_gb300 as lib
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    depth, periods_avg = 40, 5
    circ = synth.rcs(8, depth, 256, 16, gamma_diss=0.1, seed=5, delta_pp=0.01)
    layers = lib.circuit_layers(circ)
    probe = set(range(depth - 2 * periods_avg + 1, depth, 2))   # after periods 16..20
    m_max = max(k.shape[0] for layer in layers for _, k in layer)

    def run(kind, chi, k=1, mode=None, tc=False):
        if kind == "vmpo":
            g = lib.Vmpo(circ.n_sites, chi, ppt=(mode == "ppt"), sv_cutoff=1e-5 if tc else 1e-7,
                         init_vec=[1, 0, 0], tc=tc)
        else:
            g = lib.Mpdo(circ.n_sites, chi, k, m_max=m_max, prec="fp64", sv_cutoff=1e-7,
                         init_vec=[1, 0, 0])
        zs, t = [], 0.0
        for li, layer in enumerate(layers):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.apply_layer(layer)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            if li in probe:
                zs.append(g.collision() if kind == "vmpo" else
                          g.second_order(circ.n_sites // 2)["collision"])
        g.close()
        return np.array(zs), t / (depth / 2)

    z_ref, t_ref = run("mpdo", 64, 16)
    z_chk, t_chk = run("mpdo", 32, 8)
    points = []

    def add(engine, chi, k, z, t):
        points.append({"engine": engine, "chi": chi, "K": k, "s_per_period": t,
                       "collision_rel_err": float(np.mean(np.abs(z - z_ref) / z_ref)),
                       "collision": [float(x) for x in z]})

    for mode in ("naive", "ppt"):
        for chi in (8, 16, 32, 64):
            z, t = run("vmpo", chi, mode=mode)
            add(f"vmpo-{mode}", chi, None, z, t)
    z, t = run("vmpo", 128, mode="ppt", tc=True)
    add("vmpo-ppt (tensor-core form)", 128, None, z, t)
    for chi, k in ((8, 2), (16, 2), (16, 4), (32, 4)):
        z, t = run("mpdo", chi, k)
        add("mpdo", chi, k, z, t)
    line = {"metric": "collision-probability error vs update time per two-layer period "
                      "(Fig. 7 comparison)",
            "value": None, "unit": "relative error / s", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic",
            "config": {"workload": "rcs8 gamma_diss=0.1: 8 sites (d=3), depth 40, Haar U(2) on "
                                   "the qubit levels + noisy CZ brickwork (G0), post-promotion "
                                   "0.01 rad, seed 5, |0>^8; bond cut s > 1e-7 s_max",
                       "precision": "FP64 (the vMPO at chi=128: exact-slice tensor-core "
                                    "products + mixed eigensolver)",
                       "reference": "MPDO chi=64 K=16", "reference_s_per_period": t_ref,
                       "check_mpdo_32x8_vs_reference": float(np.mean(np.abs(z_chk - z_ref) /
                                                                    z_ref)),
                       "check_s_per_period": t_chk,
                       "collision_reference": [float(x) for x in z_ref]},
            "points": points}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=list(FORMS), default="mixed-tc",
                    help="mixed-tc (default): FP32 site tensors, FP64-accurate Grams and small "
                         "matrices, every large product on the tensor cores (TF32x3 for the "
                         "FP32 products, exact BF16 slices for the FP64 ones); mixed: the same "
                         "arithmetic on the CUDA cores; tf32x3 / bf16x3: complex64 with FP32 "
                         "Grams on the tensor cores; c64; fp64")
    ap.add_argument("--sv-cutoff", type=float, default=None,
                    help="bond cut s > cutoff * s_max (default: reading A4, 1e-7 for the "
                         "reduced-precision forms, 1e-14 for fp64; each form applies its "
                         "numerical floor on top)")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 comparison (single circuit and batch)")
    ap.add_argument("--no-fp64-batch", action="store_true",
                    help="skip only the batched FP64 comparison")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip measuring the FP64 / FP32 / TF32 GEMM peaks")
    ap.add_argument("--no-single", action="store_true",
                    help="skip the separate single-circuit run (workloads whose circuit takes "
                         "minutes; the reached dimensions then come from the timed handles)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--oracle-check", type=int, default=2,
                    help="circuits of the batch whose outputs are compared with the CPU oracle")
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
    ap.add_argument("--workload", choices=["chain100", "chain100deep", "chain40", "batch512",
                                           "rcs8cmp"],
                    default="chain100",
                    help="chain40 (N=40, p=2, chi=64, K=8) is the small profiling case; "
                         "chain100deep has p=8 layers (bond dimension reaches chi=256); "
                         "rcs8cmp prints Fig. 7's engine comparison (vMPO naive / PPT, MPDO)")
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
    if args.workload == "rcs8cmp":
        return run_compare(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
