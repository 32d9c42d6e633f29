#!/usr/bin/env python
"""Benchmark of the divide-and-conquer CheFSI pass on GB300.

Workload (default, `--workload si13824`): the precision-at-scale cell, 13,824 Si atoms (12^3
conventional cells, seeded displacements sigma = 0.1 bohr), global 288^3 grid (h = 0.4275 bohr),
1,728 subdomains of 72^3 points (1-cell core, 1-cell Dirichlet buffer), 528 states per subdomain
(the count that holds a subdomain's electrons, 1.2 x N_e/2 rounded up to 16; `--states literal`
runs 240), Chebyshev degree 20, V_eff the seeded stand-in potential of `synth`.  The subdomains do
not fit in HBM together: the grid runs in waves of equal size in carry mode (one worker of W
subdomain slots re-targeted to each wave, every wave starting from the subspace the previous wave
left; the core rows of every subdomain's orbitals kept on the device for the density).  One step =
one wave: restriction, projector tables and Lanczos bound of its subdomains, one CheFSI pass
(filter, projection, eigensolve, rotation, interior weights), core rows out; every completed
cycle of waves adds the Fermi level, energies and the density on the global grid.
`--workload si64` runs the 64-atom cell (8 resident subdomains of 48^3, 160 states) instead, and
`--workload si4014` the uneven 4,014-atom cell (512 subdomains of 48^3 / 60^3 / 72^3 with their own
state counts, in store-mode waves with an FP16 host store; one step = one full pass).

metric: CheFSI throughput in Gpt.vec/s = sum_alpha m N_d N_s / time, one point-vector being one
Hamiltonian application (+ recurrence) to one grid value of one vector.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CheFSI pass time & filter Gpt·vec/s, mixed vs FP64 at ΔE≤1e-5 Ha/atom"
UNIT = "Gpt*vec/s"


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=24)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp64"],
                   help="fp16 / bf16: FP32 filter + split-FP16 / split-BF16 tensor-core GEMMs; fp64: all FP64")
    p.add_argument("--fp64-steps", type=int, default=1, help="FP64 passes timed for the mixed-vs-FP64 factor")
    p.add_argument("--compare-passes", type=int, default=10,
                   help="passes of both forms from the same start before their energies are compared")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-baseline-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--sample-states", type=int, default=32)
    p.add_argument("--workload", default="si13824", choices=["si13824", "si4014", "si64"])
    p.add_argument("--states", default="consistent", choices=["consistent", "literal"],
                   help="si13824: 528 states per subdomain (consistent) or 240 (literal count, timing only)")
    p.add_argument("--budget-gb", type=float, default=250.0, help="si13824: HBM budget of the wave grid")
    p.add_argument("--fp64-cycles", type=int, default=1,
                   help="si13824: carry cycles of the FP64 and mixed forms on the 512-atom crystal of the same "
                        "subdomain geometry (mixed-vs-FP64 factor and energy difference); 0 skips")
    p.add_argument("--sample-vectors", type=int, default=16, help="si13824: vectors per oracle sample pass")
    p.add_argument("--ncell", type=int, default=12, help="si13824: crystal edge in cells (12; smaller for a quick run)")
    return p.parse_args()


def bench_workload():
    import synth
    w = synth.workload(1)
    return w, synth.veff_erf_wells(w)


def point_vectors(w) -> float:
    return float(sum(w.sub_points(a) * int(w.n_states[a]) for a in range(w.n_sub))) * w.degree


# ---------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, single thread, on a bounded sample
# ---------------------------------------------------------------------------------------------
def cpu_sample_pass(n_states: int, steps: int = 1, warmup: int = 0) -> dict:
    """Oracle CheFSI pass (filter, projection, eigensolve, rotation) on subdomain 0 of the
    workload restricted to the first n_states start vectors; returns the rate in Gpt.vec/s."""
    import synth
    from oracle import chefsi, dc, pseudo
    w, V = bench_workload()
    subs = dc.partition(w)
    H = dc.subdomain_operator(w, subs[0], V, pseudo.projector_norms(w))
    psi = synth.psi0_block(w.psi_seed, subs[0].N, int(w.n_states[0]))[:n_states]
    b = chefsi.lanczos_upper_bound(H, synth.lanczos_start(H.N))
    lam = chefsi.ritz_values(H, psi)
    times = []
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        lam, psi = chefsi.chefsi_pass(H, psi, w.degree, a=float(lam[-1]), b=b, a0=float(lam[0]))
        dc.interior_weights(psi, subs[0])
        t = time.perf_counter() - t0
        if it >= warmup:
            times.append(t)
    t = float(np.mean(times))
    units = float(H.N) * n_states * w.degree
    return {"value": units / t / 1e9, "seconds_per_pass": t, "units": units}


def run_cpu_baseline(n_states: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
                        "--sample-states", str(n_states)], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-400:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": out["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"subdomain 0 of 8, first {n_states} of 160 vectors, one full pass (degree-20 filter, "
                      f"projection, eigensolve, rotation), FP64 numpy, 1 thread; {out['seconds_per_pass']:.1f} s"}


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"xls_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device="cuda", dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM bytes (read + write) of one FP32 stencil launch on the bench workload, measured by ncu for the
# kernel source whose SHA-256 starts with the key; any other source reports null traffic
STENCIL_TRAFFIC = {"056189a407e3c6e6": 1.807340e9}


def stencil_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_2609_13115_gb300", "csrc", "k_stencil_tma.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return STENCIL_TRAFFIC.get(h)


def stencil_bytes_per_launch(w, elem: int) -> float:
    """Algorithmic HBM bytes of one filter-step stencil launch over all subdomains: read Y_k and
    Y_{k-1}, write Y_{k+1} (3 x elem per point-vector) plus V once per subdomain point."""
    tot = 0.0
    for a in range(w.n_sub):
        nd = w.sub_points(a)
        tot += 3.0 * elem * nd * int(w.n_states[a]) + elem * nd
    return tot


def run_si64(args):
    import torch
    from paper_2609_13115_gb300 import xls
    ws, rank, local = dist_setup()
    xls.load()
    w, V = bench_workload()
    stream = torch.cuda.current_stream()
    prec = {"fp16": xls.XLS_MIXED_FP16, "bf16": xls.XLS_MIXED_BF16, "fp64": xls.XLS_FP64}[args.precision]
    ng = int(np.prod(w.n))
    rho_dev = torch.zeros(ng, dtype=torch.float64, device="cuda")

    def make(p):
        g = xls.Grid(w, p, stream=stream.cuda_stream)
        g.set_hamiltonian(V)
        xls.xls_orbitals_random(g.h, w.psi_seed)
        return g

    g = make(prec)

    def step(gh):
        xls.xls_chefsi_batch(gh, w.degree, 1)
        return xls.xls_density(gh, w.n_electrons, w.kT, rho_dev)

    # passes replay CUDA graphs (one per orbital block holding the input; the warm-up captures
    # all three)
    xls.xls_set_graphs(g.h, 1)
    for _ in range(max(args.warmup, 3)):
        step(g.h)
    # the library's autotuner picks the eigensolver cluster size and the Gram K split on this
    # workload (outside the timed region); the passes after it recapture their graphs
    tune = xls.xls_autotune(g.h, 5)
    for _ in range(2):
        step(g.h)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(g.h)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    ms_step = allreduce_max(ms_step, ws)
    _, launches_pass = xls.xls_get_timings(g.h)
    mu, eb_mixed, _ = xls.xls_density(g.h, w.n_electrons, w.kT)
    # per-kernel-class times and the stage split from two further passes launched directly with
    # CUDA events around every launch (outside the timed region)
    xls.xls_set_profiling(g.h, 1)
    kms = np.zeros(8)
    kcnt = np.zeros(8)
    for _ in range(2):
        step(g.h)
        ms, cnt = xls.xls_get_kernel_times(g.h)
        kms += ms
        kcnt += cnt
    stage_ms, _ = xls.xls_get_timings(g.h)
    xls.xls_set_profiling(g.h, 0)
    # density stage: Fermi level, occupations and rho on the device (CUDA events around the call)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    xls.xls_density(g.h, w.n_electrons, w.kT, rho_dev)
    d1.record(stream)
    torch.cuda.synchronize()
    density_ms = d0.elapsed_time(d1)

    # end to end through the C ABI with host buffers, as a warm restart from orbitals kept on the
    # host between passes: H2D of every block from pinned host memory, the pass with the filter
    # bounds the previous pass left (read back with the density, passed in with the blocks, so
    # that the pass needs no Rayleigh-Ritz step of the unfiltered blocks), Fermi level and the
    # density read back to the host
    # (in the grid's own precision: FP32 blocks for the mixed paths, FP64 for the FP64 path)
    f32 = prec != xls.XLS_FP64
    hdt = torch.float32 if f32 else torch.float64
    host_in = [torch.empty((int(w.n_states[a]), w.sub_points(a)), dtype=hdt).pin_memory()
               for a in range(w.n_sub)]
    set_block = xls.xls_orbitals_set_f32 if f32 else xls.xls_orbitals_set
    for a in range(w.n_sub):
        (xls.xls_orbitals_get_f32 if f32 else xls.xls_orbitals_get)(g.h, a, host_in[a].numpy())
    rho_host = torch.empty(ng, dtype=torch.float64).pin_memory()
    bounds = xls.xls_get_bounds(g.h, w.n_sub)
    h2d = sum(t.numel() * t.element_size() for t in host_in) + bounds.size * 8
    d2h = ng * 8 + 3 * 8 + bounds.size * 8
    torch.cuda.synchronize()
    e2e_times = []
    for it in range(max(2, args.steps // 2) + 1):
        t0 = time.perf_counter()
        for a in range(w.n_sub):
            set_block(g.h, a, host_in[a].numpy())
        xls.xls_chefsi_batch(g.h, w.degree, 1, bounds)
        xls.xls_density(g.h, w.n_electrons, w.kT, rho_host.numpy())
        bounds = xls.xls_get_bounds(g.h, w.n_sub)
        if it > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = allreduce_max(float(np.mean(e2e_times)), ws)
    g.close()

    units = point_vectors(w)
    value = units * ws / (ms_step / 1e3) / 1e9
    # roofline of the dominant kernel (the stencil launches of the filter)
    elem = 8 if prec == xls.XLS_FP64 else 4
    stencil_avg_ms = kms[0] / max(kcnt[0], 1)
    bytes_launch = stencil_bytes_per_launch(w, elem)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_launch / (stencil_avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_stencil", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": stencil_traffic() if prec != xls.XLS_FP64 else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_launch": bytes_launch, "avg_launch_ms": round(stencil_avg_ms, 4)}
    kernel_share = {n: round(float(kms[i] / max(kms.sum(), 1e-9)), 4)
                    for i, n in enumerate(["stencil", "nl_project", "nl_back", "gram", "eig", "rotate", "other"])}

    # FP64 form of the same pass for the mixed-vs-FP64 factor, and the energy difference of the two
    # forms once the occupied subspace has converged (both from the same start block)
    fp64 = None
    if prec != xls.XLS_FP64 and args.fp64_steps > 0:
        g64 = make(xls.XLS_FP64)
        gm = make(prec)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        step(g64.h)
        xls.xls_autotune(g64.h, 2)
        step(g64.h)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            step(g64.h)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        for _ in range(args.compare_passes - 1 - args.fp64_steps):
            step(g64.h)
        for _ in range(args.compare_passes):
            step(gm.h)
        rho64 = torch.zeros_like(rho_dev)
        rhom = torch.zeros_like(rho_dev)
        _, eb64, es64 = xls.xls_density(g64.h, w.n_electrons, w.kT, rho64)
        _, ebm, esm = xls.xls_density(gm.h, w.n_electrons, w.kT, rhom)
        g64.close()
        gm.close()
        n_at = len(w.pos)
        fp64 = {"ms_per_step": round(ms64, 3), "mixed_speedup": round(ms64 / ms_step, 2),
                "delta_e_per_atom": abs((ebm - esm) - (eb64 - es64)) / n_at,
                "delta_e_band_per_atom": abs(ebm - eb64) / n_at,
                "rho_rel_l2": float(torch.linalg.norm(rhom - rho64) / torch.linalg.norm(rho64)),
                "passes_compared": args.compare_passes}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:   # the host baseline belongs to the 1-GPU line
        cpu = run_cpu_baseline(args.sample_states)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {xls.XLS_MIXED_FP16: "f32 filter + fp16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_MIXED_BF16: "f32 filter + bf16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "subdomains": w.n_sub, "points_per_subdomain": w.sub_points(0),
                       "states": int(w.n_states[0]), "degree": w.degree,
                       "l2": "inputs larger than L2 (each orbital block 566 MB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "autotuned": {"eig_cluster_ctas": tune[0], "gram_ctas_per_sm": tune[1],
                                     "projection_vectors_per_cta": tune[2]}},
            "filter_gpt_vec_s": round(units / (float(stage_ms[0]) / 1e3) / 1e9, 3),
            "stage_ms": dict({k: round(float(v), 3) for k, v in zip(["filter", "projection", "eig", "rotation"], stage_ms)},
                             density=round(density_ms, 3)),
            "kernel_share": kernel_share,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(units * ws / e2e_s / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches_pass + 2) * args.steps,
            "clocks": clocks,
            "fp64": fp64,
            "mu": mu, "e_band_per_atom": eb_mixed / len(w.pos),
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# The 13,824-atom cell: oracle samples on the host cores
# ---------------------------------------------------------------------------------------------
def si13824_workload(states: str, ncell: int = 12):
    import synth
    return synth.workload(3, consistent=(states == "consistent"), ncell=ncell)


def _oracle_sample(args):
    """One host process: the oracle's CheFSI pass (Lanczos bound, Rayleigh-Ritz of the start
    block, filter, projection, eigensolve, rotation, interior weights) on subdomain `sub` of the
    13,824-atom cell with the first n_vec start vectors (the oracle's operator of the subdomain
    from the atoms near it).  Returns (point-vectors, seconds of the pass)."""
    v_path, states, ncell, sub, n_vec = args
    import synth
    from oracle import chefsi, dc
    w = si13824_workload(states, ncell)
    V = np.load(v_path, mmap_mode="r")
    s = dc.partition(w)[sub]
    H = dc.subdomain_operator_local(w, s, V)
    psi = synth.psi0_block(w.psi_seed, s.N, n_vec, synth.psi0_offsets(w)[sub])
    t0 = time.perf_counter()
    b = chefsi.lanczos_upper_bound(H, synth.lanczos_start(H.N))
    lam = chefsi.ritz_values(H, psi)
    lam, psi = chefsi.chefsi_pass(H, psi, w.degree, a=float(lam[-1]), b=b, a0=float(lam[0]))
    dc.interior_weights(psi, s)
    return float(H.N) * n_vec * w.degree, time.perf_counter() - t0


def _oracle_subspace_sample(args):
    """One host process: the oracle's N_s-quadratic and -cubic steps at the full state count (the
    Gram matrices and the rotation as in chefsi.projection / chefsi.rotate, on n_pts of a
    subdomain's points, and chefsi.generalized_eig) on seeded blocks.  Returns (seconds of the
    products, seconds of the eigensolve)."""
    ns, n_pts = args
    from oracle import chefsi
    rng = np.random.default_rng(2609)
    F = rng.standard_normal((ns, n_pts))
    HF = F + 0.1 * rng.standard_normal((ns, n_pts))
    t0 = time.perf_counter()
    Ms = F @ F.T
    Hs = F @ HF.T
    Hs = 0.5 * (Hs + Hs.T)
    t1 = time.perf_counter()
    _, Y = chefsi.generalized_eig(Hs, Ms)
    t2 = time.perf_counter()
    chefsi.rotate(F, Y)
    t3 = time.perf_counter()
    return (t1 - t0) + (t3 - t2), t2 - t1


class OraclePool:
    """Host processes (spawned, one BLAS thread each) that run oracle samples side by side."""

    def __init__(self, states: str, ncell: int, V: np.ndarray, processes: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="xls_oracle_")
        self.v_path = os.path.join(self.dir, "veff.npy")
        np.save(self.v_path, V)
        self.states = states
        self.ncell = ncell
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            os.environ[k] = "1"
        self.n = processes
        self.ex = cf.ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn"))

    def run(self, subs, n_vec):
        """(total point-vectors, wall seconds, per-sample seconds) of one sample per subdomain."""
        t0 = time.perf_counter()
        out = list(self.ex.map(_oracle_sample, [(self.v_path, self.states, self.ncell, int(a), n_vec) for a in subs]))
        return sum(u for u, _ in out), time.perf_counter() - t0, [t for _, t in out]

    def subspace(self, ns, n_pts):
        """(seconds of the Gram and rotation products, seconds of the eigensolve) in one process."""
        return self.ex.submit(_oracle_subspace_sample, (int(ns), int(n_pts))).result()

    def close(self):
        import shutil
        self.ex.shutdown()
        shutil.rmtree(self.dir, ignore_errors=True)


def si13824_cpu_baseline(w, V, states, ncell, n_vec) -> dict:
    """The oracle on the host cores: one subdomain alone (one thread), then one subdomain per core
    side by side; the rate of the latter is the line's value, and the oracle's full pass of the
    cell is extrapolated from it."""
    cores = os.cpu_count() or 1
    ns, nd = int(w.n_states[0]), w.sub_points(0)
    n_pts = nd // 16
    pool = OraclePool(states, ncell, V, cores)
    try:
        u1, _, t1 = pool.run([0], n_vec)
        subs = np.linspace(0, w.n_sub - 1, cores).astype(int)
        uN, wall, _ = pool.run(subs, n_vec)
        t_prod, t_eig = pool.subspace(ns, n_pts)
    finally:
        pool.close()
    full = point_vectors(w)
    rate = uN / wall / 1e9
    # the full pass of the cell, extrapolated: the sample's pass scaled linearly in the vectors
    # (filter and H applications), plus the N_s^2 products at the full state count (timed on a
    # sixteenth of a subdomain's points, scaled by 16) and the N_s^3 eigensolve, each slowed by the
    # side-by-side factor of the sample and spread over the processes
    slow = wall / t1[0]
    per_sub = t1[0] * ns / n_vec + t_prod * nd / n_pts + t_eig
    full_s = per_sub * slow * w.n_sub / cores
    return {"value": round(rate, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": round(u1 / t1[0] / 1e9, 6),
            "sample": f"{n_vec} of {ns} start vectors of one 72^3 subdomain per process, one full "
                      f"pass each (Lanczos bound, Rayleigh-Ritz, degree-{w.degree} filter, projection, eigensolve, "
                      f"rotation), FP64 numpy, one BLAS thread per process; {cores} subdomains side by side took "
                      f"{wall:.1f} s, one alone {t1[0]:.1f} s; the Gram and rotation products at {ns} states on "
                      f"{n_pts} points {t_prod:.1f} s, the eigensolve at {ns} states {t_eig:.1f} s (one process)",
            "extrapolated_full_pass_s": round(full_s, 1),
            "extrapolated_full_pass_value": round(full / full_s / 1e9, 6)}


# ---------------------------------------------------------------------------------------------
# The 13,824-atom cell on the GPU (carry waves)
# ---------------------------------------------------------------------------------------------
def run_si13824(args):
    import torch
    ws, rank, local = dist_setup()
    w = si13824_workload(args.states, args.ncell)
    import synth
    V = synth.veff_erf_wells(w)
    from paper_2609_13115_gb300 import xls
    xls.load()
    stream = torch.cuda.current_stream()
    prec = {"fp16": xls.XLS_MIXED_FP16, "bf16": xls.XLS_MIXED_BF16, "fp64": xls.XLS_FP64}[args.precision]
    ng = int(np.prod(w.n))
    rho_dev = torch.zeros(ng, dtype=torch.float64, device="cuda")
    budget = int(args.budget_gb * 1e9)
    g = xls.Grid(w, prec, hbm_budget_bytes=budget, stream=stream.cuda_stream)
    g.set_hamiltonian(V)
    xls.xls_wave_carry(g.h, -1)
    n_waves, firsts = xls.xls_get_waves(g.h, w.n_sub)
    W = w.n_sub // n_waves
    xls.xls_orbitals_random(g.h, w.psi_seed)
    ns = int(w.n_states[0])
    nd = w.sub_points(0)
    units_wave = float(W) * nd * ns * w.degree
    state = {"k": 0, "launches": 0, "densities": 0}

    def step():
        k = state["k"] % n_waves
        xls.xls_chefsi_wave(g.h, k, w.degree, 1)
        state["launches"] += xls.xls_get_timings(g.h)[1]
        if k == n_waves - 1:   # a cycle is complete: Fermi level, energies, density (on the device)
            xls.xls_density(g.h, w.n_electrons, w.kT, rho_dev)
            state["densities"] += 1
        state["k"] += 1

    # warm-up: the first wave bootstraps (a, a0) by a Rayleigh-Ritz step of the random block; the
    # autotuner then picks the eigensolver cluster size and the Gram K split on the worker
    for _ in range(max(args.warmup, 3)):
        step()
    tune = xls.xls_autotune(g.h, 3)
    step()
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    state["launches"] = 0
    state["densities"] = 0
    k_first = state["k"]
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms_total = ev[0].elapsed_time(ev[args.steps])
    ms_total = allreduce_max(ms_total, ws)
    ms_step = ms_total / args.steps
    launches = state["launches"] + 3 * state["densities"]
    # one full pass over the cell: the last n_waves consecutive steps ending with a density, if
    # the timed steps hold a whole cycle (else the mean wave time times the wave count)
    pass_ms = None
    for end in range(args.steps - 1, n_waves - 2, -1):
        if (k_first + end) % n_waves == n_waves - 1:
            pass_ms = sum(step_ms[end - n_waves + 1:end + 1])
            break
    # complete the cycle (outside the timed region) and time the density stage alone
    while state["k"] % n_waves != 0:
        step()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    mu, eb, es = xls.xls_density(g.h, w.n_electrons, w.kT, rho_dev)
    d1.record(stream)
    torch.cuda.synchronize()
    density_ms = d0.elapsed_time(d1)
    if pass_ms is None:
        pass_ms = float(np.mean(step_ms)) * n_waves + density_ms
    # per-kernel times and the stage split of one wave with CUDA events around every launch
    xls.xls_set_profiling(g.h, 1)
    step()
    kms, kcnt = xls.xls_get_kernel_times(g.h)
    stage_ms, _ = xls.xls_get_timings(g.h)
    xls.xls_set_profiling(g.h, 0)

    # end to end through the C ABI with host buffers: every step the wave's Ritz values and weights
    # come back to the host; a cycle starts with V_eff going up from pinned host memory and ends
    # with the density coming back
    v_host = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).pin_memory()
    rho_host = torch.empty(ng, dtype=torch.float64).pin_memory()
    lam_host = np.zeros(ns)
    c_host = np.zeros(ns)
    while state["k"] % n_waves != 0:
        step()
    e2e_steps = max(3, args.steps // 4)
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        k = state["k"] % n_waves
        if k == 0:
            xls.xls_hamiltonian_set(g.h, v_host.numpy(), w.pos, w.species_index, w.species)
            h2d += v_host.numel() * 8 + w.pos.size * 8
        xls.xls_chefsi_wave(g.h, k, w.degree, 1)
        for a in range(firsts[k], firsts[k] + W):
            xls.xls_get_eigs_into(g.h, a, lam_host, c_host)
        d2h += W * ns * 16
        if k == n_waves - 1:
            xls.xls_density(g.h, w.n_electrons, w.kT, rho_host.numpy())
            d2h += ng * 8 + 24
        state["k"] += 1
    e2e_s = allreduce_max((time.perf_counter() - t0) / e2e_steps, ws)
    g.close()
    del rho_dev

    value = units_wave * ws / (ms_step / 1e3) / 1e9
    elem = 8 if prec == xls.XLS_FP64 else 4
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    stencil_avg_ms = kms[0] / max(kcnt[0], 1)
    bytes_launch = float(W) * (3.0 * elem * nd * ns + elem * nd)
    achieved = bytes_launch / (stencil_avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_stencil_tma" if prec != xls.XLS_FP64 else "k_stencil",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": stencil_traffic_13824(W, ns) if prec != xls.XLS_FP64 else None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_launch": bytes_launch, "avg_launch_ms": round(stencil_avg_ms, 4)}
    kernel_share = {n: round(float(kms[i] / max(kms.sum(), 1e-9)), 4)
                    for i, n in enumerate(["stencil", "nl_project", "nl_back", "gram", "eig", "rotate", "other"])}

    # the FP64 comparison and the host baseline belong to the 1-GPU line (scaling runs skip them)
    fp64 = None
    if args.fp64_cycles > 0 and prec != xls.XLS_FP64 and ws == 1:
        fp64 = si13824_precision(args, prec)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = si13824_cpu_baseline(w, V, args.states, args.ncell, args.sample_vectors)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {xls.XLS_MIXED_FP16: "f32 filter + fp16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_MIXED_BF16: "f32 filter + bf16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "atoms": len(w.pos), "subdomains": w.n_sub, "points_per_subdomain": nd,
                       "states": ns, "degree": w.degree, "waves": n_waves, "subdomains_per_wave": W,
                       "step": "one wave of subdomains (restriction, tables, Lanczos bound, one CheFSI pass, core "
                               "rows); Fermi level + density at each completed cycle",
                       "l2": "inputs larger than L2 (each subdomain's orbital block "
                             f"{nd * ns * elem / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "autotuned": {"eig_cluster_ctas": tune[0], "gram_ctas_per_sm": tune[1],
                                     "projection_vectors_per_cta": tune[2]}},
            "pass_ms": round(pass_ms, 1),
            # the same point-vectors over the filter stage's time alone (the filter-only rate)
            "filter_gpt_vec_s": round(units_wave / (float(stage_ms[0]) / 1e3) / 1e9, 3),
            "stage_ms_per_wave": dict({k: round(float(v), 3) for k, v in
                                       zip(["filter", "projection", "eig", "rotation"], stage_ms)},
                                      density_per_cycle=round(density_ms, 3)),
            "kernel_share": kernel_share,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(units_wave * ws / e2e_s / 1e9, 3), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "fp64": fp64,
            "mu": mu, "e_band_per_atom": eb / len(w.pos),
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def si13824_precision(args, prec) -> dict:
    """Mixed against FP64 on the 512-atom crystal (4^3 cells) cut like the 13,824-atom cell
    (64 subdomains of 72^3 with Dirichlet buffers, the same states): both forms run the same carry
    schedule from the same start (waves of 8); the last cycle is timed for the mixed-vs-FP64
    factor; band energy minus entropy term per atom and the density are compared after the
    cycles."""
    import torch
    import synth
    from paper_2609_13115_gb300 import xls
    w = synth.workload(3, consistent=(args.states == "consistent"), ncell=4)
    V = synth.veff_erf_wells(w)
    stream = torch.cuda.current_stream()
    out = {}
    for p in (xls.XLS_FP64, prec):
        # a budget below the 64 subdomains' footprint in either precision: waves of 8
        g = xls.Grid(w, p, hbm_budget_bytes=int(100e9), stream=stream.cuda_stream)
        g.set_hamiltonian(V)
        xls.xls_wave_carry(g.h, 8)
        xls.xls_orbitals_random(g.h, w.psi_seed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for c in range(args.fp64_cycles):
            if c == args.fp64_cycles - 1:
                e0.record(stream)
            xls.xls_chefsi_batch(g.h, w.degree, 1)
        e1.record(stream)
        rho = torch.zeros(int(np.prod(w.n)), dtype=torch.float64, device="cuda")
        mu, eb, es = xls.xls_density(g.h, w.n_electrons, w.kT, rho)
        torch.cuda.synchronize()
        out[p] = (e0.elapsed_time(e1), mu, eb - es, rho)
        g.close()
    (t64, mu64, e64, r64), (tm, mum, em, rm) = out[xls.XLS_FP64], out[prec]
    n_at = len(w.pos)
    return {"workload": w.name, "cycles": args.fp64_cycles, "ms_per_cycle_fp64": round(t64, 1),
            "ms_per_cycle_mixed": round(tm, 1), "mixed_speedup": round(t64 / tm, 2),
            "delta_e_per_atom": abs(em - e64) / n_at,
            "rho_rel_l2": float(torch.linalg.norm(rm - r64) / torch.linalg.norm(r64)),
            "mu_fp64": mu64, "mu_mixed": mum}


# DRAM bytes (read + write) per 72^3 subdomain with 528 states of one FP32 stencil launch, measured by ncu
# on a wave of 2 subdomains (4.699759e9 bytes) for the device code (k_stencil_tma.cu from the namespace
# to the host-side section) whose SHA-256 starts with the key; a launch over W subdomains moves W times
# this (the traffic grows with the subdomains a launch covers)
STENCIL_TRAFFIC_13824 = {"5838d36516e2b97b": 4.699759e9 / 2}


def stencil_traffic_13824(n_sub_launch: int, n_states: int):
    import hashlib
    src = open(os.path.join(ROOT, "paper_2609_13115_gb300", "csrc", "k_stencil_tma.cu"), "rb").read()
    dev = src[src.index(b"namespace xls {"):src.index(b"// ---- host side")]
    h = hashlib.sha256(dev).hexdigest()[:16]
    per_sub = STENCIL_TRAFFIC_13824.get(h)
    if per_sub is None or n_states != 528:
        return None
    return per_sub * n_sub_launch


def run_reference_si13824(args):
    """The oracle as it stands on the host cores: each step one pass per core, side by side, each
    on a different 72^3 subdomain with a few start vectors."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    w = si13824_workload(args.states, args.ncell)
    V = synth.veff_erf_wells(w)
    cores = os.cpu_count() or 1
    n_vec = 2
    pool = OraclePool(args.states, args.ncell, V, cores)
    rates, secs = [], []
    try:
        for it in range(args.warmup + args.steps):
            subs = (np.arange(cores) * 7 + it * cores) % w.n_sub
            u, wall, _ = pool.run(subs, n_vec)
            if it >= args.warmup:
                rates.append(u / wall / 1e9)
                secs.append(wall)
    finally:
        pool.close()
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.mean(secs)) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "atoms": len(w.pos), "subdomains": w.n_sub,
                       "points_per_subdomain": w.sub_points(0), "states": int(w.n_states[0]), "degree": w.degree},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(value, 6), "unit": UNIT,
                             "sample": f"per step {cores} processes side by side, each one full pass of a different "
                                       f"72^3 subdomain with {n_vec} of {int(w.n_states[0])} start vectors"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------------
# The 4,014-atom uneven cell (store-mode waves with an FP16 host store)
# ---------------------------------------------------------------------------------------------
def run_si4014(args):
    """Every step one full pass over the 512 uneven subdomains (48^3 / 60^3 / 72^3, their own state
    counts, all sizes in the same launches of a wave): the waves run in store mode, the orbitals of
    every subdomain between passes in a pinned FP16 host store and their core rows on the device,
    then the Fermi level and the density (from the core rows)."""
    import torch
    import synth
    ws, rank, local = dist_setup()
    w = synth.workload(2, consistent=(args.states == "consistent"))
    V = synth.veff_erf_wells(w)
    from paper_2609_13115_gb300 import xls
    xls.load()
    stream = torch.cuda.current_stream()
    prec = {"fp16": xls.XLS_MIXED_FP16, "bf16": xls.XLS_MIXED_BF16, "fp64": xls.XLS_FP64}[args.precision]
    ng = int(np.prod(w.n))
    rho_dev = torch.zeros(ng, dtype=torch.float64, device="cuda")
    g = xls.Grid(w, prec, hbm_budget_bytes=int(args.budget_gb * 1e9), stream=stream.cuda_stream)
    g.set_hamiltonian(V)
    xls.xls_wave_store_fp16(g.h, 1)
    n_waves, _ = xls.xls_get_waves(g.h, w.n_sub)
    xls.xls_orbitals_random(g.h, w.psi_seed)

    def step():
        xls.xls_chefsi_batch(g.h, w.degree, 1)
        return xls.xls_density(g.h, w.n_electrons, w.kT, rho_dev)

    for _ in range(max(args.warmup, 3)):
        step()
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms_step = allreduce_max(e0.elapsed_time(e1) / args.steps, ws)
    stage_ms, launches = xls.xls_get_timings(g.h)
    mu, eb, es = xls.xls_density(g.h, w.n_electrons, w.kT)
    g.close()
    units = point_vectors(w)
    if rank == 0:
        sizes = {}
        for a in range(w.n_sub):
            key = f"{int(w.sub_size(a)[0])}^3"
            sizes.setdefault(key, set()).add(int(w.n_states[a]))
        print(json.dumps({
            "metric": METRIC, "value": round(units * ws / (ms_step / 1e3) / 1e9, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {xls.XLS_MIXED_FP16: "f32 filter + fp16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_MIXED_BF16: "f32 filter + bf16x3 tensor GEMM (f64 eig/fermi)",
                      xls.XLS_FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "atoms": len(w.pos), "subdomains": w.n_sub,
                       "sizes_and_states": {k: sorted(v) for k, v in sorted(sizes.items())},
                       "degree": w.degree, "waves": n_waves, "host_store": "fp16",
                       "step": "one full pass over every wave (orbitals up from and back to the host store), "
                               "Fermi level and density"},
            "filter_gpt_vec_s": round(units / (float(stage_ms[0]) / 1e3) / 1e9, 3),
            "stage_ms": {k: round(float(v), 1) for k, v in zip(["filter", "projection", "eig", "rotation"], stage_ms)},
            "gpu_launches": int(launches) * args.steps, "clocks": clocks,
            "mu": mu, "e_band_per_atom": eb / len(w.pos)}))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = []
    for it in range(args.warmup + args.steps):
        r = cpu_sample_pass(args.sample_states)
        if it >= args.warmup:
            res.append(r)
    value = float(np.mean([r["value"] for r in res]))
    sec = float(np.mean([r["seconds_per_pass"] for r in res]))
    w, _ = bench_workload()
    cores = 1 if os.environ.get("OMP_NUM_THREADS") == "1" else (os.cpu_count() or 1)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "subdomains": w.n_sub, "points_per_subdomain": w.sub_points(0),
                       "states": int(w.n_states[0]), "degree": w.degree},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(value, 6), "unit": UNIT,
                             "sample": f"subdomain 0, first {args.sample_states} of 160 vectors, one full pass"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.cpu_baseline_worker:
        print(json.dumps(cpu_sample_pass(args.sample_states)))
        return
    if args.impl == "reference":
        if args.workload == "si13824":
            run_reference_si13824(args)
        else:
            run_reference(args)
    elif args.workload == "si13824":
        run_si13824(args)
    elif args.workload == "si4014":
        run_si4014(args)
    else:
        run_si64(args)


if __name__ == "__main__":
    main()
