#!/usr/bin/env python3
"""Benchmark of the TBPM time-evolution path on GB300.

Workload: disordered periodic graphene, 2048 x 2048 cells (8,388,608 sites,
1% vacancies -> 8,304,722 orbitals), Anderson onsite U[-0.5, 0.5] eV,
t = -2.7 eV, s = 9.5 eV, 4 random-phase states, 1024 steps of z = s tau =
pi/2 (M = 16 coefficients, 15 sparse products per step), DOS on 4096 bins.
One step of this benchmark is the whole path on that input: Hamiltonian
build on the GPU, initial states, 1024 time steps, correlation and DOS.

Metric: orbital-Chebyshev-steps/s = N_orb * states * steps * (M - 1) / time.
``value`` is the complex-FP32 form (FP64 reductions and norm carry); the
FP64 form, its speedup ratio and the DOS L1 distance between the two are in
``fp64_form``.  ``--impl reference`` times the CPU FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="disordered",
                    choices=["disordered", "batched", "graphene_dos", "differentiable", "tbg",
                             "optical", "quasi"],
                    help="disordered: 2048^2 disordered graphene, 4 states, 1024 steps "
                         "(default, the headline); batched: 32 uneven samples x 16 states, "
                         "512 steps; graphene_dos: 64x64 pristine graphene, 1 state, 1024 steps; "
                         "differentiable: 512^2 graphene, DOS loss, FP64 forward + adjoint; "
                         "tbg: twisted bilayer flake (--side nm), 6 A cutoff, 8 states; "
                         "optical: AC-conductivity correlation of 1024^2 graphene at 300 K; "
                         "quasi: quasi-eigenstates at 4 energies of 1024^2 disordered graphene")
    ap.add_argument("--side", type=float, default=200.0, help="tbg flake side in nm")
    ap.add_argument("--order", default="auto",
                    choices=["auto", "natural", "rcm", "cluster", "morton", "layers"],
                    help="row order of the build (auto: natural); tbg: 'morton' (default) or "
                         "'layers' numbering of the generated flake, or 'rcm'/'cluster' "
                         "reordering of the layer numbering")
    ap.add_argument("--no-halo", action="store_true",
                    help="tbg without --autotune: the plain wide-lane kernel instead of the "
                         "staged-gather one")
    ap.add_argument("--variant", type=int, default=None,
                    help="launch variant bits (TBPM_VARIANT_*) of the FP32 form instead of the "
                         "autotuner (group of 8 states for tbg, 4 otherwise; 64 threads)")
    ap.add_argument("--variant64", type=int, default=None,
                    help="the same for the FP64 form (group of 4 states, 64 threads)")
    ap.add_argument("--L", type=int, default=2048, help="lattice side of the disordered workload")
    ap.add_argument("--time-steps", type=int, default=1024)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shape (profiling runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def n_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def workload_inputs(args, rank):
    from tbpm_inputs import rng, workloads
    if args.workload == "batched":
        w = workloads.batched_graphene()
    elif args.workload == "graphene_dos":
        w = workloads.graphene_dos(n_steps=args.time_steps)
    elif args.workload == "tbg":
        w = workloads.twisted_bilayer_flake(side_nm=args.side, n_steps=args.time_steps)
    else:
        w = workloads.disordered_graphene(L=args.L, n_steps=args.time_steps)
    # weak scaling: rank r propagates its own states (seeds offset by the rank)
    parts = []
    for k in range(w.n_samples):
        n_k = int(w.offsets[k + 1] - w.offsets[k])
        parts.append(rng.phases(w.sample_seeds[k] + 7919 * rank, w.n_states, n_k))
    theta = np.ascontiguousarray(np.concatenate(parts, axis=1))
    return w, theta


def config_dict(w, args, world):
    cs32 = 8 * w.n_states * w.sample.n_orb / 1e6
    d = {"n_orb": int(w.sample.n_orb), "n_bonds": int(w.sample.n_hop),
         "n_samples": w.n_samples, "states_per_sample": w.n_states, "time_steps": w.n_steps,
         "z": "pi/2", "s_eV": w.s, "chebyshev_products_per_step": None,
         "dos_bins": w.n_energies,
         "parallelism": f"replicas x{world} (states sharded, no collective)"}
    if args.workload == "batched":
        d.update(workload="batched_graphene_32_samples", side_lengths=w.info["Ls"],
                 onsite_disorder_eV="U[-W/2,W/2], W ~ U[0,2] per sample",
                 l2=f"inputs larger than L2 (state vectors {cs32:.0f} MB FP32)")
    elif args.workload == "graphene_dos":
        d.update(workload="graphene_dos_64x64", onsite_disorder_eV="none",
                 l2="working set inside L2 (latency-bound; no L2 flush)")
    elif args.workload == "tbg":
        d.update(workload=f"twisted_bilayer_{args.side:g}nm", twist_deg=1.05, cutoff_A=6,
                 entries_per_row=round(2 * w.sample.n_hop / w.sample.n_orb, 1),
                 row_order={"natural": "layer by layer", "rcm": "reverse Cuthill-McKee",
                            "cluster": "RCM, then 128-row breadth-first balls (compact patches)",
                            "auto": "RCM, then 128-row breadth-first balls (compact patches)"}
                 [args.order],
                 l2=f"inputs larger than L2 (state vectors {cs32:.0f} MB FP32, matrix "
                    f"{w.sample.n_hop * 2 * 8 / 1e6:.0f} MB)")
    else:
        d.update(workload=f"disordered_graphene_{args.L}x{args.L}",
                 onsite_disorder_eV="U[-0.5,0.5]", vacancies="1%",
                 l2=f"inputs larger than L2 (state vectors {cs32:.0f} MB FP32 / "
                    f"{2 * cs32:.0f} MB FP64)")
    return d


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in Path(self.path).read_text().splitlines():
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(f[1]), max=float(f[2]), power=float(f[3]),
                                     hw=f[5], hwt=f[6], swt=f[7], pcap=f[8]))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        loaded = [r for r in rows if r["power"] > 300] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded),
                "sm_max_mhz": max(r["max"] for r in rows),
                "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(r["power"] for r in rows),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ reference --
def oracle_sample(w, theta, budget_s=15.0, rows=False):
    """Time the CPU FP64 oracle, as it stands, on a bounded sample of the same
    workload: one state, the first k time steps (k sized to ~budget_s).
    rows=False: the plain serial oracle (one core); rows=True: its twin with
    the paper's OpenMP-over-rows scheme on every core the process may use."""
    import oracle
    fn = oracle.propagate_rows if rows else oracle.propagate
    psi0 = oracle.phase_states(theta[:1])
    t0 = time.perf_counter()
    fn(w.sample, w.s, w.z, 1, psi0)
    one = time.perf_counter() - t0
    k = max(1, min(w.n_steps, int(budget_s / max(one, 1e-9))))
    t0 = time.perf_counter()
    fn(w.sample, w.s, w.z, k, psi0)
    dt = time.perf_counter() - t0
    M = oracle.n_terms(w.z)
    units = w.sample.n_orb * 1 * k * (M - 1)
    cores = oracle.threads() if rows else 1
    how = (f"C, OpenMP over rows, {cores} threads" if rows else "single-threaded C")
    return dict(value=units / dt, unit="orbital-Chebyshev-steps/s", cores=cores, kind="oracle",
                sample=f"1 state x {k} time steps of the {w.sample.n_orb}-orbital workload "
                       f"({how}, {dt:.1f} s)",
                affinity_cores=n_cores()), dt


def run_reference(args):
    """The reference arm: the oracle with the paper's OpenMP-over-rows scheme
    on all host cores, on a bounded sample of the workload per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w, theta = workload_inputs(args, 0)
    M = 16
    per_step_budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    vals = []
    times = []
    sample_desc = None
    cores = 1
    for i in range(args.warmup + args.steps):
        cb, dt = oracle_sample(w, theta, per_step_budget, rows=True)
        if i >= args.warmup:
            vals.append(cb["value"])
            times.append(dt)
            sample_desc = cb["sample"]
            cores = cb["cores"]
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": "orbital-Chebyshev-steps/s", "value": v,
            "unit": "orbital-Chebyshev-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, args, 1),
            "cpu_baseline": {"value": v, "unit": "orbital-Chebyshev-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample_desc,
                             "affinity_cores": n_cores()},
            "e2e": {"value": v, "unit": "orbital-Chebyshev-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    line["config"]["chebyshev_products_per_step"] = M - 1
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- gb300 leg --
def kernel_traffic():
    """DRAM bytes per launch of the interior term kernel from the committed
    ncu summary, valid only while the kernel source is unchanged."""
    p = ROOT / "profiles" / "term_kernel_traffic.json"
    if not p.exists():
        return None, None
    d = json.loads(p.read_text())
    src = ROOT / "paper_2209_00806_gb300" / "csrc" / "cheb_kernels.cu"
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    if d.get("source_sha256") != h:
        return None, d
    return d, d


def reduce_max_time(ms, world, device=None):
    """Slowest rank's time (the whole job's time under weak scaling)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_mean(arr, world, device=None):
    """Average of a per-rank array over the ranks: the one exchange of the
    replica decomposition (each rank's DOS comes from its own random states;
    the DOS is linear in C, so the mean of the ranks' DOS is the DOS of all
    states).  Outside the timed region."""
    if world <= 1:
        return np.asarray(arr, dtype=np.float64)
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(arr, dtype=np.float64), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy() / world


def sample_part(w, k):
    """Sample k of a (possibly batched) workload as its own bond list."""
    from tbpm_inputs import lattice
    smp = w.sample
    lo, hi = int(w.offsets[k]), int(w.offsets[k + 1])
    if w.n_samples == 1:
        return smp
    m = (smp.hop_i >= lo) & (smp.hop_i < hi)
    ons = None if smp.onsite is None else smp.onsite[lo:hi]
    return lattice.Sample(hi - lo, ons, smp.hop_i[m] - lo, smp.hop_j[m] - lo, smp.hop_v[m])


def run_gb300(args):
    import torch
    import torch.distributed as dist

    import paper_2209_00806_gb300 as tb
    from paper_2209_00806_gb300 import _native as N

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w, theta = workload_inputs(args, rank)
    smp = w.sample
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    onsite = smp.onsite if smp.onsite is not None else np.zeros(smp.n_orb)
    d_on = torch.as_tensor(onsite, device=dev)
    d_hi = torch.as_tensor(smp.hop_i, device=dev)
    d_hj = torch.as_tensor(smp.hop_j, device=dev)
    d_hv = torch.as_tensor(smp.hop_v, device=dev)
    d_th = torch.as_tensor(theta, device=dev)
    S, NT, NS = w.n_states, w.n_steps, w.n_samples
    offsets = None if NS == 1 else w.offsets
    M = len(tb.tbpm_bessel_coefficients(w.z))
    units_per_step = smp.n_orb * S * NT * (M - 1)
    prop = tb.Propagator(local, stream.cuda_stream)
    # precisions measured per workload: the first one is the headline `value`
    legs = {"disordered": [N.TBPM_FP32, N.TBPM_FP64], "batched": [N.TBPM_FP32],
            "graphene_dos": [N.TBPM_FP64], "tbg": [N.TBPM_FP32]}[args.workload]
    order = args.order if args.order != "auto" else ("cluster" if args.workload == "tbg"
                                                      else "natural")
    bflags = {"natural": 0, "rcm": N.TBPM_BUILD_REORDER_RCM,
              "cluster": N.TBPM_BUILD_REORDER_CLUSTER}[order]
    graph = args.workload == "graphene_dos"     # launch-latency bound: replay step graphs

    def one_step(precision, flags):
        prop.build(smp.n_orb, d_on, d_hi, d_hj, d_hv, w.s, sample_offsets=offsets, flags=bflags)
        prop.set_phase_states(d_th)
        N.tbpm_propagate(prop.ctx, w.z, NT, precision, None, None, flags)   # C kept on the GPU
        c = prop.correlation()                         # state average per sample (GPU)
        out = [tb.dos(c[k], w.tau, *w.e_range, w.n_energies) for k in range(NS)]
        return out[0][0], np.stack([d for _, d in out])

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    # autotune the launch shape once per precision (outside the timed region)
    tuned = {}
    prop.build(smp.n_orb, d_on, d_hi, d_hj, d_hv, w.s, sample_offsets=offsets, flags=bflags)
    prop.set_phase_states(d_th)
    for prec in legs:
        fixed = args.variant if prec == N.TBPM_FP32 else args.variant64
        if fixed is not None:
            prop.launch_config(prec, 4, 64, fixed)
            tuned[prec] = {"group": 4, "threads": 64, "variant": fixed}
        elif args.no_autotune:
            tuned[prec] = {"group": "default", "threads": 256, "variant": 1}
        else:
            tuned[prec] = prop.autotune(w.z, precision=prec, probe_steps=3)

    def timed(precision):
        flags = N.TBPM_PROP_GRAPH if graph else N.TBPM_PROP_PROFILE
        for _ in range(args.warmup):
            one_step(precision, flags)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        acc = {"ms_term": 0.0, "n_term": 0, "launches": 0, "renorm": 0, "drift": 0.0}
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                res = one_step(precision, flags)
                st = prop.stats()
                acc["ms_term"] += st["ms_term_avg"] * st["term_launches"]
                acc["n_term"] += st["term_launches"]
                acc["launches"] += st["kernel_launches"] + 13   # + builder kernels
                acc["renorm"] += st["renormalisations"]
                acc["drift"] = max(acc["drift"], st["max_norm_drift"])
            e1.record(stream)
            barrier()
        ms = reduce_max_time(e0.elapsed_time(e1), world, dev)
        ms_term = acc["ms_term"] / acc["n_term"] if acc["n_term"] else None
        return dict(ms=ms, res=res, stats=prop.stats(), ms_term=ms_term, clocks=clk.summary(),
                    launches=acc["launches"], renorm=acc["renorm"], drift=acc["drift"])

    runs = {prec: timed(prec) for prec in legs}

    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0

    def roofline(r, key):
        if r["ms_term"] is None:
            return None
        b = r["stats"]["bytes_term"]
        ach = b / (r["ms_term"] * 1e-3) / 1e9
        tr, _ = kernel_traffic()
        traffic = None
        prec = N.TBPM_FP32 if key == "fp32" else N.TBPM_FP64
        # the capture's kernel source and launch variant must be this run's
        if (tr is not None and key in tr and args.workload == "disordered" and args.L == 2048
                and tr[key].get("variant") == tuned.get(prec, {}).get("variant")):
            traffic = tr[key]["dram_bytes_per_launch_full_size"]
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "peak_source": peak_note,
                "kernel": "interior Clenshaw term", "algorithmic_bytes_per_launch": b,
                "ms_per_launch": r["ms_term"]}

    total_units = units_per_step * args.steps * world
    vals = {prec: total_units / (r["ms"] * 1e-3) for prec, r in runs.items()}
    head = legs[0]
    r0 = runs[head]
    name = {N.TBPM_FP32: "fp32", N.TBPM_FP64: "fp64"}

    # end to end through the C ABI with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        h_on = torch.from_numpy(np.ascontiguousarray(onsite)).pin_memory()
        h_hi = torch.from_numpy(np.ascontiguousarray(smp.hop_i)).pin_memory()
        h_hj = torch.from_numpy(np.ascontiguousarray(smp.hop_j)).pin_memory()
        h_hv = torch.from_numpy(np.ascontiguousarray(smp.hop_v)).pin_memory()
        h_th = torch.from_numpy(np.ascontiguousarray(theta)).pin_memory()
        h_c = torch.empty((NS, NT + 1), dtype=torch.complex128).pin_memory()
        offs = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)

        def host_step():
            N.tbpm_build_hamiltonian(prop.ctx, smp.n_orb, h_on.data_ptr(), smp.n_hop,
                                     h_hi.data_ptr(), h_hj.data_ptr(), h_hv.data_ptr(), w.s, NS,
                                     offs, N.TBPM_HOST, bflags)
            N.tbpm_set_phase_states(prop.ctx, S, h_th.data_ptr(), N.TBPM_HOST)
            N.tbpm_propagate(prop.ctx, w.z, NT, head, None, N.TBPM_HOST,
                             N.TBPM_PROP_GRAPH if graph else 0)
            N.tbpm_correlation(prop.ctx, h_c.data_ptr(), N.TBPM_HOST)   # state average (GPU)
            c = h_c.numpy()
            return [tb.dos(c[k], w.tau, *w.e_range, w.n_energies) for k in range(NS)]

        for _ in range(args.warmup):
            host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        barrier()
        dt = reduce_max_time(time.perf_counter() - t0, world, dev)
        h2d = sum(x.numel() * x.element_size() for x in (h_on, h_hi, h_hj, h_hv, h_th))
        d2h = h_c.numel() * h_c.element_size() + NS * S * (NT + 1) * 8   # mean C + norms
        e2e = {"value": total_units / dt, "unit": "orbital-Chebyshev-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * dt / args.steps, "precision": name[head]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        part = sample_part(w, 0)
        from tbpm_inputs import workloads as _wl
        wp = _wl.Workload(w.name, part, np.array([0, part.n_orb]), w.s, w.z, S, NT,
                          w.n_energies, w.e_range, w.seed, [w.sample_seeds[0]])
        cpu, _ = oracle_sample(wp, theta[:, :part.n_orb], 12.0)
        allc, _ = oracle_sample(wp, theta[:, :part.n_orb], 8.0, rows=True)
        cpu["all_cores"] = {k: allc[k] for k in ("value", "cores", "sample")}

    # DOS over the states of every rank (host-side mean of the per-rank DOS)
    d_all = combine_mean(r0["res"][1], world, dev if world > 1 and dist.get_backend() == "nccl"
                         else None)
    if rank == 0:
        cfg = config_dict(w, args, world)
        cfg["chebyshev_products_per_step"] = M - 1
        cfg["state_groups"] = r0["stats"]["group_width"]
        cfg["launch"] = {name[p]: tuned[p] for p in legs}
        line = {
            "metric": "orbital-Chebyshev-steps/s", "value": vals[head],
            "unit": "orbital-Chebyshev-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r0["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if head == N.TBPM_FP32 else "f64", "reductions": "f64",
            "data": "synthetic", "config": cfg,
            "roofline": roofline(r0, name[head]),
            "e2e": e2e, "gpu_launches": int(r0["launches"]),
            "gpu_launches_counts": "the propagation's kernels (tbpm_stats.kernel_launches); the "
                                   "Hamiltonian build's ~20 kernels per step are not counted",
            "clocks": r0["clocks"], "cpu_baseline": cpu,
        }
        de = float(r0["res"][0][1] - r0["res"][0][0])
        line["dos_all_ranks"] = {"states": S * world, "integral": float(np.sum(d_all[0]) * de)}
        if args.workload == "graphene_dos":
            # latency-bound: time per time step and per Chebyshev term of the
            # whole workload step (build, states and DOS included)
            line["latency"] = {"us_per_time_step": 1e3 * r0["ms"] / args.steps / NT,
                               "us_per_term": 1e3 * r0["ms"] / args.steps / NT / (M - 1)}
        if head == N.TBPM_FP32:
            line["fp32_renormalisations"] = r0["renorm"]
            line["fp32_max_norm_drift"] = r0["drift"]
        if N.TBPM_FP64 in runs and head != N.TBPM_FP64:
            r64 = runs[N.TBPM_FP64]
            en, d32 = r0["res"]
            _, d64 = r64["res"]
            # the FP64 term is bound by GB300's FP64 pipe, which issues an add,
            # a multiply or an FMA at one rate: the library's count of the
            # FP64 operations of one interior launch (tbpm_stats.ops_term)
            # against the FMA rate measured here by the library's probe, in
            # operations (one FMA = one operation = 2 flops)
            st64 = r64["stats"]
            ops = float(st64["ops_term"])
            alu = None
            if r64["ms_term"]:
                ach = ops / (r64["ms_term"] * 1e-3) / 1e9
                with ClockSampler(local) as pclk:
                    tf, pms = N.tbpm_fp64_fma_rate(local, 400000)
                peak = tf * 1e3 / 2
                alu = {"bound": "alu", "achieved": ach, "peak": peak,
                       "unit": "G FP64 ops/s", "frac": ach / peak, "traffic": None,
                       "peak_source": f"measured: FP64 FMA probe (tbpm_fp64_fma_rate, "
                                      f"{pms:.0f} ms, SM clock {pclk.summary().get('sm_mhz')} MHz, "
                                      f"{tf * 1e3:.1f} GFLOP/s)",
                       "ops_per_launch": ops}
            line["fp64_form"] = {"value": vals[N.TBPM_FP64], "ms_per_step": r64["ms"] / args.steps,
                                 "dtype": "f64", "roofline": roofline(r64, "fp64"),
                                 "roofline_alu": alu,
                                 "clocks": r64["clocks"], "max_norm_drift": r64["drift"]}
            line["speedup_fp32_over_fp64"] = vals[head] / vals[N.TBPM_FP64]
            line["dos_l1_fp32_vs_fp64"] = float(np.max(np.sum(np.abs(d32 - d64), axis=1)) *
                                                (en[1] - en[0]))
        print(json.dumps(line), flush=True)
    prop.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def host_mem_available():
    """MemAvailable of the host in bytes (Linux), or None."""
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def pinned_copy(t):
    """A page-locked host copy of the device tensor t, and the call that
    frees it: an exact-size cudaHostAlloc buffer (the caching pinned
    allocator would round a 30 GB request up to 32 GiB) viewed as a tensor,
    filled by one device-to-host copy."""
    import ctypes

    import torch
    rt = ctypes.CDLL("libcudart.so")
    nbytes = t.numel() * t.element_size()
    ptr = ctypes.c_void_p()
    rc = rt.cudaHostAlloc(ctypes.byref(ptr), ctypes.c_size_t(max(nbytes, 1)), ctypes.c_uint(0))
    if rc != 0:
        raise RuntimeError(f"cudaHostAlloc of {nbytes} bytes failed ({rc})")
    np_dtype = torch.empty(0, dtype=t.dtype).numpy().dtype
    buf = (ctypes.c_byte * max(nbytes, 1)).from_address(ptr.value)
    a = np.frombuffer(buf, dtype=np_dtype, count=t.numel())
    h = torch.from_numpy(a)
    h.copy_(t.reshape(-1))
    h = h.view(t.shape)

    def release():
        rt.cudaFreeHost(ptr)
    return h, release


def run_tbg(args):
    """Large twisted bilayer: the flake of side --side nm (1.05 degrees, 6 A
    Slater-Koster cutoff, ~68 entries per row, s = 12 eV, 8 FP32 states)
    generated on the GPU by lattice enumeration, numbered along a Morton
    curve of 0.5 nm cells (--order morton, the default; 'layers' is the
    layer-by-layer numbering), built FP32-only without the bond map.  One
    step = build + states + --time-steps steps + correlation + DOS; `value`
    is the propagation rate (the time-step loop is uniform, so a truncated
    run measures the full run's rate), the build is reported on its own."""
    import torch

    import paper_2209_00806_gb300 as tb
    from paper_2209_00806_gb300 import _native as N
    from tbpm_inputs import rng, tbg, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    order = args.order if args.order in ("morton", "layers") else "morton"
    bflags = N.TBPM_BUILD_NO_FP64 | N.TBPM_BUILD_NO_BOND_MAP
    if args.order in ("rcm", "cluster"):
        order = "layers"
        bflags |= {"rcm": N.TBPM_BUILD_REORDER_RCM, "cluster": N.TBPM_BUILD_REORDER_CLUSTER}[args.order]
    seed = workloads.master_seed(5)
    S, NT, s, z = 8, args.time_steps, 12.0, workloads.Z_STEP
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ds = tbg.twisted_bilayer(args.side, order=order, device=dev)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    theta = rng.phases_torch(seed + 7919 * rank, S, ds.n_orb, device=dev)
    torch.cuda.empty_cache()
    M = len(tb.tbpm_bessel_coefficients(z))
    units_per_step = ds.n_orb * S * NT * (M - 1)
    prop = tb.Propagator(local, stream.cuda_stream)
    variant = N.TBPM_VARIANT_ZIGZAG | (N.TBPM_VARIANT_HALO | N.TBPM_VARIANT_STAGED
                                       if not args.no_halo else N.TBPM_VARIANT_WIDE)
    tau = z / s

    # above 600 nm the Hamiltonian is built once, outside the timed steps, and
    # the generator's bond list (90 GB at 1.2 um) freed: the library, its
    # staged-gather copies and the states then fit the 280 GB
    rebuild = args.side <= 600
    n_orb, n_hop = ds.n_orb, ds.n_hop

    def build():
        prop.build(n_orb, None, ds.hop_i, ds.hop_j, ds.hop_v, s, flags=bflags)
        prop.set_phase_states(theta)

    torch.cuda.synchronize(dev)
    tb0 = time.perf_counter()
    build()
    torch.cuda.synchronize(dev)
    first_build_s = time.perf_counter() - tb0
    st0 = prop.stats()
    # page-locked host copies of the bonds and phases for the end-to-end leg
    # (at 1.2 um: 90.6 GB of bonds and 7 GB of phases)
    h_in, e2e_skip = None, None
    if not args.no_e2e:
        need = sum(x.numel() * x.element_size() for x in (ds.hop_i, ds.hop_j, ds.hop_v, theta))
        avail = host_mem_available()
        if avail is not None and need > 0.6 * avail:
            e2e_skip = (f"needs {need / 1e9:.1f} GB of page-locked host memory, "
                        f"{avail / 1e9:.1f} GB available")
        else:
            h_in = [pinned_copy(x) for x in (ds.hop_i, ds.hop_j, ds.hop_v, theta)]
    if not rebuild:
        del ds
        torch.cuda.empty_cache()
    # above 600 nm the launch shape is fixed (the autotuner's candidates
    # would take minutes on a 1e8-row matrix)
    if args.variant is not None or args.no_autotune or not rebuild:
        if args.variant is not None:
            variant = args.variant
        prop.launch_config(N.TBPM_FP32, 8, 64, variant)
        tuned = {"group": 8, "threads": 64, "variant": variant}
    else:
        tuned = prop.autotune(z, precision=N.TBPM_FP32, probe_steps=2)

    def one_step():
        e_b0, e_b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_b0.record(stream)
        if rebuild:
            build()
        e_b1.record(stream)
        N.tbpm_propagate(prop.ctx, z, NT, N.TBPM_FP32, None, None, N.TBPM_PROP_PROFILE)
        c = prop.correlation()
        en, d = tb.dos(c[0], tau, -s, s, 4096)
        return e_b0, e_b1, prop.stats(), d

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc = {"ms_prop": 0.0, "ms_build": 0.0, "ms_term": 0.0, "n_term": 0, "launches": 0, "drift": 0.0}
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            b0, b1, st, d = one_step()
            b1.synchronize()
            acc["ms_build"] += b0.elapsed_time(b1)
            acc["ms_prop"] += st["ms_total"]
            acc["ms_term"] += st["ms_term_avg"] * st["term_launches"]
            acc["n_term"] += st["term_launches"]
            acc["launches"] += st["kernel_launches"]
            acc["drift"] = max(acc["drift"], st["max_norm_drift"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    # end to end through the C ABI from the page-locked host buffers (bonds,
    # phases in; the averaged correlation and the norms out): every step
    # copies the whole bond list to the device and builds from it
    e2e = None
    if h_in is not None:
        h_hi, h_hj, h_hv, h_th = (h for h, _ in h_in)
        h_c = torch.empty((1, NT + 1), dtype=torch.complex128).pin_memory()

        parts = {"build": 0.0, "states": 0.0, "propagate": 0.0, "correlation_dos": 0.0}

        def host_step():
            t = [time.perf_counter()]
            N.tbpm_build_hamiltonian(prop.ctx, n_orb, None, n_hop, h_hi.data_ptr(),
                                     h_hj.data_ptr(), h_hv.data_ptr(), s, 1, None, N.TBPM_HOST,
                                     bflags)
            t.append(time.perf_counter())
            N.tbpm_set_phase_states(prop.ctx, S, h_th.data_ptr(), N.TBPM_HOST)
            torch.cuda.synchronize(dev)
            t.append(time.perf_counter())
            N.tbpm_propagate(prop.ctx, z, NT, N.TBPM_FP32, None, N.TBPM_HOST, 0)
            t.append(time.perf_counter())
            N.tbpm_correlation(prop.ctx, h_c.data_ptr(), N.TBPM_HOST)
            res = tb.dos(h_c.numpy()[0], tau, -s, s, 4096)
            t.append(time.perf_counter())
            for k, key in enumerate(parts):
                parts[key] += t[k + 1] - t[k]
            return res

        host_step()
        torch.cuda.synchronize(dev)
        for key in parts:
            parts[key] = 0.0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        h2d = sum(x.numel() * x.element_size() for x in (h_hi, h_hj, h_hv, h_th))
        d2h = h_c.numel() * h_c.element_size() + S * (NT + 1) * 8
        e2e = {"value": units_per_step * args.steps / dt, "unit": "orbital-Chebyshev-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * dt / args.steps,
               "ms_parts": {k: 1e3 * v / args.steps for k, v in parts.items()},
               "note": "whole step: H2D of bonds and phases, build, propagation, state "
                       "average and DOS"}
        del h_hi, h_hj, h_hv, h_th
        for h, unpin in h_in:
            unpin()
        h_in = None
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    ms_term = acc["ms_term"] / acc["n_term"] if acc["n_term"] else None
    roof = None
    if ms_term:
        ach = st["bytes_term"] / (ms_term * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
                "kernel": "interior Clenshaw term", "algorithmic_bytes_per_launch": st["bytes_term"],
                "ms_per_launch": ms_term}
    value = units_per_step * args.steps / (acc["ms_prop"] * 1e-3)
    line = {"metric": "orbital-Chebyshev-steps/s", "value": value,
            "unit": "orbital-Chebyshev-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "reductions": "f64",
            "data": "synthetic",
            "config": {"workload": f"twisted_bilayer_{args.side:g}nm", "n_orb": int(n_orb),
                       "n_bonds": int(n_hop),
                       "entries_per_row": round(st0["nnz_true"] / n_orb, 2),
                       "stored_entries_incl_padding": int(st0["nnz"]), "twist_deg": 1.05,
                       "cutoff_A": 6, "s_eV": s, "z": "pi/2", "states": S, "time_steps": NT,
                       "chebyshev_products_per_step": M - 1, "dos_bins": 4096,
                       "numbering": {"morton": "Morton curve of 0.5 nm cells, both layers",
                                     "layers": "layer by layer"}[order],
                       "row_order": args.order if args.order in ("rcm", "cluster") else "natural",
                       "launch": tuned, "build_flags": "FP32 only, no bond map",
                       "value_is": "propagation rate (time-step loop, CUDA events); build separate",
                       "l2": f"inputs larger than L2 (state vectors {8 * S * n_orb / 1e6:.0f} MB)",
                       "build": "inside every step" if rebuild else
                                "once before the timed steps (bond list then freed)"},
            "roofline": roof, "e2e": e2e,
            "build_ms_per_step": acc["ms_build"] / args.steps if rebuild else None,
            "first_build_s": first_build_s,
            "generator_s": gen_s,
            "value_including_build": units_per_step * args.steps / (ms * 1e-3),
            "fp32_max_norm_drift": acc["drift"],
            "gpu_launches": int(acc["launches"]), "clocks": clk.summary(),
            "dos_integral": float(np.sum(d) * (2 * s / 4096))}
    if e2e_skip:
        line["e2e_skipped"] = e2e_skip
    print(json.dumps(line), flush=True)
    prop.close()
    return 0


def run_differentiable(args):
    """One step = the DOS loss and its gradient with respect to every hopping
    and onsite energy: FP64 forward, host DOS and DOS adjoint, checkpointed
    adjoint propagation (K = 64)."""
    import torch

    import paper_2209_00806_gb300 as tb
    from paper_2209_00806_gb300 import _native as N
    from tbpm_inputs import workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    w = workloads.differentiable_graphene()
    pw = workloads.pristine_like(w)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    smp = w.sample
    S, NT = w.n_states, w.n_steps
    theta = torch.as_tensor(w.thetas()[0], device=dev)
    d = {k: torch.as_tensor(getattr(smp, k), device=dev) for k in ("hop_i", "hop_j", "hop_v", "onsite")}
    p = tb.Propagator(local, stream.cuda_stream)

    def dos_of(hv, on, flags=0):
        p.build(smp.n_orb, on, d["hop_i"], d["hop_j"], hv, w.s)
        p.set_phase_states(theta)
        N.tbpm_propagate(p.ctx, w.z, NT, N.TBPM_FP64, None, None, flags)
        return tb.dos(p.correlation()[0], w.tau, *w.e_range, w.n_energies)[1]

    target = dos_of(torch.as_tensor(pw.sample.hop_v, device=dev),
                    torch.zeros(smp.n_orb, dtype=torch.float64, device=dev))

    phases = {"fwd": [], "adj": []}

    def one_step():
        ef = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ef[0].record(stream)
        D = dos_of(d["hop_v"], d["onsite"], N.TBPM_PROP_PROFILE)
        ef[1].record(stream)
        phases["st"] = p.stats()
        loss = float(np.sum((D - target) ** 2))      # the example loss (user code)
        g = tb.dos_adjoint(2.0 * (D - target), NT, w.tau, *w.e_range)
        gbar = p.correlation_adjoint(NT, torch.as_tensor(g[None, :], device=dev))
        ef[2].record(stream)
        gh, go = p.adjoint(w.z, NT, gbar, K=64)
        ef[3].record(stream)
        ef[3].synchronize()
        phases["fwd"].append(ef[0].elapsed_time(ef[1]))
        phases["adj"].append(ef[2].elapsed_time(ef[3]))
        phases["adj_launches"] = p.stats()["kernel_launches"]
        return loss, gh, go

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            loss, gh, go = one_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    M = len(tb.tbpm_bessel_coefficients(w.z))
    units = smp.n_orb * S * NT * (M - 1) * args.steps
    # FP64 forward term: HBM and FP64-pipe rooflines (measured FP64 FMA peak);
    # the adjoint's sparse products: the forward pass, the per-segment
    # recomputation, the per-step polynomials and the conjugate terms,
    # about N (4M - 5) per state
    st = phases["st"]
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    tf, _ = N.tbpm_fp64_fma_rate(local, 400000)
    # one launch advances one state group: the library's operation count is
    # for the mean group width (3 states run as 2 + 1), as bytes_term is
    ops = float(st["ops_term"])
    ms_t = st["ms_term_avg"]
    peak = tf * 1e3 / 2
    roof = {"bound": "alu", "achieved": ops / (ms_t * 1e-3) / 1e9, "peak": peak,
            "unit": "G FP64 ops/s", "frac": ops / (ms_t * 1e-3) / 1e9 / peak,
            "traffic": None, "kernel": "FP64 interior Clenshaw term of the forward pass",
            "peak_source": "measured: FP64 FMA probe (tbpm_fp64_fma_rate), one FMA = one op",
            "hbm": {"achieved": st["bytes_term"] / (ms_t * 1e-3) / 1e9, "peak": hbm,
                    "frac": st["bytes_term"] / (ms_t * 1e-3) / 1e9 / hbm},
            "ms_per_launch": ms_t, "ops_per_launch": ops,
            "algorithmic_bytes_per_launch": st["bytes_term"]}
    adj_ms = statistics.median(phases["adj"])
    adj_units = smp.n_orb * S * NT * (4 * M - 5)
    line = {"metric": "orbital-Chebyshev-steps/s", "value": units / (ms * 1e-3),
            "unit": "orbital-Chebyshev-steps/s (forward steps of a loss+gradient evaluation)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "differentiable_graphene_512x512", "n_orb": int(smp.n_orb),
                       "n_bonds": int(smp.n_hop), "states": S, "time_steps": NT,
                       "checkpoint_every": 64, "dos_bins": w.n_energies,
                       "loss": "sum_E (D - D_pristine)^2",
                       "gradients": "all t_b and eps_i"},
            "loss": loss, "grad_norm_hop": float(torch.linalg.norm(gh)),
            "grad_norm_onsite": float(torch.linalg.norm(go)),
            "roofline": roof,
            "forward_ms": statistics.median(phases["fwd"]), "adjoint_ms": adj_ms,
            "adjoint_products_per_s": adj_units / (adj_ms * 1e-3),
            "adjoint_kernel_launches": phases["adj_launches"],
            "gpu_launches": int(p.stats()["kernel_launches"]), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    p.close()
    return 0


def run_observables(args):
    """One step = the whole optical-conductivity correlation (Fermi-operator
    preparation in FP64, FP32 propagation of psi, psi_2, psi_1x, psi_1y, the
    per-step current observer) or the whole quasi-eigenstate computation
    (forward and backward FP32 runs with the per-step accumulation).  Inputs
    resident in HBM; the matrix build is inside the step."""
    import torch

    import paper_2209_00806_gb300 as tb
    from paper_2209_00806_gb300 import _native as N
    from tbpm_inputs import lattice, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    optical = args.workload == "optical"
    w = (workloads.optical_graphene(n_steps=args.time_steps) if optical
         else workloads.quasi_graphene(n_steps=args.time_steps // 2))
    smp = w.sample
    S, NT = w.n_states, w.n_steps
    theta = torch.as_tensor(w.thetas()[0], device=dev)
    d = {k: (None if getattr(smp, k) is None else torch.as_tensor(getattr(smp, k), device=dev))
         for k in ("hop_i", "hop_j", "hop_v", "onsite")}
    p = tb.Propagator(local, stream.cuda_stream)
    M = len(tb.tbpm_bessel_coefficients(w.z))
    beta = 1.0 / (8.617333262e-5 * 300.0)
    if optical:
        dr = lattice.bond_vectors(smp)
        dx = torch.as_tensor(np.ascontiguousarray(dr[:, 0]), device=dev)
        dy = torch.as_tensor(np.ascontiguousarray(dr[:, 1]), device=dev)
        K_f = len(tb.fermi_coefficients(beta * w.s, 0.0))
        out = torch.empty((1, S, 4, NT + 1), dtype=torch.complex128, device=dev)
        # orbital-Chebyshev products: 4 lanes x (Fermi terms on 4 lanes + steps x (M - 1))
        units = smp.n_orb * S * 4 * (K_f + NT * (M - 1))
    else:
        E = np.array(w.info["energies"])
        out = torch.empty((E.shape[0], S, smp.n_orb), dtype=torch.complex128, device=dev)
        norms = np.empty((E.shape[0], S, 1))
        units = smp.n_orb * S * 2 * NT * (M - 1)

    def one_step():
        p.build(smp.n_orb, d["onsite"], d["hop_i"], d["hop_j"], d["hop_v"], w.s)
        p.set_phase_states(theta)
        if optical:
            N.tbpm_set_bond_vectors(p.ctx, dx, dy)
            N.tbpm_ac_correlation(p.ctx, w.z, NT, beta, 0.0, N.TBPM_FP32, out, None,
                                  N.TBPM_PROP_PROFILE)
        else:
            N.tbpm_quasi_eigenstates(p.ctx, w.z, NT, E, N.TBPM_FP32, out, norms, None,
                                     N.TBPM_PROP_PROFILE)

    p.build(smp.n_orb, d["onsite"], d["hop_i"], d["hop_j"], d["hop_v"], w.s)
    p.set_phase_states(theta)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st = p.stats()
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) \
        if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    roof = None
    if st["ms_term_avg"]:
        ach = st["bytes_term"] / (st["ms_term_avg"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
                "kernel": "interior Clenshaw term (last run of the step)",
                "algorithmic_bytes_per_launch": st["bytes_term"],
                "ms_per_launch": st["ms_term_avg"]}
    cfg = {"workload": f"{w.name}_{w.info['L']}x{w.info['L']}", "n_orb": int(smp.n_orb),
           "n_bonds": int(smp.n_hop), "states": S, "time_steps": NT, "z": "pi/2", "s_eV": w.s,
           "l2": "inputs larger than L2"}
    if optical:
        cfg.update(T_kelvin=300.0, mu_eV=0.0, fermi_terms=K_f, lanes="psi, f psi, (1-f) J_x psi, "
                   "(1-f) J_y psi", correlations="xx, xy, yx, yy")
    else:
        cfg.update(energies_eV=w.info["energies"], runs="forward and backward, Hann window")
    line = {"metric": "orbital-Chebyshev-steps/s", "value": units * args.steps / (ms * 1e-3),
            "unit": "orbital-Chebyshev-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "reductions": "f64",
            "data": "synthetic", "config": cfg, "roofline": roof,
            "ms_propagation_last_run": st["ms_total"],
            "gpu_launches": int(st["kernel_launches"]), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    p.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "differentiable":
        return run_differentiable(args)
    if args.workload in ("optical", "quasi"):
        return run_observables(args)
    if args.workload == "tbg":
        return run_tbg(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
