#!/usr/bin/env python3
"""Throughput benchmark of the on-the-fly property MD step on GB300.

One step = velocity-Verlet kick/drift, neighbour-list rebuild when due, LJ
pair forces with per-particle energy and virial, second kick with the
stress / heat-flux reduction, and correlator samples of the stress, heat
flux and every atom's velocity (u = 1).  Workload: the 2,048,000-atom LJ
liquid (80^3 fcc cells x 4, rho* = 0.8442, T* = 0.722, rc = 2.5, dt = 0.005)
in the mixed form (FP32 forces / fluxes / correlator products, FP64
positions, velocities, reductions and lag sums), melted before timing.
Prints one JSON line (rank 0).

--impl reference times the FP64 CPU oracle on the host cores instead.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s with on-the-fly correlators vs plain FP64 GPU; time-to-viscosity at ≤2% err"
UNIT = "atom-steps/s"
CELLS = 80  # 4 * 80^3 = 2,048,000 atoms
# skin 0.4 sigma: on the tile-window path the 2,048,000-atom step measured 0.709 ms against 0.736
# at 0.3 (cells of 2.92 instead of 2.86 sigma: longer lists, rarer rebuilds)
RHO, T_STAR, RC, DT, SKIN = 0.8442, 0.722, 2.5, 0.005, 0.4
SPEC = dict(stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=(8, 16, 2, 1))
# untimed steps of the timed system before its warm-up: twice the period of the velocity
# correlator's last block (m^(b-1) = 128 steps for b = 8, m = 2), so every block holds samples and
# the timed steps carry the push work of a long run (its pushes into the higher blocks cost ~60 %
# more per step than in the first 20 steps after the correlators start)
VACF_FILL = 256
PAIR_FLOP_PER_ATOM = 0.5 * RHO * (4.0 / 3.0) * math.pi * RC ** 3 * 50.0  # unique pairs x 50 flop


def workload_name(n, start="melted"):
    return (f"LJ liquid {n:,} atoms (fcc {round((n / 4) ** (1 / 3))}^3 x 4 {start}), rho*={RHO}, T*={T_STAR}, rc={RC} shifted, "
            f"dt={DT}, velocity Verlet NVE; on-the-fly correlators: stress xy/xz/yz and heat flux "
            f"(b=12,p=16,m=2,u=1), per-atom VACF over all atoms (b=8,p=16,m=2,u=1)")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.i0, self.i1 = 0, None

    def start(self):
        self.i0 = len(self.lines)

    def stop(self):
        time.sleep(0.15)  # let the sample taken at the end of the region arrive
        self.i1 = len(self.lines)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.i0:self.i1]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measure_fp32_peak(pkg, gpu_index, iters=40000, reps=5):
    """The FP32 FMA rate of this GPU, measured: md_fp32_peak's FMA-chain
    kernel over a grid that fills every SM, scalar FMAs and paired f32x2
    FMAs, timed with CUDA events while nvidia-smi samples the SM clock.  The
    larger of the two rates is the peak."""
    out = {}
    for name, paired in (("fma_f32", False), ("fma_f32x2", True)):
        pkg.fp32_peak(paired, iters=max(1, iters // 50), reps=1)  # clocks up, kernel loaded
        with ClockSampler(gpu_index) as clk:
            clk.start()
            flops, ms, sms = pkg.fp32_peak(paired, iters=iters, reps=reps)
            clk.stop()
        out[name] = {"tflops": flops / (ms / 1e3) / 1e12, "ms_per_launch": ms, "clocks": clk.summary()}
    best = max(("fma_f32", "fma_f32x2"), key=lambda k: out[k]["tflops"])
    out.update({"peak_tflops": out[best]["tflops"], "from": best, "sm_count": sms,
                "how": "md_fp32_peak: every SM filled with 256-thread CTAs, 8 independent FMA chains per thread, "
                       f"{iters} x 16 FMAs per chain, {reps} launches timed with CUDA events after one warm-up"})
    return out


def vacf_bytes_per_push(t, b, p, m, nseries, esz, kmin=0):
    """Algorithmic HBM bytes of push t of a grouped correlator: per series,
    block 0 reads the new sample and p-1 older ring entries and writes one;
    each higher block the push reaches reads m entries of the block below,
    p - p/m older entries (fewer while filling) and writes one.  kmin = 1
    counts the higher blocks only."""
    tot = 0
    Mk = 1
    for k in range(b):
        if k > 0:
            Mk *= m
            if t % Mk:
                break
        nk = t // Mk
        if k < kmin:
            continue
        lo = 0 if k == 0 else p // m
        nl = max(0, min(p - 1, nk - 1) - lo + 1)
        older = nl - (1 if lo == 0 and nl > 0 else 0)
        reads = (1 if k == 0 else m) + older
        tot += (reads + 1) * esz
    return tot * nseries


def vacf_bytes_blocked(done, t_end, b, p, m, nseries, esz, block=8):
    """Algorithmic HBM bytes of the velocity pushes done+1 .. t_end applied
    `block` at a time (as md_step applies them for p <= 16): per pass and
    series, block 0 reads the p-1 most recent ring entries once, reads each
    new sample from its input slot and writes it to the ring; the higher
    blocks are applied push by push (vacf_bytes_per_push with kmin = 1)."""
    tot = 0
    while done < t_end:
        nnew = min(block, t_end - done)
        tot += (min(p - 1, done) + 2 * nnew) * esz * nseries
        for t in range(done + 1, done + nnew + 1):
            tot += vacf_bytes_per_push(t, b, p, m, nseries, esz, kmin=1)
        done += nnew
    return tot


def vacf_timed_bytes(args, b, p, m, n, pre=VACF_FILL):
    """Bytes of the velocity pushes applied inside the timed region.  A
    blocked pass runs whenever a whole block of pushes waits in the input
    slots; a partial block waits across md_step calls until the next
    readout.  Nothing is read between the untimed calls (`pre` steps, then
    the warm-up) and the timed call, so the timed call applies the whole
    blocks that complete inside it: pushes (pre + warmup) // block * block + 1
    .. (pre + warmup + steps) // block * block."""
    block = min(8, p - m + 1)
    done0 = (pre + args.warmup) // block * block
    done1 = (pre + args.warmup + args.steps) // block * block
    return vacf_bytes_blocked(done0, done1, b, p, m, 3 * n, 4, block)


def pair_mode_for(pkg, precision):
    """The pair path of a Lennard-Jones form: tile windows for the mixed form,
    global Verlet lists for FP64."""
    return pkg.MD_PAIR_TILES if precision == pkg.MD_PREC_MIXED else pkg.MD_PAIR_VERLET


def melt(sysg, target_T, steps, every=10):
    for _ in range(steps // every):
        sysg.step(every)
        T = sysg.observables()["T"]
        sysg.scale_velocities(math.sqrt(target_T / T))


def prepare_state(pkg, synth, seed, cells=CELLS, melt_steps=600):
    """Melted liquid at T* (untimed): rescale to T* = 2.0 for melt_steps
    steps, then to T* = 0.722 for melt_steps steps, on the mixed path."""
    s = synth.lj_system(cells, rho=RHO, T=T_STAR, seed=seed)
    p = pkg.make_params(s["n"], s["L"], rc=RC, dt=DT, skin=SKIN, precision=pkg.MD_PREC_MIXED,
                        stress=None, heatflux=None, vacf=None)
    g = pkg.System(p, s["r"], s["v"])
    melt(g, 2.0, melt_steps)
    melt(g, T_STAR, melt_steps)
    st = g.particles()
    g.close()
    return s, st


def run_ours(args):
    import torch

    from paper_2503_07526_gb300 import replicas

    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2503_07526_gb300 as pkg
    from paper_2503_07526_gb300 import synth

    pkg.lib()
    s, st = prepare_state(pkg, synth, seed=replicas.replica_seed(1, rank), cells=args.cells,
                          melt_steps=100 if args.quick else 600)
    n, L = s["n"], s["L"]
    pair_mode = pkg.MD_PAIR_TILES if args.pair == "tiles" else pkg.MD_PAIR_VERLET
    p = pkg.make_params(n, L, rc=RC, dt=DT, skin=args.skin, precision=pkg.MD_PREC_MIXED, pair_mode=pair_mode,
                        list_build=args.list_build, **SPEC)
    g = pkg.System(p, st["r"], st["v"])
    g.step(VACF_FILL)
    g.step(args.warmup)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # --- timed region: K steps of the product launch path (8-step CUDA graphs),
    # every kernel class bracketed by CUDA events recorded inside the graphs
    g.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        clk.start()
        e0.record(stream)
        g.step(args.steps)
        e1.record(stream)
        barrier()
        clk.stop()
    ms_total = e0.elapsed_time(e1)
    ktimes = g.kernel_times()
    g.set_timing(False)
    ms_total = replicas.max_over_ranks(ms_total, dist, device="cuda")  # the slowest rank
    ms_step = ms_total / args.steps
    value = replicas.weak_scaling_rate(n, args.steps, world, ms_total / 1e3)

    # the same graphs without the event records, for reference (one untimed
    # call first captures them)
    g.step(args.steps)
    barrier()
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    barrier()
    graph_ms_step = e0.elapsed_time(e1) / args.steps
    g.close()
    if args.quick:  # profiling runs: timed region only
        if rank == 0:
            print(json.dumps({"quick": True, "n_atoms": n, "ms_per_step": ms_step, "graph_ms_per_step": graph_ms_step,
                              "kernel_ms": ktimes}), flush=True)
        return

    # --- plain FP64 GPU path on the same state (the comparison form)
    k64 = max(3, args.steps // 10)
    p64 = pkg.make_params(n, L, rc=RC, dt=DT, skin=args.skin, precision=pkg.MD_PREC_FP64, **SPEC)
    g64 = pkg.System(p64, st["r"], st["v"])
    g64.step(2)
    barrier()
    e0.record(stream)
    g64.step(k64)
    e1.record(stream)
    barrier()
    ms64 = e0.elapsed_time(e1) / k64
    g64.close()

    # --- end to end through the C ABI from host buffers (pinned host memory,
    # allocated and filled before the timed region)
    r_host = torch.from_numpy(np.ascontiguousarray(st["r"])).pin_memory()
    v_host = torch.from_numpy(np.ascontiguousarray(st["v"])).pin_memory()
    barrier()
    t0 = time.perf_counter()
    ge = pkg.System(p, r_host, v_host)  # host -> device copy of the state
    ge.step(args.steps)
    obs = ge.observables()
    for which in (pkg.MD_CORR_STRESS, pkg.MD_CORR_HEATFLUX, pkg.MD_CORR_VACF):
        ge.corr(which).read(-1)  # device -> host readout of every correlator
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ge.close()
    e2e_s = replicas.max_over_ranks(e2e_s, dist, device="cuda")
    h2d = (2 * 3 * n * 8) / args.steps
    d2h = (8 * 16 + 3 * 2 * 8 * (12 * 16 + 12 * 16 + 8 * 16)) / args.steps

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks, peak_kind = measured_peaks()
    fp32 = measure_fp32_peak(pkg, local)
    fp32_peak_tflops = fp32["peak_tflops"]
    # roofline of the dominant kernel class
    shares = {k: v[0] for k, v in ktimes.items()}
    kern_ms = sum(shares.values())
    dom = max(shares, key=shares.get)
    if dom == "vacf":
        b, pp, m, _ = SPEC["vacf"]
        achieved = vacf_timed_bytes(args, b, pp, m, n) / (ktimes["vacf"][0] / 1e3) / 1e9
        roof = {"kernel": "k_push_block0 + k_push_higher (per-atom VACF push, 8 pushes per pass)",
                "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{peak_kind} hbm_gbs"}
    else:
        flops = PAIR_FLOP_PER_ATOM * n * ktimes["pair"][1]
        achieved = flops / (ktimes["pair"][0] / 1e3) / 1e12
        kname = "k_pair_tile" if args.pair == "tiles" else "k_pair_mixed"
        roof = {"kernel": f"{kname} (LJ forces + per-particle energy and virial, mixed form)", "bound": "alu",
                "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak_tflops,
                "peak_source": f"measured in this run: md_fp32_peak ({fp32['from']}), median SM clock "
                               f"{fp32[fp32['from']]['clocks'].get('sm_mhz')} MHz"}
    roof["traffic"] = committed_traffic(roof["kernel"].split()[0])
    # secondary kernel roofline (pair ALU / VACF HBM) for completeness
    b, pp, m, _ = SPEC["vacf"]
    vacf_gbs = vacf_timed_bytes(args, b, pp, m, n) / (ktimes["vacf"][0] / 1e3) / 1e9
    pair_tf = PAIR_FLOP_PER_ATOM * n * ktimes["pair"][1] / (ktimes["pair"][0] / 1e3) / 1e12

    launches_per_step = 12  # kick_drift, 5 sort kernels, list build, pair, kick_reduce, scalar push, 2 VACF push kernels
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 forces/fluxes/products + f64 state/reductions/lag sums",
        "data": "synthetic (seeded fcc start melted at T*=2.0 then 0.722, Maxwell-Boltzmann velocities)",
        "config": {"workload": workload_name(n), "n_atoms": n, "precision": "mixed", "pair": ("tile windows (MD_PAIR_TILES)" if args.pair == "tiles" else "global Verlet lists") + f", skin {args.skin}",
                   "replicas": "one independent system per GPU" if world > 1 else "one system",
                   "l2": "inputs larger than L2 (state + neighbour lists + VACF ring about 5 GB)",
                   "timing": "CUDA events around every kernel class, recorded inside the replayed 8-step CUDA "
                             "graphs (the product launch path; velocity pushes overlap the next step), after "
                             f"{VACF_FILL} untimed steps that fill every block of the velocity correlator "
                             "(steady-state push work) and the warm-up steps"},
        "clocks": clk.summary(),
        "e2e": {"value": replicas.weak_scaling_rate(n, args.steps, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": "md_init from pinned host arrays + md_step(K) + md_observables + corr_read of all correlators"},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "kernel_ms": {k: {"total_ms": v[0], "launch_brackets": v[1], "share": v[0] / kern_ms if kern_ms else None}
                      for k, v in ktimes.items()},
        "secondary_roofline": {"pair_alu_tflops": pair_tf, "pair_frac_fp32_peak": pair_tf / fp32_peak_tflops,
                               "vacf_hbm_gbs": vacf_gbs, "vacf_frac_hbm": vacf_gbs / peaks["hbm_gbs"]},
        "graph_ms_per_step": graph_ms_step,
        "fp32_peak": fp32,
        "fp64_gpu": {"ms_per_step": ms64, "value": world * n / (ms64 / 1e3), "steps": k64,
                     "speedup_mixed_over_fp64": ms64 / ms_step},
    }
    if world == 1 and not args.no_ensemble:
        out["batched_ensemble"] = run_batched(pkg, synth, 200, torch)
        out["ionic_melt"] = run_ionic(pkg, synth, torch)
        tail, out["learned_tail"] = run_learned_tail(pkg, torch)
        out["time_to_viscosity"] = run_time_to_viscosity(pkg, synth, torch, tail=tail)
        tail.net.close()
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(st, s, budget_s=args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def c4_ensemble(pkg, synth, count=256, seed=11):
    """The batched-replica workload: count LJ replicas with sizes drawn
    log-uniformly in [500, 32,000] atoms (fcc k^3 x 4, k in [5, 20]),
    density uniform in [0.7, 0.9] and T* uniform in [0.7, 2.0]."""
    u = synth.uniform01(seed, 3 * count).reshape(3, count)
    reps, temps = [], []
    for k in range(count):
        n_target = math.exp(math.log(500) + u[0, k] * (math.log(32000) - math.log(500)))
        cells = synth.cells_for_atoms(n_target)
        rho = 0.7 + 0.2 * u[1, k]
        T = 0.7 + 1.3 * u[2, k]
        s = synth.lj_system(cells, rho=rho, T=T, seed=seed * 1000 + k)
        reps.append(dict(r=s["r"], v=s["v"], box=s["L"]))
        temps.append(T)
    return reps, np.array(temps)


def melt_replicas(g, temps, steps_hot=600, steps_cold=600, every=10):
    """Velocity rescaling per replica: all to T* = 2.0, then each to its own T*."""
    from paper_2503_07526_gb300 import learned_tail as lt

    lt.melt(g, temps, steps_hot, steps_cold, every)


def run_batched(pkg, synth, steps, torch):
    """Throughput of the 256-replica uneven ensemble in one handle (mixed
    form on the tile-window path, stress and heat-flux correlators)."""
    reps, temps = c4_ensemble(pkg, synth)
    p = pkg.make_params(1, 1.0, rc=RC, dt=DT, skin=0.2, precision=pkg.MD_PREC_MIXED, pair_mode=pkg.MD_PAIR_TILES,
                        autotune=True, stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=None)
    g = pkg.System(p, replicas=reps)  # md_init picks the cell tiles and CTA size on the ensemble itself
    melt_replicas(g, temps, 300, 300)
    g.reset_correlators()
    g.step(5)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cfg = g.config()
    g.close()
    return {"workload": "256 LJ replicas, sizes log-uniform in [500, 32000] atoms, rho* uniform in [0.7, 0.9], "
                        "T* uniform in [0.7, 2.0], rc=2.5, dt=0.005, skin 0.2, mixed form (tile windows; cell tiles and "
                        "CTA size autotuned at md_init), one handle, one graph launch per 8 steps; stress and heat-flux "
                        "correlators per replica",
            "atoms": cfg["atoms"], "replicas": cfg["replicas"], "steps": steps, "ms_per_step": ms / steps,
            "value": cfg["atoms"] * steps / (ms / 1e3), "unit": UNIT,
            "tiles": cfg["tiles"], "tile_threads": cfg["tile_threads"], "window_capacity": cfg["window_capacity"],
            "tile_extent": list(cfg["tile_extent"])}


IONIC = dict(cells=40, rho=0.031, T_K=1300.0, masses=(22.99, 35.45), A=1200.0, brho=0.32, C=10.0, rc=10.0,
             skin=1.0, alpha=0.3, mesh=128, order=8, dt_fs=1.0)
KB_EV = 8.617333262e-5           # eV / K
FS_PER_UNIT = 10.1805055         # fs per (A sqrt(amu / eV))


def run_ionic(pkg, synth, torch, steps=100, fp64_steps=10, cells=None):
    """Throughput of the ionic melt (rock salt 40^3 x 8 = 512,000 ions at
    0.031 ions/A^3, +-1 e, Na/Cl masses, Buckingham A=1200 eV, rho=0.32 A,
    C=10 eV A^6, rc=10 A, SPME alpha=0.3/A on a 128^3 mesh, order 8,
    dt = 1 fs, started from the lattice at 1300 K) in the mixed form and in
    plain FP64, with the per-kernel-class split."""
    c = IONIC
    cells = cells or c["cells"]
    s = synth.ionic_system(cells, c["rho"], KB_EV * c["T_K"], seed=9, masses=c["masses"], jitter=0.2)
    n, L = s["n"], s["L"]
    out = {"workload": f"binary ionic melt, {n} ions (rock salt {cells}^3 x 8), L = {L:.1f} A, Buckingham + SPME "
                       f"Ewald ({c['mesh']}^3 mesh, order {c['order']}, alpha {c['alpha']}/A, rc {c['rc']} A), "
                       "dt 1 fs, stress and heat-flux correlators with per-particle reciprocal energy and virial",
           "n_ions": n}
    forms = [("mixed", pkg.MD_PREC_MIXED, steps)] + ([("fp64_gpu", pkg.MD_PREC_FP64, fp64_steps)] if fp64_steps else [])
    for name, prec, k in forms:
        p = pkg.make_params(n, L, rc=c["rc"], dt=c["dt_fs"] / FS_PER_UNIT, skin=c["skin"], precision=prec,
                            masses=c["masses"], potential=pkg.MD_POT_BUCK_EWALD, charges=(1.0, -1.0),
                            buckingham=(c["A"], c["brho"], c["C"]), ewald_alpha=c["alpha"], mesh=c["mesh"],
                            order=c["order"], stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=None)
        g = pkg.System(p, s["r"], s["v"], types=s["types"])
        g.step(5)
        g.set_timing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(k)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        kt = g.kernel_times()
        g.set_timing(False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(k)
        torch.cuda.synchronize()
        sec_graph = time.perf_counter() - t0
        o = g.observables()
        g.close()
        out[name] = {"atom_steps_per_s": n * k / sec_graph, "ms_per_step": 1e3 * sec_graph / k, "steps": k,
                     "kernel_ms_per_step": {kk: v[0] / k for kk, v in kt.items()},
                     "T_K": o["T"] / KB_EV, "rebuilds": o["rebuilds"]}
    if fp64_steps:
        out["speedup_mixed_over_fp64"] = out["mixed"]["atom_steps_per_s"] / out["fp64_gpu"]["atom_steps_per_s"]
    return out


def run_learned_tail(pkg, torch):
    """Train the learned Green-Kubo tail on a replica ensemble (features from
    2,000-step runs, targets from the same replicas at 20,000 steps) and
    judge it on held-out replicas against the short-run integral."""
    from paper_2503_07526_gb300 import learned_tail as lt

    specs = lt.ensemble_specs(512, seed=5, n_range=(500, 4000))
    sync = torch.cuda.synchronize
    t0 = time.perf_counter()
    d = lt.generate(specs, 2000, 20000, sync=sync)
    gen_s = time.perf_counter() - t0
    tr, va, te = (lt.split(d, slice(a, b)) for a, b in ((0, 256), (256, 384), (384, 512)))
    tail = lt.LearnedTail(lr=1e-3, weight_decay=1e-3, seed=1)
    sync()
    t0 = time.perf_counter()
    hist = tail.fit(tr, va, epochs=30)
    sync()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    eta, kappa, ue, uk = tail.predict(te["X"], te["eta_short"], te["kappa_short"], te["steps_short"])
    infer_s = time.perf_counter() - t0
    fwd = mlp_forward_rate(tail.net, torch, rows=1 << 20, reps=5)

    def rms_rel(a, b):
        return float(np.sqrt(np.mean(((a - b) / b) ** 2)))

    return tail, {
        "workload": "512 LJ replicas, sizes log-uniform in [500, 4000] atoms, rho* uniform in [0.7, 0.9], T* uniform "
                    "in [0.7, 2.0]; features after 2,000 steps, targets (eta, kappa to t_cut = 2 tau) after 20,000 "
                    "steps; trained on 256, validated on 128, judged on 128 held-out replicas",
        "network": "132 -> 3 x 128 tanh -> 2, bfloat16 tcgen05 products, FP32 master weights, Adam, 30 epochs",
        "rms_rel_error_vs_long_run": {"eta_learned_tail": rms_rel(eta, te["eta_long"]),
                                      "eta_short_run_integral": rms_rel(te["eta_short"], te["eta_long"]),
                                      "kappa_learned_tail": rms_rel(kappa, te["kappa_long"]),
                                      "kappa_short_run_integral": rms_rel(te["kappa_short"], te["kappa_long"])},
        "network_used_fraction": {"eta": float(ue.mean()), "kappa": float(uk.mean())},
        "validation_error": list(tail.val_error), "short_run_error_coefficients": list(tail.short_coeff),
        "loss_first_last": [float(hist[0]), float(hist[-1])],
        "seconds": {"generate": gen_s, "train": train_s, "inference_128": infer_s},
        "forward_1m_rows": fwd,
        "ensemble_atom_steps_per_s": float(d["atoms"].sum() * 20000 / (d["seconds_short"] + d["seconds_long"])),
    }


def mlp_forward_rate(net, torch, rows, reps, warmup=1):
    """The network's forward pass (mlp_forward, the fused tensor-core kernel)
    on `rows` device rows of 132 FP32 features, timed with CUDA events over
    `reps` calls after `warmup`; FLOPs of the 132-128-128-128-2 products and
    the HBM bytes of the FP32 inputs and outputs set its two rooflines."""
    Xd = torch.randn(rows, net.n_in, device="cuda", dtype=torch.float32)
    for _ in range(warmup):
        net.forward(Xd)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        net.forward(Xd)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    flop = 2.0 * rows * sum(a * b for a, b in zip(net.dims[:-1], net.dims[1:]))
    hbm = 4.0 * rows * (net.n_in + net.n_out)
    peaks, peak_kind = measured_peaks()
    tf = flop / (ms / 1e3) / 1e12
    gbs = hbm / (ms / 1e3) / 1e9
    t_hbm, t_tc = hbm / (peaks["hbm_gbs"] * 1e9), flop / (peaks["bf16_tflops"] * 1e12)  # seconds at the peaks
    return {"rows": rows, "ms_per_call": ms, "tflops_algorithmic": tf,
            "frac_of_bf16_peak": tf / peaks["bf16_tflops"], "input_output_gbs": gbs,
            "frac_of_hbm": gbs / peaks["hbm_gbs"],
            "bound": "hbm" if t_hbm > t_tc else "tensor", "frac_of_roofline": max(t_hbm, t_tc) / (ms / 1e3),
            "peak_source": f"{peak_kind} bf16_tflops (burst), hbm_gbs",
            "timing": "CUDA events around whole mlp_forward calls (each ends with a status read and a "
                      "stream synchronisation)"}


def run_learned_tail_full(args):
    """The full learned-tail workload: the network trained on 4,096 replica
    runs of the batched-ensemble distribution (sizes log-uniform in
    [500, 32,000] atoms; features after 5,000 steps, targets after 50,000),
    then applied to a 16,384,000-atom box (160^3 fcc cells x 4) run for 5,000
    steps and judged against the same box's 100,000-step integral.  Opt-in
    (about half an hour on one GB300); prints one JSON line."""
    import torch

    import paper_2503_07526_gb300 as pkg
    from paper_2503_07526_gb300 import learned_tail as lt
    from paper_2503_07526_gb300 import synth

    pkg.lib()
    sync = torch.cuda.synchronize
    nrep, short, long = args.lt_replicas, 5000, 50000
    t0 = time.perf_counter()
    if args.lt_dataset:  # a training set saved by an earlier --save-dataset run
        d = dict(np.load(args.lt_dataset))
        nrep = len(d["T"])
    else:
        d = lt.generate(lt.ensemble_specs(nrep, seed=7), short, long, sync=sync)
    gen_s = time.perf_counter() - t0
    if args.save_dataset:
        np.savez(args.save_dataset, **{k: v for k, v in d.items()})
    a, b = int(nrep * 0.75), int(nrep * 0.875)
    tr, va, te = (lt.split(d, slice(x, y)) for x, y in ((0, a), (a, b), (b, nrep)))
    tail = lt.LearnedTail(lr=1e-3, weight_decay=1e-3, seed=1)
    sync()
    t0 = time.perf_counter()
    hist = tail.fit(tr, va, epochs=30)
    sync()
    train_s = time.perf_counter() - t0
    eta, kappa, ue, uk = tail.predict(te["X"], te["eta_short"], te["kappa_short"], te["steps_short"])

    def rms_rel(x, y):
        return float(np.sqrt(np.mean(((x - y) / y) ** 2)))

    held_out = {"eta_learned_tail": rms_rel(eta, te["eta_long"]),
                "eta_short_run_integral": rms_rel(te["eta_short"], te["eta_long"]),
                "kappa_learned_tail": rms_rel(kappa, te["kappa_long"]),
                "kappa_short_run_integral": rms_rel(te["kappa_short"], te["kappa_long"]),
                "network_used": [float(ue.mean()), float(uk.mean())]}
    # the judge: one large box, short run then the full-length integral
    jc, js, jl = args.lt_judge_cells, 5000, 100000
    s = synth.lj_system(jc, rho=RHO, T=T_STAR, seed=3)
    n, L = s["n"], s["L"]
    V = L ** 3
    p = pkg.make_params(n, L, rc=RC, dt=DT, skin=SKIN, precision=pkg.MD_PREC_MIXED, pair_mode=pkg.MD_PAIR_TILES,
                        stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=None)
    g = pkg.System(p, s["r"], s["v"])
    melt(g, 2.0, 600)
    melt(g, T_STAR, 600)
    g.reset_correlators()
    sync()
    t0 = time.perf_counter()
    g.step(js)
    sync()
    short_s = time.perf_counter() - t0
    ra = lt.transport(g, [V])
    X = pkg.gk_tail_features(ra["Cs"][:, :64], ra["Cq"][:, :64], [V], ra["T"], [n / V])
    je, jk, jue, juk = tail.predict(X, ra["eta"], ra["kappa"], [js])
    nete, netk = tail._net(X)
    t0 = time.perf_counter()
    g.step(jl - js)
    sync()
    long_s = time.perf_counter() - t0
    rb = lt.transport(g, [V])
    g.close()
    out = {"workload": f"learned Green-Kubo tail: {nrep} replicas x {long} steps (features at {short}), judged on "
                       f"a {n}-atom LJ box (rho*={RHO}, T*={T_STAR}) at {js} against {jl} steps",
           "training": {"seconds_generate": gen_s, "seconds_train": train_s, "atoms": int(d["atoms"].sum()),
                        "loss_first_last": [float(hist[0]), float(hist[-1])],
                        "validation_error": list(tail.val_error), "short_run_error_coefficients": list(tail.short_coeff)},
           "held_out_rms_rel_error_vs_long_run": held_out,
           "judge": {"atoms": n, "eta_full_integral": float(rb["eta"][0]), "kappa_full_integral": float(rb["kappa"][0]),
                     "eta_short_integral": float(ra["eta"][0]), "kappa_short_integral": float(ra["kappa"][0]),
                     "eta_network": float(nete[0]), "kappa_network": float(netk[0]),
                     "eta_returned": float(je[0]), "kappa_returned": float(jk[0]),
                     "network_used": [bool(jue[0]), bool(juk[0])],
                     "seconds_short": short_s, "seconds_long": long_s,
                     "atom_steps_per_s": n * jl / (short_s + long_s)}}
    print(json.dumps(out), flush=True)


TV_REFERENCE = os.path.join(ROOT, "profiles", "time_to_viscosity_reference.json")
TV_SPEC = dict(stress=(12, 16, 2, 1), heatflux=(12, 16, 2, 1), vacf=None)  # the same correlators in every form


def tv_ensemble(pkg, synth, replicas, precision, seed0=500):
    """`replicas` 4,000-atom LJ replicas at rho* = 0.8442, T* = 0.722 in one
    handle, melted (rescaled to T* = 2.0 for 2,000 steps, then to 0.722 for
    3,000) with the correlators reset after the melt."""
    reps = []
    for k in range(replicas):
        s = synth.lj_system(10, rho=RHO, T=T_STAR, seed=seed0 + k)
        reps.append(dict(r=s["r"], v=s["v"], box=s["L"]))
    p = pkg.make_params(1, 1.0, rc=RC, dt=DT, skin=0.2, precision=precision, pair_mode=pair_mode_for(pkg, precision),
                        **TV_SPEC)
    g = pkg.System(p, replicas=reps)
    melt_replicas(g, np.full(replicas, T_STAR), 2000, 3000)
    g.reset_correlators()
    return g, reps[0]["box"] ** 3, reps[0]["r"].shape[1]


def run_tv_reference(args):
    """The reference viscosity of the time-to-viscosity criterion: a long
    FP64 GPU ensemble at the state point (--tv-replicas replicas x
    --tv-steps steps, eta per replica to t_cut = 2 tau, mean and standard
    error).  Opt-in; prints one JSON line."""
    import torch

    import paper_2503_07526_gb300 as pkg
    from paper_2503_07526_gb300 import learned_tail as lt
    from paper_2503_07526_gb300 import synth

    pkg.lib()
    g, V, n = tv_ensemble(pkg, synth, args.tv_replicas, pkg.MD_PREC_FP64, seed0=100000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(args.tv_steps)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    a = lt.transport(g, np.full(args.tv_replicas, V))
    g.close()
    eta = a["eta"]
    print(json.dumps({"what": "reference Green-Kubo viscosity of the time-to-viscosity criterion: FP64 GPU ensemble, "
                              f"{args.tv_replicas} replicas of {n} LJ atoms (rho*={RHO}, T*={T_STAR}, rc={RC}, "
                              f"dt={DT}), {args.tv_steps} NVE steps each after the melt, eta of each replica to "
                              "t_cut = 2 tau (mean of xy, xz, yz)",
                      "eta": float(eta.mean()), "eta_se": float(eta.std(ddof=1) / math.sqrt(eta.size)),
                      "replicas": int(eta.size), "steps": args.tv_steps, "seconds": sec,
                      "T_mean": float(a["T"].mean())}), flush=True)


def tv_reference():
    try:
        with open(TV_REFERENCE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def run_time_to_viscosity(pkg, synth, torch, replicas=256, chunk=2000, max_steps=48000, tail=None, tail_steps=2000):
    """Time to a Green-Kubo viscosity at <= 2 % error, 4,000-atom LJ liquid
    (rho* = 0.8442, T* = 0.722; eta of each replica from its stress
    autocorrelation, mean of xy/xz/yz, integrated to t_cut = 2 tau).  The
    criterion: the ensemble mean has <= 2 % relative standard error and lies
    within 2 % of the reference eta of a long FP64 GPU ensemble (the
    committed result of --tv-reference).  Every form carries the same
    correlators (stress and heat flux; no per-atom velocity correlator).
    Measured: the mixed batch of `replicas` replicas runs `chunk` steps at a
    time until both conditions hold (production seconds, readouts included;
    at most max_steps); the single-system forms (plain FP64 and mixed, one replica at
    a time) are projected: the replica-steps that run needed times their
    measured cost per replica-step.  With a trained learned tail, the batch
    is also read after `tail_steps` steps and the network's predictions are
    judged by the same two conditions."""
    from paper_2503_07526_gb300 import learned_tail as lt

    ref = tv_reference()
    g, V, n_atoms = tv_ensemble(pkg, synth, replicas, pkg.MD_PREC_MIXED)
    Vs = np.full(replicas, V)
    sync = torch.cuda.synchronize
    learned, steps, prod_s, history = None, 0, 0.0, []
    mean = se = T_mean = 0.0
    while steps < max_steps:
        k = tail_steps if (tail is not None and steps == 0) else chunk
        sync()
        t0 = time.perf_counter()
        g.step(k)
        steps += k
        a = lt.transport(g, Vs)
        prod_s += time.perf_counter() - t0
        if tail is not None and steps == tail_steps:
            X = pkg.gk_tail_features(a["Cs"][:, :64], a["Cq"][:, :64], Vs, a["T"], np.full(replicas, n_atoms / V))
            ti = time.perf_counter()
            eta_l, _, used, _ = tail.predict(X, a["eta"], a["kappa"], np.full(replicas, tail_steps))
            learned = (eta_l, used, prod_s, time.perf_counter() - ti)
            continue
        mean, se = float(a["eta"].mean()), float(a["eta"].std(ddof=1) / math.sqrt(replicas))
        T_mean = float(a["T"].mean())
        history.append([steps, mean, se])
        # both conditions of the criterion (the run goes on while the mean is
        # still more than 2 % from the reference, even at 2 % standard error)
        if se <= 0.02 * abs(mean) and (ref is None or abs(mean - ref["eta"]) <= 0.02 * abs(ref["eta"])):
            break
    g.close()
    reached_se = se <= 0.02 * abs(mean)
    need = replicas * steps  # replica-steps the measured run took
    # cost per replica-step of one 4,000-atom system on its own (graph replay),
    # with the same correlators
    costs = {"mixed_gpu_batched_%d" % replicas: prod_s / (replicas * steps)}
    s = synth.lj_system(10, rho=RHO, T=T_STAR, seed=1)
    for name, prec in (("fp64_gpu_single", pkg.MD_PREC_FP64), ("mixed_gpu_single", pkg.MD_PREC_MIXED)):
        ps = pkg.make_params(s["n"], s["L"], rc=RC, dt=DT, skin=0.3, precision=prec, pair_mode=pair_mode_for(pkg, prec),
                             **TV_SPEC)
        gs = pkg.System(ps, s["r"], s["v"])
        gs.step(50)
        sync()
        t0 = time.perf_counter()
        gs.step(2000)
        sync()
        costs[name] = (time.perf_counter() - t0) / 2000
        gs.close()
    dev = None if ref is None else (mean - ref["eta"]) / ref["eta"]
    within = None if dev is None else abs(dev) <= 0.02
    ok = bool(reached_se and within)
    out = {"definition": "seconds of production MD (correlators included, equilibration excluded) until the "
                         "ensemble Green-Kubo viscosity has <= 2 % relative standard error and lies within 2 % of "
                         "the reference eta (long FP64 GPU ensemble); 4,000-atom LJ liquid, rho*=0.8442, T*=0.722, "
                         "eta to t_cut = 2 tau; stress and heat-flux correlators in every form",
           "reference": ref, "eta": mean, "eta_se": se, "T_mean": T_mean, "steps_per_replica": steps,
           "replicas": replicas,
           "history": history, "reached_2pct_se": bool(reached_se),
           "deviation_from_reference": dev, "within_2pct_of_reference": within,
           "replica_steps_needed": need,
           "measured": {"form": "mixed_gpu_batched_%d" % replicas, "seconds": prod_s if ok else None,
                        "seconds_run": prod_s},
           "projected_seconds": {k: (v * need if ok else None) for k, v in costs.items()},
           "cost_per_replica_step_s": costs}
    if learned is not None:
        eta_l, used, t_short, infer_s = learned
        lm, lse = float(eta_l.mean()), float(eta_l.std(ddof=1) / math.sqrt(replicas))
        ldev = None if ref is None else (lm - ref["eta"]) / ref["eta"]
        lok = bool(lse <= 0.02 * abs(lm) and ldev is not None and abs(ldev) <= 0.02)
        out["learned_tail"] = {
            "what": f"network prediction from each replica's first {tail_steps} steps of the same batch; the "
                    "mean prediction judged by the same two conditions",
            "eta_mean": lm, "eta_se": lse, "network_used_fraction": float(used.mean()),
            "deviation_from_reference": ldev, "reached": lok,
            "seconds": (t_short + infer_s) if lok else None,
            "note": "no time is claimed when the prediction misses either condition"}
    return out


def committed_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else null)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
    except OSError:
        return None
    ent = tr.get(kernel)
    if not ent:
        return None
    h = hashlib.sha256()
    for name in ent.get("sources", [ent.get("source")]):
        with open(os.path.join(ROOT, "paper_2503_07526_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return ent["bytes_per_launch"] if h.hexdigest()[:16] == ent.get("source_sha") else None


def cpu_baseline(st, s, budget_s=20.0):
    """The FP64 oracle, as it stands, on the host cores: full 2,048,000-atom
    system with the same correlators, timed over as many whole steps as fit
    in the budget after one warm-up step."""
    import oracle

    n, L = s["n"], s["L"]
    oracle.build()
    cores = oracle.num_threads()
    md = oracle.MD(st["r"], st["v"], L, rc=RC, dt=DT, cells=True)
    cs = oracle.Corr(12, 16, 2, 6)  # sigma_xy, sigma_xz, sigma_yz, q_x, q_y, q_z
    cv = oracle.Corr(8, 16, 2, 3 * n, gs=n)
    md.step(1, cs=cs, cv=cv)
    steps, t0 = 0, time.perf_counter()
    while True:
        md.step(1, cs=cs, cv=cv)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 50:
            break
    # the same oracle on one core (one whole step, continuing the same run)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    md.step(1, cs=cs, cv=cv)
    el1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": n * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} whole steps of the {n:,}-atom workload from the melted state the GPU runs "
                      f"(link-cell forces, integration, observables, stress/heat-flux and per-atom VACF "
                      f"correlators) after 1 warm-up step, {el:.1f} s",
            "single_core": {"value": n / el1, "unit": UNIT, "cores": 1,
                            "sample": f"1 further whole step of the same run on one thread, {el1:.1f} s"}}


def run_reference(args):
    """The oracle on the host cores, on this arm's workload (rank 0 only)."""
    from paper_2503_07526_gb300 import replicas

    rank, world, _ = replicas.dist_env()
    if rank != 0:
        return
    from paper_2503_07526_gb300 import synth

    import oracle

    s = synth.lj_system(CELLS, rho=RHO, T=T_STAR, seed=1)
    n, L = s["n"], s["L"]
    oracle.build()
    cores = oracle.num_threads()
    md = oracle.MD(s["r"], s["v"], L, rc=RC, dt=DT, cells=True)
    cs = oracle.Corr(12, 16, 2, 6)
    cv = oracle.Corr(8, 16, 2, 3 * n, gs=n)
    md.step(args.warmup, cs=cs, cv=cv)
    t0 = time.perf_counter()
    md.step(args.steps, cs=cs, cv=cv)
    el = time.perf_counter() - t0
    value = n * args.steps / el
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded fcc, Maxwell-Boltzmann)",
           "impl": "reference",
           "config": {"workload": workload_name(n, start="start, not melted"), "n_atoms": n, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} timed steps of the full workload from the fcc start (not melted) "
                                      f"after {args.warmup} warm-up"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the replica ensemble and time-to-viscosity")
    ap.add_argument("--cells", type=int, default=CELLS, help="fcc cells per side (4 cells^3 atoms)")
    ap.add_argument("--skin", type=float, default=SKIN, help="Verlet skin of the timed system (sigma)")
    ap.add_argument("--pair", default="tiles", choices=["tiles", "verlet"],
                    help="mixed-form pair path of the timed system: tile windows or global Verlet lists")
    ap.add_argument("--list-build", type=int, default=0,
                    help="neighbour-list build of the timed system: 0 default, 1 j-parallel, 2 i-parallel, 3 staged")
    ap.add_argument("--quick", action="store_true", help="short melt, timed region only (for profilers)")
    ap.add_argument("--ionic-only", action="store_true",
                    help="run only the ionic melt for --steps steps (mixed form; with --quick no FP64 form)")
    ap.add_argument("--learned-tail-full", action="store_true",
                    help="run only the full learned-tail workload (4,096 replicas, 16.4M-atom judge)")
    ap.add_argument("--lt-replicas", type=int, default=4096)
    ap.add_argument("--lt-judge-cells", type=int, default=160)
    ap.add_argument("--save-dataset", default=None, help="npz path for the learned-tail training set")
    ap.add_argument("--lt-dataset", default=None, help="train on this saved training set instead of generating it")
    ap.add_argument("--mlp-only", action="store_true",
                    help="time only the learned-tail network's forward pass (--mlp-rows rows, --steps calls)")
    ap.add_argument("--mlp-rows", type=int, default=1 << 20)
    ap.add_argument("--tv-reference", action="store_true",
                    help="run only the long FP64 ensemble that gives the time-to-viscosity reference eta")
    ap.add_argument("--tv-replicas", type=int, default=256)
    ap.add_argument("--tv-steps", type=int, default=20000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ionic_only:
        import torch

        import paper_2503_07526_gb300 as pkg
        from paper_2503_07526_gb300 import synth

        pkg.lib()
        print(json.dumps(run_ionic(pkg, synth, torch, steps=args.steps,
                                   fp64_steps=0 if args.quick else max(1, args.steps // 10))), flush=True)
    elif args.learned_tail_full:
        run_learned_tail_full(args)
    elif args.tv_reference:
        run_tv_reference(args)
    elif args.mlp_only:
        import torch

        import paper_2503_07526_gb300 as pkg
        from paper_2503_07526_gb300 import synth

        pkg.lib()
        net = pkg.MLP(132, 2, seed=1)
        net.set_params(synth.mlp_init(11, net.dims, bias_scale=0.2))
        print(json.dumps({"mlp_forward": mlp_forward_rate(net, torch, args.mlp_rows, args.steps, args.warmup)}),
              flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
