"""Benchmark of the (T) triples-correction energy on GB300.

Workload: the FP64 (T) energy of a synthetic alanine-chain-sized problem,
o = 50 occupied, v = 450 virtual, naux = 1500, seed 2 (the seeded generator of
paper_1609_08094_gb300.synth; vvvo alone is 36.5 GB FP64, resident in HBM).
The full problem has C(52,3) = 22100 tasks (sorted occupied triples,
Sec. 3) of equal weight (Sec. 5); a step is one pass of the whole hot path
(W contractions, fused epilogue, reductions) over a contiguous batch of
tasks, and throughput is reported in algorithmic TFLOP/s
(12 v^3 (v+o) per task with i, j, k not all equal) and triples/s.

One JSON line (rank 0) carries: the device-timed value, the end-to-end value
through the C ABI with host buffers (copies inside the timed region), the
roofline of the dominant kernel, the oracle timed on the host cores on a
sample of the same workload, clocks sampled during the timed region, the
mixed-precision (TF32x3 / BF16x3) results on the same sizes when the
tensor-core path is available, and their errors against the FP64 path.

`--impl reference` times the CPU oracle instead (the reference arm).
Under torchrun each rank processes its own batch of tasks (weak scaling, no
collective on the data path; the harness reduces timings with max).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(T) TFLOP/s, triples/s: FP64 vs mixed at ≤1e-6 rel ΔE; serving p50/p99 latency"
WORKLOAD = dict(o=50, v=450, naux=1500, seed=2)
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 (152 SMs x 2070 MHz x 2 DFMA/clk x 2 flop)
FP64_PROBE_TFLOPS = 1.20     # DFMA throughput probe on this machine's GB300
# DRAM read+write bytes of ugemm_f64_kernel per task at o=50, v=450: the
# reads of one ncu capture at o=16, v=256 (0.807 GB per task) scaled by v^3,
# plus the U writes (3 v^2 vc x 8 B); valid for this kernel version only
F64_GEMM_TRAFFIC_BYTES = {(50, 450): int(0.807e9 * (450 / 256) ** 3) + 3 * 450 * 450 * 464 * 8}
# the same for the tensor-core contractions (SM-pair kernel, FP64 emulation): DRAM
# reads plus writes per task of one ncu capture at o=16, v=256, scaled by v^3
# (the split-precision U is written as 8^3 cubes of the valid values, the
# emulation's U as [a][b][c] rows of vc)
TC_GEMM_TRAFFIC_BYTES = {
    ("bf16x3", 50, 450): int((0.2739e9 + 0.1994e9) * (450 / 256) ** 3),
    ("tf32x3", 50, 450): int((0.5524e9 + 0.2031e9) * (450 / 256) ** 3),
    ("fp64_oz", 50, 450): int(0.504e9 * (450 / 256) ** 3) + 3 * 450 * 450 * 464 * 8,
}
# batched workload: n molecules, o ~ U{4..16}, v ~ U{20..120}, naux = 3(o+v),
# per-molecule seeds seed+index; FP64 is timed on the first fp64_n of them
# (the whole set is ~44 algorithmic TFLOP, ~40 s per pass on the FP64 pipe);
# kernel shares and the unbatched FP64 comparison use the first prof_n
BATCH = dict(n=256, seed=4, fp64_n=256, prof_n=32)
# served workload: requests with o ~ U{4..40}, v ~ U{20..300}, each the
# sub-problem (a window of o occupied and v virtual orbitals) of one seeded
# o=40, v=300, naux=1020 system; Poisson arrivals at 0.7x the throughput
# measured on a closed calibration batch; mixed precision
SERVE = dict(o_max=40, v_max=300, naux=1020, seed=5, n=48, calib=100, load=0.7, prec="bf16x3")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tasks-per-step", type=int, default=4)
    ap.add_argument("--mixed-tasks-per-step", type=int, default=64)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--precs", default="tf32x3,bf16x3,fp64_oz",
                    help="tensor-core precisions to time (split precision and FP64 emulation)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--single-sm", action="store_true",
                    help="split-precision contractions on single-SM tiles (M = 128) instead of SM pairs")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-tasks", type=int, default=1)
    ap.add_argument("--err-tasks", type=int, default=16,
                    help="tasks sampled over the task list for the per-task error of the mixed legs")
    ap.add_argument("--o", type=int, default=WORKLOAD["o"])
    ap.add_argument("--v", type=int, default=WORKLOAD["v"])
    ap.add_argument("--naux", type=int, default=WORKLOAD["naux"])
    ap.add_argument("--seed", type=int, default=WORKLOAD["seed"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-n", type=int, default=BATCH["n"])
    ap.add_argument("--batch-fp64-n", type=int, default=BATCH["fp64_n"])
    ap.add_argument("--wave-mb", type=int, default=0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-mp2", action="store_true")
    ap.add_argument("--serve-n", type=int, default=SERVE["n"])
    ap.add_argument("--serve-prec", default=SERVE["prec"])
    ap.add_argument("--serve-calib", type=int, default=SERVE["calib"],
                    help="requests of the closed calibration batch that sets the arrival rate")
    ap.add_argument("--serve-err-n", type=int, default=0,
                    help="served results re-evaluated in FP64 emulation for their error "
                         "(0 = every result; else a seeded sample of this many)")
    return ap.parse_args()


def measured_peaks():
    """Measured GB300 peaks written beside the repository (HBM GB/s, dense
    BF16 TFLOP/s burst and sustained); the profiling recipe's fallback
    figures when the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16": d["bf16_tflops"],
                "bf16_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


# nominal dense tensor rates: TF32 1.1 PFLOP/s vs BF16 2.25 PFLOP/s
TF32_PER_BF16 = 1.1 / 2.25


def sorted_tasks(o):
    return [(i, j, k) for i in range(o) for j in range(i, o) for k in range(j, o)]


def sample_tasks(tasks, n, seed):
    """n task indices (i, j, k not all equal) spread over the task list:
    one seeded draw in each of n equal strata."""
    from paper_1609_08094_gb300 import synth
    u = synth.uniform(seed, 3, n)
    out = []
    for m in range(n):
        lo, hi = m * len(tasks) // n, (m + 1) * len(tasks) // n
        k = lo + int(u[m] * (hi - lo))
        while tasks[k][0] == tasks[k][1] == tasks[k][2]:
            k = k + 1 if k + 1 < len(tasks) else k - 1
        out.append(k)
    return out


def work_tasks(tasks, first, count):
    return sum(1 for t in tasks[first:first + count] if not (t[0] == t[1] == t[2]))


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    import torch
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        torch.cuda.synchronize()


def time_steps(t, tasks, first_fn, count, warmup, steps, world, stream):
    """Device time (ms) of `steps` energy_range calls after `warmup` untimed."""
    import torch
    for w in range(warmup):
        t.energy_range(first_fn(w), count)
    t.kernel_times(reset=True)
    barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for s in range(steps):
        results.append(t.energy_range(first_fn(warmup + s), count))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    barrier(world)
    return ms, results, t.kernel_times(reset=True)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch

    import oracle
    import __graft_entry__
    from paper_1609_08094_gb300 import synth, tcorr

    rank, world, local = dist_setup(args)
    __graft_entry__.build() if rank == 0 else None
    if world > 1:
        barrier(world)
    tcorr.load()
    o, v, naux, seed = args.o, args.v, args.naux, args.seed
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    t0 = time.time()
    inst = synth.make_instance(o, v, naux, seed, device=dev)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    tasks = sorted_tasks(o)
    ntask = len(tasks)
    fl_task = 12.0 * v ** 3 * (v + o)
    K, W, C = args.steps, args.warmup, args.tasks_per_step
    from paper_1609_08094_gb300 import partition

    def first_of(s):  # rank's batch at step s: disjoint across ranks (weak scaling)
        return partition.step_batch(ntask, rank, world, s, C)

    # ---- FP64, device-resident inputs -------------------------------------
    t = tcorr.Tcorr.from_instance(inst, prec="fp64", profile=True, stream=stream)
    with ClockSampler(local) as cs:
        ms, res, ktimes = time_steps(t, tasks, first_of, C, W, K, world, stream)
    clocks = cs.summary()
    ms = dist_max(ms, world)
    work = sum(work_tasks(tasks, first_of(W + s), C) for s in range(K))
    all_work = dist_max(work, world) * world if world > 1 else work
    value = all_work * fl_task / (ms * 1e-3) / 1e12
    triples_s = (K * C * world) / (ms * 1e-3)
    gemm_ms, gemm_n = ktimes["gemm"]
    gemm_flops_per_launch = work * fl_task / max(1, gemm_n)
    achieved = gemm_flops_per_launch / (gemm_ms / max(1, gemm_n) * 1e-3) / 1e12
    launches = sum(n for _, n in ktimes.values())
    shares = {k: round(m / max(1e-9, sum(mm for mm, _ in ktimes.values())), 4) for k, (m, _) in ktimes.items()}

    # parity of the timed tasks against the oracle on a sample (rank 0)
    parity = None
    cpu = None
    if rank == 0 and not args.no_cpu:
        sample = [n for n in range(first_of(W), first_of(W) + C)
                  if not (tasks[n][0] == tasks[n][1] == tasks[n][2])][: args.cpu_tasks]
        need = sorted({q for n in sample for q in tasks[n]})
        host = synth.Instance(o, v, naux, seed, inst.eps_occ.cpu().numpy(), inst.eps_vir.cpu().numpy(),
                              inst.t1.cpu().numpy(), inst.t2.cpu().numpy(), None,
                              inst.ooov.cpu().numpy(), inst.ovov.cpu().numpy())
        slices = {q: inst.vvvo[:, :, :, q].contiguous().cpu().numpy() for q in need}
        oracle.build()
        threads = oracle.max_threads()
        tc0 = time.time()
        ref = oracle.triple_energies(host, np.array([tasks[n] for n in sample]), threads, slices=slices)
        cpu_s = time.time() - tc0
        _, per = t.energy_range(sample[0], sample[-1] - sample[0] + 1, per_task=True)
        got = per[[n - sample[0] for n in sample]]
        rel = float(np.max(np.abs(got.sum(1) - ref.sum(1)) / np.abs(ref.sum(1))))
        parity = {"tasks": [list(tasks[n]) for n in sample], "max_rel_err_fp64": rel,
                  "tol": 1e-10}
        cpu = {"value": len(sample) * fl_task / cpu_s / 1e12, "unit": "TFLOP/s", "cores": threads,
               "kind": "oracle", "sample": f"{len(sample)} tasks {[list(tasks[n]) for n in sample]} "
                                          f"of the o={o}, v={v} workload ({cpu_s:.1f} s)",
               "triples_per_s": len(sample) / cpu_s}
        del host, slices
    # FP64 references of the mixed legs' errors: the first 8 tasks of their first
    # timed batch, and each task of a seeded sample spread over the task list
    Cm = args.mixed_tasks_per_step
    first_m0 = partition.step_batch(ntask, rank, world, W, Cm)
    ref8 = ref_tasks = None
    if not args.no_mixed:
        ref8 = t.energy_range(first_m0, min(Cm, 8))
        samp = sample_tasks(tasks, args.err_tasks, seed + 17)
        ref_tasks = {n: t.energy_range(n, 1)[2] for n in samp}
    t.close()

    # ---- mixed precision on the same sizes --------------------------------
    mixed = {}
    if not args.no_mixed:
        for prec in [x for x in args.precs.split(",") if x]:
            try:
                tm = tcorr.Tcorr.from_instance(inst, prec=prec, profile=True, stream=stream,
                                               single_sm=args.single_sm)
            except tcorr.TcorrError as e:
                mixed[prec] = {"unavailable": str(e)}
                continue
            Cm = args.mixed_tasks_per_step

            def first_m(s, Cm=Cm):
                return partition.step_batch(ntask, rank, world, s, Cm)
            msm, resm, kt = time_steps(tm, tasks, first_m, Cm, W, K, world, stream)
            msm = dist_max(msm, world)
            workm = sum(work_tasks(tasks, first_m(W + s), Cm) for s in range(K))
            gm, gn = kt["gemm"]
            ent = {"value": workm * world * fl_task / (msm * 1e-3) / 1e12, "unit": "TFLOP/s",
                   "triples_per_s": K * Cm * world / (msm * 1e-3), "ms_per_step": msm / K,
                   "tasks_per_step": Cm,
                   "kernel_ms_share": {k: round(m / max(1e-9, sum(mm for mm, _ in kt.values())), 4)
                                       for k, (m, _) in kt.items()},
                   "gemm_tflops": workm * fl_task / (gm * 1e-3) / 1e12 if gm > 0 else None}
            # error vs the FP64 GPU path: the sum of the first 8 tasks of the first
            # timed batch, and every task of a seeded sample spread over the task list
            em8 = tm.energy_range(first_m(W), min(Cm, 8))
            ent["rel_err_vs_fp64_first8_tasks"] = abs(em8[2] - ref8[2]) / abs(ref8[2])
            terr = [abs(tm.energy_range(n, 1)[2] - b) / abs(b) for n, b in ref_tasks.items()]
            ent["task_rel_err_vs_fp64"] = {"max": max(terr), "median": float(np.median(terr)),
                                           "tasks": len(terr), "sample": "seeded, spread over the task list"}
            pk = measured_peaks()
            peak = pk["bf16"] * (TF32_PER_BF16 if prec == "tf32x3" else 1.0)
            if prec == "fp64_oz" and ent["gemm_tflops"]:
                # 15 BF16 slice products per algorithmic flop (5 slices, pairs with i + j <= 6)
                ent["tol"] = 1e-10
                ent["roofline"] = {
                    "bound": "tensor", "kernel": "ugemm_oz_kernel (FP64 emulation, BF16 slices)",
                    "achieved": ent["gemm_tflops"], "peak": peak, "unit": "TFLOP/s",
                    "frac": ent["gemm_tflops"] / peak,
                    "traffic": TC_GEMM_TRAFFIC_BYTES.get((prec, o, v)),
                    "traffic_unit": "bytes per task (an o=16, v=256 capture scaled by v^3)",
                    "tensor_achieved": 15 * ent["gemm_tflops"],
                    "tensor_frac": 15 * ent["gemm_tflops"] / peak,
                    "fp64_pipe_peak": FP64_PEAK_TFLOPS,
                    "vs_fp64_pipe_peak": ent["gemm_tflops"] / FP64_PEAK_TFLOPS,
                    "note": "achieved counts algorithmic FP64 flops (12 v^3 (v+o) per task); the tensor "
                            "pipe executes 15 BF16 slice products per flop: tensor_achieved.  peak: BF16 "
                            "dense burst of " + pk["source"] + " peaks"}
            elif ent["gemm_tflops"]:
                ent["roofline"] = {
                    "bound": "tensor",
                    "kernel": f"{'ugemm_tc_kernel' if args.single_sm else 'ugemm_tc_pair_kernel'} ({prec})",
                    "achieved": ent["gemm_tflops"], "peak": peak, "unit": "TFLOP/s",
                    "frac": ent["gemm_tflops"] / peak,
                    "traffic": None if args.single_sm else TC_GEMM_TRAFFIC_BYTES.get((prec, o, v)),
                    "traffic_unit": "bytes per task (an o=16, v=256 capture scaled by v^3)",
                    "tensor_achieved": 3 * ent["gemm_tflops"],
                    "tensor_frac": 3 * ent["gemm_tflops"] / peak,
                    "note": ("achieved counts algorithmic flops (12 v^3 (v+o) per task); the "
                             "tensor pipe executes 3 products per flop (hi*hi, hi*lo, lo*hi): "
                             "tensor_achieved.  peak: BF16 dense burst of " + pk["source"]
                             + (" peaks x the nominal TF32/BF16 ratio" if prec == "tf32x3" else " peaks"))}
            ent["speedup_vs_fp64"] = ent["value"] / value
            mixed[prec] = ent
            tm.close()

    # ---- end to end through the C ABI with host buffers --------------------
    e2e = None
    if not args.no_e2e:
        arrays = [a.cpu().pin_memory() for a in inst.arrays()]
        h2d = sum(a.numel() * 8 for a in arrays)
        for _ in range(1):  # warm-up
            with tcorr.Tcorr(o, v, *[a.numpy() for a in arrays], prec="fp64") as te:
                te.energy_range(first_of(0), C)
        barrier(world)
        KE = max(1, min(K, 2))
        te0 = time.perf_counter()
        for s in range(KE):
            with tcorr.Tcorr(o, v, *[a.numpy() for a in arrays], prec="fp64") as te:
                te.energy_range(first_of(W + s), C)
        torch.cuda.synchronize()
        e_ms = dist_max((time.perf_counter() - te0) * 1e3, world)
        worke = sum(work_tasks(tasks, first_of(W + s), C) for s in range(KE))
        e2e = {"value": worke * world * fl_task / (e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 24, "steps": KE,
               "ms_per_step": e_ms / KE,
               "note": "per step: tcorr_create from pinned host arrays (H2D + layout prep), "
                       "tcorr_energy_range, 3-double result read, tcorr_destroy"}
        del arrays

    # the main workload's device arrays are not needed by the remaining legs
    del inst
    gc.collect()
    torch.cuda.empty_cache()

    # ---- batched: many molecules of uneven size in one graph-replayed launch sequence
    batched = None
    if not args.no_batched:
        batched = bench_batched(args, rank, world, stream)

    gc.collect()
    torch.cuda.empty_cache()
    serving = None
    if not args.no_serving:
        serving = bench_serving(args, rank, world, stream)
    gc.collect()
    torch.cuda.empty_cache()

    mp2 = None
    if not args.no_mp2:
        mp2 = bench_mp2(args, rank, world, stream)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 (T) energy, o={o} v={v} naux={naux} seed={seed}, "
                               f"{C} tasks per step per GPU",
                   "o": o, "v": v, "naux": naux, "seed": seed, "tasks_per_step": C,
                   "tasks_total": ntask, "l2": "inputs larger than L2 (one vvvo slice is "
                                                f"{v ** 3 * 8 / 1e6:.0f} MB FP64)",
                   "generate_s": round(gen_s, 1)},
        "triples_per_s": triples_s,
        "roofline": {"bound": "alu", "kernel": "ugemm_f64_kernel", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": F64_GEMM_TRAFFIC_BYTES.get((o, v)),
                     "traffic_unit": "bytes per task (an o=16, v=256 capture scaled by v^3)",
                     "peak_note": "nominal FP64 (no FP64 figure in the measured peaks); "
                                  f"DFMA probe measured {FP64_PROBE_TFLOPS} TFLOP/s"},
        "kernel_ms_share": shares,
        "gpu_launches": launches,
        "clocks": clocks,
        "parity": parity,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "mixed": mixed,
        "batched": batched,
        "serving": serving,
        "rimp2": mp2,
    }
    line["summary"] = summary(line)  # last key: a compact copy of every leg's figures
    print(json.dumps(line), flush=True)


def summary(line):
    """Every leg's headline figures in a few hundred characters (3 significant
    digits): throughput, GEMM throughput, roofline fractions, errors."""
    def r(x):
        return None if x is None else float(f"{x:.3g}")

    def get(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    out = {"fp64": {"tflops": r(line["value"]), "frac": r(line["roofline"]["frac"]),
                    "err": r(get(line, "parity", "max_rel_err_fp64"))},
           "e2e": r(get(line, "e2e", "value"))}
    for p, ent in (line.get("mixed") or {}).items():
        out[p] = {"tflops": r(ent.get("value")), "gemm": r(ent.get("gemm_tflops")),
                  "frac": r(get(ent, "roofline", "frac")), "tfrac": r(get(ent, "roofline", "tensor_frac")),
                  "err8": r(ent.get("rel_err_vs_fp64_first8_tasks")),
                  "err_task": r(get(ent, "task_rel_err_vs_fp64", "max"))}
    b = {}
    for p, ent in (get(line, "batched", "precisions") or {}).items():
        b[p] = {"tflops": r(ent.get("value")), "x_solo": r(ent.get("speedup_vs_unbatched")),
                "n": ent.get("molecules"), "err": r(get(ent, "rel_err_vs_fp64", "max"))}
    out["batched"] = b
    sv = line.get("serving") or {}
    out["serving"] = {"n": sv.get("requests"), "p50": r(get(sv, "latency_s", "p50")),
                      "p99": r(get(sv, "latency_s", "p99")), "tflops": r(get(sv, "throughput", "tflops")),
                      "err": r(get(sv, "rel_err_vs_fp64", "max")), "same": sv.get("solo_vs_mixed_identical")}
    mp = line.get("rimp2") or {}
    out["rimp2"] = {"fp64": r(mp.get("value")), "frac": r(get(mp, "roofline", "frac"))}
    for p, ent in (mp.get("mixed") or {}).items():
        out["rimp2"][p] = {"tflops": r(ent.get("value")), "err": r(ent.get("rel_err_vs_fp64"))}
    return out


def bench_batched(args, rank, world, stream):
    """The batched workload (BATCH): each rank takes its share of the
    molecules (weak scaling, no collective).  Per precision: the whole set's
    energies per step through one tcorr_batch handle (CUDA graph replay, tile
    shapes from the measured autotuner), the same molecules one handle at a
    time (the unbatched baseline, energy calls only), and the error of every
    molecule against the FP64 path."""
    import numpy as np
    import torch

    from paper_1609_08094_gb300 import synth, tcorr
    shapes_all = synth.batch_shapes(args.batch_n, BATCH["seed"])
    shapes = shapes_all[rank::world]
    t0 = time.time()
    insts = [synth.make_instance(o, v, naux, sd, device=torch.device("cuda", torch.cuda.current_device()))
             for o, v, naux, sd in shapes]
    torch.cuda.synchronize()
    gen_s = time.time() - t0

    def flops(sub):
        return sum((i.o * (i.o + 1) * (i.o + 2) // 6 - i.o) * 12.0 * i.v ** 3 * (i.v + i.o) for i in sub)

    def ntask(sub):
        return sum(i.o * (i.o + 1) * (i.o + 2) // 6 for i in sub)

    def run(prec, sub, K, W, prof=True):
        with tcorr.Batch(sub, prec=prec, tune=(prec != "fp64"), stream=stream, wave_mb=args.wave_mb) as b:
            e = None
            for _ in range(W):       # the first call captures the graph
                e = b.energy()
            barrier(world)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(K):
                e = b.energy()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = dist_max(ev0.elapsed_time(ev1), world) / K
            waves, launches = b.plan()
            tiles = sorted({b.tile(n)[0] for n in range(len(sub))})
        if not prof:
            return e, ms, waves, launches, tiles, None, None
        # kernel shares from one profiled (direct-launch) pass
        with tcorr.Batch(sub, prec=prec, tune=(prec != "fp64"), stream=stream, wave_mb=args.wave_mb,
                         profile=True) as bp:
            bp.energy()
            kt = bp.kernel_times()
        tot = sum(m for m, _ in kt.values())
        return e, ms, waves, launches, tiles, kt, tot

    def solo(prec, sub):
        """Unbatched baseline: one handle per molecule, device time of the energy calls."""
        total = 0.0
        for inst in sub:
            with tcorr.Tcorr.from_instance(inst, prec=prec, stream=stream) as t:
                t.energy()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                t.energy()
                ev1.record(stream)
                torch.cuda.synchronize()
                total += ev0.elapsed_time(ev1)
        return total

    out = {"workload": f"{args.batch_n} molecules, o ~ U{{4..16}}, v ~ U{{20..120}}, naux = 3(o+v), "
                       f"seeds {BATCH['seed']}+index; {len(shapes)} on this rank",
           "generate_s": round(gen_s, 1), "precisions": {}}
    pk = measured_peaks()
    # FP64 on every molecule (one warm-up call that captures the graph, one timed
    # call): its energies are the reference of every mixed-precision result below;
    # kernel shares and the unbatched comparison on the first prof_n molecules
    sub64 = insts[: max(1, args.batch_fp64_n // world)]
    e64, ms64, wv, nl, _, _, _ = run("fp64", sub64, K=1, W=1, prof=False)
    subp = insts[: max(1, BATCH["prof_n"] // world)]
    _, msp, _, _, _, kt, tot = run("fp64", subp, K=1, W=1)
    fl64 = flops(sub64) * world
    out["precisions"]["fp64"] = {
        "molecules": len(sub64) * world, "value": fl64 / (ms64 * 1e-3) / 1e12, "unit": "TFLOP/s",
        "triples_per_s": ntask(sub64) * world / (ms64 * 1e-3), "ms_per_step": ms64, "steps": 1,
        "waves": wv, "gpu_launches": nl,
        "kernel_ms_share": {k: round(m / max(1e-9, tot), 4) for k, (m, _) in kt.items()},
        "gemm_tflops": flops(subp) / (kt["gemm"][0] * 1e-3) / 1e12,
        "note": f"FP64 timed on {len(sub64) * world} molecules (one warm-up + one step); kernel shares "
                f"and the unbatched comparison on the first {len(subp) * world}"}
    ms_solo64 = solo("fp64", subp)
    out["precisions"]["fp64"]["unbatched_ms"] = ms_solo64
    out["precisions"]["fp64"]["speedup_vs_unbatched"] = ms_solo64 / msp
    for prec in [x for x in args.precs.split(",") if x]:
        try:
            e, ms, wv, nl, tiles, kt, tot = run(prec, insts, K=min(args.steps, 3), W=min(args.warmup, 3))
        except tcorr.TcorrError as err:
            out["precisions"][prec] = {"unavailable": str(err)}
            continue
        fl = flops(insts) * world
        peak = pk["bf16"] * (TF32_PER_BF16 if prec == "tf32x3" else 1.0)
        gemm_tf = flops(insts) / (kt["gemm"][0] * 1e-3) / 1e12
        # error of every molecule's result against its FP64 result
        rel = np.abs(e[: len(sub64), 2] - e64[:, 2]) / np.abs(e64[:, 2])
        ms_solo = solo(prec, insts)
        out["precisions"][prec] = {
            "molecules": len(insts) * world, "value": fl / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "triples_per_s": ntask(insts) * world / (ms * 1e-3), "ms_per_step": ms, "steps": min(args.steps, 3),
            "warmup": min(args.warmup, 3), "waves": wv, "gpu_launches": nl, "tiles_pb": tiles,
            "kernel_ms_share": {k: round(m / max(1e-9, tot), 4) for k, (m, _) in kt.items()},
            "roofline": {"bound": "tensor",
                         "kernel": "ugemm_oz_kernel (FP64 emulation)" if prec == "fp64_oz" else f"ugemm_tc_pair_kernel ({prec})",
                         "achieved": gemm_tf,
                         "peak": peak, "unit": "TFLOP/s", "frac": gemm_tf / peak, "traffic": None,
                         "tensor_achieved": (15 if prec == "fp64_oz" else 3) * gemm_tf,
                         "tensor_frac": (15 if prec == "fp64_oz" else 3) * gemm_tf / peak},
            "rel_err_vs_fp64": {"max": float(rel.max()), "median": float(np.median(rel)),
                                "results": int(rel.size)}, "tol": 1e-6 if prec != "fp64_oz" else 1e-10,
            "unbatched_ms": ms_solo, "speedup_vs_unbatched": ms_solo / ms,
            "speedup_vs_fp64_batched": (fl / (ms * 1e-3)) / (fl64 / (ms64 * 1e-3))}
    return out


def serve_requests(n, seed, o_max, v_max):
    """(o, v, i0, a0) of n requests: sizes uniform, windows at uniform offsets."""
    from paper_1609_08094_gb300 import synth
    u = [synth.uniform(seed, 20 + k, n) for k in range(4)]
    out = []
    for r in range(n):
        o = 4 + int(u[0][r] * (o_max - 4 + 1))
        v = 20 + int(u[1][r] * (v_max - 20 + 1))
        i0 = int(u[2][r] * (o_max - o + 1))
        a0 = int(u[3][r] * (v_max - v + 1))
        out.append((o, v, i0, a0))
    return out


def window(base, o, v, i0, a0):
    """The sub-problem of occupied i0..i0+o-1 and virtual a0..a0+v-1 (device copies)."""
    oi, va = slice(i0, i0 + o), slice(a0, a0 + v)
    arr = (base.eps_occ[oi], base.eps_vir[va], base.t1[oi, va], base.t2[oi, oi, va, va],
           base.vvvo[va, va, va, oi], base.ooov[oi, oi, oi, va], base.ovov[oi, va, oi, va])
    return (o, v, *[a.contiguous() for a in arr])


def req_flops(o, v):
    return (o * (o + 1) * (o + 2) // 6 - o) * 12.0 * v ** 3 * (v + o)


def bench_serving(args, rank, world, stream):
    """The served workload (SERVE) through tcorr_server: a closed calibration
    batch measures the saturated throughput, then a Poisson stream at 0.7x of
    it; latency = completion (observed by polling) - scheduled arrival.  Each
    rank serves its own stream (replicas)."""
    import numpy as np
    import torch

    from paper_1609_08094_gb300 import synth, tcorr
    cfg = SERVE
    t0 = time.time()
    base = synth.make_instance(cfg["o_max"], cfg["v_max"], cfg["naux"], cfg["seed"] + rank,
                               device=torch.device("cuda", torch.cuda.current_device()))
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    reqs = serve_requests(args.serve_n + args.serve_calib, cfg["seed"] + 100 * rank, cfg["o_max"], cfg["v_max"])
    calib, stream_reqs = reqs[: args.serve_calib], reqs[args.serve_calib:]
    prec = args.serve_prec
    # mean work per request of the size distribution (large sample of the same law)
    dist = serve_requests(20000, cfg["seed"] + 7, cfg["o_max"], cfg["v_max"])
    mean_fl = float(np.mean([req_flops(o, v) for o, v, _, _ in dist]))

    with tcorr.Server(prec=prec, stream=stream) as srv:
        # closed batch: everything submitted at once -> saturated throughput
        tc0 = time.perf_counter()
        ids = [srv.submit(window(base, *r)) for r in calib]
        srv.drain()
        calib_s = time.perf_counter() - tc0
        bad = [(calib[k][:2], st) for k, (state, _, st) in enumerate(srv.poll(i) for i in ids) if state != "done"]
        if bad:
            raise RuntimeError(f"calibration jobs failed ((o, v), status): {bad[:8]}")
        sat = sum(req_flops(o, v) for o, v, _, _ in calib) / calib_s   # flop/s
        lam = cfg["load"] * sat / mean_fl                                # requests/s
        gaps = -np.log(1.0 - synth.uniform(cfg["seed"] + 100 * rank, 30, len(stream_reqs))) / lam
        arrive = np.cumsum(gaps)
        barrier(world)
        st0 = srv.stats()
        t_start = time.perf_counter()
        nxt, live, done_at, res = 0, {}, {}, {}
        while len(done_at) < len(stream_reqs):
            now = time.perf_counter() - t_start
            while nxt < len(stream_reqs) and arrive[nxt] <= now:
                live[srv.submit(window(base, *stream_reqs[nxt]))] = nxt
                nxt += 1
            pending = srv.step()
            now = time.perf_counter() - t_start
            for jid, k in list(live.items()):
                state, e, status = srv.poll(jid)
                if state in ("done", "failed"):
                    done_at[k] = now
                    res[k] = (state, e, status)
                    del live[jid]
            if pending == 0 and nxt < len(stream_reqs):
                time.sleep(max(0.0, min(0.01, arrive[nxt] - (time.perf_counter() - t_start))))
        makespan = max(done_at.values())
        st1 = srv.stats()
    lat = np.array([done_at[k] - arrive[k] for k in range(len(stream_reqs))])
    ok = sum(1 for r in res.values() if r[0] == "done")
    # a sample of the served jobs again, each alone: identical energies
    same = 0
    sample = list(range(0, len(stream_reqs), max(1, len(stream_reqs) // 4)))[:4]
    with tcorr.Server(prec=prec, stream=stream) as solo:
        for k in sample:
            jid = solo.submit(window(base, *stream_reqs[k]))
            solo.drain()
            same += int(solo.poll(jid)[1] == res[k][1])
    # the error of every served result against the FP64-accurate path (FP64
    # emulation on the tensor cores, held to 1e-10 of the oracle by the tests),
    # all requests through one FP64-emulation server after the timed stream
    t_ref = time.perf_counter()
    if args.serve_err_n > 0 and args.serve_err_n < len(stream_reqs):
        pick = sorted(set(int(x) for x in synth.uniform(cfg["seed"] + 9, 31, args.serve_err_n)
                          * len(stream_reqs)))
    else:
        pick = list(range(len(stream_reqs)))
    with tcorr.Server(prec="fp64_oz", stream=stream) as ref_srv:
        rid = {k: ref_srv.submit(window(base, *stream_reqs[k])) for k in pick}
        ref_srv.drain()
        ref_e = {k: ref_srv.poll(j) for k, j in rid.items()}
    ref_s = time.perf_counter() - t_ref
    errs = np.array([abs(res[k][1][2] - ref_e[k][1][2]) / abs(ref_e[k][1][2])
                     for k in pick if res[k][0] == "done" and ref_e[k][0] == "done"])
    fl = sum(req_flops(o, v) for o, v, _, _ in stream_reqs)
    makespan = dist_max(makespan, world)
    return {"workload": f"{len(stream_reqs)} requests per GPU, o ~ U{{4..{cfg['o_max']}}}, "
                        f"v ~ U{{20..{cfg['v_max']}}}, windows of one o={cfg['o_max']} v={cfg['v_max']} "
                        f"naux={cfg['naux']} system (seed {cfg['seed']}), Poisson arrivals at "
                        f"{cfg['load']}x the calibrated saturated throughput, {prec}",
            "requests": len(stream_reqs) * world, "done": ok, "failed": len(res) - ok,
            "lambda_req_per_s": lam, "saturated_tflops": sat / 1e12, "calibration_requests": len(calib),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "throughput": {"requests_per_s": len(stream_reqs) * world / makespan,
                           "tflops": fl * world / makespan / 1e12, "makespan_s": makespan},
            "waves": st1["waves"] - st0["waves"], "peak_admitted_bytes": st1["peak_bytes"],
            "solo_vs_mixed_identical": f"{same}/{len(sample)}", "generate_s": round(gen_s, 1),
            "rel_err_vs_fp64": {"max": float(errs.max()) if errs.size else None,
                                "median": float(np.median(errs)) if errs.size else None,
                                "results": int(errs.size), "tol": 1e-6,
                                "reference": (f"{'every served request' if len(pick) == len(stream_reqs) else f'a seeded sample of {len(pick)} served requests'}"
                                              f" again in FP64 emulation ({ref_s:.0f} s)")}}


def bench_mp2(args, rank, world, stream):
    """RI-MP2 (Sec. 2.1) of the same synthetic system as the main workload
    (its occupied-virtual factors as fitting coefficients), FP64: device time
    of the fused pair kernel over all i <= j pairs per step, the oracle on the
    host cores over the whole problem, and their agreement; then the
    mixed-precision variant (TF32x3, BF16x3 on the tensor cores) with its
    error against the FP64 energy."""
    import numpy as np
    import torch

    import oracle
    from paper_1609_08094_gb300 import synth, tcorr
    o, v, naux, seed = args.o, args.v, args.naux, args.seed
    t0 = time.time()
    inst = synth.make_mp2_instance(o, v, naux, seed)
    gen_s = time.time() - t0
    dev = inst.to(torch.device("cuda", torch.cuda.current_device()))
    K, W = args.steps, args.warmup
    with tcorr.Mp2.from_instance(dev, profile=True, stream=stream) as m:
        for _ in range(W):
            m.energy()
        m.kernel_times(reset=True)
        barrier(world)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(K):
            e = m.energy()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = dist_max(ev0.elapsed_time(ev1), world) / K
        kt = m.kernel_times(reset=True)
    fl = tcorr.mp2_flops(o, v, naux)
    kern_ms = kt["gemm"][0] / max(1, kt["gemm"][1])
    out = {"workload": f"RI-MP2, o={o} v={v} naux={naux} seed={seed} (the main workload's system), FP64, "
                       "all i <= j pairs per step",
           "value": fl * world / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms, "steps": K,
           "pairs_per_s": (o * (o + 1) // 2) * world / (ms * 1e-3), "energy": e, "generate_s": round(gen_s, 1),
           "roofline": {"bound": "alu", "kernel": "mp2_pair_kernel", "achieved": fl / (kern_ms * 1e-3) / 1e12,
                        "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": fl / (kern_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                        "note": "achieved counts 2 v^2 naux flops per pair; warps whose columns lie "
                                "past v issue no FMA, so the only extra work is the padded rows of the "
                                "last diagonal tile pair and naux rounded up to 8"}}
    if rank == 0 and not args.no_cpu:
        threads = oracle.max_threads()
        tc0 = time.time()
        ref = oracle.mp2_energy(inst)
        cpu_s = time.time() - tc0
        out["parity"] = {"rel_err_vs_oracle": abs(e[2] - ref[2]) / abs(ref[2]), "tol": 1e-10,
                         "oracle_energy": ref}
        out["cpu_baseline"] = {"value": fl / cpu_s / 1e12, "unit": "TFLOP/s", "cores": threads,
                               "kind": "oracle", "sample": f"the whole problem (numpy, {cpu_s:.1f} s)"}
    # the paper's mixed-precision variant: the ERI assembly on the tensor cores
    # in split precision (4 products per algorithmic flop), error vs the FP64 path
    if not args.no_mixed:
        mixed = {}
        pk = measured_peaks()
        for prec in ("tf32x3", "bf16x3"):
            try:
                mm = tcorr.Mp2.from_instance(dev, prec=prec, profile=True, stream=stream)
            except tcorr.TcorrError as err:
                mixed[prec] = {"unavailable": str(err)}
                continue
            with mm:
                for _ in range(W):
                    mm.energy()
                mm.kernel_times(reset=True)
                barrier(world)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                for _ in range(K):
                    em = mm.energy()
                ev1.record(stream)
                torch.cuda.synchronize()
                msm = dist_max(ev0.elapsed_time(ev1), world) / K
                ktm = mm.kernel_times(reset=True)
            kms = ktm["gemm"][0] / max(1, ktm["gemm"][1])
            peak = pk["bf16"] * (TF32_PER_BF16 if prec == "tf32x3" else 1.0)
            ach = fl / (kms * 1e-3) / 1e12
            mixed[prec] = {"value": fl * world / (msm * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": msm,
                           "energy": em, "rel_err_vs_fp64": abs(em[2] - e[2]) / abs(e[2]), "tol": 1e-6,
                           "speedup_vs_fp64": ms / msm,
                           "roofline": {"bound": "tensor", "kernel": f"mp2_tc_kernel ({prec})", "achieved": ach,
                                        "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                                        "tensor_achieved": 4 * ach, "tensor_frac": 4 * ach / peak,
                                        "note": "achieved counts 2 v^2 naux flops per pair; the tensor pipe "
                                                "runs 4 split products per flop (lo*lo kept: tensor_achieved), "
                                                "plus tiles of 128 padded past v and the diagonal tile pairs "
                                                "computed as G and H both"}}
        out["mixed"] = mixed
    return out


def reference_arm(args):
    """The oracle, as it stands, on the host cores: each step one task of the
    same workload (tasks have equal weight)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1609_08094_gb300 import synth
    o, v, naux, seed = args.o, args.v, args.naux, args.seed
    tasks = [t for t in sorted_tasks(o) if not (t[0] == t[1] == t[2])]
    K, W = args.steps, args.warmup
    steps = [tasks[(97 * s) % len(tasks)] for s in range(W + K)][W:]
    need = sorted({q for t in steps for q in t})
    # only what the sampled tasks read: every block but vvvo, and vvvo slices
    inst, slices = synth.make_instance_slices(o, v, naux, seed, need)
    oracle.build()
    threads = oracle.max_threads()
    fl_task = 12.0 * v ** 3 * (v + o)
    # warm-up steps warm the process (library load, thread pool) on a small
    # instance; a full-size task takes tens of seconds on the host
    small = synth.make_instance(4, 20, 72, 1)
    for s in range(W):
        oracle.triple_energies(small, np.array([[0, 1, 2]]), threads)
    t0 = time.perf_counter()
    for s in range(K):
        oracle.triple_energies(inst, np.array([steps[s]]), threads, slices=slices)
    sec = time.perf_counter() - t0
    value = K * fl_task / sec / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": K, "warmup": W,
            "ms_per_step": sec * 1e3 / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 (T) energy, o={o} v={v} naux={naux} seed={seed}, "
                                   "1 task per step (CPU oracle)", "o": o, "v": v},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"one task per step of the o={o}, v={v} workload"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
