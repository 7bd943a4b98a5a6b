"""Throughput benchmark of the synchronous-step ACS tour construction.

Workload (the paper-scale plain ACS): two clustered instances, n=1002 and
n=2392 (20 Gaussian clusters, sigma=300, in [0,10000]^2, EUC_2D), m=128 ants,
32-NN candidate lists, beta=2, q0=0.9, rho=xi=0.1, each run once on the FP32
pheromone matrix and once on the selective pheromone memory (s=8): four
independent colonies. One bench step = one full ACS iteration (Alg. 1) of all
four colonies; the matrix and SPM contexts run concurrently on two streams.

Metric: ant-steps/s = sum over colonies of m*(n-1) per iteration / step time.
L2 is flushed (256 MiB write) between timed steps, outside the timed events.

Beside it, the JSON line carries the second half of the metric: the mean
tour-length gap at equal GPU time of the learned prior against plain ACS on
held-out n=2392 and n=5000 instances (gap_leg; --no-gap skips it).

--workload selects another configuration (n198: one n=198 instance, m=32;
batch256: 256 instances of uneven n, m=64; large16: 8 x n=10000 and
8 x n=20000, m=256); the default is the paper-scale workload above.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload: each step is one oracle iteration of one of the four
colonies in rotation.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CL = 32
MEM_NAMES = {0: "matrix", 1: "spm"}
HBM_PEAK_FALLBACK = 6800.0
BF16_PEAK_FALLBACK = 1900.0   # TFLOP/s, dense bf16 burst of an earlier GB300 measurement

# Workloads (synthetic stand-ins for the paper's TSPLIB instances). The default
# is the paper-scale configuration; the others are the single-instance, batched
# and large-scale configurations, selectable with --workload.
WORKLOADS = {
    "paper": {
        "desc": "plain ACS at paper scale: n=1002 and n=2392 clustered (20 clusters, "
                "sigma=300, [0,10000]^2, EUC_2D), m=128, 32-NN, beta=2, q0=0.9, "
                "rho=xi=0.1, FP32 matrix and SPM s=8 (4 colonies)",
        "m": 128, "memories": (0, 1),
    },
    "n198": {
        "desc": "plain ACS on one instance: n=198 uniform in [0,10000]^2, EUC_2D, m=32, "
                "32-NN, beta=2, q0=0.9, rho=xi=0.1, FP32 matrix",
        "m": 32, "memories": (0,),
    },
    "batch256": {
        "desc": "batched plain ACS: 256 instances, n uniform in [100,2500], even uniform / "
                "odd clustered in [0,10000]^2, m=64, 32-NN, FP32 matrix and SPM s=8, one "
                "launch per iteration for each memory",
        "m": 64, "memories": (0, 1),
    },
    "large16": {
        "desc": "large scale: 8 instances n=10000 and 8 instances n=20000, uniform in "
                "[0,100000]^2, m=256, 32-NN, FP32 matrix and SPM s=8, one launch per "
                "iteration for each memory",
        "m": 256, "memories": (0, 1),
    },
}
WORKLOAD = "paper"
M = WORKLOADS[WORKLOAD]["m"]
SIZES = [1002, 2392]


def make_coords(seed_offset=0):
    """Coordinates of the current workload's instances, one array each."""
    from paper_1605_02669_gb300 import instances

    if WORKLOAD == "paper":
        return [instances.clustered(n, seed=2 + seed_offset) for n in (1002, 2392)]
    if WORKLOAD == "n198":
        return [instances.uniform(198, side=10000, seed=1 + seed_offset)]
    if WORKLOAD == "batch256":
        xy, off, _, _ = instances.mixed_batch(256, 100, 2500, seed=3 + seed_offset)
        return [xy[off[b]:off[b + 1]] for b in range(256)]
    if WORKLOAD == "large16":
        return ([instances.uniform(10000, side=100000, seed=40 + i + seed_offset) for i in range(8)]
                + [instances.uniform(20000, side=100000, seed=60 + i + seed_offset)
                   for i in range(8)])
    raise ValueError(WORKLOAD)


def select_workload(name):
    global WORKLOAD, M, SIZES
    WORKLOAD = name
    M = WORKLOADS[name]["m"]
    SIZES = [c.shape[0] for c in make_coords()]


def workload_config():
    mems = WORKLOADS[WORKLOAD]["memories"]
    ncol = len(SIZES) * len(mems)
    return {
        "workload": WORKLOADS[WORKLOAD]["desc"],
        "name": WORKLOAD,
        "instances": SIZES if len(SIZES) <= 16 else "%d instances, n in [%d, %d], sum %d"
                     % (len(SIZES), min(SIZES), max(SIZES), sum(SIZES)),
        "m": M,
        "cl": CL,
        "memories": [{0: "matrix", 1: "spm_s8"}[mm] for mm in mems],
        "step": "one ACS iteration of all %d colonies" % ncol,
        "l2": "flushed between timed steps (256 MiB write)",
    }


def ant_steps_per_iter():
    return len(WORKLOADS[WORKLOAD]["memories"]) * sum(M * (n - 1) for n in SIZES)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_PEAK_FALLBACK, "bf16_tflops": BF16_PEAK_FALLBACK}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def rank_seed(rank):
    """Each rank runs its own copy of the workload: instances and Philox seed
    offset by the rank (independent units, no collective on the data path)."""
    return {"instances_seed_offset": rank, "philox_seed": 1 + rank}


# Batched workloads shard by instance across ranks (LPT on m*(n-1), global
# instance ids, no collective); the single-instance ones run one replica per
# rank with its own seed.
SHARDED = ("batch256", "large16")


def rank_share(rank, world):
    """This rank's instances: (global ids or None, coords, offsets, sizes,
    philox seed, sizes of every instance the whole job runs, scaling)."""
    from paper_1605_02669_gb300 import shard

    if WORKLOAD in SHARDED and world > 1:
        coords = make_coords()
        ids, xy, off = shard.shard_of(coords, rank, world, M)
        sizes = [coords[b].shape[0] for b in ids]
        return ids, xy, off, sizes, 1, [c.shape[0] for c in coords], "strong"
    rs = rank_seed(rank)
    coords = make_coords(seed_offset=rs["instances_seed_offset"])
    xy = np.concatenate(coords).astype(np.int32)
    off = np.zeros(len(coords) + 1, np.int64)
    off[1:] = np.cumsum([c.shape[0] for c in coords])
    sizes = [c.shape[0] for c in coords]
    return None, xy, off, sizes, rs["philox_seed"], sizes * world, "weak"


def max_over_ranks(x, world, device):
    """The job's time is the slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, total_ms):
    """Whole-job units per second: every rank processed units_per_rank."""
    return units_per_rank * world / (total_ms / 1000.0)


def run_reference(args, rank, world):
    """CPU oracle, single thread, bounded sample (one colony-iteration per step)."""
    import oracle

    if rank != 0:
        return None
    coords = make_coords()
    colonies = []
    for mem in WORKLOADS[WORKLOAD]["memories"]:
        for xy in coords[:4]:
            p = oracle.make_params(m=M, cl=CL, beta=2, q0=0.9, rho=0.1, xi=0.1, memory=mem,
                                   spm_slots=8, seed=1)
            colonies.append(oracle.Colony(xy, p))
    k = len(colonies)
    units = [M * (c.n - 1) for c in colonies]
    for i in range(args.warmup):
        colonies[i % k].run(1)
    t_total, u_total = 0.0, 0
    for i in range(args.steps):
        c = colonies[i % k]
        t0 = time.perf_counter()
        c.run(1)
        t_total += time.perf_counter() - t0
        u_total += units[i % k]
    value = u_total / t_total
    sample = ("one single-thread oracle iteration per step, rotating over %d colonies of the "
              "workload (m=%d)" % (k, M))
    return {
        "impl": "reference",
        "metric": "ant-steps/s in tour construction",
        "value": value,
        "unit": "ant-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_total / max(args.steps, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": "ant-steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "ant-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform

    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def parallel_oracle_leg(max_seconds=240.0):
    """The oracle instance-parallel over all host cores (one instance per
    thread; the ctypes calls release the GIL): one iteration of every instance
    of the batched workload on the matrix memory, as one CPU job."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    coords = make_coords()
    cores = os.cpu_count() or 1
    p = oracle.make_params(m=M, cl=CL, q0=0.9, memory=0, seed=1)
    t_setup = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        cols = list(ex.map(lambda bx: oracle.Colony(bx[1], p, instance=bx[0]), enumerate(coords)))
    t_setup = time.perf_counter() - t_setup
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda c: c.run(1), cols))
    sec = time.perf_counter() - t0
    units = sum(M * (c.n - 1) for c in cols)
    for c in cols:
        c.close()
    return {"value": units / sec, "unit": "ant-steps/s", "cores": cores, "kind": "oracle",
            "sample": "one iteration of all %d instances (matrix), one instance per thread, "
                      "%.1f s (set-up %.1f s, not timed)" % (len(coords), sec, t_setup)}


def cpu_baseline_leg(seconds_budget=15.0):
    """The oracle as it stands, one thread, on a bounded sample of the workload."""
    import oracle

    coords = make_coords()
    done_units, t_total, ran = 0, 0.0, 0
    cols = {}
    # rounds over the workload's colonies, one oracle iteration each, until the
    # budget is spent (at least one round for small workloads: 1 s)
    while t_total < (seconds_budget if ran == 0 else 1.0):
        for mem in WORKLOADS[WORKLOAD]["memories"]:
            for k, xy in enumerate(coords):
                if ran and t_total > seconds_budget:
                    break
                if (mem, k) not in cols:
                    p = oracle.make_params(m=M, cl=CL, q0=0.9, memory=mem, spm_slots=8, seed=1)
                    cols[(mem, k)] = oracle.Colony(xy, p)
                t0 = time.perf_counter()
                cols[(mem, k)].run(1)
                t_total += time.perf_counter() - t0
                done_units += M * (xy.shape[0] - 1)
                ran += 1
        if t_total > seconds_budget or len(cols) * 2 > 1000:
            break
    for c in cols.values():
        c.close()
    return {"value": done_units / t_total, "unit": "ant-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d oracle iterations over %d colonies of the workload (m=%d), "
                      "single thread, %.1f s" % (ran, len(cols), M, t_total),
            "host": host_cpu()}


KERNEL_SOURCES = ["acs_construct.cu", "acs_device.cuh", "acs_internal.cuh"]
# DRAM bytes (read + write) of one construct launch of this workload, from one
# ncu capture each (profiles/), keyed by (memory, threads per ant, cluster
# size, kernel variant) and valid only for the kernel sources they were taken on.
CAPTURED_TRAFFIC = {
    ("paper", "matrix", 32, 16, 0): {"bytes": 36764160 + 335616, "sources": "5b0c960c1c5e"},
    ("paper", "spm", 32, 16, 2): {"bytes": 16878080 + 0, "sources": "5b0c960c1c5e"},
    ("batch256", "matrix", 8, 1, 0): {"bytes": 40308651776 + 1240432896, "sources": "5b0c960c1c5e"},
    ("batch256", "spm", 8, 1, 1): {"bytes": 4615311104 + 273670912, "sources": "5b0c960c1c5e"},
}


def kernel_sources_digest():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1605_02669_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_traffic(memory, tpa, csize, mode):
    rec = CAPTURED_TRAFFIC.get((WORKLOAD, memory, tpa, csize, mode))
    if rec is None or rec["sources"] != kernel_sources_digest():
        return None
    return rec["bytes"]


def algorithmic_bytes(n, m, fallbacks, spm):
    """Bytes one iteration of one colony must touch (per ant-step, plus the
    full-scan fallback): candidate row (index 128 B + weight 128 B), the
    pheromone of the candidates (matrix gather 128 B, or the SPM record
    s*8+4 = 68 B), the local update (matrix: 2 entries written, 8 B read+write
    of one edge = 16 B; SPM: two record read-modify-writes, 2*68 B); each
    fallback selection reads the heuristic row (4n B) and the pheromone row
    (matrix, 4n B) or the record (SPM, 68 B)."""
    steps = m * (n - 1)
    if spm:
        per = 256 + 68 + 136
        fb = fallbacks * (4 * n + 68)
    else:
        per = 256 + 128 + 16
        fb = fallbacks * 8 * n
    return steps * per + fb


GAP_EVAL = [("clustered", 2392, 301), ("uniform", 5000, 302), ("clustered", 5000, 303)]
# the learned-prior configuration: 2000 generated training instances, n in
# [200, 1000], labels from 8 plain-ACS runs of 200 iterations each
GAP_TRAIN_FULL = {"instances": 2000, "runs": 8, "iters": 200}
# the benchmark's default, a quarter of the instances with 4 runs of 100
# iterations (a stated reduction, to keep the default run within minutes)
GAP_TRAIN_DEFAULT = {"instances": 500, "runs": 4, "iters": 100}


def _replica_batch(coords, reps):
    """Each held-out instance `reps` times in one batched context: replica r
    of instance i has instance id i*reps + r, so its own random stream."""
    xy = np.concatenate([c for c in coords for _ in range(reps)])
    sizes = [c.shape[0] for c in coords for _ in range(reps)]
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return xy, off, sizes


def gap_leg(iters, reps=5, ref_mult=4, train=None, log=None):
    """Tour-length gap at equal GPU time, learned prior vs plain.

    Training: generated instances (n in [200,1000], even b uniform, odd b
    clustered), labels = best-tour edge frequencies of R plain-ACS runs (m=64),
    8 epochs of Adam on the library's MLP kernels (`train` sets the instances,
    R and the run length). Evaluation on held-out instances (n=2392 clustered,
    n=5000 uniform and clustered), m=128: `reps` replicas of each instance in
    one batched context (own random streams); the plain colony runs `iters`
    iterations, the prior colony (16 of 32 candidates, w' = w*p) the same GPU
    time. L* of an instance is the best tour found by any run on it, including
    an independent reference context (prior-pruned replicas with other
    instance ids, so other random streams) that runs `ref_mult` times the
    budget. The gap of a run is
    (L - L*)/L*; reported as mean and standard deviation over the replicas.
    """
    import torch

    from paper_1605_02669_gb300 import acs, instances, prior

    train = dict(GAP_TRAIN_DEFAULT if train is None else train)
    t0 = time.perf_counter()
    params, losses = prior.train(n_instances=train["instances"], n_lo=200, n_hi=1000,
                                 runs=train["runs"], iters=train["iters"], m=64, epochs=8,
                                 batch=4096, lr=2e-3, seed=11)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    coords = [instances.clustered(n, seed=s) if k == "clustered" else instances.uniform(n, seed=s)
              for k, n, s in GAP_EVAL]
    xy, off, sizes = _replica_batch(coords, reps)
    st = torch.cuda.Stream()

    def run(mode, budget_ms=None, n_iters=None, ids=None):
        col = acs.Colony(xy, acs.params(m=128, cl=32, seed=7), offsets=off, instance_ids=ids)
        if mode == "prior":
            prior.apply(col, params, keep=16)
        col.autotune(trial_iters=1)
        col.set_stream(st.cuda_stream)     # the events below time the colony's own stream
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gpu_ms, done = 0.0, 0
        while (budget_ms is None and done < n_iters) or (budget_ms is not None and gpu_ms < budget_ms):
            ev0.record(st)
            col.run(10)
            ev1.record(st)
            ev1.synchronize()
            gpu_ms += ev0.elapsed_time(ev1)
            done += 10
        best = [int(col.best(b)[1]) for b in range(len(sizes))]
        col.close()
        return {"best": best, "iterations": done, "gpu_ms": gpu_ms}

    res = {"plain": run("plain", n_iters=iters)}
    budget = res["plain"]["gpu_ms"]
    res["prior"] = run("prior", budget_ms=budget)
    nb = len(sizes)
    ref_ids = list(range(nb, 2 * nb))
    res["reference"] = run("prior", budget_ms=ref_mult * budget, ids=ref_ids)
    out = {"metric": "tour-length gap at equal GPU time to the best tour found on the instance "
                     "(L*: any run, including an independent reference of %dx the budget)" % ref_mult,
           "unit": "fraction", "higher_is_better": False, "m": 128, "plain_iterations": iters,
           "replicas": reps, "instances": {}}
    for i, (k, n, _) in enumerate(GAP_EVAL):
        idx = range(i * reps, (i + 1) * reps)
        Lstar = min(res[mode]["best"][j] for mode in res for j in idx)
        row = {"L_star": Lstar}
        for mode in ("plain", "prior"):
            g = np.array([(res[mode]["best"][j] - Lstar) / Lstar for j in idx])
            row[mode] = {"mean": float(g.mean()), "std": float(g.std(ddof=1)) if reps > 1 else 0.0,
                         "best": int(min(res[mode]["best"][j] for j in idx))}
        out["instances"]["%s n=%d" % (k, n)] = row
    for mode in ("plain", "prior"):
        g = np.array([out["instances"][k][mode]["mean"] for k in out["instances"]])
        out[mode] = float(g.mean())
    out["iterations"] = {m_: res[m_]["iterations"] for m_ in res}
    out["gpu_ms"] = {m_: res[m_]["gpu_ms"] for m_ in res}
    out["train"] = dict(train, n=[200, 1000], epochs=8, final_loss=losses[-1], seconds=t_train,
                        full_size=train == GAP_TRAIN_FULL)
    return out


def large_prior_leg(iters=20, reps=1):
    """The large-scale configuration with the learned prior on and off: a
    prior trained at the default size scores the candidate lists of the 16
    instances (8 x n=10000, 8 x n=20000, m=256), and both colonies (matrix)
    run `iters` iterations; reports ant-steps/s and the best tour lengths."""
    import torch

    from paper_1605_02669_gb300 import acs, prior

    tr = GAP_TRAIN_DEFAULT
    params, _ = prior.train(n_instances=tr["instances"], n_lo=200, n_hi=1000, runs=tr["runs"],
                            iters=tr["iters"], m=64, epochs=8, batch=4096, lr=2e-3, seed=11)
    coords = make_coords()
    xy = np.concatenate(coords).astype(np.int32)
    off = np.zeros(len(coords) + 1, np.int64)
    off[1:] = np.cumsum([c.shape[0] for c in coords])
    st = torch.cuda.Stream()
    out = {}
    for mode in ("plain", "prior"):
        col = acs.Colony(xy, acs.params(m=M, cl=CL, seed=1), offsets=off)
        if mode == "prior":
            prior.apply(col, params, keep=16)
        col.set_stream(st.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        col.run(iters)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[mode] = {"ant_steps_per_s": sum(M * (n - 1) for n in SIZES) * iters / (ms / 1000.0),
                     "ms_per_iteration": ms / iters,
                     "best": [int(col.best(b)[1]) for b in range(len(coords))]}
        col.close()
    out["iterations"] = iters
    out["mean_best_ratio_prior_to_plain"] = float(np.mean(
        [a / b for a, b in zip(out["prior"]["best"], out["plain"]["best"])]))
    return out


SCORING_ROWS = 1 << 24   # 16.8 M candidate edges (n = 524,288 nodes x 32): 335 MB in and out, > L2
SCORING_FLOPS_USEFUL = 2 * (8 * 64 + 64 * 64 + 64)      # per edge: the three layers
SCORING_FLOPS_ISSUED = 2 * 64 * (16 + 80)                # per edge on the tensor core (K padded, bias columns)


def prior_scoring_leg(steps, warmup):
    """The learned prior's scoring kernel (tcgen05, acs_mlp_forward) on
    SCORING_ROWS seeded synthetic BF16 feature rows, timed alone with CUDA
    events on its stream. Inputs are larger than L2."""
    import torch

    from paper_1605_02669_gb300 import acs

    st = torch.cuda.Stream()
    g = torch.Generator(device="cuda").manual_seed(11)
    with torch.cuda.stream(st):
        params = (torch.randn(acs.ACS_MLP_PARAMS, device="cuda", generator=g) * 0.2).float()
        feat = torch.randn(SCORING_ROWS, 8, device="cuda", generator=g).to(torch.bfloat16).view(torch.int16)
        p = torch.empty(SCORING_ROWS, device="cuda")
    for _ in range(warmup):
        acs.acs_mlp_forward(params, feat, SCORING_ROWS, p, st.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        acs.acs_mlp_forward(params, feat, SCORING_ROWS, p, st.cuda_stream)
    e1.record(st)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0 / steps
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", BF16_PEAK_FALLBACK))
    tflops = SCORING_ROWS * SCORING_FLOPS_USEFUL / sec * 1e-12
    return {"kernel": "mlp_forward_tc_kernel (tcgen05, TMEM accumulators)", "rows": SCORING_ROWS,
            "us_per_launch": sec * 1e6, "edges_per_s": SCORING_ROWS / sec,
            "issued_tflops": SCORING_ROWS * SCORING_FLOPS_ISSUED / sec * 1e-12,
            "hbm_gbs": SCORING_ROWS * 20 / sec * 1e-9,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "peak_kind": kind + " bf16 burst",
                         "flops_per_edge": SCORING_FLOPS_USEFUL},
            "data": "synthetic N(0,1) features rounded to BF16, random N(0,0.2) weights"}


def relaxed_leg(xy, off, sizes, steps, warmup):
    """The relaxed construction (ACS-GPU-Alt, Sec. 3.1.2) on the same instances,
    pheromone matrix: no step barrier, racy local updates (not bit-exact),
    evaluation and global update in a second kernel. Timed like the main line."""
    import torch

    from paper_1605_02669_gb300 import acs

    st = torch.cuda.Stream()
    col = acs.Colony(xy, acs.params(m=M, cl=CL, seed=1, relaxed=True), offsets=off)
    col.set_stream(st.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        col.run(1)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        col.run(1)
        e1.record(st)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    units = sum(M * (n - 1) for n in sizes) * steps
    best = [int(col.best(b)[1]) for b in range(len(sizes))]
    col.close()
    return {"value": units / (total / 1000.0), "unit": "ant-steps/s",
            "ms_per_iteration": total / steps, "memory": "matrix", "best_len": best,
            "note": "relaxed construction (ACS-GPU-Alt): racy local updates, not bit-exact; "
                    "the synchronous deterministic kernels give the main value"}


def _time_iterations(cols, steps, warmup, flush=None):
    """CUDA-event time of `steps` iterations of every colony (each on its own
    stream, L2 flushed between iterations when `flush` is given)."""
    import torch

    for _ in range(warmup):
        for c, _ in cols:
            c.run(1)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        torch.cuda.synchronize()
        evs = []
        for c, st in cols:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            c.run(1)
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        total += max(e0.elapsed_time(e1) for e0, e1 in evs)
    return total


def late_window_leg(ctxs, sizes, flush, iters, steps=10):
    """Steady state: the benchmark's colonies continue for `iters` untimed
    iterations (the pheromone concentrates, the full-scan rate and the SPM hit
    pattern change), then `steps` iterations are timed like the main value."""
    import torch

    for _ in range(iters):
        for c, _ in ctxs:
            c.run(1)
    torch.cuda.synchronize()
    fb0 = [[c.stats(b)[0] for b in range(len(sizes))] for c, _ in ctxs]
    ms = _time_iterations(ctxs, steps, 0, flush)
    fb1 = [[c.stats(b)[0] for b in range(len(sizes))] for c, _ in ctxs]
    units = len(ctxs) * sum(M * (n - 1) for n in sizes) * steps
    fb = sum(b - a for x, y in zip(fb0, fb1) for a, b in zip(x, y))
    return {"value": units / (ms / 1000.0), "unit": "ant-steps/s",
            "iterations_before": int(ctxs[0][0].iteration) - steps, "timed_iterations": steps,
            "ms_per_step": ms / steps,
            "fallback_rate": fb / float(len(ctxs) * steps * sum(M * (n - 1) for n in sizes))}


def period_sweep_leg(xy, off, sizes, tuning, steps=5, warmup=3):
    """Ant-steps/s for local-update periods k = 1, 2, 4, 8, 16 (Sec. 4, the
    paper's updates limited to every k-th step) on the benchmark's instances,
    both memories, the launch shape the autotuner chose for k = 1."""
    import torch

    from paper_1605_02669_gb300 import acs

    out = []
    for k in (1, 2, 4, 8, 16):
        row = {"k": k}
        for mem in WORKLOADS[WORKLOAD]["memories"]:
            st = torch.cuda.Stream()
            col = acs.Colony(xy, acs.params(m=M, cl=CL, memory=mem, spm_slots=8, local_period=k,
                                            seed=1), offsets=off)
            t = tuning[MEM_NAMES[mem]]
            col.set_cluster_size(t["cluster_size"])
            col.set_threads_per_ant(t["threads_per_ant"])
            if mem == acs.ACS_MEM_SPM:
                col.set_spm_resident(1 if t["kernel_mode"] == 2 else 0)
            col.set_stream(st.cuda_stream)
            ms = _time_iterations([(col, st)], steps, warmup)
            row[MEM_NAMES[mem]] = sum(M * (n - 1) for n in sizes) * steps / (ms / 1000.0)
            col.close()
        out.append(row)
    return {"unit": "ant-steps/s", "iterations_timed": steps, "rows": out}


def slot_sweep_leg(xy, off, sizes, iters=50):
    """SPM hit ratio (Sec. 3.2, Fig. spm-hit-ratio: hits / (hits + misses) of
    every record update, local and global) and ant-steps/s against the slots
    per record s, over the first `iters` iterations on the benchmark's
    instances."""
    import torch

    from paper_1605_02669_gb300 import acs

    out = []
    for s in (1, 2, 4, 8, 16, 32):
        st = torch.cuda.Stream()
        col = acs.Colony(xy, acs.params(m=M, cl=CL, memory=acs.ACS_MEM_SPM, spm_slots=s, seed=1),
                         offsets=off)
        col.set_stream(st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        col.run(iters)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        stats = [col.stats(b) for b in range(len(sizes))]
        row = {"s": s, "ant_steps_per_s": sum(M * (n - 1) for n in sizes) * iters / (ms / 1000.0)}
        for n, (fb, sel, hit, miss) in zip(sizes, stats):
            row["hit_ratio_n%d" % n] = hit / float(hit + miss)
        out.append(row)
        col.close()
    return {"iterations": iters, "rows": out,
            "note": "default launch shape; counts every record update of the run"}


def run_ours(args, rank, world, local):
    import torch

    from paper_1605_02669_gb300 import acs

    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    ids, xy, off, sizes, seed, job_sizes, scaling = rank_share(rank, world)
    sA = torch.cuda.Stream()
    sB = torch.cuda.Stream()
    ctxs = []
    tuning = {}
    mems = {"both": WORKLOADS[WORKLOAD]["memories"], "matrix": (acs.ACS_MEM_MATRIX,),
            "spm": (acs.ACS_MEM_SPM,)}[args.only]
    # joint tuning of the concurrent colonies (one trial iteration on large16,
    # where an iteration takes most of a second)
    group_tune = len(mems) > 1
    for mem, st in zip(mems if sizes else (), (sA, sB)):
        p = acs.params(m=M, cl=CL, beta=2, q0=0.9, rho=0.1, xi=0.1, memory=mem, spm_slots=8,
                       seed=seed)
        col = acs.Colony(xy, p, offsets=off, instance_ids=ids)
        col.set_stream(st.cuda_stream)
        if args.tpa or args.cluster:
            if args.cluster:
                col.set_cluster_size(args.cluster)
            if args.tpa:
                col.set_threads_per_ant(args.tpa)
            if args.spm_resident >= 0 and mem == acs.ACS_MEM_SPM:
                col.set_spm_resident(args.spm_resident)
        elif not group_tune:
            # the autotuner picks lanes per ant and cluster size; the state is
            # restored afterwards, so the timed iterations are unaffected
            col.autotune(trial_iters=2)
        ctxs.append((col, st))
    if group_tune and ctxs and not (args.tpa or args.cluster):
        # the colonies run concurrently and compete for the SMs: their shapes
        # are tuned together (each alone first, then jointly)
        acs.autotune_group([c for c, _ in ctxs], trial_iters=1 if WORKLOAD == "large16" else 2)
    for (col, _), mem in zip(ctxs, mems):
        tuning[MEM_NAMES[mem]] = {"threads_per_ant": col.threads_per_ant,
                                  "cluster_size": col.cluster_size,
                                  "kernel_mode": col.kernel_mode}
    if ctxs:
        tuning["joint"] = bool(group_tune and len(ctxs) > 1 and not (args.tpa or args.cluster))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(record=None):
        # ev0/ev1 bracket the step; kev[i] brackets colony i's launch on its own stream
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in ctxs]
        evb = torch.cuda.Event()
        ev0.record(sA)
        sB.wait_event(ev0)
        for (col, st), (k0, k1) in zip(ctxs, kev):
            k0.record(st)
            col.run(1)
            k1.record(st)
        if len(ctxs) > 1:
            evb.record(sB)
            sA.wait_event(evb)
        ev1.record(sA)
        return ev0, ev1, kev

    for _ in range(args.warmup):
        flush.zero_()
        torch.cuda.synchronize()
        step()
    torch.cuda.synchronize()
    fb0 = [[c.stats(b)[0] for b in range(len(sizes))] for c, _ in ctxs]
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    events = []
    launches = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        events.append(step())
        launches += sum(acs.acs_last_launch_count(c.ctx) for c, _ in ctxs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [e0.elapsed_time(e1) for e0, e1, _ in events]
    kern_ms = [[k0.elapsed_time(k1) for k0, k1 in kev] for _, _, kev in events]
    total_ms = max_over_ranks(float(sum(step_ms)), world, "cuda")
    fb1 = [[c.stats(b)[0] for b in range(len(sizes))] for c, _ in ctxs]
    # whole-job units: every rank's replica, or the whole sharded batch
    job_units_per_step = len(mems) * sum(M * (n - 1) for n in job_sizes)
    value = job_units_per_step * args.steps / (total_ms / 1000.0)

    # roofline of each colony's construct launch (both instances in one launch);
    # the dominant kernel is the one with the longer average launch
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    roofs = []
    for i, (col, _) in enumerate(ctxs):
        spm = col.p.memory == acs.ACS_MEM_SPM
        fb = [(b - a) / args.steps for a, b in zip(fb0[i], fb1[i])]
        bytes_launch = sum(algorithmic_bytes(n, M, f, spm) for n, f in zip(sizes, fb))
        avg_s = float(np.mean([k[i] for k in kern_ms])) / 1000.0
        achieved = bytes_launch / avg_s / 1e9
        name = MEM_NAMES[col.p.memory]
        t = tuning[name]
        roofs.append({
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": kernel_traffic(name, t["threads_per_ant"], t["cluster_size"], t["kernel_mode"]),
            "kernel": "construct_kernel<%d,%d> (%s, %d instances in one launch, clusters of %d)"
                      % (t["threads_per_ant"], col.kernel_mode, name, len(sizes),
                         t["cluster_size"]),
            "peak_kind": peak_kind, "kernel_ms": 1000.0 * avg_s,
            "algorithmic_bytes_per_launch": bytes_launch,
            "fallback_rate": float(sum(fb) / (M * sum(n - 1 for n in sizes))),
        })
    roofs.sort(key=lambda r: -r["kernel_ms"])

    # end to end through the public API: host coordinates in, best tour out
    # every iteration (pinned host buffers not needed by the C ABI: it copies)
    e2e = None
    if rank == 0 and not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cols = []
        for mem in WORKLOADS[WORKLOAD]["memories"]:
            p = acs.params(m=M, cl=CL, beta=2, q0=0.9, rho=0.1, xi=0.1, memory=mem, spm_slots=8,
                           seed=seed)
            c = acs.Colony(xy, p, offsets=off, instance_ids=ids)
            # the launch shape the device leg ran with, set through the public
            # API (a caller that tuned once reuses the shape)
            t = tuning.get(MEM_NAMES[mem])
            if t:
                c.set_cluster_size(t["cluster_size"])
                c.set_threads_per_ant(t["threads_per_ant"])
                if mem == acs.ACS_MEM_SPM:
                    c.set_spm_resident(1 if t["kernel_mode"] == 2 else 0)
            cols.append(c)
        d2h = 0
        for _ in range(args.steps):
            for c in cols:
                c.run(1)
            for c in cols:
                for b in range(len(sizes)):
                    t, L = c.best(b)
                    d2h += t.nbytes + 8
        t1 = time.perf_counter()
        for c in cols:
            c.close()
        e2e = {"value": len(WORKLOADS[WORKLOAD]["memories"]) * sum(M * (n - 1) for n in sizes)
                        * args.steps / (t1 - t0), "unit": "ant-steps/s",
               "h2d_bytes_per_step": int(2 * xy.nbytes / args.steps + 2 * off.nbytes / args.steps),
               "d2h_bytes_per_step": int(d2h / args.steps),
               "includes": "context creation from host coordinates (candidate lists, "
                           "nearest-neighbour tour, pheromone init), the device leg's "
                           "launch shape set through the API, and a best-tour read "
                           "after every iteration"}

    late = None
    if rank == 0 and not args.no_late and ctxs:
        li = args.late_iters if args.late_iters is not None else \
            {"batch256": 100, "large16": 20}.get(WORKLOAD, 500)
        late = late_window_leg(ctxs, sizes, flush, li)
    if rank != 0:
        return None
    sweeps = None
    if WORKLOAD == "paper" and not args.no_sweeps:
        sweeps = {"local_period": period_sweep_leg(xy, off, sizes, tuning),
                  "spm_slots": slot_sweep_leg(xy, off, sizes)}
    gap = None if (args.no_gap or WORKLOAD != "paper") else gap_leg(
        args.gap_iters, reps=args.gap_reps,
        train=GAP_TRAIN_FULL if args.gap_full_training else GAP_TRAIN_DEFAULT)
    large_prior = None
    if WORKLOAD == "large16" and not args.no_gap:
        large_prior = large_prior_leg()
    relaxed = None if args.no_relaxed else relaxed_leg(xy, off, sizes, args.steps, args.warmup)
    scoring = None if args.no_prior_scoring else prior_scoring_leg(args.steps, args.warmup)
    cpu = None if args.no_cpu_baseline else cpu_baseline_leg()
    if cpu is not None and WORKLOAD in SHARDED and not args.no_parallel_oracle:
        cpu["all_cores"] = parallel_oracle_leg()
    return {
        "metric": "ant-steps/s in tour construction",
        "value": value,
        "unit": "ant-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": scaling,
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload_config(), parallelism=(
            "instances sharded by LPT over %d ranks" % world if scaling == "strong"
            else "one replica per rank" if world > 1 else "one GPU")),
        "iterations_per_s": 1000.0 * args.steps / total_ms,
        "roofline": roofs[0],
        "roofline_other": roofs[1:],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "tuning": tuning,
        "late_window": late,
        "sweeps": sweeps,
        "gap_at_equal_time": gap,
        "large_prior": large_prior,
        "relaxed": relaxed,
        "prior_scoring": scoring,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="paper",
                    help="paper (default, the metric's configuration), n198, batch256, large16")
    ap.add_argument("--only", choices=["both", "matrix", "spm"], default="both",
                    help="time only one memory kind (profiling runs; the metric needs both)")
    ap.add_argument("--no-gap", action="store_true",
                    help="skip the learned-prior gap leg (profiling runs)")
    ap.add_argument("--no-relaxed", action="store_true",
                    help="skip the relaxed-construction leg")
    ap.add_argument("--gap-iters", type=int, default=1000,
                    help="iterations of the plain colony in the gap leg")
    ap.add_argument("--gap-reps", type=int, default=5,
                    help="replicas (own random streams) of each held-out instance in the gap leg")
    ap.add_argument("--gap-full-training", action="store_true",
                    help="train the prior at the full configuration (2000 instances, 8 runs x "
                         "200 iterations) instead of the default quarter size")
    ap.add_argument("--no-prior-scoring", action="store_true",
                    help="skip the learned prior's scoring leg")
    ap.add_argument("--prior-scoring-only", action="store_true",
                    help="run only the learned prior's scoring leg (profiling)")
    ap.add_argument("--no-late", action="store_true", help="skip the late-window leg")
    ap.add_argument("--late-iters", type=int, default=None,
                    help="untimed iterations before the late timed window (default: 500, "
                         "batch256 100, large16 20)")
    ap.add_argument("--no-sweeps", action="store_true",
                    help="skip the local-period and SPM-slot sweeps")
    ap.add_argument("--no-parallel-oracle", action="store_true",
                    help="skip the all-cores oracle timing of the batched workloads")
    ap.add_argument("--tpa", type=int, default=0, help="pin lanes per ant instead of autotuning")
    ap.add_argument("--cluster", type=int, default=0, help="pin the cluster size instead of autotuning")
    ap.add_argument("--spm-resident", type=int, choices=[-1, 0, 1], default=-1,
                    help="with --tpa/--cluster: pin the SPM records to global memory (0) or to the "
                         "cluster's shared memory (1); -1 leaves the choice to the launch planner")
    args = ap.parse_args()
    select_workload(args.workload)
    rank, world, local = dist_setup(args)
    if args.prior_scoring_only:
        import torch

        torch.cuda.set_device(local)
        import __graft_entry__

        __graft_entry__.build()
        out = prior_scoring_leg(args.steps, args.warmup) if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
