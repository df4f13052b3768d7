#!/usr/bin/env python
"""Benchmark: pool-gradient sweeps/s at 52 spin-orbitals / 12 electrons, N = 1e6.

One step = one pass of the whole hot path on one synthetic workload:
  apply the 200-gate ansatz from the reference determinant with top-1e6
  truncation after every gate, then one pool sweep, which builds sigma = H psi
  on the state and its connected space and returns the full operator-pool
  gradient (301,600 generalized singles and doubles) and the energy.
The standalone energy kernel (sigma restricted to the state, used for
energy-only evaluations) is timed separately and reported as `energy_ms`.
`value` is steps (= pool-gradient sweeps) per second with inputs resident in
HBM; `e2e` is the same through the host-buffer C-ABI calls, host<->device
copies included.  `--impl reference` times the CPU oracle on a bounded
sample of the same workload instead.

Multi-GPU (torchrun): every rank runs its own replica of the workload (the
path has no exchange step), value = all ranks' sweeps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pool-gradient sweeps/s at 52 spin-orbitals, 12 electrons, N=1e6"
WORKLOAD = "so52_e12"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="swcs", choices=["swcs", "reference"])
    p.add_argument("--n-keep", type=int, default=1_000_000)
    p.add_argument("--cpu-sample", type=int, default=800, help="determinants in the oracle's bounded sample")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--sweep", type=int, default=0, help="0 auto, 1 hashed external table, 2 alpha-string rows")
    p.add_argument("--cluster", type=int, default=1, help="CTAs per alpha-string row cluster")
    p.add_argument("--rows-l2", type=int, default=0, help="1: cap concurrent rows to about half of L2")
    p.add_argument("--threads", type=int, default=1024, help="threads per CTA of the row sweep")
    p.add_argument("--row-clusters", type=int, default=0, help="clusters of the row sweep (0: as many as fit)")
    p.add_argument("--row-occupancy", type=int, default=2, help="resident 512-thread row-sweep CTAs per SM (1, 2 or 3)")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the 64-instance batched leg and the small configurations on the device")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    p.add_argument("--no-screen", action="store_true", help="skip the learned-screening leg")
    p.add_argument("--no-adapt", action="store_true", help="skip the ADAPT-VQE leg")
    p.add_argument("--adapt-n-keep", type=int, default=10_000, help="N_CUT of the ADAPT-VQE leg")
    p.add_argument("--adapt-iters", type=int, default=30, help="ADAPT iterations of the ADAPT-VQE leg")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        load = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ oracle sample
def oracle_sample(w, n_sample):
    """Wall time of the oracle's step (apply the ansatz truncated to n_sample
    determinants, energy, full pool gradient) on one host core."""
    import oracle as O
    t0 = time.perf_counter()
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_sample)
    O.energy(w.n_so, w.h, w.g, k, a)
    O.pool_gradients(w.n_so, w.h, w.g, k, a)
    return time.perf_counter() - t0, len(k)


def _farm_worker(inq, out, bar, name):
    sys.path.insert(0, ROOT)
    import oracle as O  # noqa: F401
    from paper_2411_07920_gb300 import inputs as I
    w = I.workload(name)
    while True:
        n = inq.get()
        if n is None:
            break
        bar.wait(timeout=900)
        t0 = time.time()
        _, nk = oracle_sample(w, n)
        out.put((t0, time.time(), nk))


class OracleFarm:
    """One single-threaded oracle process per host core (spawned, so they never
    share a CUDA context), each running the same bounded sample at the same
    time: the host's whole throughput on the oracle as it stands."""

    def __init__(self, cores, name):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.bar = ctx.Barrier(cores)
        self.out = ctx.Queue()
        self.inq = [ctx.Queue() for _ in range(cores)]
        self.procs = [ctx.Process(target=_farm_worker, args=(q, self.out, self.bar, name), daemon=True)
                      for q in self.inq]
        for p in self.procs:
            p.start()

    def run(self, n_sample):
        """(wall seconds from the first start to the last finish, determinants per sample)."""
        for q in self.inq:
            q.put(n_sample)
        res = [self.out.get(timeout=1800) for _ in self.inq]
        return max(r[1] for r in res) - min(r[0] for r in res), res[0][2]

    def close(self):
        for q in self.inq:
            q.put(None)
        for p in self.procs:
            p.join(timeout=60)


def scaling_exponent(n1, t1, n2, t2):
    return math.log(t2 / t1) / math.log(n2 / n1)


def cpu_baseline(w, n_keep, n_small, n_big, configs=True):
    """The oracle on the machine's host cores: single-threaded at two sample sizes
    (the fitted exponent carries the time to N), then one process per core on
    the larger sample at once; plus the two small configurations timed whole."""
    import oracle as O
    from paper_2411_07920_gb300 import inputs as I
    O.build()
    cores = os.cpu_count() or 1
    t1, n1 = oracle_sample(w, n_small)
    t2, n2 = oracle_sample(w, n_big)
    alpha = scaling_exponent(n1, t1, n2, t2)
    farm = OracleFarm(cores, WORKLOAD)
    try:
        tp, _ = farm.run(n_big)
    finally:
        farm.close()
    sec_per_sweep = tp * (n_keep / n2) ** alpha / cores  # cores sweeps in flight at once
    res = {"value": 1.0 / sec_per_sweep, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
           "host_cores": cores,
           "sample": (f"oracle step (apply 200 gates, energy, full pool gradient) on the same 52/12 workload "
                      f"truncated to {n2} determinants, run by {cores} single-threaded processes at once "
                      f"({tp:.1f} s wall); time per sweep carried to N={n_keep} by the exponent {alpha:.3f} "
                      f"fitted on one core at {n1} ({t1:.1f} s) and {n2} ({t2:.1f} s) determinants"),
           "single_thread": {"dets": [n1, n2], "s": [round(t1, 3), round(t2, 3)], "exponent": round(alpha, 4)},
           "parallel": {"processes": cores, "dets": n2, "wall_s": round(tp, 3)}}
    if configs:
        out = {}
        for name in ("so12_e4", "so28_e8"):
            wc = I.workload(name)
            t, nk = oracle_sample(wc, wc.n_keep)
            out[name] = {"dets": nk, "s": round(t, 3), "sweeps_per_s": round(1.0 / t, 6)}
        res["configs_single_thread"] = out
    return res


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2411_07920_gb300 import inputs as I
    import oracle as O
    O.build()
    w = I.workload(WORKLOAD, n_keep=args.n_keep)
    cores = os.cpu_count() or 1
    n_step = min(args.cpu_sample, 200)
    farm = OracleFarm(cores, WORKLOAD)
    try:
        # the exponent that carries a sample's time to N, from two sample sizes on all cores
        t_half, n_half = farm.run(max(n_step // 2, 10))
        for _ in range(args.warmup):
            t_full, nk = farm.run(n_step)
        if args.warmup < 1:
            t_full, nk = farm.run(n_step)
        alpha = scaling_exponent(n_half, t_half, nk, t_full)
        total = 0.0
        for _ in range(args.steps):
            dt, nk = farm.run(n_step)
            total += dt
    finally:
        farm.close()
    sec_per_sweep = total / args.steps * (args.n_keep / nk) ** alpha / cores
    value = 1.0 / sec_per_sweep
    sample = (f"oracle step (apply 200 gates, energy, full pool gradient) on the same 52/12 workload truncated to "
              f"{nk} determinants, run by {cores} single-threaded processes at once per step "
              f"({total / args.steps:.2f} s wall per step); time per sweep carried to N={args.n_keep} by the "
              f"exponent {alpha:.3f} fitted on all cores at {n_half} and {nk} determinants")
    line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "impl": "reference", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_sweep * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "52 spin-orbitals, 12 electrons, 200 gates, N=1e6, "
                                                        "pool 301600 (seed 3)", "l2": "n/a (CPU)"},
            "timed_region_s": round(total, 3),
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "exponent": round(alpha, 4)},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_swcs(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2411_07920_gb300 import inputs as I
    from paper_2411_07920_gb300 import swcs

    w = I.workload(WORKLOAD, n_keep=args.n_keep)
    ctx = swcs.Context()
    ctx.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    ctx.set_option("sweep", args.sweep)
    ctx.set_option("cluster", args.cluster)
    ctx.set_option("rows_l2", args.rows_l2)
    ctx.set_option("threads", args.threads)
    ctx.set_option("row_clusters", args.row_clusters)
    ctx.set_option("row_occupancy", args.row_occupancy)
    pool = ctx.pool_size()
    dev = torch.device("cuda", local)
    d_ops = torch.from_numpy(w.ops.reshape(-1).copy()).to(dev)
    d_theta = torch.from_numpy(w.theta.copy()).to(dev)
    d_g = torch.empty(pool, dtype=torch.float64, device=dev)
    d_e = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.apply_ansatz_dev(d_ops, d_theta, args.n_keep)
        ctx.pool_gradients_dev(d_g)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the timed events)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    stats = ctx.stats()
    prof = ctx.profile_read(reset=True)
    # standalone energy kernel (sigma restricted to the state), timed apart from the step
    energy_ms = []
    for _ in range(3):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx.energy_dev(d_e)
        ev1.record(stream)
        ev1.synchronize()
        energy_ms.append(ev0.elapsed_time(ev1))
    ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    ms_per_step, value = aggregate(total_ms, args.steps, world, dev)

    # hash probes of one more (untimed) step: lookups and the index slots they visit, per second of the
    # kernels that make them (gate kernel: partner lookups of the merge; row sweep: neighbour discovery)
    ctx.set_option("count_probes", 1)
    ctx.probe_counts(reset=True)
    step()
    pc = ctx.probe_counts(reset=True)
    ctx.set_option("count_probes", 0)
    g_ms = prof.get("ansatz", (0.0, 0))[0] / max(args.steps, 1)
    r_ms = prof.get("row_sweep", (0.0, 0))[0] / max(args.steps, 1)
    probes = {"gate": {"lookups": pc["gate_lookups"], "slots": pc["gate_slots"],
                       "slots_per_lookup": round(pc["gate_slots"] / max(pc["gate_lookups"], 1), 4),
                       "lookups_per_s": pc["gate_lookups"] / (g_ms / 1e3) if g_ms > 0 else None},
              "row_sweep": {"lookups": pc["row_lookups"], "slots": pc["row_slots"],
                            "slots_per_lookup": round(pc["row_slots"] / max(pc["row_lookups"], 1), 4),
                            "lookups_per_s": pc["row_lookups"] / (r_ms / 1e3) if r_ms > 0 else None}}

    # ------------------------------------------------------------ roofline of the dominant kernel
    import math
    no, nv = w.n_e // 2, w.n_so // 2 - w.n_e // 2
    n_conn = 2 * no * nv + 2 * math.comb(no, 2) * math.comb(nv, 2) + no * no * nv * nv
    n_det = args.n_keep
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    buckets = max(stats["ext_buckets"], 1)
    pairs = n_det * (n_conn + 1)
    # algorithmic bytes per connected (D, E) pair: the scatter reads the key and
    # sigma_E and writes sigma_E (24 B), the gather reads them (16 B); the row
    # sweep does both in one launch
    per_pair = {"sigma_scatter": 24.0, "pool_gather": 16.0, "row_sweep": 40.0}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if dom == "row_sweep":
        bytes_per_launch = per_pair[dom] * pairs
    elif dom in per_pair:
        bytes_per_launch = per_pair[dom] * pairs / buckets
    elif dom == "ansatz":
        # per gate: read S (16 B/det), write and re-read Phi (32 B), select reads (8 B/pass), write S (16 B)
        bytes_per_launch = (16 + 32 + 8 * max(stats["select_passes"] / max(stats["gates"], 1), 1) + 16) * \
            stats["gate_dets"] / max(dom_n, 1)
    else:
        bytes_per_launch = 16.0 * pairs
    achieved = bytes_per_launch / (dom_ms / dom_n / 1e3) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": measured_traffic(dom, args),
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    gate_ms = prof.get("ansatz", (0.0, 0))[0]
    gate_dets_per_s = stats["gate_dets"] / (gate_ms / 1e3) if gate_ms > 0 else None
    # the other two kernels of the path, on the same measured peak
    rooflines = {}
    gate_n = prof.get("ansatz", (0.0, 0))[1]
    if gate_ms > 0 and gate_n > 0:
        # per gate: read S (16 B/det), write and re-read Phi (32 B), select reads (8 B/pass), write S' (16 B),
        # with |Phi| and |S'| taken as |S|
        passes = stats["select_passes"] / max(stats["gates"], 1)
        gb = (16 + 32 + 8 * passes + 16) * stats["gate_dets"] / gate_n
        ach = gb / (gate_ms / gate_n / 1e3) / 1e9
        rooflines["gate"] = {"kernel": "ansatz", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak, "bytes_per_launch": gb, "select_passes_per_gate": passes,
                             "traffic": measured_traffic("ansatz", args)}
    if energy_ms:
        # energy <psi|H|psi>: 16 B (key and amplitude) per connection of every determinant probed in the
        # state, the bytes of the probe formulation (the row kernel in energy-only mode reads fewer)
        eb = 16.0 * n_det * (n_conn + 1)
        ach = eb / (min(energy_ms) / 1e3) / 1e9
        rooflines["energy"] = {"kernel": "row_sweep (energy only)", "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                               "unit": "GB/s", "frac": ach / hbm_peak, "bytes_per_launch": eb, "traffic": None}
    launches = int(stats["kernel_launches"])

    # ------------------------------------------------------------ end to end through the host API
    e2e = None
    if not args.no_e2e:
        h_pin = torch.from_numpy(w.h.copy()).pin_memory()
        g_pin = torch.from_numpy(w.g.reshape(-1).copy()).pin_memory()
        ops_pin = torch.from_numpy(w.ops.reshape(-1).copy()).pin_memory()
        th_pin = torch.from_numpy(w.theta.copy()).pin_memory()
        h_np, g_np, ops_np, th_np = h_pin.numpy(), g_pin.numpy(), ops_pin.numpy(), th_pin.numpy()
        t_e2e = 0.0
        for it in range(1 + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.load_hamiltonian(h_np, g_np, w.n_so, w.n_e)
            ctx.apply_ansatz(ops_np, th_np, args.n_keep)
            g_host = ctx.pool_gradients()
            e_val, _ = ctx.sweep_energy()
            dt = time.perf_counter() - t0
            if it > 0:
                t_e2e += dt
        h2d = w.h.nbytes + w.g.nbytes + w.ops.nbytes + w.theta.nbytes
        d2h = 16 + g_host.nbytes
        e2e = {"value": world * args.steps / t_e2e, "unit": "sweeps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # ------------------------------------------------------------ adjoint leg (same workload, 200 parameters)
    adjoint = None
    if not args.no_adjoint:
        ts = []
        for it in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e_adj, d_adj = ctx.energy_grad(w.ops, w.theta, args.n_keep, 20)
            ts.append(time.perf_counter() - t0)
        adjoint = {"ms": round(1e3 * min(ts[1:]), 3), "params": int(len(w.theta)), "ckpt_every": 20,
                   "energy": e_adj, "grad_norm": float(np.linalg.norm(d_adj))}

    # ------------------------------------------------------------ learned screening leg (same state)
    screen_res = None
    if not args.no_screen:
        screen_res = run_screen_leg(swcs, ctx, w, args, torch)

    # ------------------------------------------------------------ the two small configurations
    configs = None
    if not args.no_batch:
        configs = run_configs_leg(swcs, I, torch)

    # ------------------------------------------------------------ batched leg: 64 uneven instances
    batch = None
    if not args.no_batch:
        batch = run_batch_leg(swcs, I, torch)

    # ------------------------------------------------------------ ADAPT-VQE leg (same Hamiltonian, from HF)
    adapt_res = None
    if not args.no_adapt:
        adapt_res = run_adapt_leg(swcs, w, args, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, args.n_keep, max(args.cpu_sample // 4, 10), args.cpu_sample)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "52 spin-orbitals, 12 electrons, 200-gate ansatz (seed 3), "
                                       f"N={args.n_keep}, GSD pool {pool}",
                           "parallelism": f"replicas x{world}", "l2": "flushed between steps (512 MB write)"},
                "gate_dets_per_s": gate_dets_per_s, "roofline": roof, "rooflines": rooflines, "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "energy_ms": round(min(energy_ms), 3), "hash_probes": probes,
                "adjoint": adjoint, "batch": batch, "screen": screen_res, "adapt": adapt_res, "configs": configs,
                "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()},
                "ext": {"distinct": stats["ext_distinct"], "buckets": stats["ext_buckets"],
                        "capacity": stats["ext_capacity"]}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def aggregate(total_ms, steps, world, device):
    """Whole-job throughput: every rank ran `steps` replicas of the workload;
    the job time is the slowest rank's (max over ranks)."""
    import torch
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = t.item()
    return total_ms / steps, world * steps / (total_ms / 1e3)


# the launch the committed row-sweep traffic was captured on: the default workload and launch shape
TRAFFIC_CAPTURED = dict(n_keep=1_000_000, cluster=1, rows_l2=0, threads=1024, row_clusters=0)
# kernel -> (committed ncu summary, the sources of the captured kernel)
TRAFFIC_FILES = {
    "row_sweep": ("profiles/row_sweep_so52_e12_N1e6.md",
                  ["paper_2411_07920_gb300/csrc/swcs_rowsweep.cu", "paper_2411_07920_gb300/csrc/swcs_rowsweep.cuh"]),
    "ansatz": ("profiles/ansatz_so52_e12_N1e6.md",
               ["paper_2411_07920_gb300/csrc/swcs_ansatz.cu", "paper_2411_07920_gb300/csrc/swcs_select.cuh"]),
}


def source_sha16(paths):
    """sha256 prefix of the concatenated sources of a kernel."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, args):
    """DRAM bytes per launch of the dominant kernel from its committed ncu summary,
    only for the workload and launch shape that were captured and while the
    kernel's source is the one that was captured (else None)."""
    if kernel not in TRAFFIC_FILES:
        return None
    if args.sweep == 1 or any(getattr(args, k) != v for k, v in TRAFFIC_CAPTURED.items()):
        return None
    summary, srcs = TRAFFIC_FILES[kernel]
    try:
        text = open(os.path.join(ROOT, summary)).read()
        want = text.split("source_sha256:")[1].split()[0]
        traffic = int(text.split("traffic_bytes_per_launch:")[1].split()[0])
        have = source_sha16(srcs)
    except (OSError, IndexError, ValueError):
        return None
    return traffic if have == want else None


def run_screen_leg(swcs, ctx, w, args, torch, frac=0.05):
    """Train the screening network on exact pool gradients of the small
    workload families (12/4 untruncated, 20/6 and 28/8 truncated), then screen
    the 52/12 state: features, network, top 5%, subset sweep -- against the
    full sweep of the same state.  Also times the network's forward pass over
    the whole pool (tensor-core GEMMs)."""
    from paper_2411_07920_gb300 import screen
    t0 = time.perf_counter()
    X, T = screen.training_set(screen.default_specs())
    net = swcs.Mlp(32, 256)
    net.set_params(screen.init_params(seed=0))
    hist = screen.train(net, X, T)
    t_train = time.perf_counter() - t0
    ctx.apply_ansatz(w.ops, w.theta, args.n_keep)
    res = []
    for _ in range(3):
        res.append(screen.evaluate(ctx, net, frac))
    best = min(res, key=lambda r: r["t_screened"])
    best["t_full"] = min(r["t_full"] for r in res)
    best["speedup"] = best["t_full"] / best["t_screened"]
    # the same subset sweep forming sigma in full (only the contractions filtered), for comparison
    ctx.set_option("screen_scatter", 0)
    t_sigma_full = min(screen.evaluate(ctx, net, frac)["t_screened"] for _ in range(3))
    ctx.set_option("screen_scatter", 1)
    # network forward over the whole pool, device time
    P = ctx.pool_size()
    x = torch.empty((P, 32), dtype=torch.int16, device="cuda")
    ctx.pool_features_dev(x)
    y = torch.empty(P, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def timed(call):
        call(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(10):
            call(x, y)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / 10 / 1e3
    t_layers = timed(net.forward_dev)   # three launches, activations through HBM
    t_fwd = timed(net.predict_dev)      # the fused kernel the screen uses
    flops = 2.0 * P * (32 * 256 + 256 * 256 + 256)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    # one training step (five tensor-core GEMMs, transposes, reductions, Adam) on the training batch and on a
    # larger one, device time; the learning rate is 0 here, the network has served its purpose
    step_ms = {}
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for nb in (8192, 65536):
        if X.shape[0] < nb:
            continue
        xb, tb = X[:nb].contiguous(), T[:nb].contiguous()
        net.train_step_dev(xb, tb, 0.0, loss)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(20):
            net.train_step_dev(xb, tb, 0.0, loss)
        e1.record(st)
        e1.synchronize()
        step_ms[str(nb)] = round(e0.elapsed_time(e1) / 20, 4)
    net.close()
    return {"frac": frac, "subset": best["subset"], "pool": best["pool"], "recall_argmax": best["recall_argmax"],
            "recall_top10": best["recall_top10"], "same_argmax": bool(best["same_argmax"]),
            "max_abs_err_on_subset": best["max_abs_err_on_subset"], "full_ms": round(1e3 * best["t_full"], 3),
            "screened_ms": round(1e3 * best["t_screened"], 3), "speedup": round(best["speedup"], 3),
            "screened_sigma_in_full_ms": round(1e3 * t_sigma_full, 3),
            "train_s": round(t_train, 2), "train_samples": int(X.shape[0]), "train_loss": hist[-1][1],
            "train_step_ms": step_ms,
            "mlp_forward": {"kernel": "mlp_fused_kernel", "ms": round(1e3 * t_fwd, 4),
                            "tflops": round(flops / t_fwd / 1e12, 2),
                            "frac_of_bf16_peak": round(flops / t_fwd / 1e12 / bf16_peak, 4),
                            "layer_by_layer_ms": round(1e3 * t_layers, 4)}}


def run_adapt_leg(swcs, w, args, torch):
    """ADAPT-VQE with BFGS-2 over the spin-complemented pool on the benchmark
    Hamiltonian from the reference determinant at N_CUT = args.adapt_n_keep:
    wall time per iteration, split
    into the pool sweep (step 4) and the VQE over swcs_energy_grad (step 7)."""
    from paper_2411_07920_gb300 import adapt
    c = swcs.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    a = adapt.Adapt(c, args.adapt_n_keep, eps=1e-3, pool_kind="spin")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.run(args.adapt_iters, "bfgs2")
    total = time.perf_counter() - t0
    its = [it for it in a.history if it.op_index >= 0 and not it.stalled]
    t_pool = sum(it.t_pool_s for it in a.history)
    t_vqe = sum(it.t_vqe_s for it in a.history)
    res = {"workload": f"{w.n_so} spin-orbitals, {w.n_e} electrons, spin-complemented GSD pool, "
                       f"N_CUT={args.adapt_n_keep}, BFGS-2 from the reference determinant",
           "iterations": len(its), "ms_per_iteration": round(1e3 * total / max(1, len(a.history)), 3),
           "pool_ms": round(1e3 * t_pool, 3), "vqe_ms": round(1e3 * t_vqe, 3),
           "vqe_share": round(t_vqe / total, 4) if total > 0 else None,
           "energy_grad_calls": int(sum(it.energy_grad_calls for it in a.history)),
           "dets": [int(it.n_dets) for it in its], "energies": [float(it.energy) for it in its],
           "grad_norms": [float(it.grad_norm) for it in a.history]}
    c.close()
    return res


def run_configs_leg(swcs, I, torch, reps=5):
    """The two small configurations on the device: one step (apply the ansatz, pool sweep) with inputs resident,
    event-timed, with the energy and the state size."""
    out = {}
    for name in ("so12_e4", "so28_e8"):
        w = I.workload(name)
        with swcs.Context() as c:
            c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
            d_ops = torch.from_numpy(w.ops.reshape(-1).copy()).cuda()
            d_th = torch.from_numpy(w.theta.copy()).cuda()
            d_g = torch.empty(c.pool_size(), dtype=torch.float64, device="cuda")
            st = torch.cuda.current_stream()

            def step():
                c.apply_ansatz_dev(d_ops, d_th, w.n_keep)
                c.pool_gradients_dev(d_g)
            for _ in range(3):
                step()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                step()
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            e, _ = c.sweep_energy()
            out[name] = {"step_ms": round(ms, 4), "sweeps_per_s": round(1e3 / ms, 2), "energy": e,
                         "dets": int(len(c.get_state()[0])), "pool": int(c.pool_size())}
    return out


def run_batch_leg(swcs, I, torch, n_inst=64, seed0=100, reps=3):
    """64 uneven instances (n_so in U{16..40}, n_e in U{4..12}, 20-150 gates,
    N_keep log-uniform 1e3-1e5): one persistent launch for all of them
    (autotuned, settings cached in JSON) against the same per-instance kernels
    launched back to back on one stream, and against the host API called
    instance by instance; every instance's result checked against its own
    context."""
    import tempfile as tf
    specs = I.batch_specs(n_inst, seed0)
    ws = [I.batch_instance(s) for s in specs]
    b = swcs.Batch()
    for w in ws:
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    cache = os.path.join(tf.gettempdir(), "swcs_batch_tuning.json")
    b.build(autotune=True, cache_path=cache)

    def timed(call):
        call()
        b.results(0)  # synchronises
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            call()
            b.results(0)
            ts.append(time.perf_counter() - t0)
        return min(ts)
    t_launch = timed(b.run)
    res = [b.results(i) for i in range(n_inst)]
    t_back = timed(b.run_serial)
    ctxs = []
    for w in ws:
        c = swcs.Context()
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        ctxs.append(c)

    def host_api():
        for c, w in zip(ctxs, ws):
            c.apply_ansatz(w.ops, w.theta, w.n_keep)
            c.pool_gradients()
            c.sweep_energy()

    host_api()
    th = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_api()
        th.append(time.perf_counter() - t0)
    err = 0.0
    for i, (c, w) in enumerate(zip(ctxs, ws)):
        c.apply_ansatz(w.ops, w.theta, w.n_keep)
        g1 = c.pool_gradients()
        e, _, g = res[i]
        err = max(err, float(np.abs(g - g1).max()), abs(e - c.sweep_energy()[0]))
    tun = b.tuning()
    for c in ctxs:
        c.close()
    b.close()
    return {"instances": n_inst, "launch": "one persistent kernel, (instance, phase, tile) work items",
            "launch_ms": round(1e3 * t_launch, 3), "back_to_back_ms": round(1e3 * t_back, 3),
            "host_api_ms": round(1e3 * min(th), 3), "speedup_vs_back_to_back": round(t_back / t_launch, 3),
            "speedup_vs_host_api": round(min(th) / t_launch, 3), "max_abs_diff_all_instances": err,
            "autotune": tun, "tuning_from_cache": bool(getattr(b, "from_cache", False)),
            "instances_per_s": round(n_inst / t_launch, 3)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_swcs(args)


if __name__ == "__main__":
    main()
