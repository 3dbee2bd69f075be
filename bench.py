"""Benchmark of global Shepard IDW (Eq. 1) on GB300.

One step = one FP32-compensated interpolation of M = 2^20 queries against
N = 2^20 data points (p = 2), inputs resident in HBM: staging, all-pairs
sweep, FP64 combine, slow path.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (one rank per GPU, under torchrun, or started by this script
itself when ``--gpus N`` is given without a launcher): every rank
interpolates its own 2^20 queries (seeded by rank) against the same
replicated data; there is no collective on the data path (weak scaling).
Timing: barrier + synchronize on both sides of the K timed steps, max over
ranks.

Besides ``value`` (device-resident pairs/s) the line carries:
  e2e           the same metric through the host-buffer C-ABI entry point,
                host<->device copies of inputs and results inside the region;
  roofline      the all-pairs sweep kernel's pairs/s (CUDA events around each
                launch, recorded by the library) against the arithmetic-pipe
                peak min(FMA pipe / 6 ops, MUFU / 1 op) per pair;
  f64_plain     the plain FP64 form on the same GPU (query sample);
  error         max |Z - Z_64| / max |z| against the FP64 oracle on a query
                sample (the same sample the CPU baseline times);
  cpu_baseline  the FP64 oracle on the host cores (bounded query sample);
  clocks        nvidia-smi samples taken during the timed region;
  general_p, batched, adjoint, noalloc
                after the timed region: the general-power sweep (p = 3.5) on
                the same data, the 256-problem batched launch against this
                run's single-instance pairs/s, the forward and every
                gradient at N = M = 262144, p = 2.5 (dL/dq sampled against
                the oracle), and the allocation-free entry point at
                N = M = 262144 against the handle path.
``--full-check`` compares all M outputs with the oracle (minutes of host time).
``--impl reference`` times the oracle alone (the CPU reference arm).

``--config NAME`` prints one line per other workload instead (``all`` runs
the headline and every one of them): scale, clustered, adjoint, batched,
layout, paper, and the local forms.  The ``local`` and ``knn`` lines carry
rows for one-shot calls, gradients (``backward``), prepared-index calls,
and a raster of queries in sorted and caller order, plus a ``cpu_baseline``
of the oracle; ``--members`` and ``--data`` pick their cases.
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

METRIC = ("pairs/s at N=M=2^20 p=2: FP32-comp vs FP64 plain, error ≤2e-6, "
          "% pipe roofline")
UNIT = "pairs/s"
N_DEFAULT = 1 << 20
# Doc values for compute capability 10.x (per SM per clock): 128 FP32 FMA
# lanes, 16 MUFU lanes.  The measured rates are reported beside them.
FFMA_PER_SM_CLK = 128.0
MUFU_PER_SM_CLK = 16.0
FMA_OPS_PER_PAIR = 6.0   # 2 FADD (dx, dy), FMUL, FFMA (d^2), FADD (S0), FFMA (S1)
MUFU_OPS_PER_PAIR = 1.0  # rcp(d^2) at p = 2
# Sharing one reciprocal between two pairs trades half a MUFU op per pair for
# 1.5 FMA-pipe ops (1/(da db), then db r and da r).
SHARED_FMA_PER_PAIR = 1.5
SHARED_MUFU_SAVED_PER_PAIR = 0.5
SWEEP_SOURCES = ("idw_fwd_f32.cu", "idw_f32_common.cuh", "idw_device.cuh", "idw_internal.h")
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "sweep_p2_n1048576_dram.md")


# Algorithmic cost per pair evaluation of each sweep (compensation, loads
# and loop overhead not credited): FP32 FMA-pipe ops and MUFU ops by kind.
#   p = 2      d^2 (2 FADD, FMUL, FFMA), S0 FADD, S1 FFMA; rcp
#   general p  the same plus t = -(p/2) log2 d^2 (FMUL); lg2, ex2
#   adjoint    one sweep's term (general p): d^2 (4), the two exponents (2
#              FMUL), z - Z, (z - Z) v, two FFMA for the x / y sums, and for
#              dL/dp (z - Z) w, log2 d^2 + shift, an FFMA; lg2 and two ex2
#              (w and v = w / d^2).  The adjoint evaluates each pair twice
#              (query sweep and data sweep).
SWEEP_COSTS = {
    "pow2": {"fma": 6.0, "mufu": {"mufu_rcp": 1.0}},
    "general": {"fma": 7.0, "mufu": {"mufu_lg2": 1.0, "mufu_ex2": 1.0}},
    "adjoint_general": {"fma": 13.0, "mufu": {"mufu_lg2": 1.0, "mufu_ex2": 2.0}},
}


def pipe_peak_pairs_s(kind, rates, sms, mhz, evaluations_per_pair=1.0):
    """min(FMA pipe, MUFU pipe) pairs/s of a sweep from the measured per-SM
    per-clock pipe rates (MUFU ops of different kinds share the pipe, so
    their issue times add)."""
    c = SWEEP_COSTS[kind]
    ffma = max(rates["ffma"], rates["ffma2"])
    mufu_clk = sum(n / rates[k] for k, n in c["mufu"].items())
    per_sm_clk = min(ffma / c["fma"], 1.0 / mufu_clk)
    return sms * mhz * 1e6 * per_sm_clk / evaluations_per_pair


def roofline_block(kind, achieved, rates, sms, mhz, kernel, evaluations_per_pair=1.0,
                   traffic=None, algorithmic_bytes=None):
    """The roofline object of a non-headline line: the measured-rate pipe
    bound of its sweep at the sampled clock."""
    peak = pipe_peak_pairs_s(kind, rates, sms, mhz, evaluations_per_pair)
    c = SWEEP_COSTS[kind]
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpairs/s",
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "algorithmic_bytes_per_launch": algorithmic_bytes, "kernel": kernel,
            "peak_basis": f"min(FMA pipe / {c['fma']:g} ops, MUFU pipe / "
                          + " + ".join(f"{n:g} {k[5:]}" for k, n in c["mufu"].items())
                          + f") per pair evaluation, measured per-SM-per-clock rates x {sms} "
                          f"SMs x {mhz} MHz" + (f", {evaluations_per_pair:g} evaluations per pair"
                                                if evaluations_per_pair != 1.0 else "")}


def lp_pairs_per_sm_clk(ffma, mufu):
    """Best pairs per SM per clock when any fraction f of the pairs may share
    reciprocals: max r s.t. r (6 + 1.5 f) <= ffma and r (1 - f / 2) <= mufu."""
    best = 0.0
    for i in range(1001):
        f = i / 1000.0
        best = max(best, min(ffma / (FMA_OPS_PER_PAIR + SHARED_FMA_PER_PAIR * f),
                             mufu / (MUFU_OPS_PER_PAIR - SHARED_MUFU_SAVED_PER_PAIR * f)))
    return best


def sweep_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1402_4986_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current sweep sources (else None)."""
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    vals = dict(line.split(":", 1) for line in text.splitlines()
                if line.startswith(("traffic_bytes_per_launch:", "sweep_source_sha256:")))
    if vals.get("sweep_source_sha256:".rstrip(":"), "").strip() != sweep_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--full-check", action="store_true",
                    help="headline only: after the timed region, compare every one of the M "
                         "outputs with the FP64 oracle on all host cores (minutes) and report "
                         "the maximum error")
    ap.add_argument("--members", type=float, nargs="*", default=None,
                    help="local / knn workloads only: these neighbour counts (K, or k) "
                         "instead of the default sweep")
    ap.add_argument("--data", choices=["uniform", "clustered"], default="uniform",
                    help="local / knn workloads with --members: the data distribution")
    ap.add_argument("--config", default="headline",
                    choices=["headline", "scale", "clustered", "adjoint", "batched", "layout",
                             "paper", "local", "knn", "all"],
                    help="headline = the N=M=2^20 line; the others measure the other "
                         "workloads (one JSON line each)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args, rank):
    """CPU reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    import synthetic
    prob = synthetic.config_scale(args.n)
    data, q = prob["data"], prob["queries"]
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.idw(data, q[:32], 2.0)
    rate = 32 * args.n / (time.perf_counter() - t)
    total_steps = args.steps + args.warmup
    per_step = max(8, int(min(150.0 / total_steps, 8.0) * rate / args.n))
    rng = np.random.default_rng(0)
    times = []
    for s in range(total_steps):
        idx = rng.choice(q.shape[0], per_step, replace=False)
        t = time.perf_counter()
        oracle.idw(data, q[idx], 2.0, threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    pairs = per_step * args.n
    value = pairs * len(times) / sum(times)
    sample = f"{per_step} random queries x all {args.n} data points per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"global Shepard IDW, N=M={args.n}, p=2, uniform [0,1)^2, "
                               "wave field (FP64 CPU oracle on a query sample)",
                   "n": args.n, "m": args.n, "p": 2.0},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import synthetic
    import paper_1402_4986_gb300 as idw
    from paper_1402_4986_gb300 import build as libbuild
    libbuild.build()

    n = m = args.n
    prob = synthetic.config_scale(n)
    data_np = prob["data"]
    # Weak scaling: rank r interpolates its own query set against the same data.
    q_np = prob["queries"] if rank == 0 else synthetic.uniform_xy(
        np.random.default_rng(9000 + rank), m)
    data = torch.from_numpy(data_np).cuda()
    q = torch.from_numpy(q_np).cuda()
    out = torch.empty(m, device="cuda")
    h = idw.get_handle(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        idw.interpolate(data, q, 2.0, out=out, handle=h)
    idw.sync_status(handle=h)

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed region: K device-resident steps
    idw.profile_read(handle=h)
    idw.profile_enable(True, handle=h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)   # evict inputs from L2 between steps
        ev[k][0].record(stream)
        idw.interpolate(data, q, 2.0, out=out, handle=h)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier()
    clocks = sampler.stop()
    idw.profile_enable(False, handle=h)
    sweep_ms, sweep_launches = idw.profile_read(handle=h)
    idw.sync_status(handle=h)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if dist is not None:
        t = torch.tensor([total_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t)
    pairs_step = float(n) * m
    value = ws * pairs_step * args.steps / total_s
    Z_dev = out.cpu().numpy()

    # ---- end to end: host buffers through the C ABI, copies inside the region
    d_host = torch.from_numpy(data_np).pin_memory()
    q_host = torch.from_numpy(q_np).pin_memory()
    o_host = torch.empty(m, dtype=torch.float32).pin_memory()
    idw.interpolate_host(d_host, q_host, 2.0, out=o_host, handle=h)
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        idw.interpolate_host(d_host, q_host, 2.0, out=o_host, handle=h)
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t)
    e2e = {"value": ws * pairs_step * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(data_np.nbytes + q_np.nbytes),
           "d2h_bytes_per_step": int(o_host.numel() * 4)}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- FP64 plain form, same GPU, query sample (it runs ~100x slower)
    m64 = 8192
    d64 = data.double()
    q64 = q[:m64].double()
    idw.interpolate(d64, q64[:1024], 2.0, "f64", handle=h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    idw.interpolate(d64, q64, 2.0, "f64", handle=h)
    e1.record(stream)
    torch.cuda.synchronize()
    f64_value = float(n) * m64 / (e0.elapsed_time(e1) / 1e3)

    # ---- pipe roofline of the sweep kernel
    rates = idw.measure_pipe_rates(local)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    clk_mhz = clocks.get("sm_mhz") or 0.0
    sweep_avg_s = sweep_ms / max(1, sweep_launches) / 1e3
    achieved = pairs_step / sweep_avg_s

    def peak(ffma, mufu, mhz):
        return sms * mhz * 1e6 * min(ffma / FMA_OPS_PER_PAIR, mufu / MUFU_OPS_PER_PAIR)

    peak_doc = peak(FFMA_PER_SM_CLK, MUFU_PER_SM_CLK, clk_mhz)
    peak_meas = peak(max(rates["ffma"], rates["ffma2"]), rates["mufu_rcp"], clk_mhz)
    lp = sms * clk_mhz * 1e6 * lp_pairs_per_sm_clk(FFMA_PER_SM_CLK, MUFU_PER_SM_CLK)
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_doc / 1e9,
            "unit": "Gpairs/s", "frac": achieved / peak_doc if peak_doc else None,
            "traffic": recorded_traffic(),
            "algorithmic_bytes_per_launch": 12 * n + 8 * m + 4 * m,
            "lp_bound": lp / 1e9, "frac_of_lp_bound": achieved / lp if lp else None,
            "lp_basis": "max pairs/s when a fraction f of pairs shares reciprocals: "
                        "r (6 + 1.5 f) <= 128 FMA lanes and r (1 - f/2) <= 16 MUFU lanes "
                        "per SM per clock",
            "kernel": "sweep_kernel<p = 2> (all-pairs sweep)",
            "peak_basis": "min(128 FFMA / 6 ops, 16 MUFU / 1 op) per SM per clock x "
                          f"{sms} SMs x median SM clock {clk_mhz} MHz under load",
            "peak_measured_rates": peak_meas / 1e9,
            "frac_of_measured_rates": achieved / peak_meas if peak_meas else None,
            "peak_at_2070mhz": peak(FFMA_PER_SM_CLK, MUFU_PER_SM_CLK, 2070.0) / 1e9,
            "pipe_rates_per_sm_clk": rates,
            "sweep_ms_avg": sweep_avg_s * 1e3, "sweep_launches": sweep_launches}

    extras = headline_extras(args, idw, h, data, q, data_np, q_np, value / ws, rates, sms,
                             clk_mhz)

    # ---- FP64 oracle on the host: error check + CPU baseline on one sample
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        oracle.idw(data_np, q_np[:32], 2.0, threads=cores)
        rate = 32 * n / (time.perf_counter() - t)
        S = int(min(max(256, args.cpu_seconds * rate / n), m))
        idx = np.sort(np.random.default_rng(1).choice(m, S, replace=False))
        t = time.perf_counter()
        Z64, _ = oracle.idw(data_np, q_np[idx], 2.0, threads=cores)
        cpu_s = time.perf_counter() - t
        err = float(np.max(np.abs(Z_dev[idx].astype(np.float64) - Z64)) /
                    np.max(np.abs(data_np[:, 2])))
        cpu = {"value": S * n / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{S} random queries x all {n} data points ({cpu_s:.1f} s)"}

    full = None
    if args.full_check:
        import oracle
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        Zall, _ = oracle.idw(data_np, q_np, 2.0, threads=cores)
        full = {"queries": int(m), "max_error_vs_fp64_oracle": float(
                    np.max(np.abs(Z_dev.astype(np.float64) - Zall)) / np.max(np.abs(data_np[:, 2]))),
                "oracle_s": time.perf_counter() - t, "cores": cores}

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"global Shepard IDW, N=M={n} per GPU, p=2, uniform [0,1)^2 "
                               "points, z = sin(2 pi x) cos(2 pi y) + 0.1 N(0,1), "
                               "FP32-compensated (FP64 combine)",
                   "n": n, "m": m, "p": 2.0, "parallelism": f"query shards x{ws}, data replicated",
                   "l2": "flushed between steps (256 MiB write; inputs are 36 MiB)"},
        "e2e": e2e, "gpu_launches": 4 * args.steps,
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "error_vs_fp64_oracle": err,
        **({"full_check": full} if full else {}),
        "f64_plain": {"value": f64_value, "unit": UNIT,
                      "sample": f"{m64} queries x all {n} data points"},
        "speedup_vs_f64_plain": value / ws / f64_value,
        "wall_s_timed_region": wall,
        **extras,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                    "max": max(step_ms)},
    }
    print(json.dumps(res), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def headline_extras(args, idw, h, data, q, data_np, q_np, single_pairs_s, rates, sms, mhz):
    """Compact summaries of the other workloads, measured in the same run
    after the headline's timed region: the general-power sweep on the same
    N = M = 2^20 data (p = 3.5), the batched workload (256 uneven problems
    in one persistent launch) against this run's single-instance pairs/s,
    the forward and adjoint at N = M = 262144, p = 2.5, and the
    allocation-free entry point at N = M = 262144."""
    import ctypes
    import torch
    import synthetic
    out = {}
    n, m = data.shape[0], q.shape[0]
    pairs = float(n) * m
    o = torch.empty(m, device="cuda")
    # General power: the lg2/ex2 sweep.
    p = 3.5
    idw.interpolate(data, q, p, out=o, handle=h)
    idw.profile_read(handle=h)
    idw.profile_enable(True, handle=h)
    ms = _events_ms(lambda: idw.interpolate(data, q, p, out=o, handle=h), 3, warm=0)
    idw.profile_enable(False, handle=h)
    sweep_ms, launches = idw.profile_read(handle=h)
    achieved = pairs / (sweep_ms / max(1, launches) / 1e3)
    gen = {"p": p, "pairs_s": pairs / (ms / 1e3), "call_ms": ms,
           "roofline": roofline_block("general", achieved, rates, sms, mhz,
                                      "sweep_kernel<general p> (all-pairs sweep)")}
    if not args.no_cpu_baseline:
        import oracle
        idx = np.sort(np.random.default_rng(11).choice(m, 512, replace=False))
        Z64, _ = oracle.idw(data_np, q_np[idx], p, threads=os.cpu_count() or 1)
        gen["error_vs_fp64_oracle"] = float(
            np.max(np.abs(o.cpu().numpy()[idx].astype(np.float64) - Z64)) /
            np.max(np.abs(data_np[:, 2])))
        gen["error_sample_queries"] = len(idx)
    # The same sweep with one log2 in 16 on the FMA pipe (IDW_OPT_FMA_LOG2).
    hf = idw.Handle(torch.cuda.current_device())
    idw.set_option("fma_log2", 1, handle=hf)
    fms = _events_ms(lambda: idw.interpolate(data, q, p, out=o, handle=hf), 3)
    hf.close()
    gen["fma_log2_1_in_16"] = {"pairs_s": pairs / (fms / 1e3), "call_ms": fms,
                               "vs_mufu_lg2": ms / fms}
    out["general_p"] = gen
    # Batched: 256 uneven problems, one persistent launch.
    batch = synthetic.config_batch()
    bd = [torch.from_numpy(i["data"]).cuda() for i in batch["instances"]]
    bq = [torch.from_numpy(i["queries"]).cuda() for i in batch["instances"]]
    bo = [torch.empty(x.shape[0], device="cuda") for x in bq]
    bpairs = float(sum(x.shape[0] * y.shape[0] for x, y in zip(bd, bq)))
    idw.profile_read(handle=h)
    idw.profile_enable(True, handle=h)
    bms = _events_ms(lambda: idw.interpolate_batched(bd, bq, 2.0, outs=bo, handle=h), 5)
    idw.profile_enable(False, handle=h)
    bsweep, blaunch = idw.profile_read(handle=h)
    out["batched"] = {
        "instances": len(bd), "total_pairs": bpairs, "persistent_ms": bms,
        "persistent_pairs_s": bpairs / (bms / 1e3),
        "single_large_instance_pairs_s": single_pairs_s,
        "persistent_vs_single": bpairs / (bms / 1e3) / single_pairs_s,
        "roofline": roofline_block("pow2", bpairs / (bsweep / max(1, blaunch) / 1e3), rates, sms,
                                   mhz, "sweep_kernel<p = 2, batch table> (one persistent launch)")}
    del bd, bq, bo
    # Differentiation: forward with saved S0, then every gradient, N = M = 262144,
    # p = 2.5; dL/dq of 256 sampled queries against the FP64 oracle (each
    # query's dL/dq depends on its own row of Eq. 1 only).
    ap = synthetic.config_adjoint()
    ad = torch.from_numpy(ap["data"]).cuda()
    aq = torch.from_numpy(ap["queries"]).cuda()
    ag = torch.from_numpy(ap["grad_out"]).cuda()
    saved = {}

    def adj_fwd():
        saved["Z"], saved["s0"], saved["hit"] = idw.interpolate_saved(ad, aq, ap["p"], handle=h)

    def adj_bwd():
        saved["g"] = idw.backward(ad, aq, ap["p"], saved["Z"], saved["s0"], saved["hit"], ag,
                                  handle=h)

    f_ms = _events_ms(adj_fwd, 3)
    b_ms = _events_ms(adj_bwd, 3)
    apairs = float(ad.shape[0]) * aq.shape[0]
    adj = {"n": ad.shape[0], "m": aq.shape[0], "p": ap["p"], "forward_ms": f_ms,
           "backward_ms": b_ms, "backward_over_forward": b_ms / f_ms,
           "backward_pair_evaluations_s": 2 * apairs / (b_ms / 1e3),
           "roofline": roofline_block("adjoint_general", apairs / (b_ms / 1e3), rates, sms, mhz,
                                      "query sweep + data sweep (whole backward call)",
                                      evaluations_per_pair=2.0)}
    if not args.no_cpu_baseline:
        import oracle
        idx = np.sort(np.random.default_rng(12).choice(aq.shape[0], 256, replace=False))
        G = oracle.idw_grad(ap["data"], ap["queries"][idx], ap["p"], ap["grad_out"][idx],
                            threads=os.cpu_count() or 1)
        gq = saved["g"][2].cpu().numpy()[idx]
        adj["grad_q_error_vs_fp64_oracle"] = float(
            np.max(np.abs(gq - G["grad_q"])) / np.max(np.abs(G["grad_q"])))
        adj["error_sample_queries"] = len(idx)
    out["adjoint"] = adj
    del ad, aq, ag, saved
    # The allocation-free entry point against the handle path, N = M = 262144.
    sp = synthetic.config_scale(262144)
    sd = torch.from_numpy(sp["data"]).cuda()
    sq = torch.from_numpy(sp["queries"]).cuda()
    so = torch.empty(sq.shape[0], device="cuda")
    lib = h.lib
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def noalloc():
        rc = lib.idw_interpolate_noalloc(sd.data_ptr(), sd.shape[0], sq.data_ptr(), sq.shape[0],
                                         2.0, so.data_ptr(), st)
        if rc != 0:
            raise RuntimeError(f"idw_interpolate_noalloc: status {rc}")

    na_ms = _events_ms(noalloc, 10, warm=2)
    if lib.idw_noalloc_sync_status(st) != 0:
        raise RuntimeError("idw_interpolate_noalloc reported a device timeout")
    hd_ms = _events_ms(lambda: idw.interpolate(sd, sq, 2.0, out=so, handle=h), 10, warm=2)
    p2 = float(sd.shape[0]) * sq.shape[0]
    out["noalloc"] = {"n": sd.shape[0], "m": sq.shape[0], "p": 2.0, "ms": na_ms,
                      "pairs_s": p2 / (na_ms / 1e3), "handle_path_ms": hd_ms,
                      "noalloc_vs_handle": hd_ms / na_ms}
    return out


# ------------------------------------------------------------ other workloads

def _events_ms(fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _timed_with_sweep(idw, h, fn, reps, warm=1):
    """(call ms, sweep-kernel ms) per call, each averaged over ``reps`` calls
    on handle ``h``: the calls timed as a user runs them, then the sweep
    alone from the CUDA events the library records around it when profiling
    is on (which launches the sweep without programmatic dependent launch,
    so the call time is taken with profiling off)."""
    ms = _events_ms(fn, reps, warm=warm)
    idw.profile_read(handle=h)
    idw.profile_enable(True, handle=h)
    _events_ms(fn, reps, warm=0)
    idw.profile_enable(False, handle=h)
    sweep_ms, launches = idw.profile_read(handle=h)
    return ms, sweep_ms / max(1, launches)


def _pipe_context():
    """Measured pipe rates, SM count and the SM clock for the roofline of the
    non-headline lines (the clock: the current nvidia-smi reading under load
    is not sampled here, so the maximum SM clock is used, which makes the
    fractions conservative)."""
    import torch
    import paper_1402_4986_gb300 as idw
    dev = torch.cuda.current_device()
    rates = idw.measure_pipe_rates(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(dev)], capture_output=True, text=True, timeout=10).stdout
        mhz = float(out.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    return rates, sms, mhz


def _raster_order_rows(idw, d, form, arg, label):
    """The same data queried on a 1024 x 1024 raster of cell centres (rows
    in order): one-shot and prepared-index calls with the queries sorted
    into cells (default) and in the caller's order."""
    import torch
    g = (torch.arange(1024, device="cuda", dtype=torch.float64) + 0.5) / 1024
    yy, xx = torch.meshgrid(g, g, indexing="ij")
    q = torch.stack([xx.reshape(-1), yy.reshape(-1)], 1).float().contiguous()
    out = torch.empty(q.shape[0], device="cuda")
    rows = []
    for order in (0, 1):
        h = idw.Handle(torch.cuda.current_device())
        idw.set_option("local_query_order", order, handle=h)
        if form == "local":
            one = lambda: idw.interpolate_local(d, q, 2.0, arg, out=out, handle=h)
            ix = idw.LocalIndex(d, radius=arg, handle=h)
            call = lambda: ix.interpolate(q, 2.0, out=out)
        else:
            one = lambda: idw.interpolate_knn(d, q, 2.0, arg, out=out, handle=h)
            ix = idw.LocalIndex(d, k=arg, handle=h)
            call = lambda: ix.knn(q, 2.0, out=out)
        for kind, fn in (("one-shot", one), ("prepared index", call)):
            ms = _events_ms(fn, 10, warm=3)
            rows.append({"data": "uniform", "queries": "raster 1024 x 1024", "call": kind,
                         "query_order": "caller" if order else "sorted", label: arg, "p": 2.0,
                         "ms": ms, "queries_s": q.shape[0] / (ms / 1e3)})
        ix.close()
        h.close()
    return rows


def _oracle_queries_s(args, fn, m, label):
    """The FP64 oracle timed on the host cores over a bounded random sample
    of the workload's queries (about a third of --cpu-seconds)."""
    if args.no_cpu_baseline:
        return None
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    fn(np.arange(64), cores)
    rate = 64 / (time.perf_counter() - t)
    S = int(min(max(256, args.cpu_seconds / 3 * rate), m))
    idx = np.sort(np.random.default_rng(9).choice(m, S, replace=False))
    t = time.perf_counter()
    fn(idx, cores)
    cpu_s = time.perf_counter() - t
    return {"value": S / cpu_s, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{S} random queries of {label} ({cpu_s:.1f} s)"}


def _emit(workload, rows, **extra):
    line = {"metric": "pairs/s", "unit": UNIT, "data": "synthetic", "dtype": "f32",
            "config": {"workload": workload}, "rows": rows}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_scale(args):
    """Paper-shaped sweep N = M, FP32-compensated vs plain FP64, p = 2."""
    import torch
    import oracle
    import synthetic
    import paper_1402_4986_gb300 as idw
    rows = []
    rates, sms, mhz = _pipe_context()
    h = idw.get_handle()
    for n in synthetic.SCALE_SWEEP:
        prob = synthetic.config_scale(n)
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        out = torch.empty(n, device="cuda")
        pairs = float(n) * n
        reps = max(3, int(2e11 / pairs))
        ms, sweep_ms = _timed_with_sweep(idw, h, lambda: idw.interpolate(d, q, 2.0, out=out,
                                                                          handle=h), reps)
        m64 = min(n, 8192)
        d64, q64 = d.double(), q[:m64].double()
        ms64 = _events_ms(lambda: idw.interpolate(d64, q64, 2.0, "f64"), 2)
        idx = np.random.default_rng(3).choice(n, min(n, 512), replace=False)
        Z64, _ = oracle.idw(prob["data"], prob["queries"][idx], 2.0)
        err = float(np.max(np.abs(out.cpu().numpy()[idx] - Z64)) /
                    np.max(np.abs(prob["data"][:, 2])))
        rows.append({"n": n, "m": n, "f32c_pairs_s": pairs / (ms / 1e3),
                     "f32c_ms": ms, "f64_pairs_s": float(n) * m64 / (ms64 / 1e3),
                     "speedup_vs_f64": (pairs / ms) / (float(n) * m64 / ms64),
                     "error_vs_fp64_oracle": err, "error_sample_queries": len(idx),
                     "roofline": roofline_block("pow2", pairs / (sweep_ms / 1e3), rates, sms, mhz,
                                                "sweep_kernel<p = 2>")})
    _emit("paper-shaped scale sweep N=M, uniform [0,1)^2, wave field, p=2 (FP64 arm on "
          "min(N, 8192) queries)", rows)


def run_clustered(args):
    """Gaussian-mixture data, 1024^2 query grid, p in {1.5, 2, 3.5}."""
    import torch
    import oracle
    import synthetic
    import paper_1402_4986_gb300 as idw
    prob = synthetic.config_clustered()
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    n, m = d.shape[0], q.shape[0]
    out = torch.empty(m, device="cuda")
    idx = np.random.default_rng(4).choice(m, 1024, replace=False)
    rows = []
    rates, sms, mhz = _pipe_context()
    h = idw.get_handle()
    for p in prob["p_values"]:
        ms, sweep_ms = _timed_with_sweep(idw, h, lambda: idw.interpolate(d, q, p, out=out,
                                                                          handle=h), 5)
        Z64, _ = oracle.idw(prob["data"], prob["queries"][idx], p)
        err = float(np.max(np.abs(out.cpu().numpy()[idx] - Z64)) /
                    np.max(np.abs(prob["data"][:, 2])))
        rows.append({"p": p, "pairs_s": float(n) * m / (ms / 1e3), "ms": ms,
                     "path": "rcp" if p == 2.0 else "log2/exp2",
                     "error_vs_fp64_oracle": err, "error_sample_queries": len(idx),
                     "roofline": roofline_block("pow2" if p == 2.0 else "general",
                                                float(n) * m / (sweep_ms / 1e3), rates, sms, mhz,
                                                "sweep_kernel")})
    # p = 2 through the log2/exp2 form as well.
    hg = idw.Handle(torch.cuda.current_device())
    idw.set_option("force_general_power", 1, handle=hg)
    ms, sweep_ms = _timed_with_sweep(idw, hg, lambda: idw.interpolate(d, q, 2.0, out=out,
                                                                       handle=hg), 5)
    Z64, _ = oracle.idw(prob["data"], prob["queries"][idx], 2.0)
    err = float(np.max(np.abs(out.cpu().numpy()[idx] - Z64)) / np.max(np.abs(prob["data"][:, 2])))
    hg.close()
    rows.append({"p": 2.0, "pairs_s": float(n) * m / (ms / 1e3), "ms": ms, "path": "log2/exp2",
                 "error_vs_fp64_oracle": err, "error_sample_queries": len(idx),
                 "roofline": roofline_block("general", float(n) * m / (sweep_ms / 1e3), rates, sms,
                                            mhz, "sweep_kernel<general p>")})
    _emit("clustered: N=262144 from 64 Gaussian blobs (sigma 0.01), z = exp(-4 r^2) + "
          "0.05 N(0,1), queries on a 1024^2 grid", rows)


def run_adjoint(args):
    """Forward + adjoint at N = M = 262144, p = 2.5."""
    import torch
    import synthetic
    import paper_1402_4986_gb300 as idw
    prob = synthetic.config_adjoint()
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    g = torch.from_numpy(prob["grad_out"]).cuda()
    p = prob["p"]
    n, m = d.shape[0], q.shape[0]
    state = {}

    def fwd():
        state["Z"], state["s0"], state["hit"] = idw.interpolate_saved(d, q, p)

    def bwd():
        idw.backward(d, q, p, state["Z"], state["s0"], state["hit"], g)

    fwd_ms = _events_ms(fwd, 3)
    bwd_ms = _events_ms(bwd, 3)
    pairs = float(n) * m
    rates, sms, mhz = _pipe_context()
    _emit("adjoint: N=M=262144 uniform [0,1)^2, wave field, p=2.5, upstream grad N(0,1); "
          "backward = query sweep + data sweep (2 pair evaluations per pair)",
          [{"forward_ms": fwd_ms, "forward_pairs_s": pairs / (fwd_ms / 1e3),
            "backward_ms": bwd_ms, "backward_pairs_s": pairs / (bwd_ms / 1e3),
            "backward_pair_evaluations_s": 2 * pairs / (bwd_ms / 1e3),
            "backward_over_forward": bwd_ms / fwd_ms,
            "roofline": roofline_block("adjoint_general", pairs / (bwd_ms / 1e3), rates, sms, mhz,
                                       "query sweep + data sweep (whole backward call)",
                                       evaluations_per_pair=2.0),
            "forward_roofline": roofline_block("general", pairs / (fwd_ms / 1e3), rates, sms, mhz,
                                               "sweep_kernel<general p> (whole forward call)")}])


def run_batched(args, headline_pairs_s=None):
    """256 uneven problems: one persistent launch vs a per-instance loop."""
    import torch
    import synthetic
    import paper_1402_4986_gb300 as idw
    batch = synthetic.config_batch()
    inst = batch["instances"]
    d = [torch.from_numpy(i["data"]).cuda() for i in inst]
    q = [torch.from_numpy(i["queries"]).cuda() for i in inst]
    outs = [torch.empty(x.shape[0], device="cuda") for x in q]
    pairs = float(sum(x.shape[0] * y.shape[0] for x, y in zip(d, q)))

    def batched():
        idw.interpolate_batched(d, q, 2.0, outs=outs)

    def loop():
        for dk, qk, ok in zip(d, q, outs):
            idw.interpolate(dk, qk, 2.0, out=ok)

    rates, sms, mhz = _pipe_context()
    hb = idw.get_handle()
    ms_b, sweep_b = _timed_with_sweep(idw, hb, batched, 5)
    ms_l = _events_ms(loop, 3)
    # Autotuned: the first call of the size class times every sweep variant.
    ht = idw.Handle(torch.cuda.current_device())
    idw.set_option("autotune", 1, handle=ht)
    t0 = time.perf_counter()
    idw.interpolate_batched(d, q, 2.0, outs=outs, handle=ht)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    ms_t = _events_ms(lambda: idw.interpolate_batched(d, q, 2.0, outs=outs, handle=ht), 5)
    tuned_variant = idw.get_option("last_variant", handle=ht)
    per_variant = {}
    for v in range(6):
        idw.set_option("sweep_variant", v, handle=ht)
        per_variant[v] = pairs / (_events_ms(
            lambda: idw.interpolate_batched(d, q, 2.0, outs=outs, handle=ht), 3) / 1e3)
    ht.close()
    graph = torch.cuda.CUDAGraph()
    batched()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batched()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(graph):
        batched()
    ms_g = _events_ms(graph.replay, 5)
    if headline_pairs_s is None:
        big = synthetic.config_scale(1 << 20)
        bd = torch.from_numpy(big["data"]).cuda()
        bq = torch.from_numpy(big["queries"]).cuda()
        bo = torch.empty(bq.shape[0], device="cuda")
        headline_pairs_s = float(1 << 40) / (_events_ms(
            lambda: idw.interpolate(bd, bq, 2.0, out=bo), 3) / 1e3)
    row = {"instances": len(inst), "total_pairs": pairs,
           "persistent_ms": ms_b, "persistent_pairs_s": pairs / (ms_b / 1e3),
           "graph_replay_ms": ms_g, "graph_replay_pairs_s": pairs / (ms_g / 1e3),
           "loop_ms": ms_l, "loop_pairs_s": pairs / (ms_l / 1e3),
           "autotuned_variant": tuned_variant, "autotuned_pairs_s": pairs / (ms_t / 1e3),
           "autotune_first_call_s": tune_s, "pairs_s_per_variant": per_variant,
           "single_large_instance_pairs_s": headline_pairs_s,
           "persistent_vs_single": (pairs / (ms_b / 1e3)) / headline_pairs_s,
           "persistent_vs_loop": ms_l / ms_b,
           "roofline": roofline_block("pow2", pairs / (sweep_b / 1e3), rates, sms, mhz,
                                      "sweep_kernel<p = 2, batch table> (one persistent launch)")}
    # Small problems, where a per-instance loop pays a call's fixed latency
    # for little arithmetic: 256 problems, N_i, M_i log-uniform in [256, 8192].
    del d, q, outs, graph
    small = synthetic.config_batch(count=256, lo=256, hi=8192)["instances"]
    sd = [torch.from_numpy(i["data"]).cuda() for i in small]
    sq = [torch.from_numpy(i["queries"]).cuda() for i in small]
    so = [torch.empty(x.shape[0], device="cuda") for x in sq]
    spairs = float(sum(x.shape[0] * y.shape[0] for x, y in zip(sd, sq)))
    ms_sb = _events_ms(lambda: idw.interpolate_batched(sd, sq, 2.0, outs=so), 10, warm=2)
    small_default = idw.get_option("last_variant")

    def small_loop():
        for dk, qk, ok in zip(sd, sq, so):
            idw.interpolate(dk, qk, 2.0, out=ok)

    ms_sl = _events_ms(small_loop, 3)
    hv = idw.Handle(torch.cuda.current_device())
    small_variants = {}
    for v in range(6):
        idw.set_option("sweep_variant", v, handle=hv)
        small_variants[v] = spairs / (_events_ms(
            lambda: idw.interpolate_batched(sd, sq, 2.0, outs=so, handle=hv), 5, warm=2) / 1e3)
    hv.close()
    small_row = {"instances": len(small), "sizes": "N_i, M_i log-uniform in [256, 8192]",
                 "total_pairs": spairs, "persistent_ms": ms_sb,
                 "persistent_pairs_s": spairs / (ms_sb / 1e3), "loop_ms": ms_sl,
                 "loop_pairs_s": spairs / (ms_sl / 1e3), "persistent_vs_loop": ms_sl / ms_sb,
                 "default_variant": small_default,
                 "pairs_s_per_variant": small_variants}
    _emit("batched: 256 problems, N_i, M_i log-uniform in [1024, 262144] (seeded), uniform "
          "[0,1)^2, p=2, FP32-compensated; one persistent launch (also graph-captured) vs a "
          "loop of per-instance calls; single large instance = N=M=2^20; second row: 256 "
          "small problems, N_i, M_i log-uniform in [256, 8192]", [row, small_row])


def run_layout(args):
    """Staging-layout ablation of the single-problem sweep (Sec. 2.2, 3.3)."""
    import torch
    import synthetic
    import paper_1402_4986_gb300 as idw
    names = {0: "duplicated pairs (x,x,y,y)+(z,z), 24 B/point",
             1: "aligned AoS (x,y,z,pad), 16 B/point", 2: "SoA x[],y[],z[], 12 B/point"}
    rows = []
    for n in (100_000, 1 << 20):
        prob = synthetic.config_scale(n)
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        out = torch.empty(n, device="cuda")
        for p in (2.0, 3.5):
            for layout in (0, 1, 2):
                h = idw.Handle(torch.cuda.current_device())
                idw.set_option("sweep_variant", 0, handle=h)
                idw.set_option("staging_layout", layout, handle=h)
                reps = 3 if n > 200_000 else 20
                ms = _events_ms(lambda: idw.interpolate(d, q, p, out=out, handle=h), reps)
                idw.profile_enable(True, handle=h)
                idw.interpolate(d, q, p, out=out, handle=h)
                sweep_ms, _ = idw.profile_read(handle=h)
                h.close()
                rows.append({"n": n, "m": n, "p": p, "layout": layout, "layout_name": names[layout],
                             "pairs_s": float(n) * n / (ms / 1e3), "call_ms": ms,
                             "sweep_ms": sweep_ms})
    # The plain FP64 form in the paper's FP64 layouts (Sec. 3.5, 4.1.2).
    f64_names = {-1: "Hybrid (x,y) pairs + z[], 24 B/point", 1: "AoaS (x,y,z,pad), 32 B/point",
                 2: "SoA x[],y[],z[], 24 B/point"}
    for n in (100_000, 1 << 20):
        prob = synthetic.config_scale(n)
        d = torch.from_numpy(prob["data"]).cuda().double()
        m = min(n, 65536)
        q = torch.from_numpy(prob["queries"][:m]).cuda().double()
        out = torch.empty(m, device="cuda", dtype=torch.float64)
        for p in (2.0, 3.5):
            for layout in (-1, 1, 2):
                h = idw.Handle(torch.cuda.current_device())
                idw.set_option("staging_layout", layout, handle=h)
                ms = _events_ms(lambda: idw.interpolate(d, q, p, "f64", out=out, handle=h), 2)
                h.close()
                rows.append({"n": n, "m": m, "p": p, "precision": "f64", "layout": layout,
                             "layout_name": f64_names[layout],
                             "pairs_s": float(n) * m / (ms / 1e3), "call_ms": ms})
    _emit("staging-layout ablation: same sweep (variant 0) on data tiles staged as duplicated "
          "pairs, aligned AoS or SoA; N=M, uniform [0,1)^2, wave field; then the plain FP64 "
          "form staged as Hybrid, AoaS or SoA (M = min(N, 65536))", rows)


def run_paper(args):
    """The paper's naive and tiled kernels in its layouts vs this library, at
    the paper's sizes (N = M, 1K = 1024, Sec. 4.1), p = 2."""
    import torch
    import synthetic
    import paper_1402_4986_gb300 as idw
    rows = []
    for n, fp64_too in ((10 * 1024, True), (100 * 1024, True), (1000 * 1024, False)):
        prob = synthetic.config_scale(n)
        d32 = torch.from_numpy(prob["data"]).cuda()
        q32 = torch.from_numpy(prob["queries"]).cuda()
        pairs = float(n) * n
        reps = 1 if n > 500_000 else 3
        ms = _events_ms(lambda: idw.interpolate(d32, q32, 2.0), reps)
        rows.append({"n": n, "precision": "f32", "kernel": "this library (compensated)",
                     "layout": "staged", "pairs_s": pairs / (ms / 1e3)})
        for prec, d, q, layouts in (
                ("f32", d32, q32, ("soa", "aos", "aoas")),
                ("f64", d32.double(), q32.double(), ("soa", "aos", "aoas", "hybrid"))):
            if prec == "f64" and not fp64_too:
                continue
            if prec == "f64":
                ms = _events_ms(lambda: idw.interpolate(d, q, 2.0, "f64"), 1)
                rows.append({"n": n, "precision": "f64", "kernel": "this library (plain FP64)",
                             "layout": "hybrid", "pairs_s": pairs / (ms / 1e3)})
            for kernel in ("naive", "tiled"):
                for layout in layouts:
                    pr = "f32c" if prec == "f32" else "f64"
                    ms = _events_ms(lambda: idw.paper_interpolate(d, q, 2.0, kernel=kernel,
                                                                  layout=layout, precision=pr),
                                    1 if (prec == "f64" or n > 500_000) else reps)
                    rows.append({"n": n, "precision": prec, "kernel": kernel, "layout": layout,
                                 "pairs_s": pairs / (ms / 1e3)})
    _emit("the paper's naive and tiled kernels (plain sums) in its layouts vs this library; "
          "N = M in {10K, 100K, 1000K}, 1K = 1024, uniform [0,1)^2, wave field, p = 2", rows)


def run_local(args):
    """Local (radius-limited) form: N = M = 2^20, R for K neighbours on
    average, uniform and clustered data, p in {2, 3.5}.  A one-shot call
    sorts the data and the queries into the grid and gathers; a call on a
    prepared index (built once, timed apart) sorts only the queries."""
    import torch
    import oracle
    import synthetic
    import paper_1402_4986_gb300 as idw
    rows = []
    cases = ((False, 32.0), (False, 8.0), (False, 128.0), (True, 32.0))
    if args.members:
        cases = tuple((args.data == "clustered", float(k)) for k in args.members)
    for clustered, members in cases:
        prob = synthetic.config_local(members=members, clustered=clustered)
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        n, m, R = d.shape[0], q.shape[0], prob["radius"]
        out = torch.empty(m, device="cuda")
        idx = np.random.default_rng(5).choice(m, 256, replace=False)
        for p in (2.0, 3.5):
            ms = _events_ms(lambda: idw.interpolate_local(d, q, p, R, out=out), 10, warm=3)
            _, cnt = idw.interpolate_local(d, q, p, R, counts=True)
            c = cnt.cpu().numpy()
            pairs = float(c[c > 0].sum())
            Z64, _, c64 = oracle.idw_local(prob["data"], prob["queries"][idx], p, R)
            Zs = out.cpu().numpy()[idx].astype(np.float64)
            ok = ~np.isnan(Z64)
            err = float(np.max(np.abs(Zs[ok] - Z64[ok])) / np.max(np.abs(prob["data"][:, 2])))
            rows.append({"data": "clustered" if clustered else "uniform", "call": "one-shot",
                         "n": n, "m": m,
                         "radius": R, "mean_members": pairs / m, "p": p, "ms": ms,
                         "queries_s": m / (ms / 1e3), "member_pairs_s": pairs / (ms / 1e3),
                         "empty_queries": int((c == 0).sum()),
                         "counts_match_oracle": bool(np.array_equal(c[idx], c64)),
                         "error_vs_fp64_oracle": err, "error_sample_queries": len(idx)})
        mms = _events_ms(lambda: idw.interpolate_modified(d, q, 2.0, R, out=out), 10, warm=3)
        Zm64, _, _ = oracle.idw_modified(prob["data"], prob["queries"][idx], 2.0, R)
        okm = ~np.isnan(Zm64)
        merr = float(np.max(np.abs(out.cpu().numpy()[idx][okm] - Zm64[okm]), initial=0.0) /
                     np.max(np.abs(prob["data"][:, 2])))
        rows.append({"data": "clustered" if clustered else "uniform", "call": "modified Shepard",
                     "n": n, "m": m, "radius": R, "p": 2.0, "ms": mms,
                     "queries_s": m / (mms / 1e3), "error_vs_fp64_oracle": merr,
                     "error_sample_queries": len(idx)})
        gout = torch.from_numpy(np.random.default_rng(7).standard_normal(m).astype(np.float32)).cuda()
        mbms = _events_ms(lambda: idw.local_backward(d, q, 2.0, R, gout, modified=True), 10, warm=3)
        rows.append({"data": "clustered" if clustered else "uniform",
                     "call": "modified Shepard backward", "n": n, "m": m, "radius": R, "p": 2.0,
                     "ms": mbms, "queries_s": m / (mbms / 1e3)})
        bms = _events_ms(lambda: idw.local_backward(d, q, 2.0, R, gout), 10, warm=3)
        _, _, gq, _ = idw.local_backward(d, q, 2.0, R, gout)
        sub = np.sort(idx[:128])
        Gs = oracle.idw_local_grad(prob["data"], prob["queries"][sub], 2.0, R,
                                   gout.cpu().numpy()[sub])
        gerr = float(np.max(np.abs(gq.cpu().numpy()[sub] - Gs["grad_q"])) /
                     np.max(np.abs(Gs["grad_q"])))
        rows.append({"data": "clustered" if clustered else "uniform", "call": "backward",
                     "n": n, "m": m, "radius": R, "p": 2.0, "ms": bms,
                     "queries_s": m / (bms / 1e3), "grad_q_error_vs_fp64_oracle": gerr,
                     "error_sample_queries": len(sub)})
        build_ms = _events_ms(lambda: idw.LocalIndex(d, radius=R).close(), 3, warm=1)
        ix = idw.LocalIndex(d, radius=R)
        ms = _events_ms(lambda: ix.interpolate(q, 2.0, out=out), 10, warm=3)
        _, cix = ix.interpolate(q, 2.0, counts=True)
        rows.append({"data": "clustered" if clustered else "uniform", "call": "prepared index",
                     "n": n, "m": m, "radius": R, "p": 2.0, "ms": ms,
                     "queries_s": m / (ms / 1e3), "index_build_ms": build_ms,
                     "counts_match_one_shot": bool(torch.equal(cix, cnt))})
        ix.close()
    base = synthetic.config_local(members=32.0)
    rows += _raster_order_rows(idw, torch.from_numpy(base["data"]).cuda(), "local",
                               base["radius"], "radius")
    cpu = _oracle_queries_s(
        args, lambda ix, c: oracle.idw_local(base["data"], base["queries"][ix], 2.0,
                                             base["radius"], threads=c),
        base["queries"].shape[0], "the uniform K = 32, p = 2 workload, each against all N points")
    _emit("local (radius-limited) Eq. 1: N = M = 2^20, queries uniform on [0,1)^2, "
          "R = sqrt(K / (pi N)); data uniform (wave field) or 64 Gaussian blobs (bump field); "
          "a one-shot call's time includes the grid build, a prepared index's call sorts the "
          "queries only (index_build_ms: building it, allocation included); backward = every "
          "gradient (z, data xy, query xy, p) including its grid build", rows,
          metric="local queries/s", unit="queries/s", cpu_baseline=cpu)


def run_knn(args):
    """k-nearest-neighbour form: N = M = 2^20, k in {8, 32, 64}, uniform and
    clustered data, p in {2, 3.5}.  Each call builds the grid and searches."""
    import torch
    import oracle
    import synthetic
    import paper_1402_4986_gb300 as idw
    rows = []
    ks = tuple(int(k) for k in args.members) if args.members else (8, 32, 64)
    cases = ([(args.data == "clustered", k) for k in ks] if args.members
             else [(False, k) for k in ks] + [(True, 32)])
    for clustered, k in cases:
        prob = synthetic.config_local(clustered=clustered)
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        n, m = d.shape[0], q.shape[0]
        out = torch.empty(m, device="cuda")
        idx = np.random.default_rng(6).choice(m, 128, replace=False)
        for p in (2.0, 3.5):
            ms = _events_ms(lambda: idw.interpolate_knn(d, q, p, k, out=out), 10, warm=3)
            r = oracle.idw_knn(prob["data"], prob["queries"][idx], p, k)
            _, nbr = idw.interpolate_knn(d, q, p, k, neighbours=True)
            err = float(np.max(np.abs(out.cpu().numpy()[idx] - r["Z"])) /
                        np.max(np.abs(prob["data"][:, 2])))
            rows.append({"data": "clustered" if clustered else "uniform", "call": "one-shot",
                         "n": n, "m": m, "k": k,
                         "p": p, "ms": ms, "queries_s": m / (ms / 1e3),
                         "neighbour_pairs_s": float(m) * k / (ms / 1e3),
                         "neighbours_match_oracle": bool(np.array_equal(
                             nbr.cpu().numpy()[idx], r["nbr"])),
                         "error_vs_fp64_oracle": err, "error_sample_queries": len(idx)})
        # The same call with the lanes of each warp kept in step
        # (IDW_OPT_KNN_SEARCH = 1): the same selection, another schedule.
        hs = idw.Handle(torch.cuda.current_device())
        idw.set_option("knn_search", 1, handle=hs)
        sms = _events_ms(lambda: idw.interpolate_knn(d, q, 2.0, k, out=out, handle=hs), 10, warm=3)
        _, nbs = idw.interpolate_knn(d, q, 2.0, k, neighbours=True, handle=hs)
        _, nbr2 = idw.interpolate_knn(d, q, 2.0, k, neighbours=True)
        hs.close()
        rows.append({"data": "clustered" if clustered else "uniform",
                     "call": "one-shot, lockstep search", "n": n, "m": m, "k": k, "p": 2.0,
                     "ms": sms, "queries_s": m / (sms / 1e3),
                     "vs_default_search": sms / rows[-2]["ms"],
                     "neighbours_match_default_search": bool(torch.equal(nbs, nbr2))})
        gout = torch.from_numpy(np.random.default_rng(8).standard_normal(m).astype(np.float32)).cuda()
        bms = _events_ms(lambda: idw.knn_backward(d, q, 2.0, k, gout), 10, warm=3)
        _, _, gq, _ = idw.knn_backward(d, q, 2.0, k, gout)
        Gs = oracle.idw_knn_grad(prob["data"], prob["queries"][np.sort(idx)], 2.0, k,
                                 gout.cpu().numpy()[np.sort(idx)])
        # Relative to the largest |dL/dq| (absolute where every one is 0: at
        # k = 1, Z is the nearest point's z and does not move with q).
        gscale = float(np.max(np.abs(Gs["grad_q"])))
        gerr = float(np.max(np.abs(gq.cpu().numpy()[np.sort(idx)] - Gs["grad_q"]))) / (
            gscale if gscale > 0 else 1.0)
        rows.append({"data": "clustered" if clustered else "uniform", "call": "backward",
                     "n": n, "m": m, "k": k, "p": 2.0, "ms": bms, "queries_s": m / (bms / 1e3),
                     "grad_q_error_vs_fp64_oracle": gerr, "error_sample_queries": len(idx)})
        # The deterministic mode: selections sorted by point, fixed-order sums.
        hd = idw.Handle(torch.cuda.current_device())
        idw.set_option("deterministic", 1, handle=hd)
        dms = _events_ms(lambda: idw.knn_backward(d, q, 2.0, k, gout, handle=hd), 10, warm=3)
        r1 = idw.knn_backward(d, q, 2.0, k, gout, handle=hd)
        r1 = [t.clone() for t in r1]
        r2 = idw.knn_backward(d, q, 2.0, k, gout, handle=hd)
        hd.close()
        rows.append({"data": "clustered" if clustered else "uniform",
                     "call": "backward (deterministic)", "n": n, "m": m, "k": k, "p": 2.0,
                     "ms": dms, "queries_s": m / (dms / 1e3), "vs_atomic_backward": dms / bms,
                     "bitwise_repeatable": all(bool(torch.equal(a, b)) for a, b in zip(r1, r2))})
        build_ms = _events_ms(lambda: idw.LocalIndex(d, k=k).close(), 3, warm=1)
        ix = idw.LocalIndex(d, k=k)
        ms = _events_ms(lambda: ix.knn(q, 2.0, k, out=out), 10, warm=3)
        _, nix = ix.knn(q, 2.0, k, neighbours=True)
        rows.append({"data": "clustered" if clustered else "uniform", "call": "prepared index",
                     "n": n, "m": m, "k": k, "p": 2.0, "ms": ms, "queries_s": m / (ms / 1e3),
                     "index_build_ms": build_ms,
                     "neighbours_match_one_shot": bool(torch.equal(nix, nbr))})
        ix.close()
    base = synthetic.config_local()
    rows += _raster_order_rows(idw, torch.from_numpy(base["data"]).cuda(), "knn", 32, "k")
    cpu = _oracle_queries_s(
        args, lambda ix, c: oracle.idw_knn(base["data"], base["queries"][ix], 2.0, 32, threads=c),
        base["queries"].shape[0], "the uniform k = 32, p = 2 workload, each against all N points")
    _emit("k-nearest-neighbour Eq. 1: N = M = 2^20, queries uniform on [0,1)^2; data uniform "
          "(wave field) or 64 Gaussian blobs (bump field); a one-shot call's time includes the "
          "grid build, a prepared index's call sorts the queries only (index_build_ms: building "
          "it, allocation included); backward = every gradient (z, data xy, query xy, p) "
          "including its search", rows, metric="knn queries/s", unit="queries/s",
          cpu_baseline=cpu)


def spawn_ranks(args):
    """``--gpus N`` without an external launcher: start N copies of this script
    as ranks 0..N-1 (one GPU each, NCCL rendezvous on 127.0.0.1) and wait for
    them; rank 0 prints the JSON line."""
    import socket
    import torch
    visible = torch.cuda.device_count()
    if visible < args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} needs {args.gpus} visible GPUs, found {visible}")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = []
    for r in range(args.gpus):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(args.gpus),
                   LOCAL_WORLD_SIZE=str(args.gpus), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), *sys.argv[1:]],
                                      env=env))
    rc = 0
    for pr in procs:
        rc = max(rc, pr.wait())
    sys.exit(rc)


def main():
    args = parse()
    if "WORLD_SIZE" not in os.environ and args.gpus > 1 and args.impl == "ours":
        spawn_ranks(args)
    ws, rank, local = dist_env()
    if "WORLD_SIZE" in os.environ and args.impl == "ours" and ws != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started {ws} ranks")
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.config in ("headline", "all"):
        run_ours(args, ws, rank, local)
    if rank != 0 or args.config == "headline":
        return
    import torch
    torch.cuda.set_device(local)
    from paper_1402_4986_gb300 import build as libbuild
    libbuild.build()
    for name, fn in (("scale", run_scale), ("clustered", run_clustered),
                     ("adjoint", run_adjoint), ("batched", run_batched),
                     ("layout", run_layout), ("paper", run_paper), ("local", run_local),
                     ("knn", run_knn)):
        if args.config in (name, "all"):
            fn(args)


if __name__ == "__main__":
    main()
