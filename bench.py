"""Benchmark of the Horseshoe-probit Gibbs sweep on GB300.

Workload (default): N = 1,000,000 rows, p = 1000, X iid N(0,1) stored FP32
(4 GB), 10 nonzero coefficients U[1,3] with random sign, y = 1{x beta + eps > 0},
seed 0 -- the paper's N = 1e6, p = 1000 synthetic problem (Sect. 6.1, Eq. 13)
with random sparse beta.  One step = one full Gibbs sweep (X-stream, reduce,
lambda/tau, Cholesky + inverse, beta tail, nu/xi, commit).  X (4 GB) is far
larger than L2 (129 MB), so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (rank 0 only).  Under torchrun each rank runs an
independent chain (distinct Philox chain id) on its own GPU: weak scaling,
no collective on the data path; the barrier and max-over-ranks timing use
torch.distributed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gibbs sweeps/sec at N=1e6,p=1000 (1 chain and K chains); % HBM roofline"
WORKLOADS = {
    "c1s": dict(N=200_000, p=1000, nz=10, dt="f32",
                name="horseshoe-probit sweep, N=2e5, p=1000, X iid N(0,1) fp32 (profiling case, 800 MB)"),
    "c1": dict(N=1_000_000, p=1000, nz=10, dt="f32",
               name="horseshoe-probit sweep, N=1e6, p=1000, X iid N(0,1) fp32, 10 nonzeros U[1,3], 1 chain"),
    "c0": dict(N=10_000, p=100, nz=5, dt="f64",
               name="horseshoe-probit sweep, N=1e4, p=100, X iid N(0,1) fp64, 5 nonzeros U[1,3], 1 chain"),
    "c2": dict(N=1_000_000, p=1000, nz=10, dt="bf16",
               name="horseshoe-probit sweep of K chains, N=1e6, p=1000, X iid N(0,1) bf16, 10 nonzeros U[1,3]"),
    "c2s": dict(N=200_000, p=1000, nz=10, dt="bf16",
                name="horseshoe-probit sweep of K chains, N=2e5, p=1000, X iid N(0,1) bf16 (profiling case, 400 MB)"),
    "c4": dict(N=4_000_000, p=4000, nz=20, dt="fp8", design="ar1", mag=(0.5, 2.0),
               name="horseshoe-probit sweep, N=4e6, p=4000, X rows N(0, Toeplitz 0.5^|i-j|) fp8 e4m3 with column "
                    "scales (16 GB), 20 nonzeros U[0.5,2], 1 chain"),
    "c4s": dict(N=200_000, p=4000, nz=20, dt="fp8", design="ar1", mag=(0.5, 2.0),
                name="horseshoe-probit sweep, N=2e5, p=4000, X rows N(0, Toeplitz 0.5^|i-j|) fp8 e4m3 with column "
                     "scales (profiling case, 800 MB)"),
}
UNEVEN = dict(n=64, N=(10_000, 200_000), p=(50, 2000), K=4, dt="bf16", nz_frac=0.01,
              name="uneven multi-problem batch: 64 probit problems, N log-uniform [1e4, 2e5], p log-uniform "
                   "[50, 2000], X iid N(0,1) bf16, 1% nonzeros U[1,3], 4 chains each, one graph launch per sweep")
XSTREAM_SOURCES = ["paper_1608_04329_gb300/csrc/xstream.cu", "paper_1608_04329_gb300/csrc/hs_common.cuh"]
XSTREAM_K_SOURCES = ["paper_1608_04329_gb300/csrc/xstream_k.cu", "paper_1608_04329_gb300/csrc/hs_common.cuh"]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return dist, rank, ws, local


def max_over_ranks(dist, value: float) -> float:
    """Max of a float over ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms; the samples
    whose own timestamps fall in the timed region are kept (nvidia-smi's
    output reaches the pipe in blocks, so arrival times say nothing)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []          # (arrival time, line)
        self.window = None       # (t0, t1) of the timed region, host wall clock

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts only once samples are flowing (nvidia-smi takes a moment to start)
            t_end = time.monotonic() + 3.0
            while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, start: bool):
        """Host wall-clock time of the start (start=True) or end of the timed region."""
        now = time.time()
        self.window = (now, None) if start else (self.window[0] if self.window else now, now)

    @staticmethod
    def _stamp(field: str):
        import datetime
        try:
            return datetime.datetime.strptime(field.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for _, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 10:
                rows.append((self._stamp(f[0]), f[1:]))
        if self.window and self.window[1] is not None:
            # samples stamped inside the timed region (one sampling period of slack on each side)
            t0, t1 = self.window
            inside = [r for ts, r in rows if ts is not None and t0 - 0.02 <= ts <= t1 + 0.02]
            if not inside:  # none in a region shorter than the period: the nearest after its start
                later = sorted((ts, r) for ts, r in rows if ts is not None and ts >= t0)
                inside = [later[0][1]] if later else []
        else:
            inside = [r for _, r in rows]
        for f in inside:
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _alu_peak(torch, local):
    """FP32-pair FMAs per second the CUDA cores can issue: SMs x 128 FP32 lanes x
    max SM clock / 12 FP32 instructions per pair-FMA."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "measured"
    except (OSError, KeyError, ValueError):
        mhz, src = 2070.0, "nominal"
    return sms * 128 * mhz * 1e6 / 12.0, f"SMs x 128 FP32 lanes x {src} max SM clock / 12 FP32 instructions per pair-FMA"


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1e12, "measured"
    except (OSError, KeyError, ValueError):
        return 1.9e15, "fallback"


def factor_work(p: int, tensor: bool = True):
    """Algorithmic work of one chain's factorization of the p x p precision
    matrix (P = 32 ceil(p / 32) padded rows, which are skipped).  Block-column
    form (blocks of 128 columns): the CUDA cores do the updates inside each
    block column in FP32 pairs; the tensor cores apply the rank-128 updates of
    the rest as 21 BF16 digit-pair products per multiply-add.  Returns
    (CUDA-core pair-FMAs, tensor-core flops)."""
    if not tensor:
        return p ** 3 / 6.0, 0.0
    alu, mac = 0.0, 0.0
    for c0 in range(0, p, 128):
        c1 = min(c0 + 128, p)
        for j in range(c0, c1):
            alu += (p - j) * (j - c0)          # column j's updates from the block's earlier columns
        r = p - c1
        mac += r * (r + 1) / 2.0 * (c1 - c0)   # trailing lower triangle, rank c1 - c0
    return alu, 2.0 * 21.0 * mac


def _traffic(workload: str, record: str = "xstream_traffic.json", sources=XSTREAM_SOURCES):
    """DRAM bytes per X-stream launch from the committed ncu summary, or None
    when the kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", record)
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("sources_sha256") != sources_sha256(sources) or rec.get("workload") != workload:
        return None
    return rec.get("dram_bytes_per_launch")


# DRAM-traffic records of the X-stream kernels (profiles/*_traffic.json):
# captured at the profiling size, scaled by rows to the full workload.
TRAFFIC_RECORDS = {
    "c1s": dict(record="xstream_traffic.json", sources=XSTREAM_SOURCES, kernel_regex="xstream_kernel",
                full="c1", row_bytes=lambda p: 4 * p + 1),
    "c2s": dict(record="xstream_k_traffic.json", sources=XSTREAM_K_SOURCES, kernel_regex="xstream_k_kernel",
                full="c2", row_bytes=lambda p: 2 * p + 1),
}


def sources_sha256(sources) -> str:
    h = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _ncu_bytes(value: str, unit: str) -> float:
    scale = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12}[unit.strip().lower()]
    return float(value.replace(",", "")) * scale


def write_traffic_record(csv_path: str, workload: str, command: str) -> dict:
    """Turn an ncu CSV (dram__bytes_read.sum and dram__bytes_write.sum of the
    X-stream kernel at the profiling size) into the committed traffic record:
    bytes of the last captured launch, scaled by rows to the full workload,
    tagged with the hash of the kernel's sources."""
    import csv
    import re
    spec = TRAFFIC_RECORDS[workload]
    wl, full = WORKLOADS[workload], WORKLOADS[spec["full"]]
    launches = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if r]
    head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[head]
    ik, im, iu, iv, iid = (cols.index("Kernel Name"), cols.index("Metric Name"), cols.index("Metric Unit"),
                           cols.index("Metric Value"), cols.index("ID"))
    for r in rows[head + 1:]:
        if len(r) <= iv or not re.search(spec["kernel_regex"], r[ik]):
            continue
        if r[im] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            launches.setdefault(int(r[iid]), {})[r[im]] = _ncu_bytes(r[iv], r[iu])
    if not launches:
        raise SystemExit(f"no launch of {spec['kernel_regex']} with DRAM counters in {csv_path}")
    last = launches[max(launches)]
    rd, wr = last["dram__bytes_read.sum"], last["dram__bytes_write.sum"]
    scale = full["N"] / wl["N"]
    rec = {"kernel": spec["kernel_regex"], "workload": spec["full"],
           "dram_bytes_per_launch": int(round((rd + wr) * scale)),
           "captured_on": f"N={wl['N']}, p={wl['p']} {wl['dt']} (X larger than L2); scaled by rows to N={full['N']}",
           "captured_read_bytes": rd, "captured_write_bytes": wr,
           "algorithmic_bytes_per_launch": full["N"] * spec["row_bytes"](full["p"]),
           "sources": spec["sources"], "sources_sha256": sources_sha256(spec["sources"]), "command": command}
    rec["traffic_over_algorithmic"] = rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"]
    with open(os.path.join(ROOT, "profiles", spec["record"]), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def make_data(wl):
    import hs_synth
    return hs_synth.make_problem(wl["N"], wl["p"], wl["nz"], wl["dt"], seed=0, design=wl.get("design", "iid"),
                                 mag=wl.get("mag", (1.0, 3.0)))


def run_config(wl, args, ws, x_nbytes):
    """The ``config`` object of the bench line (the same for both arms)."""
    return {"workload": wl["name"], "N": wl["N"], "p": wl["p"], "x_dtype": wl["dt"],
            "chains_per_gpu": 1, "cholesky": args.chol, "graph": bool(args.graph),
            "l2": f"inputs larger than L2 (X {x_nbytes / 1e9:.1f} GB), no flush",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def cpu_oracle_rate(d, wl, n_sweeps: int, budget_s: float = 30.0, warmup: int = 1):
    """Oracle sweeps/s on the host (full workload, first n_sweeps sweeps after
    ``warmup`` untimed ones)."""
    import oracle
    X = oracle.fmt.stored_to_f64(d["X"], d["x_dtype"], d["scales"])
    t0 = time.perf_counter()
    G = oracle.gram(X)
    t_gram = time.perf_counter() - t0
    st = oracle.init_state(wl["p"])
    for _ in range(max(warmup, 1)):
        st = oracle.sweep_once(st, X, d["y"], G, 0)  # warm-up
    done, t = 0, 0.0
    while done < n_sweeps and t < budget_s:
        t1 = time.perf_counter()
        st = oracle.sweep_once(st, X, d["y"], G, 0)
        t += time.perf_counter() - t1
        done += 1
    return done / t, done, t, t_gram


def run_reference(args, wl, dist, rank):
    if rank != 0:
        return 0
    d = make_data(wl)
    n = args.steps
    rate, done, t, t_gram = cpu_oracle_rate(d, wl, n_sweeps=n, budget_s=args.ref_budget, warmup=args.warmup)
    cores = os.cpu_count()
    sample = (f"{done} oracle sweeps of the full workload (of {n} requested; capped at "
              f"{args.ref_budget:.0f} s), after an untimed Gram ({t_gram:.1f} s) and {args.warmup} warm-up sweeps")
    line = {"metric": METRIC, "value": rate, "unit": "sweeps/s", "n_gpus": 0, "steps": done,
            "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(wl, args, 1, d["X"].nbytes),
            "impl": "reference",
            "cpu_baseline": {"value": rate, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_k_chains(args, wk, pkg, torch, dist, ws, rank, local, chol, one_chain_value, dk=None, K=None):
    """K chains on one X: chain-sweeps/s, the X-stream roofline and the
    factorization's floors.  BF16 X takes the tensor-core X-stream (one pass
    for every chain); other types one pass per chain."""
    peak, peak_kind = _peaks()
    K = K or args.k_chains
    if dk is None:
        dk = make_data(wk)
    sk = pkg.HSProbit(dk["X"], dk["y"], seed=0, chain=32 * rank, device=local, use_graph=bool(args.graph),
                      chol_arith=chol, num_chains=K, ring_size=max(args.k_steps + 3, 16), scales=dk["scales"])
    shape = sk.launch_shape()
    streamk = torch.cuda.ExternalStream(sk.stream(), device=local)
    sk.sweep(3)
    sk.set_profiling(bool(args.profile))
    barrier(dist)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.mark(True)
        k0.record(streamk)
        sk.sweep(args.k_steps)
        k1.record(streamk)
        torch.cuda.synchronize()
        clk.mark(False)
    barrier(dist)
    kms = max_over_ranks(dist, k0.elapsed_time(k1))
    kgroups = {g: sk.kernel_time(g) for g in ("xstream", "reduce", "shrink", "cholesky", "tail")}
    klaunches = sk.launches_per_sweep()
    sk.set_profiling(False)
    sk.close()
    kx_ms, kx_n = kgroups["xstream"]
    eb = {"f64": 8, "f32": 4, "bf16": 2, "fp8": 1}[wk["dt"]]
    tensor_xs = shape["xk_chains"] > 0
    # algorithmic bytes: X once for all chains on the tensor cores, else once per chain
    kbytes = (1 if tensor_xs else K) * wk["N"] * (wk["p"] * eb + 1)
    kroof = None
    if kx_n > 0:
        kavg = kx_ms / kx_n
        kach = kbytes / (kavg / 1e3) / 1e9
        if tensor_xs:
            rec = _traffic("c2" if wk["N"] == WORKLOADS["c2"]["N"] else "c2s", "xstream_k_traffic.json",
                           XSTREAM_K_SOURCES)
            kern = f"xstream_k<{shape['xk_chains']}, {shape['xk_stages']}> (B prep + tensor-core X-stream)"
        else:
            rec = _traffic(args.workload) if wk is WORKLOADS.get(args.workload) else None
            rec = K * rec if rec else None
            kern = f"xstream ({K} one-chain passes)"
        kroof = {"bound": "hbm", "achieved": kach, "peak": peak, "unit": "GB/s", "frac": kach / peak,
                 "traffic": rec, "peak_source": peak_kind, "kernel": kern, "avg_launch_ms": kavg}
        if tensor_xs:
            kc = shape["xk_chains"]
            fpad = (wk["p"] + 127) // 128 * 128
            kroof["tensor_tflops"] = 4.0 * wk["N"] * fpad * 2 * kc / (kavg / 1e3) / 1e12
    # the K factorizations: block columns of FP32-pair panel work on the CUDA
    # cores and rank-128 digit products on the tensor cores, chained block
    # column after block column; the floors are each unit's share at its peak
    kc_ms, kc_n = kgroups["cholesky"]
    kchol = None
    if kc_n > 0:
        alu_peak, alu_src = _alu_peak(torch, local)
        tc_peak, tc_src = _bf16_peak()
        alu, tflop = factor_work(wk["p"])
        cavg = kc_ms / kc_n
        t_alu = K * alu / alu_peak * 1e3
        t_tc = K * tflop / tc_peak * 1e3
        kchol = {"bound": "latency", "achieved_ms": cavg, "alu_floor_ms": t_alu, "tensor_floor_ms": t_tc,
                 "frac": max(t_alu, t_tc) / cavg, "traffic": None,
                 "kernel": "chol_persistent_kernel + chol_trail_kernel per block column (K chains, factor only)",
                 "work": {"cuda_core_pair_fma": K * alu, "tensor_flop": K * tflop,
                          "all_pair_fma_equivalent": K * wk["p"] ** 3 / 6.0},
                 "alu_peak_pair_fma_s": alu_peak, "alu_peak_source": alu_src,
                 "tensor_peak_flop_s": tc_peak, "tensor_peak_source": f"{tc_src} cuBLAS bf16",
                 "note": "the block columns run one after another (each waits for its diagonal chain), "
                         "so the sum of the floors is not reachable; frac = the larger floor / achieved"}
    kvalue = ws * K * args.k_steps / (kms / 1e3)
    return {"value": kvalue, "unit": "chain-sweeps/s", "K": K, "x_dtype": wk["dt"], "launch_shape": shape,
            "steps": args.k_steps, "warmup": 3, "ms_per_sweep": kms / args.k_steps,
            "vs_one_chain_fp32": (kvalue / one_chain_value) if one_chain_value else None,
            "kernel_ms_per_sweep": {g: (v[0] / max(v[1], 1)) for g, v in kgroups.items()},
            "gpu_launches_per_sweep": klaunches, "roofline": kroof, "factorization_roofline": kchol,
            "clocks": clk.summary(),
            "workload": wk["name"]}


def run_uneven_batch(args, pkg, torch, dist, ws, rank, local, chol):
    """Many problems of uneven N and p, K chains each, swept by one graph per
    sweep after the batch tuner has picked the launch shapes."""
    import hs_synth
    u = UNEVEN
    peak, peak_kind = _peaks()
    t_gen = time.perf_counter()
    sizes = hs_synth.uneven_sizes(u["n"], u["N"], u["p"], seed=0)
    ds = [hs_synth.make_problem(N, p, max(1, round(u["nz_frac"] * p)), u["dt"], seed=1000 + m)
          for m, (N, p) in enumerate(sizes)]
    t_gen = time.perf_counter() - t_gen
    x_bytes = sum(d["X"].nbytes for d in ds)
    y_bytes = sum(d["y"].nbytes for d in ds)
    root = torch.cuda.Stream(device=local)
    t0 = time.perf_counter()
    b = pkg.HSProbitBatch([(d["X"], d["y"]) for d in ds], seed=0, num_chains=u["K"], chol_arith=chol,
                          problem=u["n"] * rank, device=local, stream=root.cuda_stream,
                          ring_size=max(args.c3_steps + 8, 16))
    t_init = time.perf_counter() - t0
    b.sweep(3)  # warm-up
    t0 = time.perf_counter()
    best = b.tune(3)
    t_tune = time.perf_counter() - t0
    trials = b.tune_trials()
    shapes = [b.problem(m).launch_shape() for m in range(len(ds))]
    b.sweep(3)  # warm-up of the tuned graph
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees these sweeps only
    with ClockSampler(local) as clk:
        clk.mark(True)
        e0.record(root)
        b.sweep(args.c3_steps)
        e1.record(root)
        torch.cuda.synchronize()
        clk.mark(False)
    torch.cuda.profiler.stop()
    barrier(dist)
    ms = max_over_ranks(dist, e0.elapsed_time(e1))
    ms_sweep = ms / args.c3_steps
    # e2e through the public API: per step one batch sweep and every chain's newest draw read back
    for m in range(len(ds)):
        for c in range(u["K"]):
            b.problem(m).draws(chain=c)  # read what the timed sweeps left, before the clock starts
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(max(1, args.c3_steps // 5)):
        b.sweep(1)
        for m in range(len(ds)):
            for c in range(u["K"]):
                dr = b.problem(m).draws(chain=c)
                d2h += sum(v.nbytes for v in dr.values())
    n_e2e = max(1, args.c3_steps // 5)
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0)
    launches = sum(b.problem(m).launches_per_sweep() for m in range(len(ds)))
    b.close()
    sweeps_s = ws * args.c3_steps / (ms / 1e3)
    # floors of a sweep: X read once (HBM); the K factorizations' panel work on
    # the CUDA cores and trailing digit products on the tensor cores
    t_hbm = (x_bytes + y_bytes) / (peak * 1e9) * 1e3
    alu_peak, alu_src = _alu_peak(torch, local)
    tc_peak, tc_src = _bf16_peak()
    work = [factor_work(p) for _, p in sizes]
    pair_fmas = u["K"] * sum(a for a, _ in work)
    tflop = u["K"] * sum(t for _, t in work)
    t_alu = pair_fmas / alu_peak * 1e3
    t_tc = tflop / tc_peak * 1e3
    bound = max(t_hbm, t_alu, t_tc)
    return {"value": sweeps_s * u["n"] * u["K"], "unit": "chain-sweeps/s", "batch_sweeps_per_s": sweeps_s,
            "problems": u["n"], "K": u["K"], "steps": args.c3_steps, "warmup": 6, "ms_per_sweep": ms_sweep,
            "workload": u["name"],
            "realised": {"sum_x_bytes": x_bytes, "sum_4p3_over_3_flop": sum(4.0 * p ** 3 / 3.0 for _, p in sizes),
                         "sum_K_p3_over_6": u["K"] * sum(float(p) ** 3 / 6.0 for _, p in sizes), "N_min_max": [min(n for n, _ in sizes),
                                                                                max(n for n, _ in sizes)],
                         "p_min_max": [min(p for _, p in sizes), max(p for _, p in sizes)]},
            "roofline": {"bound": ("hbm", "alu", "tensor")[[t_hbm, t_alu, t_tc].index(bound)],
                         "achieved_ms": ms_sweep, "bound_ms": bound, "frac": bound / ms_sweep, "hbm_ms": t_hbm,
                         "alu_ms": t_alu, "tensor_ms": t_tc, "hbm_peak_gbs": peak, "peak_source": peak_kind,
                         "cuda_core_pair_fma": pair_fmas, "tensor_flop": tflop, "alu_peak": alu_src,
                         "tensor_peak": f"{tc_src} cuBLAS bf16 {tc_peak / 1e12:.0f} TFLOP/s",
                         "note": "floors of the three units; each problem's block columns run one after "
                                 "another, so latency, not any floor, is what the sweep meets",
                         # context: the same factorizations as native FP64 Cholesky (sum K p^3 / 3 FMAs)
                         # on GB300's FP64 pipe at its nominal 1.25 TFLOP/s
                         "fp64_pipe_ms": sum(u["K"] * 2.0 * float(p) ** 3 / 3.0 for _, p in sizes) / 1.25e12 * 1e3},
            "tuner": {"best_ms_per_sweep": best, "trials": trials, "tune_s": t_tune,
                      "xk_chains": sorted({sh["xk_chains"] for sh in shapes}),
                      "xk_stages": sorted({sh["xk_stages"] for sh in shapes})},
            "e2e": {"value": ws * n_e2e * u["n"] * u["K"] / t_e2e, "unit": "chain-sweeps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(d2h / n_e2e),
                    "includes": "per step one batch sweep and the D2H of every chain's newest draw; inputs were "
                                f"copied from host once at init ({t_init:.1f} s, {(x_bytes + y_bytes) / 1e9:.2f} GB)"},
            "gpu_launches_per_sweep": launches, "init_s": t_init, "gen_s": t_gen, "clocks": clk.summary()}


def run_c3_line(args, dist, rank, ws, local):
    """``--workload c3``: the uneven batch alone, as its own bench line (our
    arm), or the oracle on a bounded sample of its problems (reference arm)."""
    import hs_synth
    u = UNEVEN
    metric = "chain-sweeps/s of the uneven 64-problem batch (K = 4 each)"
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        sizes = hs_synth.uneven_sizes(u["n"], u["N"], u["p"], seed=0)
        done, t, used = 0, 0.0, 0
        for m, (N, p) in enumerate(sizes):
            if t >= args.ref_budget:
                break
            d = hs_synth.make_problem(N, p, max(1, round(u["nz_frac"] * p)), u["dt"], seed=1000 + m)
            X = oracle.fmt.stored_to_f64(d["X"], d["x_dtype"], d["scales"])
            G = oracle.gram(X)  # untimed, as the library's init
            for c in range(u["K"]):
                st = oracle.init_state(p)
                t0 = time.perf_counter()
                oracle.sweep_once(st, X, d["y"], G, 0, chain=c, problem=m)
                t += time.perf_counter() - t0
                done += 1
            used += 1
        rate = done / t
        line = {"metric": metric, "value": rate, "unit": "chain-sweeps/s", "n_gpus": 0, "steps": done,
                "warmup": 0, "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": u["name"]}, "impl": "reference",
                "cpu_baseline": {"value": rate, "unit": "chain-sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"one FP64 oracle sweep of each of the {u['K']} chains of the first "
                                           f"{used} problems (Gram untimed), within {args.ref_budget:.0f} s"},
                "e2e": {"value": rate, "unit": "chain-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import torch
    import paper_1608_04329_gb300 as pkg
    pkg.load_library()
    torch.cuda.set_device(local)
    chol = pkg.CHOL_F64 if args.chol == "f64" else pkg.CHOL_DF32
    c3 = run_uneven_batch(args, pkg, torch, dist, ws, rank, local, chol)
    if rank == 0:
        line = {"metric": metric, "value": c3["value"], "unit": c3["unit"], "n_gpus": ws, "steps": c3["steps"],
                "warmup": c3["warmup"], "ms_per_step": c3["ms_per_sweep"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": c3["workload"], "l2": "inputs larger than L2 (2.9 GB of X), no flush"},
                "roofline": c3["roofline"], "e2e": c3["e2e"], "gpu_launches": c3["gpu_launches_per_sweep"] * c3["steps"],
                "clocks": c3["clocks"], "uneven_batch": c3}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_tn_compare(d, pkg, torch, local, reps=20):
    """The latent draw alone, both samplers, on this workload's mu* = y* x_i beta_true
    (N draws): time per launch (CUDA events), proposals per draw, and how long a
    warp runs for its slowest lane (mean over warps of the max attempts / mean)."""
    X = torch.from_numpy(d["X"]).to(f"cuda:{local}")
    bt = torch.from_numpy(d["beta_true"]).to(device=X.device, dtype=X.dtype)
    ys = torch.from_numpy(d["y"]).to(X.device).to(X.dtype) * 2.0 - 1.0
    mu = (ys * (X @ bt)).float().contiguous()
    del X
    out = {"workload": "mu* = y* x_i beta_true of the benchmark data (N draws), FP32, one thread per draw"}
    for name, meth in (("inverse_cdf", pkg.TN_INVCDF), ("rejection", pkg.TN_REJECTION)):
        for _ in range(3):
            z, t = pkg.tn_sample(mu, seed=0, sweep=1, method=meth)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            z, t = pkg.tn_sample(mu, seed=0, sweep=1 + r, method=meth)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tt = t.double()
        n = tt.numel() // 32 * 32
        warp_max = tt[:n].view(-1, 32).max(dim=1).values.mean().item()
        out[name] = {"ms_per_launch": ms, "draws_per_s": mu.numel() / (ms / 1e3), "mean_attempts": tt.mean().item(),
                     "warp_wait_factor": warp_max / tt[:n].mean().item()}
    out["rejection_over_inverse_cdf_time"] = out["rejection"]["ms_per_launch"] / out["inverse_cdf"]["ms_per_launch"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS) + ["c3"],
                    help="c3: the uneven multi-problem batch alone")
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--chol", default="df32", choices=["f64", "df32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=3)
    ap.add_argument("--profile", type=int, default=1,
                    help="1: CUDA events around each kernel group in the timed region (eager launches)")
    ap.add_argument("--ref-budget", type=float, default=120.0)
    ap.add_argument("--k-chains", type=int, default=32,
                    help="also time the batched form: K chains on BF16 X (0: skip)")
    ap.add_argument("--k-steps", type=int, default=20)
    ap.add_argument("--no-tn", action="store_true", help="skip the standalone sampler comparison")
    ap.add_argument("--no-c3", action="store_true", help="skip the uneven multi-problem batch")
    ap.add_argument("--c4-chains", type=int, default=8, help="chains of the large correlated workload's K-chain leg")
    ap.add_argument("--c3-steps", type=int, default=50, help="timed sweeps of the uneven batch")
    ap.add_argument("--traffic-from", default=None, metavar="CSV",
                    help="write profiles/<kernel>_traffic.json from an ncu CSV of --workload c1s or c2s and exit")
    ap.add_argument("--traffic-command", default="", help="the ncu command that made the CSV (recorded)")
    args = ap.parse_args(argv)
    if args.traffic_from:
        print(json.dumps(write_traffic_record(args.traffic_from, args.workload, args.traffic_command)))
        return 0
    dist, rank, ws, local = _dist()
    if args.workload == "c3":
        return run_c3_line(args, dist, rank, ws, local)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        rc = run_reference(args, wl, dist, rank)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    import torch
    import paper_1608_04329_gb300 as pkg
    pkg.load_library()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    torch.cuda.set_device(local)
    chol = pkg.CHOL_F64 if args.chol == "f64" else pkg.CHOL_DF32
    if wl["dt"] == "bf16":
        # the batched form alone (profiling and K-chain runs)
        kch = run_k_chains(args, wl, pkg, torch, dist, ws, rank, local, chol, None)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": kch["value"], "unit": kch["unit"], "n_gpus": ws,
                              "steps": args.k_steps, "warmup": 3, "ms_per_step": kch["ms_per_sweep"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                              "data": "synthetic", "config": {"workload": wl["name"], "K": args.k_chains},
                              "k_chains": kch}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0
    d = make_data(wl)
    s = pkg.HSProbit(d["X"], d["y"], seed=0, chain=rank, device=local, use_graph=bool(args.graph), scales=d["scales"],
                     chol_arith=chol, ring_size=max(args.steps + args.warmup, 16))
    stream = torch.cuda.ExternalStream(s.stream(), device=local)
    s.sweep(args.warmup)

    # ---- device-timed region: K sweeps, inputs resident in HBM ----
    s.set_profiling(bool(args.profile))
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.mark(True)
        e0.record(stream)
        s.sweep(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark(False)
    barrier(dist)
    ms_local = e0.elapsed_time(e1)
    ms = max_over_ranks(dist, ms_local)
    value = ws * args.steps / (ms / 1e3)
    xs_ms, xs_n = s.kernel_time("xstream")
    groups = {g: s.kernel_time(g) for g in ("xstream", "reduce", "shrink", "cholesky", "tail")}
    launches = s.launches_per_sweep() * args.steps
    s.set_profiling(False)
    s.close()

    # ---- roofline of the X-stream kernel ----
    bytes_per_launch = wl["N"] * (wl["p"] * {"f64": 8, "f32": 4, "bf16": 2, "fp8": 1}[wl["dt"]] + 1)
    peak, peak_kind = _peaks()
    if xs_n > 0:
        avg_ms = xs_ms / xs_n
        achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": _traffic(args.workload), "peak_source": peak_kind,
                    "kernel": "xstream", "avg_launch_ms": avg_ms}
    else:
        roofline = None

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        Xp = torch.from_numpy(d["X"]).pin_memory()
        yp = torch.from_numpy(d["y"]).pin_memory()
        Xh, yh = Xp.numpy(), yp.numpy()
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = pkg.HSProbit(Xh, yh, seed=1, chain=rank, device=local, use_graph=bool(args.graph), chol_arith=chol,
                          scales=d["scales"])
        t_init = time.perf_counter() - t0
        d2h = 0
        for _ in range(args.steps):
            s2.sweep(1)
            dr = s2.draws()
            d2h += sum(v.nbytes for v in dr.values())
        s2.close()
        t_e2e = max_over_ranks(dist, time.perf_counter() - t0)
        e2e = {"value": ws * args.steps / t_e2e, "unit": "sweeps/s",
               "h2d_bytes_per_step": int((d["X"].nbytes + d["y"].nbytes) / args.steps),
               "d2h_bytes_per_step": int(d2h / args.steps), "init_s": t_init,
               "includes": "init from pinned host X and y (H2D copy + Gram on the tensor cores) amortised over the steps, "
                           "then per step one sweep and the D2H of its draw (beta, lambda^-2, tau^-2)"}

    # ---- K chains on BF16 X (tensor-core X-stream), same N and p ----
    kch = None
    if args.workload in ("c4", "c4s") and args.c4_chains > 1:
        # the large correlated workload's own K chains on its FP8 X
        kch = run_k_chains(args, wl, pkg, torch, dist, ws, rank, local, chol, value, dk=d, K=args.c4_chains)
    elif args.k_chains > 1:
        kch = run_k_chains(args, WORKLOADS["c2"], pkg, torch, dist, ws, rank, local, chol, value)

    c3 = None
    if not args.no_c3 and wl is WORKLOADS["c1"]:
        c3 = run_uneven_batch(args, pkg, torch, dist, ws, rank, local, chol)

    tnc = None
    if rank == 0 and not args.no_tn and wl["dt"] in ("f32", "f64"):
        tnc = run_tn_compare(d, pkg, torch, local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, done, t, t_gram = cpu_oracle_rate(d, wl, n_sweeps=args.cpu_sweeps)
        cpu = {"value": rate, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} FP64 oracle sweeps of the full workload after one warm-up sweep "
                         f"(Gram {t_gram:.1f} s untimed), numpy/scipy with all host cores"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if wl["dt"] != "f64" else "f64",
                "data": "synthetic",
                "config": run_config(wl, args, ws, d["X"].nbytes),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "kernel_ms_per_sweep": {g: (v[0] / max(v[1], 1)) for g, v in groups.items()},
                "hbm_roofline_frac_whole_sweep": (bytes_per_launch / (ms / args.steps / 1e3) / 1e9) / 8000.0,
                "k_chains": kch, "uneven_batch": c3, "tn_samplers": tnc}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
