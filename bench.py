"""Benchmark of the sparse Tucker (HOOI) hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload skew-20M]

A step is one HOOI sweep (Algorithm 2): TTMc + QRP for every mode, then the core
tensor and the fit, on a seeded synthetic tensor resident in HBM.  The metric is
nonzeros processed per second per mode: value = N_modes * nnz / (time of one sweep),
whole job over all ranks.  Each rank runs an independent replica (weak scaling;
the method has no exchange step between independent decompositions).

Besides the JSON line's required keys it reports the per-phase split of a sweep,
TTMc nonzeros/s per mode, the roofline of the dominant kernel, the BF16-factor form,
the one-off initialisation, the end-to-end rate through the C ABI from pinned host
buffers, and the FP64 oracle timed on the host cores on a bounded sample.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sparse TTMc nonzeros/sec per mode and HOOI iteration time (s), % of HBM roofline"
UNIT = "nonzeros/s per mode (N_modes * nnz / HOOI sweep time)"
FP64_PEAK_TFLOPS_NOMINAL = 1.25
L2_BYTES = 129 * 1024 * 1024


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def file_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on the current source."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2010_10638_gb300", "csrc", vals.get("source", "ttmc.cu"))
    if "source_sha" not in vals or not os.path.exists(src) or file_sha(src) != vals["source_sha"]:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_model():
    """The host CPU's model name (x86 'model name', or the Arm implementer/part codes)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model", "Hardware"):
        for line in info.splitlines():
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = sorted({line.split(":", 1)[1].strip() for line in info.splitlines() if line.startswith("CPU part")})
    impl = sorted({line.split(":", 1)[1].strip() for line in info.splitlines() if line.startswith("CPU implementer")})
    return f"Arm implementer {','.join(impl)} part {','.join(parts)}" if parts else "unknown"


def oracle_coalesced(inst, sample_nnz=None):
    """The workload's listed entries (the first `sample_nnz`, or all), coalesced by the oracle."""
    import oracle
    n = inst.workload.nnz if sample_nnz is None else min(sample_nnz, inst.workload.nnz)
    coords = np.ascontiguousarray(inst.coords[:, :n])
    return oracle.coalesce(coords, inst.vals[:n].astype(np.float64))


def oracle_sweep(inst, cc, cv, threads=1):
    """Seconds of one oracle HOOI sweep (TTMc + QRP per mode, core, fit) on coalesced entries."""
    import oracle
    w = inst.workload
    t0 = time.perf_counter()
    oracle.hooi(w.dims, w.ranks, cc, cv, inst.U0, 1, coalesced=True, threads=threads)
    return time.perf_counter() - t0


def oracle_sample(inst, sample_nnz, threads=1):
    """The oracle on a bounded sample: one HOOI sweep over the first `sample_nnz` listed
    entries of the same workload (same dims, ranks, initial factors).  Returns (seconds, nnz)."""
    cc, cv = oracle_coalesced(inst, sample_nnz)
    return oracle_sweep(inst, cc, cv, threads), cc.shape[1]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over all ranks of the default process group (identity
    without one).  Runs on NCCL with a CUDA device, or on gloo with the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def time_ttmc_modes(T, torch, ctx, dims, dev, stream, flush, reps=10):
    """Median CUDA-event duration of ttmc_mode for every mode (L2 flushed before each)."""
    out = []
    for n in range(len(dims)):
        Y = torch.empty((dims[n], ctx.P(n)), dtype=torch.float32, device=dev)
        T.ttmc_mode(ctx, n, Y, stream=stream)
        evs = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            T.ttmc_mode(ctx, n, Y, stream=stream)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        out.append(statistics.median(a.elapsed_time(b) for a, b in evs))
        del Y
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    import oracle
    from paper_2010_10638_gb300 import synth
    oracle.build()
    inst = synth.make(args.workload)
    w = inst.workload
    N = len(w.dims)
    steps = max(1, min(args.steps, 5))
    warm = min(args.warmup, 1)
    threads = os.cpu_count() or 1
    cc, cv = oracle_coalesced(inst, None if args.oracle_full else args.oracle_nnz)
    nz = cc.shape[1]
    for _ in range(warm):
        oracle_sweep(inst, cc, cv, threads)
    times = [oracle_sweep(inst, cc, cv, threads) for _ in range(steps)]
    tstep = sum(times) / len(times)
    value = N * nz / tstep
    desc = (f"one oracle HOOI sweep (C, FP64, {threads} threads split by output column, results equal to the "
            f"serial oracle bit for bit) over {'all' if args.oracle_full else f'the first {args.oracle_nnz:,} listed'} "
            f"entries of {w.name} ({nz:,} after coalescing), same dims/ranks/initial factors; {steps} timed of "
            f"{args.steps} requested steps; CPU: {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": tstep * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "ranks": list(w.ranks)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_mine(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2010_10638_gb300 import build as libbuild
    from paper_2010_10638_gb300 import synth, tucker as T
    if rank == 0 or world == 1:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    T.load()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T.tucker_lib_setup(local)  # once per process: memory pool, first allocation, init kernels loaded
    lib_setup_s = time.perf_counter() - t0

    inst = synth.make(args.workload)
    w = inst.workload
    N, Z = len(w.dims), w.nnz
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        coords_d = torch.as_tensor(inst.coords.astype(np.int32)).to(dev)
        vals_d = torch.as_tensor(inst.vals).to(dev)
        U0_d = [torch.as_tensor(u).to(dev) for u in inst.U0]
        torch.cuda.synchronize()
        # one-off initialisation (a1), timed separately
        t0 = time.perf_counter()
        ctx = T.tucker_init(w.dims, coords_d, vals_d, w.ranks, U0_d, fit_device=True, stream=stream)
        torch.cuda.synchronize()
        init_s = time.perf_counter() - t0
        Zc = T.tucker_nnz(ctx)
        fit_buf = torch.zeros(1, dtype=torch.float64, device=dev)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

        # the timed step: one sweep replayed from a CUDA graph of the whole iteration (the
        # first call runs one sweep eagerly and captures the next)
        for _ in range(args.warmup):
            T.tucker_hooi_graph(ctx, 1, fit_buf, stream=stream)
        torch.cuda.synchronize()

        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        launches0 = T.tucker_kernel_launches()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
                starts[i].record(stream)
                T.tucker_hooi_graph(ctx, 1, fit_buf, stream=stream)
                ends[i].record(stream)
            torch.cuda.synchronize()
        launches = T.tucker_kernel_launches() - launches0
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms_per_step = sum(step_ms) / len(step_ms)
        fit = float(fit_buf.item())

        # max over ranks
        ms_per_step = max_over_ranks(ms_per_step, dev)

        # the same sweep launched kernel by kernel (hooi_iter), for comparison
        eager = []
        for i in range(20):
            flush.fill_(float(i))
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            T.hooi_iter(ctx, fit_buf, stream=stream)
            b_.record(stream)
            eager.append((a_, b_))
        torch.cuda.synchronize()
        eager_ms = statistics.median(a_.elapsed_time(b_) for a_, b_ in eager)

        # per-phase split of a sweep (profiling pass, events inside the library)
        T.tucker_set_profiling(ctx, True)
        phase = []
        for _ in range(5):
            flush.fill_(0.0)
            T.hooi_iter(ctx, fit_buf, stream=stream)
            phase.append(T.tucker_phase_times(ctx))
        T.tucker_set_profiling(ctx, False)
        phase_ms = [statistics.median(p[i] for p in phase) for i in range(2 * N + 1)]

        # TTMc alone, per mode: launch durations with events on the launching stream
        ttmc_ms = time_ttmc_modes(T, torch, ctx, w.dims, dev, stream, flush)

        # BF16-factor form on the same workload
        bf16 = None
        if not args.no_bf16:
            ctxb = T.tucker_init(w.dims, coords_d, vals_d, w.ranks, U0_d, bf16=True, fit_device=True, stream=stream)
            bms = time_ttmc_modes(T, torch, ctxb, w.dims, dev, stream, flush)
            for _ in range(2):
                T.hooi_iter(ctxb, fit_buf, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                T.hooi_iter(ctxb, fit_buf, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            sweep_b = e0.elapsed_time(e1) / 5
            bf16 = {"ttmc_ms_per_mode": bms, "ttmc_nnz_per_s_per_mode": [Zc / (t * 1e-3) for t in bms],
                    "hooi_s_per_iter": sweep_b * 1e-3, "value": N * Zc / (sweep_b * 1e-3),
                    "hbm_frac_per_mode": [b_ / (t * 1e-3) / 1e9 / peaks()[0] for b_, t in
                                          zip([4.0 * N * Zc + 4.0 * w.dims[n] * ctx.P(n) + 4.0 * (w.dims[n] + 1)
                                               for n in range(N)], bms)]}
            T.tucker_free(ctxb)

    # ---- the differentiation form: loss + adjoint on the completion workload
    adjoint = None
    if not args.no_adjoint:
        ci = synth.make("completion-10M")
        cw = ci.workload
        with torch.cuda.stream(stream):
            ctxa = T.tucker_init(cw.dims, torch.as_tensor(ci.coords.astype(np.int32)).to(dev),
                                 torch.as_tensor(ci.vals).to(dev), cw.ranks, [torch.as_tensor(u).to(dev) for u in ci.U0],
                                 stream=stream)
            rng = np.random.default_rng(7)
            Ua = [torch.as_tensor((ci.model["U"][m] + 0.1 * rng.standard_normal(ci.model["U"][m].shape))
                                  .astype(np.float32)).to(dev) for m in range(len(cw.dims))]
            Ga = torch.as_tensor(ci.model["G"].astype(np.float32)).to(dev)
            lossb = torch.empty(1, dtype=torch.float64, device=dev)
            dUa = [torch.empty_like(u) for u in Ua]
            dGa = torch.empty_like(Ga)
            for _ in range(3):
                T.tucker_loss_grad(ctxa, Ua, Ga, lossb, dUa, dGa, stream=stream)
            evs = []
            for i in range(10):
                flush.fill_(float(i))
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                T.tucker_loss_grad(ctxa, Ua, Ga, lossb, dUa, dGa, stream=stream)
                b_.record(stream)
                evs.append((a_, b_))
            torch.cuda.synchronize()
            ams = statistics.median(a_.elapsed_time(b_) for a_, b_ in evs)
            Za = T.tucker_nnz(ctxa)
            adjoint = {"workload": cw.name, "dims": list(cw.dims), "nnz": Za, "ranks": list(cw.ranks),
                       "ms_per_loss_and_grad": ams, "nnz_per_s": Za / (ams * 1e-3), "loss": float(lossb.item()),
                       "precision": "FP32 (loss accumulated in FP64)"}
            T.tucker_free(ctxa)

    # ---- end to end through the C ABI from pinned host buffers: the whole decomposition
    # job of the workload (init + its sweeps + read back fit, core and factors)
    e2e = None
    if not args.no_e2e:
        import torch as _t
        coords_h = _t.from_numpy(inst.coords.astype(np.uint32).view(np.int32)).pin_memory()
        vals_h = _t.from_numpy(inst.vals).pin_memory()
        U0_h = _t.from_numpy(np.concatenate([u.reshape(-1) for u in inst.U0])).pin_memory()
        Uh = [_t.empty((w.dims[n], w.ranks[n]), dtype=_t.float64).pin_memory() for n in range(N)]
        Gh = _t.empty(w.ranks, dtype=_t.float64).pin_memory()
        h2d = coords_h.numel() * 4 + vals_h.numel() * 4 + U0_h.numel() * 8
        d2h = 8 + Gh.numel() * 8 + sum(u.numel() * 8 for u in Uh)
        lib = T.load()
        import ctypes
        dims_a = (ctypes.c_int64 * N)(*w.dims)
        ranks_a = (ctypes.c_int * N)(*w.ranks)
        ts = []
        for rep in range(1 + max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = ctypes.c_void_p()
            rc = lib.tucker_init(ctypes.byref(h), N, dims_a, Z, coords_h.data_ptr(), vals_h.data_ptr(), ranks_a,
                                 U0_h.data_ptr(), 0, T.TUCKER_F_HOST_INPUT, _stream(stream))
            assert rc == 0, rc
            f = ctypes.c_double()
            for _ in range(w.iters - 1):
                assert lib.hooi_iter(h, None, _stream(stream)) == 0
            assert lib.hooi_iter(h, ctypes.addressof(f), _stream(stream)) == 0
            with torch.cuda.stream(stream):
                Gd = torch.empty(w.ranks, dtype=torch.float64, device=dev)
                assert lib.core_tensor(h, Gd.data_ptr(), _stream(stream)) == 0
                Gh.copy_(Gd, non_blocking=True)
                for n in range(N):
                    Ud = torch.empty((w.dims[n], w.ranks[n]), dtype=torch.float64, device=dev)
                    assert lib.tucker_get_factor(h, n, Ud.data_ptr(), _stream(stream)) == 0
                    Uh[n].copy_(Ud, non_blocking=True)
            stream.synchronize()
            t1 = time.perf_counter()
            lib.tucker_free(h)
            if rep > 0:
                ts.append(t1 - t0)
        tj = statistics.median(ts)
        e2e = {"value": N * Zc * w.iters / tj, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "job_s": tj,
               "step": f"tucker_init from pinned host COO + {w.iters} hooi_iter + fit/core/factors read back"}

    # ---- roofline of the dominant kernel
    hbm_peak, hbm_src = peaks()
    with torch.cuda.stream(stream):
        fp32_peak = T.tucker_fp32_fma_tflops(20000, stream=stream)
    ttmc_total = sum(phase_ms[2 * n] for n in range(N))
    qrp_total = sum(phase_ms[2 * n + 1] for n in range(N))
    flops = [2.0 * ctx.P(n) * Zc for n in range(N)]
    bytes_alg = [4.0 * N * Zc + 4.0 * w.dims[n] * ctx.P(n) + 4.0 * (w.dims[n] + 1) for n in range(N)]
    ttmc_avg_ms = sum(ttmc_ms) / N
    ttmc_flops = sum(flops) / N
    ttmc_bytes = sum(bytes_alg) / N
    forms = []
    for n in range(N):
        mi = T.tucker_mode_info(ctx, n)
        forms.append("fiber form (ttmc_fibsum_kernel + ttmc_pipe_kernel over fibers, "
                     f"{mi['fibers'] / max(Zc, 1):.2f} fibers per nonzero)" if mi["fibers_on"]
                     else "nonzero form (ttmc_pipe_kernel)")
    ttmc_roof = {"kernel": "FP32 TTMc per mode: " + "; ".join(f"mode {n + 1} {f}" for n, f in enumerate(forms)),
                 "bound": "alu",
                 "achieved": ttmc_flops / (ttmc_avg_ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                 "frac": ttmc_flops / (ttmc_avg_ms * 1e-3) / 1e12 / fp32_peak,
                 "traffic": profile_traffic("ttmc_fp32_skew-20M"),
                 "peak_source": "measured in this run: FP32 FMA throughput kernel (tucker_fp32_fma_tflops)",
                 "binding_unit": "L1/shared-memory path (operand and row loads) and instruction issue; see profiles/",
                 "hbm_view": {"achieved_gbs": ttmc_bytes / (ttmc_avg_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                              "frac": ttmc_bytes / (ttmc_avg_ms * 1e-3) / 1e9 / hbm_peak,
                              "peak_source": hbm_src, "alg_bytes_per_launch": ttmc_bytes},
                 "alg_flops_per_launch": ttmc_flops, "avg_launch_ms": ttmc_avg_ms}
    # QRP: one launch per mode; for the tall unfoldings its memory work is k + 1 passes
    # over the FP32 Y_(n) (initial norms + one A^T v per reflector) plus V and Q (FP64).
    big = [n for n in range(N) if w.dims[n] == max(w.dims)]
    qbytes = []
    for n in big:
        m_, n_, k_ = w.dims[n], ctx.P(n), w.ranks[n]
        qbytes.append((k_ + 1) * m_ * n_ * 4.0 + 2.0 * m_ * k_ * 8.0)
    q_ms = sum(phase_ms[2 * n + 1] for n in big) / len(big)
    q_bytes = sum(qbytes) / len(qbytes)
    one_pass = sum(w.dims[n] * ctx.P(n) * 4.0 + 2.0 * w.dims[n] * w.ranks[n] * 8.0 for n in big) / len(big)
    k_q = w.ranks[big[0]]
    qrp_roof = {"kernel": f"qrp_cluster_kernel<float> on the {max(w.dims)} x {ctx.P(big[0])} unfoldings",
                "bound": "latency",
                "achieved": one_pass / (q_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": one_pass / (q_ms * 1e-3) / 1e9 / hbm_peak,
                "traffic": None,
                "peak_source": hbm_src, "dram_bytes_per_launch": one_pass, "avg_launch_ms": q_ms,
                "us_per_reflector": q_ms * 1e3 / k_q,
                "note": "DRAM traffic is about one pass over the FP32 Y plus V and Q (the other k passes of the "
                        "column sums read shared memory and L2); the step is bound by the k dependent reflector "
                        "steps (one grid barrier, a cluster reduction and FP64 dependent chains each), not by a "
                        "memory or arithmetic roof; traffic is not captured (the kernel is kept off ncu)"}
    dominant = ttmc_roof if ttmc_total >= qrp_total else qrp_roof

    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        cc, cv = oracle_coalesced(inst, None if args.oracle_full else args.oracle_nnz)
        t_all = oracle_sweep(inst, cc, cv, threads)
        t1, nz1 = oracle_sample(inst, args.oracle_single_nnz, threads=1)
        cpu = {"value": N * cc.shape[1] / t_all, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"one oracle HOOI sweep (C, FP64, {threads} threads split by output column, equal to the "
                         f"serial oracle bit for bit) over {cc.shape[1]:,} coalesced entries of {w.name}; "
                         f"{t_all:.1f} s",
               "cpu_model": cpu_model(),
               "single_thread": {"value": N * nz1 / t1, "cores": 1,
                                 "sample": f"one serial oracle sweep over the first {args.oracle_single_nnz:,} listed "
                                           f"entries ({nz1:,} after coalescing); {t1:.1f} s"}}

    paper = {}
    if rank == 0 and not args.no_paper:
        import oracle
        oracle.build()
        paper["fig7_sparsity_sweep"] = fig7_rows(T, torch, os.cpu_count() or 1)
        paper["table3_core_ttm"] = table3_rows(T, torch, os.cpu_count() or 1)

    clocks = clk.summary()
    value = world * N * Zc / (ms_per_step * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "nnz_coalesced": Zc,
                       "ranks": list(w.ranks), "l2": "flushed between timed steps (256 MiB write)",
                       "precision": "TTMc FP32 (FP32 products and sums); QRP: FP64 storage, norms, reflectors, R "
                                    "and T, with A^T y summed in double-float FP32 pairs around a power-of-two "
                                    "offset (about 2^-49 s1 per product) and Q formed as double-float sums; core "
                                    "on the tensor cores: Y (FP32) and U_N (FP64) cut into four exact 8-bit "
                                    "fixed-point slices per column, BF16 products summed exactly (integer) in "
                                    "FP32 tensor memory, levels combined in 64-bit integers, row ranges and fit "
                                    "in FP64", "replicas": world},
            "hooi_s_per_iter": ms_per_step * 1e-3,
            "step": "one HOOI sweep (TTMc + QRP per mode, core, fit) replayed from a CUDA graph of the whole iteration",
            "eager_ms_per_step": eager_ms,
            "phases_ms": {"ttmc": [phase_ms[2 * n] for n in range(N)], "qrp": [phase_ms[2 * n + 1] for n in range(N)],
                          "core_fit": phase_ms[2 * N]},
            "ttmc_nnz_per_s_per_mode": [Zc / (t * 1e-3) for t in ttmc_ms],
            "roofline": dominant, "roofline_other": qrp_roof if dominant is ttmc_roof else ttmc_roof,
            "init_s": init_s, "lib_setup_s": lib_setup_s, "fit_after_warmup_and_steps": fit,
            "bf16_factor_form": bf16, "adjoint_form": adjoint, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clocks, "gpu_launches": int(launches), **paper}
    if rank == 0:
        print(json.dumps(line), flush=True)
    T.tucker_free(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- paper experiments
def _gpu_sweeps(T, torch, inst, iters, profile=False):
    """init + `iters` HOOI sweeps on the GPU; returns (init_s, per-sweep ms list, fits, ctx)."""
    w = inst.workload
    coords = torch.as_tensor(inst.coords.astype(np.int32)).cuda()
    vals = torch.as_tensor(inst.vals).cuda()
    U0 = [torch.as_tensor(u).cuda() for u in inst.U0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = T.tucker_init(w.dims, coords, vals, w.ranks, U0)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    if profile:
        T.tucker_set_profiling(ctx, True)
    ms, fits, phases = [], [], []
    for _ in range(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fits.append(T.hooi_iter(ctx))
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        if profile:
            phases.append(T.tucker_phase_times(ctx))
    return init_s, ms, fits, ctx, phases


def fig7_rows(T, torch, threads=1):
    """Section IV-C, Fig. 7: whole decompositions of 200^3 random tensors, ranks 16, over a
    range of sparsities; GPU (init + sweeps) beside the FP64 oracle on the host."""
    import oracle
    from paper_2010_10638_gb300 import synth
    rows = []
    for i in range(len(synth.FIG7_DENSITIES)):
        inst = synth.make(synth.fig7_workload(i))
        w = inst.workload
        _, _, _, ctx, _ = _gpu_sweeps(T, torch, inst, 2)  # warm-up (first-use set-up of the kernels)
        T.tucker_free(ctx)
        init_s, ms, fits, ctx, _ = _gpu_sweeps(T, torch, inst, w.iters)
        T.tucker_free(ctx)
        t0 = time.perf_counter()
        ref = oracle.hooi(w.dims, w.ranks, inst.coords, inst.vals.astype(np.float64), inst.U0, w.iters,
                          threads=threads)
        t_or = time.perf_counter() - t0
        gpu_s = init_s + sum(ms) * 1e-3
        rows.append({"sparsity": w.nnz / float(np.prod(w.dims)), "nnz": w.nnz, "sweeps": w.iters,
                     "gpu_s": gpu_s, "gpu_init_s": init_s, "gpu_sweep_ms": float(np.median(ms)),
                     "oracle_s": t_or, "oracle_cores": threads, "speedup_vs_oracle": t_or / gpu_s,
                     "max_fit_diff_vs_oracle": float(np.max(np.abs(np.asarray(fits) - np.asarray(ref.fits)))),
                     "fit_gpu": fits[-1], "fit_oracle": float(ref.fits[-1])})
    return {"experiment": "fig7 sparsity sweep (Section IV-C)", "dims": [200, 200, 200], "ranks": [16, 16, 16],
            "data": "synthetic, distinct uniform coordinates, U(0,1) values", "rows": rows}


def table3_rows(T, torch, threads=1):
    """Table III: the dense core TTM, a 32 x 32 x I3 tensor times a 32 x I3 factor, as the
    core step of one sweep on a fully listed 32 x 32 x I3 tensor (ranks 32); the core
    phase is timed with CUDA events inside hooi_iter, beside the oracle's core on the
    same Y_(3) and U_3 (and its difference from the GPU's core)."""
    import oracle
    from paper_2010_10638_gb300 import synth
    rows = []
    for i in range(len(synth.TABLE3_I3)):
        inst = synth.make(synth.table3_workload(i))
        w = inst.workload
        _, _, _, ctx, phases = _gpu_sweeps(T, torch, inst, 12, profile=True)
        core_ms = float(np.median([p[-1] for p in phases[2:]]))
        Y3 = T.ttmc_mode(ctx, 2).cpu().numpy().astype(np.float64)
        U3 = T.tucker_get_factor(ctx, 2).cpu().numpy()
        Gg = T.core_tensor(ctx).cpu().numpy()
        T.tucker_free(ctx)
        reps = 20
        t0 = time.perf_counter()
        for _ in range(reps):
            Go = oracle.core(Y3, U3, w.ranks, threads)
        t_or = (time.perf_counter() - t0) / reps
        flops = 2.0 * 32 * 32 * w.dims[2] * 32
        rows.append({"I3": w.dims[2], "core_fit_ms": core_ms, "gflops": flops / (core_ms * 1e-3) / 1e9,
                     "oracle_ms": t_or * 1e3, "oracle_cores": threads,
                     "core_rel_diff_vs_oracle": float(np.linalg.norm(Gg - Go) / np.linalg.norm(Go))})
    return {"experiment": "table3 core TTM (Section IV-A)", "shape": "(32 x 32 x I3) x_3 (32 x I3)^T -> 32 x 32 x 32",
            "note": "core_fit_ms is the core step of hooi_iter (core tensor, its norm and the fit); the oracle's "
                    "core is computed from the GPU's Y_(3) and U_3", "rows": rows}


def run_fig7(args):
    import torch
    import oracle
    from paper_2010_10638_gb300 import build as libbuild, tucker as T
    libbuild.build()
    T.load()
    oracle.build()
    print(json.dumps(fig7_rows(T, torch, os.cpu_count() or 1)), flush=True)
    return 0


def run_table3(args):
    import torch
    import oracle
    from paper_2010_10638_gb300 import build as libbuild, tucker as T
    libbuild.build()
    T.load()
    oracle.build()
    print(json.dumps(table3_rows(T, torch, os.cpu_count() or 1)), flush=True)
    return 0


def run_configs(args):
    """Every workload recipe at full size: GPU sweep and per-mode TTMc times (CUDA events),
    HBM and arithmetic fractions of the TTMc, and the oracle's time per sweep (one sweep on
    at most `oracle_nnz` entries, scaled by the nonzero count).  Parity at these sizes is
    the GPU test suite's (sampled rows against the oracle, componentwise bound)."""
    import torch
    import oracle
    from paper_2010_10638_gb300 import build as libbuild, synth, tucker as T
    libbuild.build()
    T.load()
    oracle.build()
    hbm_peak, _ = peaks()
    bf16_peak = 1918.6
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f).get("bf16_tflops", bf16_peak))
    except (OSError, ValueError):
        pass
    rows = []
    fp32_peak = T.tucker_fp32_fma_tflops(20000)
    for name in ("tiny-100^3", "zipf-10k^3", "order4-5M", "skew-20M"):
        inst = synth.make(name)
        w = inst.workload
        N = len(w.dims)
        for bf16 in ((False, True) if name in ("order4-5M", "skew-20M") else (False,)):
            ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                                torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0],
                                bf16=bf16)
            Zc = T.tucker_nnz(ctx)
            T.tucker_set_profiling(ctx, True)
            T.hooi_iter(ctx)
            for _ in range(3):
                T.hooi_iter(ctx)
            ph = []
            for _ in range(10):
                T.hooi_iter(ctx)
                ph.append(T.tucker_phase_times(ctx))
            med = [float(np.median([p_[i] for p_ in ph])) for i in range(2 * N + 1)]
            sweep_ms = sum(med)
            ttmc_ms = [med[2 * n] for n in range(N)]
            flops = [2.0 * ctx.P(n) * Zc for n in range(N)]
            bytes_alg = [4.0 * N * Zc + 4.0 * w.dims[n] * ctx.P(n) + 4.0 * (w.dims[n] + 1) for n in range(N)]
            gbs = sum(bytes_alg) / (sum(ttmc_ms) * 1e-3) / 1e9
            tflops = sum(flops) / (sum(ttmc_ms) * 1e-3) / 1e12
            T.tucker_free(ctx)
            row = {"config": name, "form": "bf16 factors" if bf16 else "fp32", "nnz": Zc,
                   "ttmc_nnz_per_s_per_mode": [Zc / (m_ * 1e-3) for m_ in ttmc_ms], "ttmc_ms": ttmc_ms,
                   "hooi_s_per_iter": sweep_ms * 1e-3, "ttmc_hbm_gbs": gbs, "ttmc_hbm_frac": gbs / hbm_peak}
            if bf16:
                row["ttmc_tensor_frac"] = tflops / bf16_peak
            else:
                row["ttmc_fp32_frac"] = tflops / fp32_peak
            if not bf16:
                threads = os.cpu_count() or 1
                cc, cv = oracle_coalesced(inst)
                row["oracle_s_per_iter"] = oracle_sweep(inst, cc, cv, threads)
                row["oracle_note"] = (f"one full sweep on {threads} threads (column-split oracle, equal to the serial "
                                      f"one bit for bit)")
                row["oracle_cores"] = threads
            rows.append(row)
    print(json.dumps({"experiment": "all workload recipes", "rows": rows}), flush=True)
    return 0


def _stream(s):
    return int(s.cuda_stream)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="skew-20M")
    ap.add_argument("--oracle-nnz", type=int, default=1_000_000,
                    help="entries the threaded oracle sweeps when --oracle-full is off")
    ap.add_argument("--oracle-full", type=int, default=1, help="1: the threaded oracle sweeps the whole workload")
    ap.add_argument("--oracle-single-nnz", type=int, default=1_000_000,
                    help="entries of the single-thread oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper", action="store_true", help="leave the Fig. 7 and Table III curves out of the line")
    ap.add_argument("--fig7", action="store_true", help="Fig. 7 sparsity sweep (200^3, ranks 16) instead")
    ap.add_argument("--table3", action="store_true", help="Table III core TTM shapes instead")
    ap.add_argument("--configs", action="store_true", help="every workload recipe at full size instead")
    args = ap.parse_args()
    if args.configs:
        return run_configs(args)
    if args.fig7:
        return run_fig7(args)
    if args.table3:
        return run_table3(args)
    if args.warmup < 3 and args.impl == "mine":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
