"""Benchmark: beyond-Limber C_l sets per second on one or more GB300s.

Workload: the 3x2pt data vector with 5 clustering + 5 lensing tomographic bins
(55 spectra), 64 log-spaced ells in 2..1000, n_chi = 128, n_R = 128 in
R in [0.2, 1.8], Chebyshev order 64, for a batch of seeded synthetic
cosmologies (each with its own P(k), kernels and growth).  One step is one
pass of the whole hot path — Chebyshev fit, weights, contraction (a) and
quadrature (b) — over the batch.  The basis precompute is excluded, as in the
paper's timings.

The headline value is the mixed-precision batched path (tcgen05 BF16 five-slice
exact split when the plan supports it); the plain FP64 GPU path is measured
beside it with the headline's error against the FP64 result stated.  Usage:

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl blast|reference]
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "C_l-sets/sec (3x2pt, all bin pairs) mixed vs FP64 at ≤1e-4 rel err; p50/p99 latency"
UNIT = "C_l-sets/s"
WORKLOADS = {
    "c1": ("3x2pt, 5 clustering + 5 lensing bins (55 spectra), 64 log-spaced ells 2..1000, "
           "n_chi=128, n_R=128 (R in [0.2,1.8]), Chebyshev order 64, n_kquad=65537"),
    "c2": ("3x2pt precision grid, 10 clustering + 10 lensing bins (210 spectra), 100 log-spaced ells 2..2000, "
           "n_chi=256, n_R=192 (R in [0.2,1.8]), Chebyshev order 96, n_kquad=65537"),
    "c3": ("ragged batch on the 10+10-bin grid: every cosmology with its own bin counts (2..10 of each kind) "
           "and its own set of 16..100 of the 100 ells, n_chi=256, n_R=192, Chebyshev order 96"),
}
WORKLOAD = WORKLOADS["c1"]


def workload_config(batch, world, name="c1"):
    """The workload both arms report (the arithmetic type is the line's dtype)."""
    return {"workload": WORKLOADS[name], "batch_per_gpu": batch,
            "l2": "inputs larger than L2 (basis tables 0.8-14 GB per step)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# --------------------------------------------------------------------------- replicas
# The path shards by cosmology: every rank evaluates its own batch on its own
# GPU with no exchange; the job's time is the slowest rank's.
def replica_request_ids(rank, batch):
    """Seeded cosmology indices of a rank's batch (disjoint across ranks)."""
    return [1 + i + rank * batch for i in range(batch)]


def max_over_ranks(x, world, device=None):
    """The largest value over ranks (an all-reduce MAX); x itself at world 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, batch, steps, seconds):
    """C_l-sets per second of the whole job: every rank's batches over the slowest rank's time."""
    return world * batch * steps / seconds


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- oracle (CPU) timing
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OracleSample:
    """The FP64 oracle's per-cosmology evaluation (fit + contraction +
    quadrature; the basis is excluded as in the paper) on a workload's grid,
    for a subset of ells.  The oracle's basis for these grids would take hours
    to build on the host, and its evaluation loops cost the same whatever the
    basis values are, so the sample feeds it a seeded random basis of the right
    shape.  c1: 4 cosmologies x every 4th of the 64 ells; c2: 2 cosmologies x
    every 10th of the 100 ells; c3: 2 ragged requests (own bin counts), the
    sample ells inside each request's own ell set, scaled by its size."""

    def __init__(self, n_req=None, workload="c1", seed=7):
        import oracle
        from paper_2410_03632_gb300 import synth
        grid = "c1" if workload == "c1" else "c2"
        spec = synth.plan_spec(grid)
        stride = 4 if grid == "c1" else 10
        n_req = n_req or (4 if grid == "c1" else 2)
        self.g = oracle.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min,
                             spec.R_max, spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
        sub_idx = np.arange(0, spec.ells.size, stride)
        rng = np.random.default_rng(seed)
        self.T = rng.standard_normal((3, sub_idx.size, spec.n_cheb, spec.n_chi * spec.n_R))
        self.items = []  # (request, sample-ell positions, the C_l-set fraction it evaluates)
        self._Tsel = {}
        for i in range(n_req):
            if workload == "c3":
                rq, sel = synth.ragged_request(self.g.chi, self.g.R, 1 + i, spec.ells.size)
                pos = [k for k, e in enumerate(sub_idx) if e in set(sel)]
                self.items.append((rq, pos, len(pos) / len(sel)))
                self._Tsel[i] = np.ascontiguousarray(self.T[:, pos])  # built here, not in the timed pass
            else:
                rq = synth.config_request(grid, self.g.chi, self.g.R, 1 + i)
                self.items.append((rq, list(range(sub_idx.size)), sub_idx.size / spec.ells.size))
        self.sub = spec.ells[sub_idx]
        self.sets = sum(f for _, _, f in self.items)  # C_l-sets one run evaluates
        own = " (those within each request's own ell set)" if workload == "c3" else ""
        self.desc = (f"{workload}: {n_req} cosmologies x every {stride}th of the {spec.ells.size} ells{own} "
                     f"on the {grid} grid, oracle fit + contraction + quadrature, seeded random basis of the "
                     f"right shape; scaled to full C_l-sets")

    def run(self, threads):
        """Seconds for one pass over the sample with `threads` OpenMP threads."""
        t0 = time.perf_counter()
        for i, (rq, pos, _) in enumerate(self.items):
            if not pos:
                continue
            a = self.g.fit(rq.k_tab, rq.p_tab)
            T = self._Tsel.get(i, self.T)
            self.g.cl(T, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi,
                      rq.growth_chi, rq.growth_Rchi, ell_subset=self.sub[pos], nthreads=threads)
        return time.perf_counter() - t0


def cpu_baseline(reps=10, workload="c1"):
    """Oracle throughput on the host cores at 1 thread and at every core: the
    median of `reps` passes after one warm-up pass, in C_l-sets/s."""
    smp = OracleSample(workload=workload)
    cores = os.cpu_count() or 1
    res = {}
    for th in (1, cores):
        smp.run(th)
        ts = [smp.run(th) for _ in range(reps)]
        res[th] = (smp.sets / statistics.median(ts), sum(ts))
    return {"value": res[cores][0], "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1_thread": res[1][0], "nproc": cores, "cpu_model": cpu_model(),
            "statistic": f"median of {reps} passes after 1 warm-up, per thread count",
            "seconds": res[1][1] + res[cores][1], "sample": smp.desc}


def run_reference(args):
    """The oracle as it stands on the host cores: each step is one pass over a
    bounded sample of the workload (one cosmology, a subset of its ells; see
    OracleSample), scaled to C_l-sets."""
    rank, _, world = env_rank()
    if rank != 0:
        return
    smp = OracleSample(n_req=1, workload=args.workload)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        smp.run(cores)
    secs = sum(smp.run(cores) for _ in range(args.steps))
    value = args.steps * smp.sets / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.batch, world, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": smp.desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def alu_peaks():
    """CUDA-core FMA peaks (TFLOP/s) measured by the probe library's own kernels:
    FP64, FP32 scalar and FP32 packed pairs."""
    import ctypes
    from paper_2410_03632_gb300 import build as _b
    L = ctypes.CDLL(_b.build_probe())
    L.peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]
    out = {}
    for kind, name, iters in ((0, "fp64_tflops", 8000), (1, "fp32_tflops", 200000), (2, "fp32x2_tflops", 100000)):
        tf, ms = ctypes.c_double(), ctypes.c_double()
        if L.peak_probe(kind, iters, ctypes.byref(tf), ctypes.byref(ms)) == 0:
            out[name] = tf.value
    out["how"] = ("own kernels: 8 independent dependent-FMA chains per thread, 8 blocks of 256 threads "
                  "per SM, one timed launch after a warm-up (CUDA events)")
    return out


# --------------------------------------------------------------------------- GPU arm
def traffic_for(kernel_file, kernel_name, workload="c1", batch=256):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json for the
    current source of the kernel and this workload and batch (None when the
    source changed since or no capture covers the workload)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, "paper_2410_03632_gb300", "csrc", kernel_file), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    for rec in json.load(open(path)):
        if (rec.get("kernel") == kernel_name and rec.get("src_sha") == sha and rec.get("workload") == workload
                and rec.get("batch") == batch):
            return rec.get("bytes_per_launch_full")
    return None


def run_blast(args):
    import torch
    import torch.distributed as dist
    from paper_2410_03632_gb300 import blast as bl
    from paper_2410_03632_gb300 import synth
    from tests.metrics import eij

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = args.workload
    spec = synth.plan_spec("c1" if wl == "c1" else "c2")
    if args.n_ell:  # the same grid on fewer ells: a smaller case for profiler captures
        import dataclasses
        spec = dataclasses.replace(spec, ells=synth.ell_list(args.n_ell, 2, int(spec.ells[-1])))
    plan = bl.Plan(spec, device=local)
    cache = args.basis_cache
    if cache and os.path.exists(cache):
        bl.blast_basis_load(plan.h, cache, bl.BASIS_ALL)
    else:
        plan.precompute(bl.BASIS_ALL)
        if cache and rank == 0:
            bl.blast_basis_save(plan.h, cache)
    chi, R, _ = plan.nodes()
    B = args.batch
    if wl == "c3":
        made = [synth.ragged_request(chi, R, i, plan.L) for i in replica_request_ids(rank, B)]
        rqs, sels = [m[0] for m in made], [m[1] for m in made]
    else:
        rqs = [synth.config_request(wl, chi, R, i) for i in replica_request_ids(rank, B)]
        sels = [None] * B
    fields = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]
    dev_arrays = [{f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).to(dev) for f in fields} for rq in rqs]
    reqs = [plan.request(rq, ell_sel=sl, device_arrays=d) for rq, sl, d in zip(rqs, sels, dev_arrays)]
    P = bl.blast_npairs(spec.max_clust, spec.max_lens)
    shapes = [(bl.blast_npairs(rq.n_clust, rq.n_lens), plan.L if sl is None else len(sl)) for rq, sl in zip(rqs, sels)]
    outs = [torch.empty(sh, dtype=torch.float64, device=dev) for sh in shapes]
    out_ptrs = [o.data_ptr() for o in outs]
    stream = torch.cuda.current_stream(dev)

    have_tc = bl.blast_cl_batch(plan.h, reqs[:2], bl.BLAST_BF16S, out_ptrs[:2], 1, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    tuned = None
    if have_tc and not args.no_autotune:  # launch parameters picked on this batch (outside the timed region)
        t0 = time.perf_counter()
        rc = bl.blast_autotune(plan.h, reqs, args.tune_cache, stream.cuda_stream)
        if rc == 0:
            g_, w_, n_ = bl.blast_tuned_params(plan.h)
            tuned = {"contract_ctas": g_, "reduce_warps": w_, "reduce_stages": n_,
                     "seconds": time.perf_counter() - t0}
    prec_main = bl.BLAST_BF16S if have_tc else bl.BLAST_FP32
    dtype_main = "bf16 5-slice exact split (tcgen05)" if have_tc else "f32"

    def step(prec):
        rc = bl.blast_cl_batch(plan.h, reqs, prec, out_ptrs, 1, stream.cuda_stream)
        if rc != 0:
            raise RuntimeError(f"blast_cl_batch failed: {bl.blast_status_str(rc)}")

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(prec, K, W, profile=False):
        for _ in range(W):
            step(prec)
        torch.cuda.synchronize()
        barrier()
        bl.blast_profile_reset(plan.h)
        bl.blast_profile_enable(plan.h, profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        prof = {}
        for c, name in enumerate(bl.KERNEL_CLASS_NAMES):
            prof[name] = bl.blast_profile_read(plan.h, c)
        bl.blast_profile_enable(plan.h, False)
        return ms, prof

    clk = ClockSampler(local)
    clk.start()
    ms_main, prof_main = timed(prec_main, args.steps, args.warmup, profile=True)
    clocks = clk.stop()
    C_main = [o.cpu().numpy() for o in outs]

    # the same batch captured once as a CUDA graph and launched K times
    graph = None
    g = bl.blast_graph_create(plan.h, reqs, prec_main, out_ptrs)
    try:
        for _ in range(args.warmup):
            if bl.blast_graph_launch(g, stream.cuda_stream) != 0:
                raise RuntimeError("blast_graph_launch failed")
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bl.blast_graph_launch(g, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_g = max_over_ranks(e0.elapsed_time(e1), world, dev)
        same = all(np.array_equal(o.cpu().numpy(), c) for o, c in zip(outs, C_main))
        graph = {"value": job_throughput(world, B, args.steps, ms_g * 1e-3), "unit": UNIT,
                 "ms_per_step": ms_g / args.steps, "bitwise_equal_to_calls": same,
                 "reserved_bytes": bl.blast_graph_reserved(g),
                 "what": "blast_graph_create once (descriptors staged, work space owned by the graph), then "
                         "blast_graph_launch per step on the same device buffers"}
    finally:
        bl.blast_graph_destroy(g)
    k64 = max(2, min(20, args.steps // 4))  # FP64 steps: ~150 ms each at the benchmark batch
    ms_64, prof_64 = timed(bl.BLAST_FP64, k64, 1, profile=True)
    C_64 = [o.cpu().numpy() for o in outs]
    e_all = [eij(a, b, rq.n_clust, rq.n_lens) for a, b, rq in zip(C_main, C_64, rqs)]
    err = max(float(np.max(e))for e in e_all)
    # worst e_ij per (ell, pair type) over the batch (the precision table)
    from tests.metrics import pair_list
    table = {}
    for e, rq, sl in zip(e_all, rqs, sels):
        types = np.array([t for t, _, _ in pair_list(rq.n_clust, rq.n_lens)])
        cols = range(plan.L) if sl is None else sl
        for k, col in enumerate(cols):
            for t in range(3):
                if np.any(types == t):
                    key = (int(spec.ells[col]), t)
                    table[key] = max(table.get(key, 0.0), float(np.max(e[types == t, k])))

    # contraction kernel roofline (dominant kernel of the step)
    kname = "contract_tc" if have_tc else "contract"
    kms, klaunch = prof_main[kname]
    avg_ms = kms / max(1, klaunch)
    L, N, Q, X = plan.L, plan.N, plan.Q, plan.X
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    # contraction (a), one multiply-add per product, over each cosmology's own ells
    method_flops = sum(2.0 * 3 * (L if sl is None else len(sl)) * N * Q for sl in sels)
    if have_tc:
        # the roofline flops: the method's products with the split-MMA allowance x3;
        # the kernel is timed alone in its launch, so the burst BF16 peak applies
        flops = method_flops * 3
        peak = peaks.get("bf16_tflops", 1900.0)
        achieved = flops / (avg_ms * 1e-3) / 1e12
        # what the tensor cores actually execute: 15 BF16 slice products per
        # product, K padded to the swizzle row, cosmologies padded to the tile
        slice_flops = 2.0 * 3 * L * (-(-N // 64) * 64) * Q * (-(-B // 128) * 128) * 15
        slice_rate = slice_flops / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_kind": "bf16 burst, of measured",
                "flops_per_launch": flops, "flops_def": "2*3*L*N*Q*B x3 (split-MMA allowance)",
                "traffic": traffic_for("contract_tc.cu", "contract_tc", wl, B),
                "slice_mma": {"achieved": slice_rate, "frac": slice_rate / peak, "flops_per_launch": slice_flops,
                              "def": "15 BF16 slice products per product, K padded to 64, M padded to 128"}}
    else:
        ntr = 10
        alg_bytes = 3 * L * N * Q * 4 + B * (ntr * Q * 4 + N * 4 + 3 * L * X * 5 * 4)
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": "hbm copy, of measured", "traffic": traffic_for("eval.cu", "k_contract<float>", wl, B)}
    roof["kernel"] = kname
    roof["avg_launch_ms"] = avg_ms
    roof["launches"] = klaunch
    # the other kernels against their own bounds
    alu = alu_peaks()
    kern = {}
    rms, rl = prof_main["reduce"]
    if rl and have_tc:
        MT = max(spec.max_clust, spec.max_lens)
        Bp = -(-B // 128) * 128
        # R-tile partial pairs of every padded cosmology, chi weights (hi, lo) of the
        # A-side kind per type, and the C_l written
        red_bytes = (Bp * 3 * L * X * (plan.Rn // 32) * MT * 8 + 3 * Bp * X * MT * 8
                     + sum(sh[0] * sh[1] for sh in shapes) * 8)
        gbs = red_bytes / (rms / rl * 1e-3) / 1e9
        kern["reduce"] = {"bound": "hbm", "bytes_per_launch": red_bytes, "achieved": gbs,
                          "peak": peaks.get("hbm_gbs"), "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                          "unit": "GB/s"}
    cms, cl64 = prof_64["contract"]
    if cl64:
        tf = method_flops / (cms / cl64 * 1e-3) / 1e12
        kern["contract_fp64"] = {"bound": "alu", "achieved": tf, "peak": alu.get("fp64_tflops"),
                                 "frac": tf / alu["fp64_tflops"] if alu.get("fp64_tflops") else None,
                                 "unit": "TFLOP/s", "peak_kind": "FP64 FMA, measured by the probe kernels"}

    # single-request latency (p50 / p99) of the mixed path
    # the comparator of the serving numbers: requests one at a time in FP64
    lat = []
    one_prec = bl.BLAST_FP64
    for i in range(3):
        bl.blast_cl(plan.h, reqs[0], one_prec, out_ptrs[0], 1, stream.cuda_stream)
    torch.cuda.synchronize()
    for i in range(50):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bl.blast_cl(plan.h, reqs[i % B], one_prec, out_ptrs[i % B], 1, stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    lat.sort()

    # end to end through the C ABI with host buffers (pinned)
    host = []
    h2d = 0
    for rq in rqs:
        d = {}
        for f in fields:
            arr = np.ascontiguousarray(getattr(rq, f))
            t = torch.empty(arr.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = arr
            d[f] = t
            h2d += arr.nbytes
        host.append(d)
    hreqs = [plan.request(rq, ell_sel=sl, device_arrays=None) for rq, sl in zip(rqs, sels)]
    for hr, d in zip(hreqs, host):  # point the host request at pinned copies
        hr.kern_chi, hr.kern_Rchi = d["kern_chi"].data_ptr(), d["kern_Rchi"].data_ptr()
        hr.growth_chi, hr.growth_Rchi = d["growth_chi"].data_ptr(), d["growth_Rchi"].data_ptr()
        hr.k_tab, hr.p_tab = d["k_tab"].data_ptr(), d["p_tab"].data_ptr()
        hr._keep = d
    houts = [torch.empty(sh, dtype=torch.float64, pin_memory=True) for sh in shapes]
    hptrs = [o.data_ptr() for o in houts]
    d2h = sum(o.numel() * 8 for o in houts)

    def e2e_step():
        rc = bl.blast_cl_batch(plan.h, hreqs, prec_main, hptrs, 0, stream.cuda_stream)
        if rc != 0:
            raise RuntimeError(bl.blast_status_str(rc))
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)

    serve = None
    if args.serve_seconds > 0 and rank == 0 and wl == "c1":
        serve = serve_latency(plan, rqs, prec_main, dtype_main, args.serve_rate, args.serve_seconds)

    mixed = None
    if args.serve_mix and rank == 0 and wl == "c1":
        mixed = serve_mix(plan, rqs, prec_main, dtype_main, args.serve_rate, max(args.serve_seconds, 1.0),
                          basis_cache=args.basis_cache_mix)

    launches = sum(prof_main[n][1] for n in bl.KERNEL_CLASS_NAMES)
    value = job_throughput(world, B, args.steps, ms_main * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_main / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_main, "data": "synthetic",
        "config": dict(workload_config(B, world, wl), **({"n_ell_override": args.n_ell} if args.n_ell else {})),
        "fp64": {"value": job_throughput(world, B, k64, ms_64 * 1e-3), "unit": UNIT, "ms_per_step": ms_64 / k64,
                 "dtype": "f64"},
        "err_vs_fp64": {"max_eij": err, "bound": 1e-4,
                        "def": "|C-C_fp64|/sqrt(C_ii C_jj), every cosmology of the batch, all pairs and ells",
                        "by_ell_type": {f"{l}:{'gg gs ss'.split()[t]}": v for (l, t), v in sorted(table.items())}
                        if wl != "c1" else None},
        "graph": graph,
        "latency_ms": serve,
        "serving_mix": mixed,
        "sequential_fp64_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                               "req_per_s": 1e3 * len(lat) / sum(lat),
                               "what": "one blast_cl call per cosmology, FP64 path, device inputs, back to back"},
        "roofline": roof,
        "autotune": tuned,
        "kernel_bounds": kern,
        "alu_peaks": alu,
        "e2e": {"value": job_throughput(world, B, args.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernels_ms_per_step": {n: prof_main[n][0] / args.steps for n in bl.KERNEL_CLASS_NAMES
                                if prof_main[n][1]},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(workload=wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def serve_stream(srv, lanes, weights, rate, seconds, prec, seed=2000):
    """Drive a server with seeded Poisson arrivals at ``rate`` requests/s for
    ``seconds``: arrival i goes to lane l with probability weights[l] and takes
    the lane's next request (cycling over lanes[l], a list of (blast_request,
    output shape)); host inputs.  Latency = from the submit call to the end of
    the poll that returns the C_l (a poller thread per lane, in submit order).
    Returns p50/p99 overall and per lane."""
    import queue
    import threading

    from paper_2410_03632_gb300 import blast as bl
    n = max(1, int(rate * seconds))
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    w = np.asarray(weights, float)
    pick = rng.choice(len(lanes), size=n, p=w / w.sum())
    sub_t, done_t, status = [0.0] * n, [0.0] * n, [0] * n
    qs = [queue.Queue() for _ in lanes]
    outs = [np.empty(max(sh[0] * sh[1] for _, sh in ln)) for ln in lanes]

    def poller(li):
        while True:
            item = qs[li].get()
            if item is None:
                return
            i, t = item
            status[i], _ = bl.blast_poll(srv.h, t, outs[li].ctypes.data, -1)
            done_t[i] = time.perf_counter()

    th = [threading.Thread(target=poller, args=(li,)) for li in range(len(lanes))]
    for t in th:
        t.start()
    nxt_req = [0] * len(lanes)
    t0 = time.perf_counter()
    nxt, busy = t0, 0
    for i in range(n):
        nxt += gaps[i]
        while True:
            d = nxt - time.perf_counter()
            if d <= 0:
                break
            time.sleep(min(d, 5e-4))
        li = int(pick[i])
        r = lanes[li][nxt_req[li] % len(lanes[li])][0]
        nxt_req[li] += 1
        sub_t[i] = time.perf_counter()
        rc, t = bl.blast_submit(srv.h, li, r, prec)
        while rc == bl.BLAST_EBUSY:  # admission pushed back: the wait counts as latency
            busy += 1
            time.sleep(1e-4)
            rc, t = bl.blast_submit(srv.h, li, r, prec)
        if rc != 0:
            raise RuntimeError(f"blast_submit: {bl.blast_status_str(rc)}")
        qs[li].put((i, t))
    for q in qs:
        q.put(None)
    for t in th:
        t.join()
    bad = [(int(pick[i]), bl.blast_status_str(status[i])) for i in range(n) if status[i]]
    if bad:
        from collections import Counter
        raise RuntimeError(f"blast_poll failed for {len(bad)} of {n} requests: {dict(Counter(bad))}")
    wall = max(done_t) - t0

    def pct(ix):
        lat = sorted((done_t[i] - sub_t[i]) * 1e3 for i in ix)
        if not lat:
            return None
        return {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "max": lat[-1],
                "requests": len(lat)}

    res = pct(range(n))
    res.update({"offered_req_s": rate, "served_req_s": n / wall, "busy_retries": busy,
                "lanes": [pct([i for i in range(n) if pick[i] == li]) for li in range(len(lanes))]})
    return res


def serve_latency(plan, rqs, prec, prec_name, rate, seconds, seed=2000):
    """Serving latency of the 3x2pt grid alone through blast_submit / blast_poll."""
    from paper_2410_03632_gb300 import blast as bl
    srv = bl.Server([plan], hbm_budget=32 << 30, max_slots=256)
    try:
        lane = [(plan.request(rq), (bl.blast_npairs(rq.n_clust, rq.n_lens), plan.L)) for rq in rqs]
        res = serve_stream(srv, [lane], [1.0], rate, seconds, prec, seed)
    finally:
        srv.close()
    res.pop("lanes")
    res.update({"precision": prec_name,
                "what": "server (blast_submit/blast_poll, continuous batching, max 256 per batch), seeded Poisson "
                        "arrivals, host inputs; submit to completed poll"})
    return res


def serve_mix(plan1, rqs1, prec, prec_name, rate, seconds, basis_cache=None, max_slots=256):
    """Serving of a request stream that mixes the three workloads in size: a
    third 5+5-bin requests on the 3x2pt grid, a third 10+10-bin requests and a
    third ragged requests (own bin counts and ell sets) on the 10+10-bin order-96
    grid; both plans resident, one server lane each.  Each lane's stream is also
    served alone (same lane rate, the other lane idle) and every request kind is
    timed one by one on the FP64 path, which the server's latencies are set
    against."""
    import torch

    from paper_2410_03632_gb300 import blast as bl
    from paper_2410_03632_gb300 import synth
    t0 = time.perf_counter()
    plan2 = bl.Plan(synth.plan_spec("c2"), device=plan1.device)
    if basis_cache and os.path.exists(basis_cache):
        bl.blast_basis_load(plan2.h, basis_cache, bl.BASIS_ALL)
    else:
        plan2.precompute(bl.BASIS_ALL)
        if basis_cache:
            bl.blast_basis_save(plan2.h, basis_cache)
    basis_s = time.perf_counter() - t0
    chi2, R2, _ = plan2.nodes()
    L2 = plan2.L
    kinds = {"c1": [], "c2": [], "c3": []}
    for rq in rqs1[:16]:
        kinds["c1"].append((plan1.request(rq), (bl.blast_npairs(rq.n_clust, rq.n_lens), plan1.L)))
    for i in range(16):
        rq = synth.config_request("c2", chi2, R2, 5000 + i)
        kinds["c2"].append((plan2.request(rq), (bl.blast_npairs(rq.n_clust, rq.n_lens), L2)))
        rq3, sel = synth.ragged_request(chi2, R2, 5000 + i, L2)
        kinds["c3"].append((plan2.request(rq3, ell_sel=sel), (bl.blast_npairs(rq3.n_clust, rq3.n_lens), len(sel))))
    lane2 = [x for pair in zip(kinds["c2"], kinds["c3"]) for x in pair]  # alternating 10+10 and ragged

    # sequential FP64 comparator: one blast_cl per request, host inputs and outputs
    seq = {}
    for name, items in kinds.items():
        pl = plan1 if name == "c1" else plan2
        out = np.empty(max(sh[0] * sh[1] for _, sh in items))
        lat = []
        for k in range(3 + 24):
            r, _ = items[k % len(items)]
            a = time.perf_counter()
            rc = bl.blast_cl(pl.h, r, bl.BLAST_FP64, out.ctypes.data, 0, None)
            if rc != 0:
                raise RuntimeError(bl.blast_status_str(rc))
            if k >= 3:
                lat.append((time.perf_counter() - a) * 1e3)
        lat.sort()
        seq[name] = {"p50": lat[len(lat) // 2], "p99": lat[-1], "req_per_s": 1e3 * len(lat) / sum(lat)}
    torch.cuda.synchronize()

    srv = bl.Server([plan1, plan2], hbm_budget=64 << 30, max_slots=max_slots)
    try:
        reserved = srv.reserved()
        serve_stream(srv, [kinds["c1"], lane2], [1.0, 2.0], min(rate, 500.0), 0.5, prec, seed=1)  # warm-up
        alone1 = serve_stream(srv, [kinds["c1"], lane2], [1.0, 0.0], rate / 3.0, seconds, prec, seed=2002)
        alone2 = serve_stream(srv, [kinds["c1"], lane2], [0.0, 1.0], 2.0 * rate / 3.0, seconds, prec, seed=2003)
        mix = serve_stream(srv, [kinds["c1"], lane2], [1.0, 2.0], rate, seconds, prec, seed=2001)
    finally:
        srv.close()
        plan2.close()
    return {"mix": mix, "alone": [alone1["lanes"][0], alone2["lanes"][1]],
            "alone_served_req_s": [alone1["served_req_s"], alone2["served_req_s"]],
            "sequential_fp64_ms": seq, "server_reserved_bytes": reserved, "precision": prec_name,
            "basis_seconds_10x10_grid": basis_s, "max_slots": max_slots,
            "what": ("two resident plans (3x2pt 5+5 grid; 10+10 order-96 grid), one server lane each; seeded Poisson "
                     "arrivals, a third each 5+5, 10+10 and ragged requests; lane 0 = 5+5, lane 1 = 10+10 and "
                     "ragged alternating; 'alone' = the lane's own stream with the other lane idle; latency from "
                     "submit to completed poll, host inputs; sequential_fp64 = one blast_cl per request, host "
                     "inputs and outputs")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--impl", default="blast", choices=["blast", "reference"])
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS),
                    help="c1: the 3x2pt 5+5-bin grid (default); c2: the 10+10-bin order-96 grid; "
                         "c3: ragged bins and ell sets on the c2 grid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="offered request rate of the serving-latency run (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="length of the serving-latency run (0 = skip)")
    ap.add_argument("--serve-mix", action="store_true",
                    help="also serve a stream mixing the 5+5, 10+10 and ragged workloads over two resident plans "
                         "(computes the 10+10 grid's basis: minutes)")
    ap.add_argument("--n-ell", type=int, default=0,
                    help="evaluate the workload's grid on this many log-spaced ells instead (profiler captures)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch parameters")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (read, then appended)")
    ap.add_argument("--basis-cache-mix", default=None, help="basis file of the 10+10 grid for --serve-mix")
    ap.add_argument("--basis-cache", default=None,
                    help="file to load the FP64 basis from (or save it to after computing it)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_blast(args)


if __name__ == "__main__":
    main()
