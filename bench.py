#!/usr/bin/env python3
"""Benchmark: on-the-fly M-scheme H*X for 48Cr in the pf shell (4 protons + 4
neutrons, M=0, dim 1,963,461, seeded random isospin-coupled TBMEs).

A step is one block product Y = H X over k interleaved FP32 vectors through
the library's fused CUDA kernel (the FP32-mixed block path); `value` counts
vector-matvecs per second (k per step), whole job.  The same run also times
the plain FP64 single-vector path and reports the speedup, the end-to-end
rate through the host-buffer C-ABI call, a roofline line for the kernel and
the CPU oracle timed on a bounded sample of rows.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank works on its own GPU on its own copy of
the workload (the product has no exchange step on one basis; see the design
notes), and the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "48Cr-pf H·x matvecs/s & HBM GB/s vs peak: FP32-mixed block vs FP64, ≤1e-4 MeV"
UNIT = "vector-matvecs/s"
WORKLOAD = dict(space="pf", Z=4, N=4, twoM=0, parity=+1)
WORKLOAD_NAME = "pf shell 4p4n M=0 (48Cr), dim 1963461, 195 seeded random TBMEs"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def sample_rows(dim, frac, nchunks=64):
    """A bounded sample of basis rows: nchunks contiguous runs spread evenly
    through the basis, frac of all rows in total (every sector region is
    represented in proportion)."""
    n = max(nchunks, int(dim * frac))
    per = max(1, n // nchunks)
    starts = (np.arange(nchunks, dtype=np.int64) * dim) // nchunks
    rows = (starts[:, None] + np.arange(per, dtype=np.int64)[None, :]).reshape(-1)
    return np.unique(rows[rows < dim])


def csr_sample(frac=0.10):
    """The oracle of the workload with a sample of rows of its explicit FP64 H
    stored (CSR, built from bit operations on all host cores).  Returns
    (oracle, rows, nnz, build seconds)."""
    import oracle as O
    from paper_1801_08432_gb300 import inputs as I
    orbits, spe, tb = I.space(WORKLOAD["space"])
    o = O.Oracle(orbits, WORKLOAD["Z"], WORKLOAD["N"], WORKLOAD["twoM"], 0).set_interaction(spe, tb)
    rows = sample_rows(o.dim, frac)
    t0 = time.perf_counter()
    nnz = o.build_rows(rows)
    return o, rows, nnz, time.perf_counter() - t0


def host_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(budget_s=12.0, seed=5):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    its explicit-matrix product (CSR, FP64, OpenMP over all host cores) over a
    10 % row sample of H, repeated for about budget_s seconds.  The sample's
    rows are built first (reported, not timed); value = rows/s / dim."""
    from paper_1801_08432_gb300 import inputs as I
    o, rows, nnz, build_s = csr_sample()
    x = I.random_block(o.dim, 1, seed=seed)[:, 0]
    o.spmv_rows(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        o.spmv_rows(x)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    rows_per_s = reps * len(rows) / dt
    return {"value": rows_per_s / o.dim, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "method": "explicit CSR SpMV, FP64, OpenMP over all host cores",
            "sample": "%d of %d rows of H (64 runs spread over the basis, %d stored elements, built in %.1f s, "
                      "not timed); their product repeated %d times in %.1f s = %.0f rows/s; value = rows/s / dim"
                      % (len(rows), o.dim, nnz, build_s, reps, dt, rows_per_s),
            "csr_build_s": round(build_s, 2), "csr_sample_rows": int(len(rows)), "csr_sample_nnz": int(nnz),
            "nproc": os.cpu_count()}


def reference_arm(args):
    """The reference arm: the oracle as it stands on the host cores.  Each step
    is one product of the sampled rows of the explicit FP64 H (CSR, OpenMP),
    timed on its own; value = rows per second / dim."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1801_08432_gb300 import inputs as I
    o, rows, nnz, build_s = csr_sample()
    x = I.random_block(o.dim, 1, seed=5)[:, 0]
    for _ in range(args.warmup):
        o.spmv_rows(x)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.spmv_rows(x)
        ts.append(time.perf_counter() - t0)
    t = float(np.sum(ts))
    v = args.steps * len(rows) / t / o.dim
    sample = ("%d of %d rows of H (64 runs spread over the basis, %d stored elements, built in %.1f s before the "
              "steps); each step one product of them" % (len(rows), o.dim, nnz, build_s))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD_NAME, "k": 1, "sample": "10 % of the rows of H per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "method": "explicit CSR SpMV, FP64, OpenMP over all host cores",
                             "sample": sample, "csr_build_s": round(build_s, 2)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_lanczos(args):
    """The oracle's whole FP64 run on the workload: the explicit H (CSR) built
    on all host cores, then its Lanczos with full reorthogonalization from the
    seeded pivot for the bench's iteration count; one JSON line with the
    times (not part of the default run: ~40 GB of host memory)."""
    import oracle as O
    from paper_1801_08432_gb300 import inputs as I
    orbits, spe, tb = I.space(WORKLOAD["space"])
    o = O.Oracle(orbits, WORKLOAD["Z"], WORKLOAD["N"], WORKLOAD["twoM"], 0).set_interaction(spe, tb)
    t0 = time.perf_counter()
    nnz = o.build_matrix()
    build_s = time.perf_counter() - t0
    x = I.random_block(o.dim, 1, seed=5)[:, 0]
    o.spmv(x)
    t0 = time.perf_counter()
    for _ in range(5):
        o.spmv(x)
    spmv_s = (time.perf_counter() - t0) / 5
    p = I.random_block(o.dim, 1, seed=I.PIVOT_SEED)[:, 0]
    t0 = time.perf_counter()
    ev = o.lanczos(p, args.cpu_lanczos, nkeep=5)
    lan_s = time.perf_counter() - t0
    print(json.dumps({"cpu_lanczos": True, "workload": WORKLOAD_NAME, "cores": host_cores(), "nnz": nnz,
                      "csr_build_s": round(build_s, 1), "spmv_s": round(spmv_s, 3),
                      "vector_matvecs_per_s": 1.0 / spmv_s, "iterations": args.cpu_lanczos,
                      "lanczos_s": round(lan_s, 1), "evals_mev": [round(float(e), 9) for e in ev]}), flush=True)
    return 0


def aggregate_max(values, dist=None):
    """Element-wise max over ranks (the job time is the slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def reorth_bytes(dim, k, s, n_iter, passes):
    """Compulsory HBM bytes of the vector work between H X and the next
    block in n_iter block-Lanczos iterations (blocks of dim * k * s bytes):
    alpha (V_n^T W reads 2 blocks; W -= V_n A_n reads 2, writes 1), each
    Gram-Schmidt pass against the n + 1 stored blocks (dots read n + 2
    blocks; the update reads n + 2 and writes 1), the Gram matrix W^T W (1)
    and the normalization (read 1, write 1): 8 + passes (2 n + 5) blocks in
    iteration n."""
    blocks = sum(8 + passes * (2 * n + 5) for n in range(n_iter))
    return float(blocks) * dim * k * s


def reorth_bytes_thick(dim, k, s, niter, tb, restarts, passes):
    """reorth_bytes for thick-restart cycles: the first cycle runs iterations
    0 .. niter - 1, each later one tb .. niter - 1 (tb = Ritz blocks kept);
    each restart forms tb Ritz blocks from niter stored ones (read niter + 1,
    write 1 per Ritz block) and moves tb + 1 blocks (read and write)."""
    blocks = sum(8 + passes * (2 * n + 5) for n in range(niter))
    blocks += restarts * sum(8 + passes * (2 * n + 5) for n in range(tb, niter))
    blocks += restarts * (tb * (niter + 2) + 2 * (tb + 1))
    return float(blocks) * dim * k * s


def lanczos_check(ctx, N, I, torch, stream):
    """FP32-mixed block Lanczos (k=8) against FP64 single-vector Lanczos on the
    same space: lowest 5 eigenvalues after the FP64 refinement, residuals and
    the time split."""
    out = {}
    hbm_gbs = (peaks() or {}).get("hbm_gbs", 6800.0)
    runs = {"fp64_k1": (1, N.BS_F64, 300), "fp32_k8": (8, N.BS_F32, 80)}
    for name, (k, dt, niter) in runs.items():
        p = torch.from_numpy(I.random_block(ctx.dim, k, seed=I.PIVOT_SEED)).to(
            "cuda", torch.float64 if dt == N.BS_F64 else torch.float32)
        ev, rep = ctx.lanczos(p, k, dt, niter, 5, refine=True, stream=stream)
        nit = rep["iterations"]
        rb = reorth_bytes(ctx.dim, k, 8 if dt == N.BS_F64 else 4, nit, 2)
        out[name] = {"k": k, "block_iterations": nit, "vector_matvecs": nit * k,
                     "evals_mev": [round(float(e), 9) for e in ev], "residual_mev": rep["residual"],
                     "ms_total": round(rep["ms_total"], 1), "ms_matvec": round(rep["ms_matvec"], 1),
                     "ms_reorth_alpha_gram": round(rep["ms_reorth"], 1), "delta_conv": rep["delta_conv"],
                     "reorth_alg_bytes": rb, "reorth_gbs": round(rb / (rep["ms_reorth"] / 1000.0) / 1e9, 1),
                     "reorth_hbm_frac": round(rb / (rep["ms_reorth"] / 1000.0) / 1e9 / hbm_gbs, 3)}
    # thick-restart block Lanczos (FP32, k = 8): 16 block iterations per cycle,
    # 24 Ritz vectors kept, restarted until the residual estimates of the
    # lowest five are <= 1e-3 MeV; 20 stored blocks instead of 81
    p = torch.from_numpy(I.random_block(ctx.dim, 8, seed=I.PIVOT_SEED)).to("cuda", torch.float32)
    niter, nthick = 16, 24
    ev, rep = ctx.lanczos(p, 8, N.BS_F32, niter, 5, refine=True, stream=stream, nthick=nthick,
                          max_restarts=80, tol=1e-3)
    out["fp32_k8_thick"] = {"k": 8, "block_iterations_per_cycle": niter, "nthick": nthick,
                            "restarts": rep["restarts"], "block_products": rep["matvec_blocks"],
                            "vector_matvecs": rep["matvec_blocks"] * 8,
                            "stored_blocks": niter + 1 + nthick // 8,
                            "stored_gb": round((niter + 1 + nthick // 8) * ctx.dim * 8 * 4 / 1e9, 2),
                            "evals_mev": [round(float(e), 9) for e in ev], "residual_mev": rep["residual"],
                            "resid_est_mev": rep["resid_est"], "ms_total": round(rep["ms_total"], 1),
                            "ms_matvec": round(rep["ms_matvec"], 1),
                            "ms_reorth_alpha_gram_restart": round(rep["ms_reorth"], 1)}
    rb = reorth_bytes_thick(ctx.dim, 8, 4, niter, nthick // 8, rep["restarts"], 2)
    out["fp32_k8_thick"]["reorth_alg_bytes"] = rb
    out["fp32_k8_thick"]["reorth_gbs"] = round(rb / (rep["ms_reorth"] / 1000.0) / 1e9, 1)
    out["fp32_k8_thick"]["reorth_hbm_frac"] = round(rb / (rep["ms_reorth"] / 1000.0) / 1e9 / hbm_gbs, 3)
    # compare the pairs both runs converged (FP64 residual <= 1e-3 MeV bounds the
    # eigenvalue error by r^2/gap)
    t, b = out["fp32_k8_thick"], out["fp64_k1"]
    pairs = [i for i in range(5) if t["residual_mev"][i] <= 1e-3 and b["residual_mev"][i] <= 1e-3]
    d = [abs(t["evals_mev"][i] - b["evals_mev"][i]) for i in pairs]
    t["max_abs_diff_vs_fp64_k1_mev"] = max(d) if d else None
    a = out["fp32_k8"]
    pairs = [i for i in range(5) if a["residual_mev"][i] <= 1e-3 and b["residual_mev"][i] <= 1e-3]
    d = [abs(a["evals_mev"][i] - b["evals_mev"][i]) for i in pairs]
    out["compared_levels"] = pairs
    out["max_abs_diff_mev"] = max(d) if d else None
    out["within_1e-4_mev"] = bool(d) and max(d) <= 1e-4
    out["speedup_fp32_k8_vs_fp64_k1_wall"] = out["fp64_k1"]["ms_total"] / out["fp32_k8"]["ms_total"]
    # against the FP64 oracle's levels (tests/golden/cr48_levels.txt, written by
    # the oracle alone): every converged level of each GPU run
    gold = os.path.join(ROOT, "tests", "golden", "cr48_levels.txt")
    if os.path.exists(gold):
        ev_o = [float(l.split()[1]) for l in open(gold) if l.strip() and not l.startswith("#")]
        for name in ("fp64_k1", "fp32_k8", "fp32_k8_thick"):
            r = out[name]
            lv = [i for i in range(5) if r["residual_mev"][i] <= 1e-3]
            d = [abs(r["evals_mev"][i] - ev_o[i]) for i in lv]
            r["vs_oracle_levels"] = lv
            r["max_abs_diff_vs_oracle_mev"] = max(d) if d else None
        a = out["fp32_k8"]
        out["fp32_k8_within_1e-4_mev_of_oracle"] = (a["max_abs_diff_vs_oracle_mev"] is not None and
                                                    a["max_abs_diff_vs_oracle_mev"] <= 1e-4)
    return out


KERNEL_SOURCES = {1: "bs_hx.cu", 2: "bs_hx_row.cu", 3: "bs_hx_row.cu", 4: "bs_hx_row.cu", 5: "bs_hx_row.cu",
                  6: "bs_hx_pipe.cu", 7: "bs_hx_pipe.cu", 8: "bs_hx_pipe.cu", 9: "bs_hx_pipe.cu", 10: "bs_hx_pipe.cu",
                  11: "bs_hx_core.cu", 12: "bs_hx_core.cu", 13: "bs_hx_core.cu", 14: "bs_hx_core.cu",
                  15: "bs_hx_core.cu", 16: "bs_hx_core.cu", 17: "bs_hx_core.cu", 18: "bs_hx_core.cu",
                  19: "bs_hx_core.cu", 20: "bs_hx_core.cu"}
# ncu summaries of the dominant kernel per mode (the pn-core kernel in 11..20)
PROFILES = {1: "hx_fused_pf4p4n_k8.md", 2: "hx_row_pf4p4n_k8.md", 6: "hx_pipe_pf4p4n_k8.md",
            11: "hx_core_pf4p4n_k8.md", 12: "hx_core_pf4p4n_k8.md", 13: "hx_core_pf4p4n_k8.md",
            14: "hx_core_pf4p4n_k8.md", 15: "hx_core_pf4p4n_k8.md", 16: "hx_core_pf4p4n_k8.md",
            17: "hx_core_pf4p4n_k8.md", 18: "hx_core_pf4p4n_k8.md", 19: "hx_core_pf4p4n_k8.md",
            20: "hx_core_pf4p4n_k8.md"}


def launches_per_product(mode):
    """Kernels one H x launches in a kernel mode: the core-grouped modes run the
    pn kernel (and in 13 to 16 and 18 to 20 the pp kernel) and the like-particle
    kernel; the row-tile like-particle kernel of 13 to 16, 19 and 20 also adds the
    partial vectors, the pipelined one of 11, 12, 17 and 18 is followed by the
    ordered sum; every other mode is one kernel."""
    return {11: 3, 12: 3, 13: 3, 14: 3, 15: 3, 16: 3, 17: 3, 18: 4, 19: 3, 20: 3}.get(mode, 1)


def traffic_from_profile(k, mode):
    """DRAM bytes per launch from the committed ncu summary of the kernel mode
    the bench timed, if it was taken on the current kernel source; else None."""
    if mode not in PROFILES:
        return None
    src = os.path.join(ROOT, "paper_1801_08432_gb300", "csrc", KERNEL_SOURCES[mode])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", PROFILES[mode])
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.strip().split()
        # "traffic k=<k> src=<sha> dram_bytes=<n>"
        if len(f) == 4 and f[0] == "traffic" and f[1] == "k=%d" % k and f[2] == "src=" + sha:
            return int(f[3].split("=")[1])
    return None


def fe52_product(N, I, torch, device, mode=18, nrep=3):
    """The largest workload (pf 6p6n M=0, 52Fe, dim 109,954,620) at its block
    size k = 4: set-up (basis, decoupling, tables, upload) timed on the host,
    then one warm-up and nrep timed FP32 block products H X in the
    core-grouped mode the autotuner picks for its wide neutron sectors (the
    pipelined nn kernel after the pp-core kernel), CUDA events around each product and around its
    pn-core kernel.  Reported beside the main line, not part of its value."""
    orbits, spe, tb = I.space("pf")
    t0 = time.time()
    ctx = N.make(orbits, spe, tb, 6, 6, 0, +1, device=device)
    setup_s = time.time() - t0
    dim, k = ctx.dim, 4
    stats = ctx.table("stats", np.int64)
    ctx.set_kernel(mode)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    g = torch.Generator(device="cuda").manual_seed(52)
    x = torch.randn((dim, k), device="cuda", dtype=torch.float32, generator=g)
    y = torch.empty_like(x)
    with torch.cuda.stream(stream):
        ctx.apply_H(x, y, k, N.BS_F32, sp)
    stream.synchronize()
    ctx.time_kernel(nrep)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nrep)]
    for i in range(nrep):
        ev[i][0].record(stream)
        with torch.cuda.stream(stream):
            ctx.apply_H(x, y, k, N.BS_F32, sp)
        ev[i][1].record(stream)
    stream.synchronize()
    ms = [a.elapsed_time(b) for (a, b) in ev]
    kern = [float(t) for t in ctx.kernel_times()]
    ctx.time_kernel(0)
    ctx.sync_status()
    del x, y
    ctx.close()
    torch.cuda.empty_cache()
    hx_ms = float(np.mean(ms))
    kern_ms = float(np.mean(kern))
    return {"workload": "pf shell 6p6n M=0 (52Fe), dim %d, 195 seeded random TBMEs" % dim, "k": k,
            "kernel_mode": mode, "set_up_s": round(setup_s, 1), "products": nrep,
            "hx_ms_per_block_product": round(hx_ms, 2), "vector_matvecs_per_s": k / (hx_ms / 1000.0),
            "pn_core_kernel_ms": round(kern_ms, 2),
            "pn_core_tflops": 2.0 * float(stats[8]) * k / (kern_ms / 1000.0) / 1e12,
            "product_tflops": 2.0 * float(stats[5]) * k / (hx_ms / 1000.0) / 1e12,
            "note": "L2 not flushed: the 1.76 GB vectors exceed it"}


def fe52_run(args):
    """The pf 6p6n space (52Fe, M=0, dim 109,954,620): FP32 block Lanczos with
    k = 4 interleaved vectors, 50 block iterations kept on the device, FP64
    refinement of the 5 lowest pairs.  Its eigenvalues have no feasible
    oracle (the explicit H would be ~1.4 TB): the FP64 residuals are reported
    instead.  One JSON line."""
    import torch
    from paper_1801_08432_gb300 import _native as N
    from paper_1801_08432_gb300 import build as B
    from paper_1801_08432_gb300 import inputs as I

    torch.cuda.set_device(0)
    B.build()
    orbits, spe, tb = I.space("pf")
    t0 = time.time()
    ctx = N.make(orbits, spe, tb, 6, 6, 0, +1, device=0)
    setup_s = time.time() - t0
    dim, k = ctx.dim, 4
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    mode, mode_ms = ctx.autotune(k, N.BS_F32, sp, times=True)
    g = torch.Generator(device="cuda").manual_seed(52)
    x = torch.randn((dim, k), device="cuda", dtype=torch.float32, generator=g)
    y = torch.empty_like(x)
    with torch.cuda.stream(stream):
        for _ in range(2):
            ctx.apply_H(x, y, k, N.BS_F32, sp)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    nrep = 5
    ctx.time_kernel(nrep)
    ev[0].record(stream)
    with torch.cuda.stream(stream):
        for _ in range(nrep):
            ctx.apply_H(x, y, k, N.BS_F32, sp)
    ev[1].record(stream)
    stream.synchronize()
    hx_ms = ev[0].elapsed_time(ev[1]) / nrep
    kern_ms = float(np.mean(ctx.kernel_times()))
    ctx.time_kernel(0)
    del x, y
    torch.cuda.empty_cache()
    stats = ctx.table("stats", np.int64)
    p = torch.from_numpy(I.random_block(dim, k, seed=I.PIVOT_SEED)).to("cuda", torch.float32)
    if args.thick:
        # thick restart: 20 block iterations per cycle, 3 k Ritz vectors kept,
        # until the residual estimates of the lowest five are <= 1e-3 MeV
        ev5, rep = ctx.lanczos(p, k, N.BS_F32, 20, 5, refine=True, stream=sp, nthick=3 * k,
                               max_restarts=args.thick, tol=1e-3)
    else:
        ev5, rep = ctx.lanczos(p, k, N.BS_F32, 50, 5, refine=True, stream=sp)
    nit = rep["iterations"]
    rb = (reorth_bytes_thick(dim, k, 4, 20, 3, rep["restarts"], 2) if args.thick else
          reorth_bytes(dim, k, 4, nit, 2))
    hbm_gbs = (peaks() or {}).get("hbm_gbs", 6800.0)
    line = {"workload": "pf shell 6p6n M=0 (52Fe), dim %d, 195 seeded random TBMEs" % dim, "k": k,
            "set_up_s": round(setup_s, 1), "kernel_mode": mode, "ms_per_mode_f32": mode_ms,
            "hx_ms_per_block_product": round(hx_ms, 2), "vector_matvecs_per_s": k / (hx_ms / 1000.0),
            "dominant_kernel_ms": round(kern_ms, 2),
            "dominant_kernel_tflops": 2.0 * float(stats[8]) * k / (kern_ms / 1000.0) / 1e12,
            "lanczos": {"block_iterations": nit, "ms_total": round(rep["ms_total"], 1),
                        "ms_matvec": round(rep["ms_matvec"], 1), "ms_reorth_alpha_gram": round(rep["ms_reorth"], 1),
                        "reorth_alg_bytes": rb, "reorth_gbs": round(rb / (rep["ms_reorth"] / 1000.0) / 1e9, 1),
                        "reorth_hbm_frac": round(rb / (rep["ms_reorth"] / 1000.0) / 1e9 / hbm_gbs, 3),
                        "evals_mev": [round(float(e), 6) for e in ev5], "residual_mev": rep["residual"],
                        "delta_conv": rep["delta_conv"], "restarts": rep["restarts"],
                        "block_products": rep["matvec_blocks"], "resid_est_mev": rep["resid_est"],
                        "stored_blocks": (20 + 1 + 3) if args.thick else 51}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def ours(args):
    import torch
    from paper_1801_08432_gb300 import _native as N
    from paper_1801_08432_gb300 import build as B
    from paper_1801_08432_gb300 import inputs as I

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    orbits, spe, tb = I.space(WORKLOAD["space"])
    t0 = time.time()
    ctx = N.make(orbits, spe, tb, WORKLOAD["Z"], WORKLOAD["N"], WORKLOAD["twoM"], WORKLOAD["parity"], device=local)
    setup_s = time.time() - t0
    dim = ctx.dim
    stats = ctx.table("stats", np.int64)
    ops = float(stats[5])
    tbytes = 0
    for name, sz in (("pp_src", 4), ("pp_coef", 8), ("nn_src", 4), ("nn_coef", 8), ("p1_ent", 4), ("n1_ent", 4),
                     ("p1_ptr", 8), ("n1_ptr", 8), ("pp_ptr", 8), ("nn_ptr", 8), ("wpn", 8)):
        n = len(ctx.table(name, np.uint8))
        tbytes += n if sz != 8 or not name.endswith(("coef", "wpn")) else n // 2   # FP32 coefficients
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def bar():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(k, dtype, steps, warmup, kernel_events=False):
        tdt = torch.float32 if dtype == N.BS_F32 else torch.float64
        g = torch.Generator(device="cuda").manual_seed(1234 + k)
        x = torch.randn((dim, k), device="cuda", dtype=tdt, generator=g)
        y = torch.empty_like(x)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                ctx.apply_H(x, y, k, dtype, sp)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if kernel_events:
            ctx.time_kernel(steps)    # events around the dominant kernel, on the launching stream
        bar()
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()                        # > L2: the next launch starts cold
                ev[i][0].record(stream)
                ctx.apply_H(x, y, k, dtype, sp)
                ev[i][1].record(stream)
        stream.synchronize()
        bar()
        ms = [a.elapsed_time(b) for (a, b) in ev]
        if kernel_events:
            timed.kernel_ms = [float(t) for t in ctx.kernel_times()]
            ctx.time_kernel(0)
        return ms, x, y

    # autotune: kernel variant per (k, dtype) in the library, then k here
    tune = {}
    modes = {}
    mode_ms = {}
    if args.mode:
        ctx.set_kernel(args.mode)
    if args.profile_lanczos:
        # only an FP32 block Lanczos of that many block iterations (for ncu of the reorthogonalization kernels)
        k = args.k or 8
        if args.mode:
            ctx.set_kernel(args.mode)
        p = torch.from_numpy(I.random_block(dim, k, seed=I.PIVOT_SEED)).to("cuda", torch.float32)
        ev, rep = ctx.lanczos(p, k, N.BS_F32, args.profile_lanczos, 5, refine=False, stream=sp)
        rb = reorth_bytes(dim, k, 4, rep["iterations"], 2)
        if rank == 0:
            print(json.dumps({"profile_lanczos": True, "k": k, "iterations": rep["iterations"],
                              "ms_reorth_alpha_gram": rep["ms_reorth"], "ms_matvec": rep["ms_matvec"],
                              "reorth_gbs": rb / (rep["ms_reorth"] / 1000.0) / 1e9}), flush=True)
        ctx.close()
        return 0
    if args.profile_only:
        # a fixed kernel mode and k, warm-up launches then the timed ones, nothing else (for ncu)
        ms, _, _ = timed(args.k or 8, N.BS_F32, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"profile_only": True, "mode": args.mode, "k": args.k or 8, "ms": ms}), flush=True)
        ctx.close()
        return 0
    if args.tune_load:
        # replay a recorded tuning: the same kernel choices, no timing (so that a
        # profiled run, whose serialized launches would skew the autotuner, runs
        # the kernels the plain run chose)
        rec = json.load(open(args.tune_load))
        kbest = int(rec["kbest"])
        modes = {int(k): int(m) for k, m in rec["f32"].items()}
        mode_ms = {int(k): v for k, v in rec["ms_per_mode_f32"].items()}
        tune = {int(k): v for k, v in rec["autotune_k"].items()}
        mode64, ms64modes = int(rec["f64_k1"]), rec["ms_per_mode_f64_k1"]
        for k, m in modes.items():
            ctx.set_tuned(k, N.BS_F32, m)
        ctx.set_tuned(1, N.BS_F64, mode64)
    else:
        if args.k:
            kbest = args.k
            modes[kbest], mode_ms[kbest] = ctx.autotune(kbest, N.BS_F32, sp, times=True)
            if args.mode:
                ctx.set_kernel(args.mode)
        else:
            for k in (1, 2, 4, 8):
                modes[k], mode_ms[k] = ctx.autotune(k, N.BS_F32, sp, times=True)
                ms, _, _ = timed(k, N.BS_F32, 3, 2)
                tune[k] = k / (min(ms) / 1000.0)
            kbest = max(tune, key=tune.get)
        mode64, ms64modes = ctx.autotune(1, N.BS_F64, sp, times=True)
    if args.tune_save and rank == 0:
        json.dump({"workload": WORKLOAD_NAME, "kbest": kbest, "f32": modes, "ms_per_mode_f32": mode_ms,
                   "autotune_k": tune, "f64_k1": mode64, "ms_per_mode_f64_k1": ms64modes},
                  open(args.tune_save, "w"), indent=1)

    sampler = ClockSampler(local)
    sampler.start()
    ms32, _, _ = timed(kbest, N.BS_F32, args.steps, args.warmup, kernel_events=True)
    clocks = sampler.stop()
    kern_ms = timed.kernel_ms
    ms64, _, _ = timed(1, N.BS_F64, max(3, args.steps // 2), max(3, args.warmup))

    # end to end through the host-buffer call: pinned host input, H*X, result back;
    # at least 80 calls, so that the two-slot pipeline's fill and drain (one copy in,
    # one copy out) are a small part of the timed region
    n_e2e = max(args.steps, 80)
    xh = torch.randn((dim, kbest), dtype=torch.float32).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xa = xh.numpy()
    ya = yh.numpy()
    for _ in range(2):
        ctx.apply_H_host(xa, ya, kbest, N.BS_F32, sp)
    bar()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ctx.apply_H_host(xa, ya, kbest, N.BS_F32, sp)
    bar()
    e2e_s = time.perf_counter() - t0
    # the same through the asynchronous host-buffer call: two streams and two staging
    # slots, so that one step's copies in and out run while the other's product does
    # (every step still copies its input block in and its result block out)
    xs = [xh, torch.randn((dim, kbest), dtype=torch.float32).pin_memory()]
    ys = [yh, torch.empty_like(xh).pin_memory()]
    sts = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i in range(4):
        ctx.apply_H_host_async(xs[i % 2], ys[i % 2], kbest, N.BS_F32, sts[i % 2].cuda_stream, i % 2)
    for st in sts:
        st.synchronize()
    bar()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        ctx.apply_H_host_async(xs[i % 2], ys[i % 2], kbest, N.BS_F32, sts[i % 2].cuda_stream, i % 2)
    for st in sts:
        st.synchronize()
    bar()
    e2e_pipe_s = time.perf_counter() - t0

    t_ms = float(np.sum(ms32))
    t_max, e2e_max, e2e_pipe_max = aggregate_max([t_ms, e2e_s, e2e_pipe_s], dist)
    value = world * args.steps * kbest / (t_max / 1000.0)
    avg_launch_s = t_ms / args.steps / 1000.0
    fp64_rate = 1.0 / (float(np.mean(ms64)) / 1000.0)
    fp32_rate_single = kbest / avg_launch_s
    pk = peaks()
    sm_mhz_max = (pk or {}).get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_mhz_max * 1e6 / 1e12       # TFLOP/s, FMA = 2 FLOP
    mode_used = args.mode or modes.get(kbest, 0)
    core = 11 <= mode_used <= 20
    # dominant kernel: the pn-core kernel of the core-grouped modes (its own
    # multiply-adds), else the one kernel of the product (all of them)
    dom_ops = float(stats[8]) if core else ops
    flops = 2.0 * dom_ops * kbest
    dom_s = float(np.mean(kern_ms)) / 1000.0
    achieved = flops / dom_s / 1e12
    alg_bytes = 2.0 * dim * kbest * 4 + tbytes
    hbm_peak = (pk or {}).get("hbm_gbs", 6800.0)
    traffic = traffic_from_profile(kbest, args.mode or modes.get(kbest, 0))
    # measured on-chip ceiling of the product's inner step (bs_gather_ceiling:
    # random k-float gathers from shared memory or L2, each applied to 1, 2
    # or 4 rows by packed FP32 FMAs), outside the timed region
    ceil = {}
    if kbest in (4, 8):
        for where, name in ((0, "smem"), (1, "l2")):
            for rows in (1, 2, 4):
                ceil["ceil_%s_rows%d" % (name, rows)] = ctx.gather_ceiling(where, kbest, rows, sp) / 1e3
    gathers = float(stats[11]) if len(stats) > 11 else 0.0
    rpg = float(stats[8]) / gathers if core and gathers > 0 else None
    if rpg is not None and ceil:
        # linear in the rows between the measured 1-, 2- and 4-row rates
        lo, hi = (1, 2) if rpg <= 2 else (2, 4)
        c_lo, c_hi = ceil["ceil_smem_rows%d" % lo], ceil["ceil_smem_rows%d" % hi]
        ceiling = c_lo + (min(rpg, 4.0) - lo) / (hi - lo) * (c_hi - c_lo)
        peak, peak_note = ceiling, ("measured shared-memory gather + FMA ceiling (bs_gather_ceiling, k = %d) at the "
                                    "kernel's %.3f rows per gathered element, between the measured %d- and %d-row "
                                    "rates" % (kbest, rpg, lo, hi))
    else:
        peak, peak_note = fp32_peak, "FP32 FMA issue (derived)"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "k": kbest, "kernel_mode": mode_used,
                   "path": "FP32-mixed block H*X (core-grouped kernels)" if core else "FP32-mixed block H*X (one kernel)",
                   "l2": "flushed: 256 MB write before every timed launch", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "set_up_s": round(setup_s, 2)},
        "roofline": dict({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                          "frac": achieved / peak, "traffic": traffic,
                          "kernel": "hx_core_kernel (pn term by proton cores)" if core else "the single H x kernel",
                          "kernel_ms": dom_s * 1000.0, "flop_per_launch": flops, "peak_note": peak_note,
                          "rows_per_gather": rpg,
                          "fma_issue_peak": fp32_peak, "frac_fma_issue": achieved / fp32_peak,
                          "fma_issue_note": "FP32 FMA issue: %d SMs x 128 lanes x 2 FLOP x %.0f MHz (derived, not "
                                            "measured)" % (nsm, sm_mhz_max),
                          "product_flop": 2.0 * ops * kbest, "product_ms": avg_launch_s * 1000.0,
                          "product_tflops": 2.0 * ops * kbest / avg_launch_s / 1e12,
                          "product_launches": launches_per_product(mode_used)}, **ceil),
        "hbm": {"algorithmic_bytes_per_launch": alg_bytes, "gbs": alg_bytes / avg_launch_s / 1e9,
                "peak_gbs": hbm_peak, "frac": alg_bytes / avg_launch_s / 1e9 / hbm_peak,
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)" if pk else "fallback"},
        "fp64_single_vector": {"value": fp64_rate, "unit": UNIT, "ms_per_matvec": float(np.mean(ms64))},
        "speedup_fp32_block_vs_fp64": fp32_rate_single / fp64_rate,
        "autotune_k": {str(k): v for k, v in tune.items()},
        "kernel_mode": {"f32": {str(k): m for k, m in modes.items()}, "f64_k1": mode64,
                        "ms_per_mode_f32": {str(k): v for k, v in mode_ms.items()}, "ms_per_mode_f64_k1": ms64modes},
        "e2e": {"value": world * n_e2e * kbest / e2e_pipe_max, "unit": UNIT,
                "h2d_bytes_per_step": dim * kbest * 4, "d2h_bytes_per_step": dim * kbest * 4,
                "steps": n_e2e,
                "call": "bs_apply_H_host_async on two streams and two staging slots (pinned host buffers)",
                "value_synchronous": world * n_e2e * kbest / e2e_max,
                "call_synchronous": "bs_apply_H_host, which returns after its copy out"},
        "gpu_launches": args.steps * launches_per_product(mode_used),
        "clocks": clocks,
    }
    if not args.no_lanczos:
        line["lanczos"] = lanczos_check(ctx, N, I, torch, sp)
    ctx.close()
    if not args.no_fe52 and rank == 0:
        line["fe52"] = fe52_product(N, I, torch, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--k", type=int, default=0, help="fix k instead of autotuning it")
    ap.add_argument("--no-lanczos", action="store_true", help="skip the Lanczos accuracy check")
    ap.add_argument("--no-fe52", action="store_true", help="skip the pf 6p6n (52Fe) product key")
    ap.add_argument("--mode", type=int, default=0, help="fix the H x kernel mode (bs_set_kernel) instead of autotuning")
    ap.add_argument("--profile-only", action="store_true", help="only the FP32 H*X launches (for ncu)")
    ap.add_argument("--fe52", action="store_true", help="only the pf 6p6n (52Fe) block Lanczos, k = 4, 50 iterations")
    ap.add_argument("--thick", type=int, default=0,
                    help="with --fe52: thick-restart block Lanczos with at most this many restarts")
    ap.add_argument("--tune-save", default="", help="write the autotuned kernel modes and k to this JSON file")
    ap.add_argument("--tune-load", default="", help="replay kernel modes and k from a --tune-save file instead of autotuning")
    ap.add_argument("--profile-lanczos", type=int, default=0,
                    help="only an FP32 block Lanczos of this many block iterations (for ncu)")
    ap.add_argument("--cpu-lanczos", type=int, default=0,
                    help="only the oracle's full FP64 run on the host: build H, then this many Lanczos iterations")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.cpu_lanczos:
        return cpu_lanczos(args)
    if args.fe52:
        return fe52_run(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
