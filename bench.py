#!/usr/bin/env python
"""Benchmark of the BOBA hot path on the GB300.

One step = one pass of the whole path over one synthetic graph resident in HBM:
BOBA reorder (key init, first occurrence, rank, relabel), then the COO->CSR
build of the reordered graph and ``--spmv-iters`` SpMV products y = A x.

Printed (rank 0, one JSON line):
  value        reorder throughput, Gedges/s = m / (device time of the reorder
               phase), summed over all ranks (each rank reorders its own copy)
  ms_per_step  device time of the whole step (reorder + CSR + SpMV)
  e2e          the same metric through the public API with the inputs in
               pinned host memory: H2D of src/dst, reorder, D2H of perm and
               the relabelled edges, all inside the timed region
  roofline     the step's dominant kernel: algorithmic bytes per launch over
               its mean event-timed duration, against the measured HBM copy
               bandwidth
  cpu_baseline the CPU oracle (single-threaded C) on a bounded sample
  spmv_error   relative L2 error of the timed fp32 SpMV against the fp64
               oracle product, on the BOBA and the random order (the oracle
               runs in spawned worker processes beside the GPU-only legs, on
               the synthetic input, never on anything the GPU produced)
  perm_only    the permutation alone (no edge rewrite), the figure the
               paper times
  configs2     the low-skew workloads (4096^2 grid, Erdos-Renyi 2^24 / 2^27)
  latency      the R-MAT scale-14 graph (L2-resident): one reorder's latency
  gather_ceiling  random 4-byte loads per second from global, shared and
               cluster-distributed shared memory, the ceiling of the two
               lookup passes of the reorder

``--impl reference`` times the CPU oracle instead (the method has no other
implementation to run), on the same workload, metric and unit.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("BOBA reorder Gedges/s + % HBM roofline (plain vs batched); "
          "SpMV GB/s BOBA vs random")
# The paper's own reorder times (Sec. 1.2.4, Sec. 5.3, Table 2), on an NVIDIA
# V100 32 GB with CUDA 11.6; the paper times the permutation only.  Context
# beside `perm_only`, not a target (other hardware, other inputs).
PAPER_REPORTED = {
    "hardware": "NVIDIA V100 32 GB (80 SMs), CUDA 11.6",
    "what": "BOBA permutation (no edge rewrite), the datasets' native edge order",
    "kron_g500-logn20": {"edges": 89_000_000, "ms": 17.0, "gedges_s": 5.2},
    "arabic-2005": {"edges": 639_900_000, "ms": 224.0, "gedges_s": 2.9},
}
FALLBACK_HBM_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0          # GB300 HBM3e nominal, reported beside the measured peak
L2_FLUSH_BYTES = 512 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_info():
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model, os.cpu_count() or 1


# ---------------------------------------------------------------------------
# algorithmic (compulsory) bytes per launch of each kernel
# ---------------------------------------------------------------------------

def algorithmic_bytes(m: int, n: int, nnz: int):
    """Bytes each kernel must move to or from HBM at the least.

    Arrays of n (or 2m-bit) words that fit in L2 between kernels are still
    counted once where they are produced or consumed for the first time.
    """
    bitmap = (2 * m + 7) // 8
    bits = max(1, (n - 1).bit_length())
    passes = (bits + 7) // 8
    # radix passes: keys and values in and out (16m); the last one writes no
    # keys but val and the row ends (12m + 4n); mean over the passes of a build
    pass_mean = ((passes - 1) * 16 * m + 12 * m + 4 * n) / passes if passes > 1 else 16 * m
    return {
        "reorder.init": 4 * n + bitmap,            # write key, clear bitmap
        "reorder.first": 8 * m + 4 * n,            # stream I ++ J, final keys
        "reorder.mark": 4 * n + bitmap,            # read keys, bitmap
        "reorder.scan": bitmap + bitmap // 8,      # read bitmap, write group prefix
        "reorder.emit": 4 * n + 4 * n + 4 * n,     # keys in, label + perm out
        "reorder.relabel": 16 * m + 4 * n,         # src,dst in; src_out,dst_out out; label
        "csr.hist": 4 * m,                         # read dst (outdeg is counted in pass 0)
        "csr.pass": int(pass_mean),
        "spmv": 8 * nnz + 16 * n,
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.uuid = device_uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# fp64 oracle products, computed in spawned worker processes
# ---------------------------------------------------------------------------

def oracle_y(workload_name, order):
    """y = A x in fp64 by the oracle for a workload in `order` ("boba": the
    oracle's own BOBA relabelling of the synthetic input; "random": the input
    order), with the x the bench uses.  Runs in a worker process; only synth/
    and oracle/ are used."""
    import synth
    import oracle
    w = synth.WORKLOADS[workload_name]
    I, J = w.generate()
    if order == "boba":
        _, I, J = oracle.reorder(I, J, w.n)
    rp, col, val = oracle.coo_to_csr(I, J, w.n)
    del I, J
    x = synth.uniform_f32(w.n, seed=w.seed)
    return oracle.spmv_f64(rp, col, val, x)


def start_oracle_jobs(names, workers=4):
    """Start the oracle products for `names` x (boba, random) in spawned
    processes (spawned, not forked, so starting them after CUDA use is safe)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    futs = {(nm, o): ex.submit(oracle_y, nm, o) for nm in names for o in ("boba", "random")}
    return ex, futs


def rel_l2(y32, y64):
    y32 = np.asarray(y32, dtype=np.float64)
    nrm = float(np.linalg.norm(y64))
    return float(np.linalg.norm(y32 - y64) / nrm) if nrm > 0 else float(np.linalg.norm(y32))


def spmv_errors(futs, name, ys, timeout=900):
    """{order: rel-L2 of the GPU y against the oracle} for the orders in ys."""
    out = {}
    for order, y in ys.items():
        f = futs.get((name, order)) if futs else None
        if f is None or y is None:
            out[order] = None
            continue
        try:
            out[order] = round(rel_l2(y, f.result(timeout=timeout)), 10)
        except Exception as exc:                     # report, do not hide
            out[order] = "oracle failed: " + str(exc)[:120]
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import synth
    import paper_2306_10410_gb300 as boba
    from paper_2306_10410_gb300 import build as bb

    world, rank, local = dist_env()
    w = synth.WORKLOADS[args.workload]
    # the oracle's fp64 products run in spawned worker processes beside the
    # GPU-only legs; they start after the host-buffer (e2e) leg, whose copies
    # they would slow down through the host's memory
    oracle_names = []
    if args.spmv_error and rank == 0 and args.spmv_iters > 0:
        oracle_names.append(w.name)
        if args.configs2 and world == 1:
            oracle_names += [synth.GRID4096.name, synth.ER24.name]
    oracle_ex, oracle_futs = None, {}
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    bb.build()
    boba.load()

    m, n = w.m, w.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # inputs: generated on the host into pinned memory, then made resident in HBM
    src_h = torch.empty(m, dtype=torch.int32, pin_memory=True)
    dst_h = torch.empty(m, dtype=torch.int32, pin_memory=True)
    w.generate(out=(src_h.numpy(), dst_h.numpy()))
    src = src_h.to(dev)
    dst = dst_h.to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    label = torch.empty(n, dtype=torch.int32, device=dev)
    so = torch.empty(m, dtype=torch.int32, device=dev)
    do = torch.empty(m, dtype=torch.int32, device=dev)
    ws_r = torch.empty(boba.boba_reorder_workspace_bytes(m, n), dtype=torch.uint8, device=dev)

    have_csr = boba.boba_coo_to_csr_workspace_bytes(m, n) > 0
    if have_csr:
        row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        col = torch.empty(m, dtype=torch.int32, device=dev)
        val = torch.empty(m, dtype=torch.float32, device=dev)
        ws_c = torch.empty(boba.boba_coo_to_csr_workspace_bytes(m, n), dtype=torch.uint8,
                           device=dev)
        ws_s = torch.empty(max(256, boba.boba_spmv_workspace_bytes(n, m)), dtype=torch.uint8,
                           device=dev)
        x = torch.from_numpy(synth.uniform_f32(n, seed=w.seed)).to(dev)
        y = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def reorder():
        boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, label, ws_r,
                                        ws_r.numel(), stream), "reorder")

    def csr():
        boba.check(boba.boba_coo_to_csr(so, do, m, n, row_ptr, col, val, ws_c, ws_c.numel(),
                                        stream), "csr")

    def spmv():
        boba.check(boba.boba_spmv_csr(row_ptr, col, val, x, y, n, m, ws_s, ws_s.numel(),
                                      stream), "spmv")

    def step(ev):
        ev[0].record(stream)
        reorder()
        ev[1].record(stream)
        if have_csr:
            csr()
            ev[2].record(stream)
            for _ in range(args.spmv_iters):
                spmv()
        ev[3].record(stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    tuning = None
    if args.tune_spec:
        # fixed variants (reproducible profiling): "first=5,relabel=3,spmv=5"
        fam = {"first": boba.TUNE_FIRST, "relabel": boba.TUNE_RELABEL, "spmv": boba.TUNE_SPMV,
               "csr": boba.TUNE_CSR}
        tuning = {}
        for item in args.tune_spec.split(","):
            k, v = item.split("=")
            size = m
            boba.load().boba_tune_set(fam[k], size, int(v))
            tuning[k] = int(v)
    elif args.tune:
        # autotune launch shapes on this workload (every variant checked bit-identical)
        tuning = boba.tune_reorder(src, dst, n, reps=3)
        if have_csr:
            reorder()
            tuning.update(boba.tune_csr(so, do, n, reps=2))
            csr()
            tuning.update(boba.tune_spmv(row_ptr, col, val, x, reps=3))
        boba.stream_status(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    boba.stream_status(stream)

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None)
    sampler.start()
    time.sleep(0.3)
    evs = []
    barrier()
    with boba.kernel_timing() as kt:
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush between steps (not timed)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            step(ev)
            evs.append(ev)
        barrier()
    clocks = sampler.stop()
    boba.stream_status(stream)
    # the last product of the last step: the timed SpMV on the BOBA order
    y_boba = y.cpu().numpy() if have_csr and args.spmv_iters > 0 else None

    # the permutation alone (src_out = dst_out = NULL): what the paper times
    t_perm = []
    for _ in range(max(3, min(args.steps, 5)) + 1):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, None, None, label, ws_r,
                                        ws_r.numel(), stream), "reorder (perm only)")
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        t_perm.append(ev[0].elapsed_time(ev[1]))
    boba.stream_status(stream)
    perm_ms = statistics.median(t_perm[1:])

    t_reorder = [e[0].elapsed_time(e[1]) for e in evs]
    t_step = [e[0].elapsed_time(e[3]) for e in evs]
    t_csr = [e[1].elapsed_time(e[2]) for e in evs] if have_csr else []
    t_spmv = [e[2].elapsed_time(e[3]) for e in evs] if have_csr else []
    reorder_ms = sum(t_reorder) / len(t_reorder)
    step_ms = sum(t_step) / len(t_step)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([reorder_ms, step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        reorder_ms, step_ms = t.tolist()
    value = world * m / (reorder_ms * 1e-3) / 1e9

    # per-kernel roofline
    hbm, peak_kind = peaks()
    alg = algorithmic_bytes(m, n, m)
    kern = {}
    for name, (tot_ms, launches) in kt.result.items():
        mean_ms = tot_ms / max(1, launches)
        a = alg.get(name)
        gbs = (a / (mean_ms * 1e-3) / 1e9) if a else None
        kern[name] = {"launches": launches, "mean_ms": round(mean_ms, 5),
                      "share": None, "alg_bytes": a,
                      "achieved_gbs": round(gbs, 1) if gbs else None,
                      "frac": round(gbs / hbm, 4) if gbs else None}
    tot_all = sum(v[0] for v in kt.result.values())
    for name, (tot_ms, _) in kt.result.items():
        kern[name]["share"] = round(tot_ms / tot_all, 4) if tot_all else None
    dom = max(kt.result.items(), key=lambda kv: kv[1][0])[0] if kt.result else None
    launches = sum(v[1] for v in kt.result.values())
    traffic = load_traffic(dom, args.workload)
    roof = None
    if dom and kern[dom]["achieved_gbs"]:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["achieved_gbs"],
                "peak": hbm, "unit": "GB/s", "frac": kern[dom]["frac"], "traffic": traffic,
                "peak_source": peak_kind, "peak_nominal": HBM_NOMINAL_GBS,
                "frac_nominal": round(kern[dom]["achieved_gbs"] / HBM_NOMINAL_GBS, 4)}
    # end-to-end through the public API with host buffers
    e2e = None if args.no_e2e else run_e2e(args, boba, torch, dev, stream, src_h, dst_h, m, n,
                                           world)
    if oracle_names:
        oracle_ex, oracle_futs = start_oracle_jobs(oracle_names)

    # SpMV and CSR on the BOBA order vs the random (input) order, same kernels
    compare = None
    y_random = None
    if have_csr:
        compare = compare_orders(args, boba, torch, dev, stream, src, dst, so, do, m, n,
                                 row_ptr, col, val, ws_c, ws_s, x, y, flush)
        y_random = compare.pop("_y_random", None)
    if compare is not None:
        # the whole pipeline on each order (Sec. 5.6): what a user pays to go
        # from the edge list to spmv_iters products, and how many products it
        # takes for the reorder to pay for itself
        r, o, it = compare["random"], compare["boba"], args.spmv_iters
        gain = r["spmv_ms"] - o["spmv_ms"]
        compare["pipeline"] = {
            "spmv_iters": it,
            "random_csr_spmv_ms": round(r["csr_ms"] + it * r["spmv_ms"], 3),
            "boba_reorder_csr_spmv_ms": round(reorder_ms + o["csr_ms"] + it * o["spmv_ms"], 3),
            "break_even_spmv_iters": (round((reorder_ms + o["csr_ms"] - r["csr_ms"]) / gain, 1)
                                      if gain > 0 else None)}
    full = 24 * m + 4 * n
    reorder_traffic = reorder_dram_traffic(args.workload, m, n)
    reorder_roof = {"alg_bytes": full, "achieved_gbs": round(full / (reorder_ms * 1e-3) / 1e9, 1),
                    "frac": round(full / (reorder_ms * 1e-3) / 1e9 / hbm, 4),
                    "frac_nominal": round(full / (reorder_ms * 1e-3) / 1e9 / HBM_NOMINAL_GBS, 4),
                    "peak": hbm, "peak_source": peak_kind, "traffic": reorder_traffic}
    perm_bytes = 8 * m + 4 * n
    perm_only = {"ms": round(perm_ms, 4), "gedges_s": round(m / (perm_ms * 1e-3) / 1e9, 3),
                 "alg_bytes": perm_bytes,
                 "achieved_gbs": round(perm_bytes / (perm_ms * 1e-3) / 1e9, 1),
                 "frac": round(perm_bytes / (perm_ms * 1e-3) / 1e9 / hbm, 4),
                 "frac_nominal": round(perm_bytes / (perm_ms * 1e-3) / 1e9 / HBM_NOMINAL_GBS, 4)}
    target = {"reorder_frac_of_hbm": 0.60, "reorder_frac": reorder_roof["frac"],
              "met": bool(reorder_roof["frac"] >= 0.60),
              "note": "the reorder looks up one entry of an n-sized array per endpoint twice "
                      "(key, then label); see gather_ceiling for the rate those lookups allow"}

    variants = None
    if args.tune and not args.tune_spec and world == 1:
        variants = time_reorder_variants(boba, torch, dev, stream, flush, src, dst, m, n, perm,
                                         so, do, ws_r, tuning)
    gather = None
    if args.gather and world == 1:
        gather = run_gather_probe(args, boba, torch, dev, stream, reorder_ms, m, kt.result)
    latency = None
    if args.latency and world == 1:
        latency = run_latency(args, boba, torch, dev, stream)
    configs2 = None
    if args.configs2 and world == 1:
        configs2 = run_configs2(args, boba, torch, dev, stream, flush, oracle_futs)
    # the unit that binds the dominant kernel, measured: its random loads
    # against the probe's ceiling (see gather_ceiling / lookup_roofline)
    if roof is not None and gather and (gather.get("lookups_frac_of_ceiling") or {}).get(dom):
        roof["limiter"] = {"unit": "L1TEX-to-crossbar request port (random loads that miss L1)",
                           "frac_of_measured_ceiling": gather["lookups_frac_of_ceiling"][dom]}
    spmv_err = None
    if oracle_futs:
        spmv_err = spmv_errors(oracle_futs, w.name, {"boba": y_boba, "random": y_random})
        spmv_err["bound"] = 1e-5
        spmv_err["kernel"] = f"tuned SpMV variant {(tuning or {}).get('spmv', 0)} (the timed one)"

    if oracle_ex is not None:
        oracle_ex.shutdown(wait=True, cancel_futures=True)
        oracle_ex = None

    serving = None
    if args.serve and world == 1:
        from paper_2306_10410_gb300 import serve as sv
        req_pool = sv.request_pool(args.serve_pool, 0xB0BA0004)
        serving = sv.serve_workload(n_requests=args.serve_requests, load=0.8,
                                    budget_bytes=120 << 30, spmv_iters=10, pool=req_pool)
        serving = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in serving.items()}
        serving["workload"] = ("Poisson stream of BOBA + CSR + 10x SpMV requests, R-MAT or grid, "
                               "m log-uniform in [1e4, 1e8], offered load 0.8, HBM budget 120 GB")
        # saturation (every request submitted at once) against the same list run
        # one request at a time through the per-graph entry points, same outputs;
        # three alternating pairs, the median of the paired ratios reported
        cmp_ = sv.serve_vs_sequential(n_requests=2 * args.serve_pool, budget_bytes=120 << 30,
                                      spmv_iters=10, pool=req_pool)
        del req_pool

        def rnd(d):
            return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}
        serving["saturated"] = rnd(cmp_["saturated"])
        serving["sequential"] = rnd(cmp_["sequential"])
        serving["saturated_gedges_s"] = round(cmp_["saturated"]["gedges_s_wall"], 4)
        serving["sequential_gedges_s"] = round(cmp_["sequential"]["gedges_s_wall"], 4)
        serving["speedup_served_vs_sequential"] = round(cmp_["speedup_served_vs_sequential"], 3)
        serving["comparison_rounds_gedges_s"] = {
            k: [round(v, 4) for v in vs] for k, vs in cmp_["rounds_gedges_s"].items()}
        serving["identical"] = cmp_["identical"]
        serving["saturated_requests"] = cmp_["n_requests"]

    batched = None
    if args.batched and world == 1:
        del src_h, dst_h
        batched = run_batched(args, boba, torch, dev, stream, flush, n_batch=args.batch_graphs)

    result = {
        "metric": METRIC, "value": round(value, 3),
        "value_hbm_frac": reorder_roof["frac"], "unit": "Gedges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": w.name, "m": m, "n": n, "kind": w.kind, "seed": w.seed,
                   "spmv_iters": args.spmv_iters if have_csr else 0,
                   "l2": "flushed between steps (512 MiB write); inputs 8m bytes > L2",
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"reorder": round(reorder_ms, 4),
                      "csr": round(statistics.mean(t_csr), 4) if t_csr else None,
                      "spmv_total": round(statistics.mean(t_spmv), 4) if t_spmv else None},
        "reorder_roofline": reorder_roof,
        "target": target,
        "perm_only": perm_only,
        "paper_reported": PAPER_REPORTED,
        "spmv_rel_l2_vs_fp64": spmv_err,
        "gather_ceiling": gather,
        "lookup_roofline": lookup_roofline(gather),
        "reorder_variants_ms": variants,
        "latency": latency,
        "configs2": configs2,
        "tuning": tuning,
        "orders": compare,
        "roofline": roof,
        "kernels": kern,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def compare_orders(args, boba, torch, dev, stream, src, dst, so, do, m, n, row_ptr, col, val,
                   ws_c, ws_s, x, y, flush):
    """CSR build and SpMV GB/s on the random input order vs the BOBA order (Sec. 5.6)."""
    out = {}
    spmv_bytes = 8 * m + 16 * n
    for name, (s_, d_) in (("random", (src, dst)), ("boba", (so, do))):
        t_csr, t_spmv = [], []
        for rep in range(max(3, min(args.steps, 5)) + 1):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            boba.check(boba.boba_coo_to_csr(s_, d_, m, n, row_ptr, col, val, ws_c, ws_c.numel(),
                                            stream), "csr")
            ev[1].record(stream)
            for _ in range(args.spmv_iters):
                boba.check(boba.boba_spmv_csr(row_ptr, col, val, x, y, n, m, ws_s, ws_s.numel(),
                                              stream), "spmv")
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            if rep:                                  # first repetition is warm-up
                t_csr.append(ev[0].elapsed_time(ev[1]))
                t_spmv.append(ev[1].elapsed_time(ev[2]) / max(1, args.spmv_iters))
        boba.stream_status(stream)
        if name == "random" and args.spmv_iters > 0:
            out["_y_random"] = y.cpu().numpy()         # the timed kernel's product
        ms = statistics.median(t_spmv)
        out[name] = {"csr_ms": round(statistics.median(t_csr), 4), "spmv_ms": round(ms, 4),
                     "spmv_gbs": round(spmv_bytes / (ms * 1e-3) / 1e9, 1)}
    out["spmv_speedup_boba_vs_random"] = round(out["random"]["spmv_ms"] / out["boba"]["spmv_ms"], 3)
    # Sec. 5.6: sort (or bin) the randomly ordered edges by destination, then BOBA
    s2, d2 = torch.empty_like(src), torch.empty_like(dst)
    s3, d3 = torch.empty_like(src), torch.empty_like(dst)
    perm2 = torch.empty(n, dtype=torch.int32, device=dev)
    ws_sort = torch.empty(boba.boba_sort_by_dst_workspace_bytes(m, n), dtype=torch.uint8,
                          device=dev)
    ws_r2 = torch.empty(boba.boba_reorder_workspace_bytes(m, n), dtype=torch.uint8, device=dev)
    for name, top in (("boba_dst_sorted", 0), ("boba_dst_binned", 1)):
        ts, tr, tsp = [], [], []
        for rep in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            flush.zero_()
            ev[0].record(stream)
            boba.check(boba.boba_sort_by_dst(src, dst, m, n, s2, d2, top, ws_sort,
                                             ws_sort.numel(), stream), "sort")
            ev[1].record(stream)
            boba.check(boba.boba_reorder_ex(s2, d2, m, n, perm2, s3, d3, None, ws_r2,
                                            ws_r2.numel(), stream), "reorder")
            ev[2].record(stream)
            boba.check(boba.boba_coo_to_csr(s3, d3, m, n, row_ptr, col, val, ws_c, ws_c.numel(),
                                            stream), "csr")
            for _ in range(args.spmv_iters):
                boba.check(boba.boba_spmv_csr(row_ptr, col, val, x, y, n, m, ws_s, ws_s.numel(),
                                              stream), "spmv")
            ev[3].record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                ts.append(ev[0].elapsed_time(ev[1]))
                tr.append(ev[1].elapsed_time(ev[2]))
                tsp.append(ev[2].elapsed_time(ev[3]))
        v, _ = boba.nbr(row_ptr, col, ids_per_line=32)
        out[name] = {"sort_ms": round(statistics.median(ts), 4),
                     "reorder_ms": round(statistics.median(tr), 4),
                     "csr_plus_spmv_ms": round(statistics.median(tsp), 4), "nbr32": round(v, 5)}
    # the other readings (Fig. 1 interleaved, Alg. 2's racy store): reorder
    # time, and the locality and SpMV of the order they give
    for name, variant in (("boba_interleaved", 1), ("boba_racy", 2)):
        tr = []
        for rep in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            flush.zero_()
            ev[0].record(stream)
            boba.check(boba.boba_reorder_variant(src, dst, m, n, perm2, s3, d3, variant, ws_r2,
                                                 ws_r2.numel(), stream), "variant")
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                tr.append(ev[0].elapsed_time(ev[1]))
        boba.check(boba.boba_coo_to_csr(s3, d3, m, n, row_ptr, col, val, ws_c, ws_c.numel(),
                                        stream), "csr")
        ts = []
        for rep in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            boba.check(boba.boba_spmv_csr(row_ptr, col, val, x, y, n, m, ws_s, ws_s.numel(),
                                          stream), "spmv")
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                ts.append(ev[0].elapsed_time(ev[1]))
        v, _ = boba.nbr(row_ptr, col, ids_per_line=32)
        out[name] = {"reorder_ms": round(statistics.median(tr), 4),
                     "spmv_ms": round(statistics.median(ts), 4), "nbr32": round(v, 5)}
    del s2, d2, s3, d3, ws_sort, ws_r2
    boba.stream_status(stream)
    # NBR spatial-locality metric (Sec. 5.2) of the two CSRs, lines of 32 IDs, and
    # PageRank (Sec. 5.1 applications) on each: spmv_iters fixed steps, then the
    # steps needed for an L1 change below 1e-6
    ws_pr = torch.empty(boba.boba_pagerank_workspace_bytes(n, m), dtype=torch.uint8, device=dev)
    pr = torch.empty(n, dtype=torch.float32, device=dev)
    pr_steps = torch.zeros(1, dtype=torch.int32, device=dev)
    pr_res = torch.zeros(1, dtype=torch.float64, device=dev)
    k = max(1, args.spmv_iters)
    for name, (s_, d_) in (("random", (src, dst)), ("boba", (so, do))):
        boba.check(boba.boba_coo_to_csr(s_, d_, m, n, row_ptr, col, val, ws_c, ws_c.numel(),
                                        stream), "csr")
        v, cnt = boba.nbr(row_ptr, col, ids_per_line=32)
        out[name]["nbr32"] = round(v, 5)
        t_pr = []
        for rep in range(4):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            boba.check(boba.boba_pagerank(row_ptr, col, val, n, m, 0.85, k, 0.0, pr, pr_steps,
                                          pr_res, ws_pr, ws_pr.numel(), stream), "pagerank")
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                t_pr.append(ev[0].elapsed_time(ev[1]) / k)
        with boba.kernel_timing() as kt:                 # per-kernel split of fixed steps
            boba.check(boba.boba_pagerank(row_ptr, col, val, n, m, 0.85, k, 0.0, pr, pr_steps,
                                          pr_res, ws_pr, ws_pr.numel(), stream), "pagerank")
            boba.stream_status(stream)
        out[name]["pagerank_kernels_ms"] = {
            kname: round(t / max(1, c), 4) for kname, (t, c) in kt.result.items()}
        boba.check(boba.boba_pagerank(row_ptr, col, val, n, m, 0.85, 1000, 1e-6, pr, pr_steps,
                                      pr_res, ws_pr, ws_pr.numel(), stream), "pagerank")
        boba.stream_status(stream)
        out[name]["pagerank_ms_per_step"] = round(statistics.median(t_pr), 4)
        out[name]["pagerank_steps_to_1e-6"] = int(pr_steps.item())
    del ws_pr, pr
    out["pagerank_speedup_boba_vs_random"] = round(
        out["random"]["pagerank_ms_per_step"] / out["boba"]["pagerank_ms_per_step"], 3)
    out["csr_speedup_boba_vs_random"] = round(out["random"]["csr_ms"] / out["boba"]["csr_ms"], 3)
    out["spmv_bytes_per_launch"] = spmv_bytes
    return out


def run_batched(args, boba, torch, dev, stream, flush, n_batch=4096, seed=None):
    """The batched workload: n_batch R-MAT graphs (n log-uniform in [2^8, 2^18),
    edge factor 4..32) reordered in one persistent launch, against one launch
    sequence per graph (eager, and replayed from a CUDA graph).  Outputs of the
    two forms are compared bit for bit."""
    import synth
    seed = synth.SEED_BASE + 3 if seed is None else seed
    n_g, m_g = synth.batch_sizes(n_batch, seed)
    eo = np.zeros(n_batch + 1, np.int64); eo[1:] = np.cumsum(m_g)
    vo = np.zeros(n_batch + 1, np.int64); vo[1:] = np.cumsum(n_g)
    E, V = int(eo[-1]), int(vo[-1])
    src_h = torch.empty(E, dtype=torch.int32, pin_memory=True)
    dst_h = torch.empty(E, dtype=torch.int32, pin_memory=True)
    synth.rmat_batch(n_batch, seed, out=(src_h.numpy(), dst_h.numpy()))
    src, dst = src_h.to(dev), dst_h.to(dev)
    del src_h, dst_h
    eo_d, vo_d = torch.from_numpy(eo).to(dev), torch.from_numpy(vo).to(dev)
    max_m, max_n = int(m_g.max()), int(n_g.max())
    perm = torch.empty(V, dtype=torch.int32, device=dev)
    so, do = torch.empty_like(src), torch.empty_like(dst)
    ws = torch.empty(boba.boba_reorder_batched_workspace_bytes(n_batch, max_m, max_n, E, V),
                     dtype=torch.uint8, device=dev)

    def batched(st):
        boba.check(boba.boba_reorder_batched(src, dst, eo_d, vo_d, n_batch, max_m, max_n, E, V,
                                             perm, so, do, ws, ws.numel(), st), "batched")

    # one launch sequence per graph, outputs into separate buffers
    perm1 = torch.empty_like(perm)
    so1, do1 = torch.empty_like(src), torch.empty_like(dst)
    ws1 = torch.empty(boba.boba_reorder_workspace_bytes(max_m, max_n), dtype=torch.uint8,
                      device=dev)
    views = [(src[eo[g]:eo[g + 1]], dst[eo[g]:eo[g + 1]], int(m_g[g]), int(n_g[g]),
              perm1[vo[g]:vo[g + 1]], so1[eo[g]:eo[g + 1]], do1[eo[g]:eo[g + 1]])
             for g in range(n_batch)]

    def per_graph(st):
        for s_, d_, mg, ng, p_, o1, o2 in views:
            boba.check(boba.boba_reorder_ex(s_, d_, mg, ng, p_, o1, o2, None, ws1, ws1.numel(),
                                            st), "per-graph")

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    reps = max(3, min(args.steps, 5))
    tuned = None
    if args.tune:
        tuned = boba.tune_batched(src, dst, eo_d, vo_d, max_m, max_n, reps=2)
        ws = torch.empty(boba.boba_reorder_batched_workspace_bytes(n_batch, max_m, max_n, E, V),
                         dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        batched(stream)
    t_batched = timed(batched, reps)
    flush.zero_()
    with boba.kernel_timing() as kt:                # per-kernel split of one batched call
        batched(stream)
        torch.cuda.synchronize(dev)
    split = {k: round(t, 3) for k, (t, _) in sorted(kt.result.items())}
    per_graph(stream)
    t_pergraph = timed(per_graph, reps)
    boba.stream_status(stream)
    identical = bool(torch.equal(perm, perm1) and torch.equal(so, so1) and torch.equal(do, do1))

    # every schedule of the batched call, each checked against the per-graph
    # outputs: 0 is the one persistent launch (8-block clusters, keys in
    # distributed shared memory), 1..8 the split schedules (a persistent launch
    # for the small graphs, six grid-wide phase launches for the large ones)
    sched = {}
    names = {0: "cluster: plan + one persistent launch", 1: "split, sliced first <= 8, relabel <= 1",
             2: "split, sliced first and relabel <= 8", 3: "split, sliced first <= 8, relabel <= 2",
             4: "split, global phases", 5: "split, sliced first <= 3",
             6: "split as 1, global relabel in per-SM runs of 2^21 edges (default)",
             7: "split as 6, global first-occurrence in per-SM runs too",
             8: "split as 7, sliced first <= 1"}
    for mode in range(9):
        boba.boba_batched_set_mode(mode)
        need = boba.boba_reorder_batched_workspace_bytes(n_batch, max_m, max_n, E, V)
        if need > ws.numel():
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        perm.fill_(-1)
        batched(stream)
        boba.stream_status(stream)
        same = bool(torch.equal(perm, perm1) and torch.equal(so, so1) and torch.equal(do, do1))
        with boba.kernel_timing() as kt2:
            batched(stream)
            torch.cuda.synchronize(dev)
        t = timed(batched, reps)
        sched[mode] = {"form": names[mode], "ms": round(t, 3),
                       "gedges_s": round(E / (t * 1e-3) / 1e9, 3),
                       "launches": sum(c for _, c in kt2.result.values()),
                       "bit_identical": same}
        identical = identical and same
    boba.boba_batched_set_mode(-1)
    boba.stream_status(stream)

    # both forms captured once into a CUDA graph and replayed
    t_graph = {}
    for name, fn in (("batched", batched), ("per_graph", per_graph)):
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn(torch.cuda.current_stream(dev))
            torch.cuda.synchronize(dev)
            for _ in range(2):
                g.replay()
            torch.cuda.synchronize(dev)
            t_graph[name] = round(timed(lambda st, g=g: g.replay(), reps), 3)
            del g
        except Exception as exc:                 # report why capture was not possible
            t_graph[name] = "capture failed: " + str(exc)[:160]
    boba.stream_status(stream)
    identical = identical and bool(torch.equal(perm, perm1) and torch.equal(so, so1))
    return {"workload": f"rmat_batch{n_batch}", "graphs": n_batch, "edges": E, "vertices": V,
            "max_m": max_m, "max_n": max_n,
            "batched_ms": round(t_batched, 3),
            "batched_gedges_s": round(E / (t_batched * 1e-3) / 1e9, 3),
            "roofline": {"alg_bytes": 24 * E + 4 * V,
                         "achieved_gbs": round((24 * E + 4 * V) / (t_batched * 1e-3) / 1e9, 1),
                         "frac": round((24 * E + 4 * V) / (t_batched * 1e-3) / 1e9
                                       / peaks()[0], 4)},
            "per_graph_ms": round(t_pergraph, 3),
            "per_graph_gedges_s": round(E / (t_pergraph * 1e-3) / 1e9, 3),
            "speedup_batched_vs_per_graph": round(t_pergraph / t_batched, 3),
            "kernels_ms": split,
            "schedules": sched,
            "cuda_graph_ms": t_graph,
            "schedule": {0: "split, sliced first <= 8 slices, relabel <= 1, global relabel in "
                            "per-SM runs", 1: "cluster",
                         2: "split, sliced first and relabel <= 8 slices",
                         3: "split, sliced first <= 8 slices, relabel <= 2",
                         4: "split, global phases", 5: "split, sliced first <= 3 slices",
                         6: "split, sliced first <= 8 slices, relabel <= 1, grid-stride relabel",
                         7: "split as 0, global first and relabel in per-SM runs",
                         8: "split, sliced first and relabel <= 1, the rest in per-SM runs"}.get(
                (tuned or {}).get("batched", 0)),
            "bit_identical": identical}


def run_e2e(args, boba, torch, dev, stream, src_h, dst_h, m, n, world):
    """Same metric through the C ABI with the graph in pinned host memory:
    boba_reorder_host copies the edges in, reorders and copies perm and the
    relabelled edges out, all inside the timed region.

    Steps alternate between two streams, each with its own workspace and host
    output buffers, as a caller streaming graphs would: the input copies of
    step k+1 then run while step k's results are copied out.  The timed region
    spans all K steps; the latency of one call alone is reported beside it."""
    streams = [stream, torch.cuda.Stream(dev)]
    outs = [(torch.empty(n, dtype=torch.int32, pin_memory=True),
             torch.empty(m, dtype=torch.int32, pin_memory=True),
             torch.empty(m, dtype=torch.int32, pin_memory=True)) for _ in range(2)]
    nbytes = boba.boba_reorder_host_workspace_bytes(m, n)
    wss = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]

    def one(k):
        s = streams[k % 2]
        perm_h, so_h, do_h = outs[k % 2]
        boba.check(boba.boba_reorder_host(src_h, dst_h, m, n, perm_h, so_h, do_h, wss[k % 2],
                                          nbytes, s), "reorder_host")

    for k in range(max(2, args.warmup)):
        one(k)
    torch.cuda.synchronize(dev)
    # one call alone: its latency
    lat = []
    for k in range(3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(streams[0])
        one(0)
        ev[1].record(streams[0])
        torch.cuda.synchronize(dev)
        lat.append(ev[0].elapsed_time(ev[1]))
    # K steps back to back on alternating streams; nine rounds, the median
    # round is reported (the host link is shared with the machine's other work,
    # and rounds come out either near the link's bound or about twice it)
    steps = max(2, min(args.steps, 10))
    rounds = []
    for _ in range(9):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(streams[0])
        streams[1].wait_event(ev0)
        for k in range(steps):
            one(k)
        done1 = torch.cuda.Event()
        done1.record(streams[1])
        streams[0].wait_event(done1)
        ev1.record(streams[0])
        torch.cuda.synchronize(dev)
        rounds.append(ev0.elapsed_time(ev1) / steps)
    boba.stream_status(stream)
    ok = all(torch.equal(outs[0][i], outs[1][i]) for i in range(3))
    ms = statistics.median(rounds)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    return {"value": round(world * m / (ms * 1e-3) / 1e9, 3), "unit": "Gedges/s",
            "ms_per_step": round(ms, 3), "h2d_bytes_per_step": 8 * m,
            "d2h_bytes_per_step": 8 * m + 4 * n,
            "single_call_ms": round(statistics.median(lat), 3),
            "rounds_ms_per_step": [round(r, 3) for r in rounds],
            "best_round_gedges_s": round(world * m / (min(rounds) * 1e-3) / 1e9, 3),
            "outputs_equal_across_streams": ok,
            "api": "boba_reorder_host (chunked, copies overlapped with kernels); "
                   "steps alternate over 2 streams so step k+1's input copies overlap "
                   "step k's output copies"}


def run_gather_probe(args, boba, torch, dev, stream, reorder_ms, m, kernel_times):
    """Random 4-byte loads per second (boba_probe_gather) from a 64 MiB table in
    global memory -- the size of the key and label arrays at n = 2^24 -- and
    from smaller and larger tables, from one block's shared memory and from the
    distributed shared memory of 8- and 16-block clusters; beside them the
    lookups per second the reorder's two lookup passes reached."""
    import ctypes
    cases = [("global_64MiB", 0, 1 << 24, 0), ("global_4MiB", 0, 1 << 20, 0),
             ("global_128KiB", 0, 1 << 15, 0),
             ("global_1GiB", 0, 1 << 28, 0), ("shared_128KiB", 1, 1 << 15, 0),
             ("cluster8_1MiB", 2, 1 << 18, 8), ("cluster16_2MiB", 2, 1 << 19, 16)]
    table = torch.randint(0, 1 << 30, (1 << 28,), dtype=torch.int32, device=dev)
    out_words = 152 * 64 * 256
    out = torch.empty(out_words, dtype=torch.int32, device=dev)
    res = {}
    for name, mode, words, cl in cases:
        issued = ctypes.c_int64(0)
        per_thread = 2048
        times = []
        rc = 0
        for rep in range(4):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            rc = boba.boba_probe_gather(mode, table, words, per_thread, cl, out, out_words,
                                        issued, stream)
            ev[1].record(stream)
            if rc != 0:
                break
            torch.cuda.synchronize(dev)
            if rep:
                times.append(ev[0].elapsed_time(ev[1]))
        if rc != 0:
            res[name] = {"unavailable": boba.boba_status_string(rc)}
            continue
        boba.stream_status(stream)
        ms = statistics.median(times)
        res[name] = {"loads_per_s": round(issued.value / (ms * 1e-3), 0), "ms": round(ms, 4),
                     "loads": issued.value}
    del table, out
    # the reorder: 2m lookups in the first-occurrence pass, 2m in the relabel
    look = {}
    for k in ("reorder.first", "reorder.relabel"):
        if k in kernel_times:
            tot, launches = kernel_times[k]
            look[k] = round(2 * m / (tot / max(1, launches) * 1e-3), 0)
    if "spmv" in kernel_times:
        tot, launches = kernel_times["spmv"]
        look["spmv"] = round(m / (tot / max(1, launches) * 1e-3), 0)
    g64 = res.get("global_64MiB", {}).get("loads_per_s")
    if g64:
        look_frac = {k: round(v / g64, 4) for k, v in look.items()}
    else:
        look_frac = None
    return {"probe": res, "reorder_lookups_per_s": look, "lookups_frac_of_ceiling": look_frac,
            "reorder_lookup_bound_ms": round(4 * m / g64 * 1e3, 4) if g64 else None,
            "reorder_ms": round(reorder_ms, 4),
            "note": "reorder_lookup_bound_ms = 4m lookups at the global_64MiB rate, with no "
                    "stream traffic: the least time any one-lookup-per-endpoint design needs"}


def lookup_roofline(gather):
    """The lookup passes against the measured random-load ceiling: random loads
    per second each reached over the probe's rate from a 64 MiB table."""
    if not gather or not gather.get("lookups_frac_of_ceiling"):
        return None
    peak = gather["probe"]["global_64MiB"]["loads_per_s"]
    return {"bound": "random 4-byte loads (L1TEX/L2 request rate)", "unit": "loads/s",
            "peak": peak, "peak_source": "boba_probe_gather, 64 MiB table, measured in this run",
            "achieved": gather["reorder_lookups_per_s"],
            "frac": gather["lookups_frac_of_ceiling"]}


def time_reorder_variants(boba, torch, dev, stream, flush, src, dst, m, n, perm, so, do, ws,
                          tuning, reps=5):
    """Device time of the first-occurrence and relabel kernels for every variant
    (0..5 launch shapes, 6 warp-aggregated, 7 bulk-copied streams), the other family
    at its tuned choice; restores the tuned choices."""
    out = {}
    for fam_name, fam, key in (("first", boba.TUNE_FIRST, "reorder.first"),
                               ("relabel", boba.TUNE_RELABEL, "reorder.relabel")):
        res = {}
        for v in range(8):
            boba.load().boba_tune_set(fam, m, v)
            boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws, ws.numel(),
                                            stream), "reorder")
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                with boba.kernel_timing() as kt:
                    boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws,
                                                    ws.numel(), stream), "reorder")
                    torch.cuda.synchronize(dev)
                tot += kt.result[key][0]
            res[v] = round(tot / reps, 4)
        boba.load().boba_tune_set(fam, m, (tuning or {}).get(fam_name, 0))
        out[fam_name] = res
    boba.stream_status(stream)
    return out


def run_latency(args, boba, torch, dev, stream):
    """R-MAT scale 14 / 2^18 edges (fits in L2): the latency of one reorder,
    eager and replayed from a CUDA graph, and of reorder + CSR + SpMV."""
    import synth
    w = synth.RMAT14
    I, J = w.generate()
    src, dst = torch.from_numpy(I).to(dev), torch.from_numpy(J).to(dev)
    m, n = w.m, w.n
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    so, do = torch.empty_like(src), torch.empty_like(dst)
    ws = torch.empty(boba.boba_reorder_workspace_bytes(m, n), dtype=torch.uint8, device=dev)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(m, dtype=torch.int32, device=dev)
    val = torch.empty(m, dtype=torch.float32, device=dev)
    wc = torch.empty(boba.boba_coo_to_csr_workspace_bytes(m, n), dtype=torch.uint8, device=dev)
    wsp = torch.empty(max(256, boba.boba_spmv_workspace_bytes(n, m)), dtype=torch.uint8,
                      device=dev)
    x = torch.from_numpy(synth.uniform_f32(n, seed=w.seed)).to(dev)
    y = torch.empty(n, dtype=torch.float32, device=dev)

    def reorder(st):
        boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws, ws.numel(), st),
                   "reorder")

    def pipeline(st):
        reorder(st)
        boba.check(boba.boba_coo_to_csr(so, do, m, n, row_ptr, col, val, wc, wc.numel(), st),
                   "csr")
        boba.check(boba.boba_spmv_csr(row_ptr, col, val, x, y, n, m, wsp, wsp.numel(), st),
                   "spmv")

    def lat(fn, reps=50):
        for _ in range(3):
            fn(stream)
        torch.cuda.synchronize(dev)
        out = []
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            fn(stream)
            ev[1].record(stream)
            ev[1].synchronize()
            out.append(ev[0].elapsed_time(ev[1]))
        return statistics.median(out)

    res = {"workload": w.name, "m": m, "n": n,
           "reorder_us": round(lat(reorder) * 1e3, 2),
           "reorder_csr_spmv_us": round(lat(pipeline) * 1e3, 2)}
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            reorder(torch.cuda.current_stream(dev))
        torch.cuda.synchronize(dev)
        res["reorder_graph_replay_us"] = round(lat(lambda st: g.replay()) * 1e3, 2)
        del g
    except Exception as exc:
        res["reorder_graph_replay_us"] = "capture failed: " + str(exc)[:120]
    boba.stream_status(stream)
    res["reorder_gedges_s"] = round(m / (res["reorder_us"] * 1e-6) / 1e9, 3)
    res["note"] = "inputs stay in L2 (2 MiB); this is latency, not a roofline figure"
    return res


def run_configs2(args, boba, torch, dev, stream, flush, oracle_futs):
    """The low-skew workloads: a 4096 x 4096 grid (both edge directions) and an
    Erdos-Renyi graph with n = 2^24, m = 2^27, each relabelled at random with
    edges shuffled: reorder (full and perm only), CSR and SpMV on the random and
    the BOBA order, and the SpMV error against the fp64 oracle."""
    import synth
    hbm, _ = peaks()
    res = {}
    for w in (synth.GRID4096, synth.ER24):
        m, n = w.m, w.n
        I, J = w.generate()
        src, dst = torch.from_numpy(I).to(dev), torch.from_numpy(J).to(dev)
        del I, J
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        so, do = torch.empty_like(src), torch.empty_like(dst)
        ws = torch.empty(boba.boba_reorder_workspace_bytes(m, n), dtype=torch.uint8, device=dev)
        row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        col = torch.empty(m, dtype=torch.int32, device=dev)
        val = torch.empty(m, dtype=torch.float32, device=dev)
        wc = torch.empty(boba.boba_coo_to_csr_workspace_bytes(m, n), dtype=torch.uint8,
                         device=dev)
        wsp = torch.empty(max(256, boba.boba_spmv_workspace_bytes(n, m)), dtype=torch.uint8,
                          device=dev)
        x = torch.from_numpy(synth.uniform_f32(n, seed=w.seed)).to(dev)
        y = torch.empty(n, dtype=torch.float32, device=dev)
        tuning = None
        if args.tune:
            tuning = boba.tune_reorder(src, dst, n, reps=3)
            boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws, ws.numel(),
                                            stream), "reorder")
            tuning.update(boba.tune_csr(so, do, n, reps=2))
            boba.check(boba.boba_coo_to_csr(so, do, m, n, row_ptr, col, val, wc, wc.numel(),
                                            stream), "csr")
            tuning.update(boba.tune_spmv(row_ptr, col, val, x, reps=3))
            boba.stream_status(stream)

        def timed(fn, reps=5):
            out = []
            for rep in range(reps + 1):
                flush.zero_()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(stream)
                fn()
                ev[1].record(stream)
                torch.cuda.synchronize(dev)
                if rep:
                    out.append(ev[0].elapsed_time(ev[1]))
            boba.stream_status(stream)
            return statistics.median(out)

        t_full = timed(lambda: boba.check(boba.boba_reorder_ex(
            src, dst, m, n, perm, so, do, None, ws, ws.numel(), stream), "reorder"))
        t_perm = timed(lambda: boba.check(boba.boba_reorder_ex(
            src, dst, m, n, perm, None, None, None, ws, ws.numel(), stream), "reorder"))
        boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws, ws.numel(),
                                        stream), "reorder")
        r = {"m": m, "n": n, "tuning": tuning,
             "reorder_ms": round(t_full, 4), "gedges_s": round(m / (t_full * 1e-3) / 1e9, 3),
             "frac": round((24 * m + 4 * n) / (t_full * 1e-3) / 1e9 / hbm, 4),
             "perm_only_ms": round(t_perm, 4),
             "perm_only_gedges_s": round(m / (t_perm * 1e-3) / 1e9, 3),
             "perm_only_frac": round((8 * m + 4 * n) / (t_perm * 1e-3) / 1e9 / hbm, 4)}
        ys = {}
        for order, (s_, d_) in (("random", (src, dst)), ("boba", (so, do))):
            t_csr = timed(lambda: boba.check(boba.boba_coo_to_csr(
                s_, d_, m, n, row_ptr, col, val, wc, wc.numel(), stream), "csr"), reps=3)
            t_spmv = timed(lambda: boba.check(boba.boba_spmv_csr(
                row_ptr, col, val, x, y, n, m, wsp, wsp.numel(), stream), "spmv"))
            ys[order] = y.cpu().numpy()
            nbr32, _ = boba.nbr(row_ptr, col, ids_per_line=32)
            r[order] = {"csr_ms": round(t_csr, 4), "spmv_ms": round(t_spmv, 4),
                        "spmv_gbs": round((8 * m + 16 * n) / (t_spmv * 1e-3) / 1e9, 1),
                        "nbr32": round(nbr32, 5)}
        r["spmv_speedup_boba_vs_random"] = round(r["random"]["spmv_ms"] / r["boba"]["spmv_ms"], 3)
        r["spmv_rel_l2_vs_fp64"] = spmv_errors(oracle_futs, w.name, ys)
        res[w.name] = r
        del src, dst, perm, so, do, ws, row_ptr, col, val, wc, wsp, x, y
        torch.cuda.empty_cache()
    return res


def reorder_dram_traffic(workload, m=None, n=None):
    """DRAM bytes per launch of the reorder's two lookup kernels from the
    committed ncu summary, beside their algorithmic bytes."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f).get(workload, {})
    except Exception:
        return None
    out = {}
    alg = algorithmic_bytes(m, n, m) if m else {}
    for k in ("reorder.first", "reorder.relabel"):
        if d.get(k) is None:
            continue
        out[k] = {"dram_bytes": d[k], "alg_bytes": alg.get(k),
                  "ratio": round(d[k] / alg[k], 3) if alg.get(k) else None}
    return out or None


def load_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d.get(workload, {}).get(kernel)
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the CPU oracle (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, m_sample):
    # a prefix of the shuffled edge list is a uniform sample of its edges
    return w.generate(edge_range=(0, m_sample))


def time_oracle(I, J, n):
    import oracle
    t = time.perf_counter()
    perm, label = oracle.boba_perm(I, J, n)
    oracle.relabel(I, J, label, n)
    return time.perf_counter() - t


def cpu_baseline(w, args):
    m_s = min(w.m, args.cpu_sample_edges)
    I, J = oracle_sample(w, m_s)
    times = [time_oracle(I, J, w.n) for _ in range(2)]
    t = statistics.median(times)
    model, cores = cpu_info()
    return {"value": round(m_s / t / 1e9, 5), "unit": "Gedges/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m_s} edges of {w.name} (n={w.n}), reorder (perm + relabel), "
                      f"median of 2 runs; host {model}, {cores} cores visible, 1 used"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    w = synth.WORKLOADS[args.workload]
    m_s = min(w.m, args.cpu_sample_edges)
    I, J = oracle_sample(w, m_s)
    for _ in range(args.warmup):
        time_oracle(I, J, w.n)
    times = [time_oracle(I, J, w.n) for _ in range(args.steps)]
    t = statistics.mean(times)
    v = m_s / t / 1e9
    model, cores = cpu_info()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "Gedges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "sample_edges": m_s},
        "cpu_baseline": {"value": round(v, 5), "unit": "Gedges/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {m_s} edges of {w.name}, reorder (perm + relabel) "
                                   f"per step; host {model}, {cores} cores visible, 1 used"},
        "e2e": {"value": round(v, 5), "unit": "Gedges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rmat24_m2^28",
                    help="one of: " + ", ".join(sorted(__import__("synth").WORKLOADS)))
    ap.add_argument("--spmv-iters", type=int, default=20)
    ap.add_argument("--cpu-sample-edges", type=int, default=1 << 27)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batched", type=int, default=1,
                    help="1: also time the batched workload (4096 graphs) vs per-graph launches")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--tune", type=int, default=1,
                    help="1: autotune launch variants on the workload before timing")
    ap.add_argument("--tune-spec", default="",
                    help="set variants instead of tuning, e.g. first=5,relabel=3,spmv=5")
    ap.add_argument("--serve", type=int, default=1,
                    help="1: also run the serving workload (Poisson requests, HBM budget)")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--spmv-error", type=int, default=1,
                    help="1: report the SpMV's rel-L2 error against the fp64 oracle")
    ap.add_argument("--configs2", type=int, default=1,
                    help="1: also run the grid 4096^2 and ER 2^24 / 2^27 workloads")
    ap.add_argument("--latency", type=int, default=1,
                    help="1: also time one reorder of R-MAT scale 14 (latency)")
    ap.add_argument("--gather", type=int, default=1,
                    help="1: also measure the random-load ceiling (boba_probe_gather)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)        # at least 3 untimed warm-up steps
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: relaunch this command under torch.distributed.run
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1",
               "--master-port", os.environ.get("MASTER_PORT", "29533"),
               os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; using {world}",
              file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
