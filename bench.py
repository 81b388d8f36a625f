#!/usr/bin/env python
"""Throughput benchmark of the D2Q9 MRT lattice Boltzmann library on GB300.

Default workload (one JSON line): 512 independent periodic lattices, areas
log-uniform in [32^2, 1024^2] (6.7e7 nodes), per-lattice relaxation rates,
Gaussian pulses, FP32 deviation storage.  One benchmark step = the whole
batch advanced 500 time steps (500 batched fused step launches replayed from
CUDA graphs) followed by the FP64 drift check of every lattice (one batched
reduction).

  value      MLUPS with the populations resident in HBM
  e2e        MLUPS through the C ABI with host buffers: every step uploads
             the initial fields (rho, ux, uy) from pinned host memory
             (packed batch I/O), steps, and downloads rho, ux, uy
  roofline   the batched step kernel: algorithmic 72 B per lattice update
             over its average launch time against the measured HBM copy
             bandwidth
  fp64_plain the plain FP64 path on one 8192^2 lattice, for comparison
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the workload

--batch-dtype f16 / bf16 runs the same batch in 16-bit deviation storage.
Other workloads: --workload large (one 8192^2 lattice, per storage type),
--workload serving (Poisson request stream through lbm_submit/poll),
--workload vn (von Neumann eigenvalue sweep), --workload opt (the
free-parameter cost functions and their minimization), --workload source
(the section 5.1 point source on 101 x 101, three schemes) and --workload
oracle (the CPU oracle alone: one thread and all cores).
--impl reference times the CPU oracle on the same metric.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs as inp  # noqa: E402

BYTES_PER_LU = {"f64": 144, "f64dev": 144, "f32": 72, "f16": 36, "bf16": 36}
KERNEL_SOURCES = ["csrc/step_impl.cuh", "csrc/d2q9_pull.cuh", "csrc/collide.cuh",
                  "csrc/step_f32.cu", "csrc/step_f16.cu", "csrc/step_bf16.cu", "csrc/step_f64.cu",
                  "csrc/step_f64dev.cu", "csrc/resident.cuh"]


def parser():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="batched",
                   choices=["batched", "large", "serving", "vn", "opt", "source", "oracle",
                            "slabs", "small"])
    p.add_argument("--lattices", type=int, default=512)
    p.add_argument("--lbm-steps", type=int, default=500)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="batched workload alone (no FP16 batch, config 3, serving keys)")
    p.add_argument("--requests", type=int, default=10000)
    p.add_argument("--policy", default="fifo", choices=["fifo", "shortest"])
    p.add_argument("--max-nodes", type=int, default=0, help="server resident-node cap")
    p.add_argument("--size", type=int, default=8192, help="side of the large lattice")
    p.add_argument("--dtypes", default="f32,f16,bf16,f64,f64dev", help="storage types (large)")
    p.add_argument("--batch-dtype", default="f32", choices=["f32", "f16", "bf16"],
                   help="storage type of the batched workload")
    p.add_argument("--batch-variant", type=int, default=-1,
                   help="pin the batched launch variant (default: tuned)")
    return p


def parse(argv=None):
    return parser().parse_args(argv)


# ------------------------------------------------------------ environment
def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_specs(args, rank, world=None):
    """The lattices of one rank.  The workload is `lattices` lattices per GPU
    (weak scaling: N GPUs step N x 512 independent lattices), drawn as one
    seeded set and placed on the ranks by bytes (multi_gpu.partition_by_bytes:
    largest first onto the least-loaded rank); no data crosses ranks while
    they step.  With one rank this is the 512-lattice workload itself."""
    from paper_1107_4543_gb300 import multi_gpu

    if world is None:
        world = dist()[0]
    specs = inp.batch_specs(args.lattices * world, seed=1107 + 4, steps=args.lbm_steps)
    if world == 1:
        return specs
    sizes = [multi_gpu.lattice_bytes(sp["nx"], sp["ny"], 1) for sp in specs]
    return [specs[i] for i in multi_gpu.partition_by_bytes(sizes, world)[rank]]


def reduce_max(x, device="cuda"):
    """Max of a float over the ranks (the timing rule: the slowest rank)."""
    import torch

    if not torch.distributed.is_initialized() or torch.distributed.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, device="cuda"):
    """Sum of a float over the ranks."""
    import torch

    if not torch.distributed.is_initialized() or torch.distributed.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_mlups(units_all_ranks, seconds):
    """Whole-job throughput: the units all ranks processed over the max time."""
    return units_all_ranks / seconds / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def traffic_record(kernel):
    """DRAM bytes per lattice update from the committed ncu summary, or None
    when the kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha") != sources_sha():
        return None
    return rec


def code_of(text):
    """C++ source with its comments and blank space removed (string
    literals kept), so that a comment edit does not count as a kernel
    change."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            i = text.find("*/", i + 2)
            i = n if i < 0 else i + 2
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def sources_sha():
    """Hash of the step kernels' code (comments and spacing ignored): a
    traffic record taken at other code is not reported."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1107_4543_gb300", rel), encoding="utf-8") as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()[:16]


# -------------------------------------------------------------- CPU oracle
def cpu_oracle_mlups(specs, target_s=20.0, threads=None, lattices=4):
    """The FP64 oracle (as it stands) on a bounded sample of the workload:
    the first `lattices` lattices of the list, each stepped for about
    target_s / lattices seconds (at most the workload's step count).
    Returns (MLUPS, cores, sample description)."""
    import oracle as orc

    threads = threads or os.cpu_count() or 1
    orc.set_threads(threads)
    nodes = 0
    t_total = 0.0
    used = []
    for spec in specs[:lattices]:
        rho, ux, uy = inp.batch_fields(spec)
        f = orc.init_eq(rho, ux, uy)
        s = inp.s_paper(spec["rates"])
        f = orc.run(f, s, 1)  # thread start-up outside the estimate
        t0 = time.perf_counter()
        f = orc.run(f, s, 4)
        per_step = (time.perf_counter() - t0) / 4
        n = spec["nx"] * spec["ny"]
        steps = int(max(2, min(spec.get("steps", 500), (target_s / lattices) / max(per_step, 1e-9))))
        t0 = time.perf_counter()
        orc.run(f, s, steps)
        t_total += time.perf_counter() - t0
        nodes += n * steps
        used.append("%dx%d x %d steps" % (spec["nx"], spec["ny"], steps))
    return nodes / t_total / 1e6, threads, "; ".join(used)


# ------------------------------------------------------------- GPU workloads
def setup_batch(L, torch, specs, dtype, stream):
    hs = []
    fields = []
    for spec in specs:
        h = L.lbm_create(spec["nx"], spec["ny"], inp.s_ll(spec["rates"]), 1.0, (0.0, 0.0),
                         L.DTYPES[dtype])
        L.lbm_set_stream(h, stream)
        rho, ux, uy = inp.batch_fields(spec)
        pinned = []
        for a in (rho, ux, uy):
            t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = a
            pinned.append(t.numpy())
        L.lbm_init_field(h, *pinned)
        hs.append(h)
        fields.append(pinned)
    return hs, fields


def fp64_plain(L, torch, stream, n=8192, steps=20, dtype=None):
    """An FP64 path on one n x n lattice (Gaussian pulse), MLUPS: the plain
    one (bit-identical to the FP64 oracle) or, with dtype LBM_F64DEV, FP64
    deviations collided with fused multiply-adds."""
    r = inp.rates("OPT")
    h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F64 if dtype is None else dtype)
    try:
        L.lbm_set_stream(h, stream)
        L.lbm_init_analytic(h, L.LBM_INIT_GAUSSIAN, (1e-3, 20.0, n / 2, n / 2))
        L.lbm_step(h, 4)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        L.lbm_step(h, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        L.lbm_destroy(h)
    return n * n * steps / (ms * 1e-3) / 1e6, ms / steps


_HOST_ARRAYS = {}


def host_arrays(kind, n):
    """Three page-locked huge-page host arrays of n doubles, slices of one
    lbm_host_alloc array (one allocation fills whole huge pages with less
    padding than three), kept for the rest of the process."""
    from paper_1107_4543_gb300 import lbm as L

    key = (kind, n)
    if key not in _HOST_ARRAYS:
        stride = (n + 511) // 512 * 512  # each field on a 4 KiB boundary
        whole = L.host_array(3 * stride)
        _HOST_ARRAYS[key] = tuple(whole[c * stride:c * stride + n] for c in range(3))
    return _HOST_ARRAYS[key]


def huge_page_share(arrays):
    """Share of the arrays' bytes that the kernel backs with transparent huge
    pages (from /proc/self/smaps; None where that cannot be read)."""
    try:
        spans = [(a.ctypes.data, a.ctypes.data + a.nbytes) for a in arrays]
        huge = total = 0
        cur = None
        with open("/proc/self/smaps") as fh:
            for line in fh:
                head = line.split()[0]
                if "-" in head and not head.endswith(":"):
                    lo, hi = (int(x, 16) for x in head.split("-"))
                    cur = (lo, hi) if any(lo < e and s < hi for s, e in spans) else None
                elif cur and line.startswith("AnonHugePages:"):
                    huge += int(line.split()[1]) * 1024
                    total += cur[1] - cur[0]
        return round(huge / total, 3) if total else None
    except OSError:
        return None


def bench_batched(args, L, torch, rank, ws):
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    specs = rank_specs(args, rank)
    bdt = args.batch_dtype
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    # the end-to-end host arrays first, before other host allocations can
    # break up the memory their huge pages need
    host_arrays("in", nodes)
    host_arrays("out", nodes)
    hs, fields = setup_batch(L, torch, specs, bdt, stream)
    b = L.lbm_batch_create(hs)
    if args.batch_variant >= 0:
        L.lbm_batch_set_variant(b, args.batch_variant)
    lbm_steps = args.lbm_steps
    # members held in shared memory for all the steps of a call (one launch
    # beside the per-step launches; no per-step HBM traffic)
    resident = L.lbm_batch_resident(b)
    res_nodes = sum(s["nx"] * s["ny"] for s, r in zip(specs, resident) if r)
    step_nodes = nodes - res_nodes  # the per-step kernel's lattice updates
    # one resident launch per non-empty size class (up to a third, a half,
    # all of a block's shared memory) per call
    optin = torch.cuda.get_device_properties(dev).shared_memory_per_block_optin
    esize = {"f32": 4, "f16": 2, "bf16": 2}[bdt]
    res_classes = len({0 if rb <= optin // 3 else (1 if rb <= optin // 2 else 2)
                       for rb in (2 * 9 * s["nx"] * s["ny"] * esize
                                  for s, r in zip(specs, resident) if r)})
    # one launch per call refreshes the batch's slots of the constant table
    # (a single storage type here) when it holds any
    table_fills = int(L.lbm_batch_const_table(b).any())

    def one_step():
        L.lbm_batch_step(b, lbm_steps)
        L.lbm_batch_drift(b, len(hs))

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    variant = L.lbm_batch_get_variant(b)
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(dev)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]
    ev[0].record()
    for k in range(args.steps):
        ev[2 * k + 1].record()
        L.lbm_batch_step(b, lbm_steps)
        ev[2 * k + 2].record()
        L.lbm_batch_drift(b, len(hs))
    ev[-1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(args.steps)]
    total_ms = reduce_max(total_ms)
    if ws > 1:
        torch.distributed.barrier()
    lu_per_step = nodes * lbm_steps
    lu_job = reduce_sum(lu_per_step * args.steps)  # every rank's lattice updates
    value = job_mlups(lu_job, total_ms * 1e-3)
    launch_ms = float(np.mean(step_ms)) / lbm_steps  # one batched kernel per time step
    # batched steps, the resident launches, the constant-table refresh and
    # one drift launch pair
    launches = args.steps * (lbm_steps + 2 + res_classes + table_fills)

    # e2e: host fields in, moments out, through the public API: one
    # lbm_batch_solve_packed call per benchmark step (upload of the fields
    # from page-locked host arrays, equilibrium init, the 500 steps, the
    # drift sums, moments, download), queued back to back so that one
    # solve's copies overlap its neighbours' stepping; lbm_batch_wait ends
    # the timed region and reports the device time per phase (median over
    # the timed solves)
    # page-locked host memory on huge pages (lbm_host_alloc; copies from
    # ordinary page-locked memory slowed to 17 - 80 GB/s on a host that had
    # run for a while), allocated once per process and shared by the
    # workloads of equal size
    fin = host_arrays("in", nodes)
    for c in range(3):
        np.concatenate([f[c].ravel() for f in fields], out=fin[c])
    fout = host_arrays("out", nodes)
    dout = np.zeros((len(hs), 4))

    def e2e_solve():
        L.lbm_batch_solve_packed(b, lbm_steps, fin, fout, dout)

    def e2e_wait():
        return L.lbm_batch_wait(b)

    for _ in range(2):
        e2e_solve()
    e2e_wait()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_solve()
    phases = e2e_wait()
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0)
    e2e_value = job_mlups(lu_job, e2e_s)
    L.lbm_batch_destroy(b)
    h2d = 3 * 8 * nodes
    d2h = 3 * 8 * nodes + 4 * 8 * len(hs)

    fp64 = None
    if not args.no_fp64:
        mlups64, ms64 = fp64_plain(L, torch, stream)
        mlupsd, msd = fp64_plain(L, torch, stream, dtype=L.LBM_F64DEV)
        fp64 = {"workload": "single 8192x8192 lattice, plain FP64 full populations "
                            "(bit-identical to the FP64 oracle)",
                "mlups": round(mlups64, 1), "ms_per_lbm_step": round(ms64, 3),
                "fp64_fma": {"workload": "the same lattice in FP64 deviation storage, FP64 "
                                         "collision with fused multiply-adds (within 1e-12 of "
                                         "the extended-precision oracle)",
                             "mlups": round(mlupsd, 1), "ms_per_lbm_step": round(msd, 3)}}
    for h in hs:
        L.lbm_destroy(h)

    peak, peak_kind = peaks()
    kname = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16"}[bdt]
    sname = {"f32": "FP32", "f16": "FP16", "bf16": "BF16"}[bdt]
    achieved = BYTES_PER_LU[bdt] * step_nodes / (launch_ms * 1e-3) / 1e9
    tr = traffic_record("k_step_batch<%s>" % kname)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                # ncu DRAM bytes per lattice update of a smaller capture of the
                # same kernel, scaled to this launch's lattice updates
                "traffic": (round(tr["dram_bytes_per_lu"] * step_nodes) if tr else None),
                "kernel": "k_step_batch<%s> (launch variant %d)" % (kname, variant),
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": BYTES_PER_LU[bdt] * step_nodes,
                "avg_launch_ms": round(launch_ms, 4),
                # against GB300's nominal 7.9 TB/s HBM3e, and the DRAM bytes
                # ncu counted (traffic) over the same launch time
                "nominal_peak": NOMINAL_HBM_GBS,
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "achieved_dram": (round(tr["dram_bytes_per_lu"] * step_nodes / (launch_ms * 1e-3) / 1e9, 1)
                                  if tr else None),
                "dram_frac_of_nominal": (round(tr["dram_bytes_per_lu"] * step_nodes / (launch_ms * 1e-3)
                                               / 1e9 / NOMINAL_HBM_GBS, 4) if tr else None)}
    line = {
        "metric": "MLUPS (lattice updates/s, millions), batched %s-deviation D2Q9 MRT" % sname,
        "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": bdt,
        "data": "synthetic (seeded Gaussian pulses, per-lattice relaxation rates)",
        "config": {"workload": "batched-%d-lattices-%sdev-%d-steps" % (
                       args.lattices, {"f32": "fp32", "f16": "fp16", "bf16": "bf16"}[bdt],
                       lbm_steps),
                   "lattices_per_gpu": len(specs), "nodes_per_gpu": nodes,
                   "resident_lattices": int(resident.sum()), "resident_nodes": res_nodes,
                   "lbm_steps_per_step": lbm_steps, "storage": "%s deviation" % sname.lower(),
                   "l2": "working set %.1f GB per time step > L2 (129 MB)" % (
                       BYTES_PER_LU[bdt] * nodes / 1e9),
                   "parallelism": "independent lattices placed on the GPUs by bytes "
                                  "(weak scaling: 512 lattices per GPU)"},
        "e2e": {"value": round(e2e_value, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_s * 1e3 / args.steps, 3),
                "api": ("lbm_batch_solve_packed per step (page-locked host fields in, moments "
                        "and drift out), successive solves overlapped, lbm_batch_wait at the "
                        "end"),
                # device time of each phase, median over the timed solves (events on the
                # streams that ran them; the copies overlap the neighbouring
                # solves' steps)
                "phases_ms": {k: round(phases[k], 3) for k in L.BATCH_PHASES},
                "h2d_gbs": round(h2d / max(phases["h2d_ms"], 1e-9) / 1e6, 1),
                "d2h_gbs": round(d2h / max(phases["d2h_ms"], 1e-9) / 1e6, 1),
                "host_huge_page_share": {"in": huge_page_share(fin),
                                         "out": huge_page_share(fout)}},
        "roofline": roofline,
        "fp64_plain": fp64,
        "gpu_launches": launches,
        "clocks": clk,
    }
    return line, specs


def large_one(L, torch, stream, n, dtype, lbm_steps, reps, warmup):
    """One n x n lattice (optimized rates, device-side Gaussian pulse A = 1e-3,
    b = 20) in one storage type: `reps` timed runs of lbm_steps steps after
    `warmup` untimed ones (CUDA events on the launching stream).  Returns
    (MLUPS, ms per time step)."""
    r = inp.rates("OPT")
    h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
    try:
        L.lbm_set_stream(h, stream)
        L.lbm_init_analytic(h, L.LBM_INIT_GAUSSIAN, (1e-3, 20.0, n / 2, n / 2))
        for _ in range(warmup):
            L.lbm_step(h, min(lbm_steps, 50))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            L.lbm_step(h, lbm_steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        L.lbm_destroy(h)
    return n * n * lbm_steps * reps / (ms * 1e-3) / 1e6, ms / (lbm_steps * reps)


def bench_large(args, L, torch, rank, ws):
    """One 8192^2 lattice per storage type; prints one line per type."""
    stream = torch.cuda.current_stream()
    n = args.size
    lines = []
    peak, peak_kind = peaks()
    for dtype in args.dtypes.split(","):
        lbm_steps = 50 if not dtype.startswith("f64") else 10
        mlups, launch_ms = large_one(L, torch, stream, n, dtype, lbm_steps, args.steps,
                                     args.warmup)
        achieved = BYTES_PER_LU[dtype] * n * n / (launch_ms * 1e-3) / 1e9
        lines.append({"metric": "MLUPS, single %dx%d lattice" % (n, n), "value": round(mlups, 1),
                      "unit": "MLUPS", "dtype": dtype, "n_gpus": ws, "steps": args.steps,
                      "warmup": args.warmup, "higher_is_better": True,
                      "config": {"workload": "single-%dx%d-%s" % (n, n, dtype)},
                      "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                                   "unit": "GB/s", "frac": round(achieved / peak, 4),
                                   "peak_source": peak_kind}})
    return lines


def config3_record(L, torch):
    """Config 3 at its stated size: one 8192^2 lattice, 1000 time steps, per
    storage type (FP32, FP16, BF16 deviation and plain FP64), each with the
    roofline of its step kernel (algorithmic bytes per lattice update over
    the average step time against the measured HBM copy rate; FP64 is bound
    by GB300's FP64 pipe, its fraction is of the same HBM peak)."""
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    n, steps = 8192, 1000
    out = {"workload": "single-8192x8192-1000-steps", "note": "one timed run of 1000 steps "
           "after 2 x 50 warm-up steps; 2.4-9.7 GB of populations per type (> L2)"}
    kern = {"f32": "k_step_dev<float>", "f16": "k_step_dev<__half>",
            "bf16": "k_step_dev<__nv_bfloat16>", "f64": "k_step_f64",
            "f64dev": "k_step_dev<double>"}
    for dtype in ("f32", "f16", "bf16", "f64", "f64dev"):
        mlups, ms = large_one(L, torch, stream, n, dtype, steps, 1, 2)
        achieved = BYTES_PER_LU[dtype] * n * n / (ms * 1e-3) / 1e9
        out[dtype] = {"mlups": round(mlups, 1), "ms_per_lbm_step": round(ms, 4),
                      "roofline": {"bound": "hbm" if not dtype.startswith("f64") else "fp64-alu",
                                   "kernel": kern[dtype], "achieved": round(achieved, 1),
                                   "peak": peak, "unit": "GB/s",
                                   "frac": round(achieved / peak, 4), "peak_source": peak_kind}}
    return out


def bench_serving(args, L, torch):
    """Poisson request stream through lbm_submit / lbm_poll."""
    reqs = inp.request_stream(args.requests, seed=1107 + 5)
    srv = L.lbm_server_create(150 * 10**9, 100)
    L.lbm_server_set_policy(srv, L.LBM_SERVE_SHORTEST if args.policy == "shortest"
                            else L.LBM_SERVE_FIFO, args.max_nodes)
    ids = {}
    t0 = time.perf_counter()
    k = 0
    pending = {}
    lat = []
    failed = 0
    # the admitted-concurrency trace: every 2 s, [time s, resident lattices,
    # resident GB, requests waiting for admission]
    trace = []
    next_sample = 0.0
    while k < len(reqs) or pending:
        now = time.perf_counter() - t0
        if now >= next_sample:
            st = L.lbm_server_stats(srv)
            trace.append([round(now, 1), st["resident"], round(st["resident_bytes"] / 1e9, 2),
                          st["submitted"] - st["admitted"]])
            next_sample += 2.0
        while k < len(reqs) and reqs[k]["arrival"] <= now:
            q = reqs[k]
            init = q["init"]
            if init["kind"] == "gaussian":
                kind, params = L.LBM_INIT_GAUSSIAN, (init["amp"], init["b"], init["xc"], init["yc"])
            else:
                kind, params = L.LBM_INIT_PLANE, (init["amp"], init["m"])
            req, _ = L.make_request(q["nx"], q["ny"], inp.s_ll(q["rates"]), q["steps"],
                                    dtype=q["dtype"], init_kind=kind, init_params=params)
            pending[L.lbm_submit(srv, req)] = q
            k += 1
        for rid in L.lbm_server_done(srv):
            try:
                _, _, _, _, latency = L.lbm_poll(srv, rid)
                lat.append(latency)
            except L.LbmError:
                failed += 1
            del pending[rid]
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    st = L.lbm_server_stats(srv)
    L.lbm_server_destroy(srv)
    lu = sum(q["nx"] * q["ny"] * q["steps"] for q in reqs)
    return {"metric": "served MLUPS and solve latency", "value": round(lu / wall / 1e6, 1),
            "unit": "MLUPS", "higher_is_better": True,
            "config": {"workload": "serving-poisson-%d-requests" % len(reqs),
                       "policy": args.policy, "max_resident_nodes": args.max_nodes,
                       "hbm_budget_gb": 150, "chunk_steps": 100},
            "latency_s": {"p50": round(float(np.percentile(lat, 50)), 3),
                          "p99": round(float(np.percentile(lat, 99)), 3),
                          "definition": "submit to moments on the host"},
            "requests": {"completed": len(lat), "failed": failed},
            "peak_resident_lattices": st["peak_resident"],
            "wall_s": round(wall, 2),
            "admitted_trace": {"columns": ["t_s", "resident_lattices", "resident_gb", "queued"],
                               "every_s": 2.0, "samples": trace},
            "server": st}


def bench_slabs(args, L, torch):
    """One n x n FP32 lattice split into 1, 2 and 4 y-slabs on this one GPU
    (lbm_slabs_*), against the unsplit lattice: MLUPS per split, i.e. what
    the boundary-row launches and the halo copies cost when nothing is
    gained from more devices."""
    n, steps = args.size, 200
    r = inp.rates("OPT")
    fields = inp.gaussian_pulse(n, n, 1e-3, 20.0)
    stream = torch.cuda.current_stream()
    out = {}
    mlups, _ = large_one(L, torch, stream, n, "f32", steps, 1, 1)
    out["unsplit"] = round(mlups, 1)
    for k in (1, 2, 4):
        s = L.lbm_slabs_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.LBM_F32DEV, k)
        try:
            L.lbm_slabs_init_field(s, *fields)
            L.lbm_slabs_step(s, 20)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.lbm_slabs_step(s, steps)
            L.lbm_slabs_drift(s)  # synchronizes every slab
            dt = time.perf_counter() - t0
        finally:
            L.lbm_slabs_destroy(s)
        out["slabs_%d" % k] = round(n * n * steps / dt / 1e6, 1)
    return {"metric": "MLUPS, one %dx%d FP32 lattice split into y-slabs on one GPU" % (n, n),
            "value": out["slabs_2"], "unit": "MLUPS", "higher_is_better": True,
            "config": {"workload": "slabs-%dx%d-fp32-%d-steps" % (n, n, steps)},
            "per_split": out,
            "note": "host-timed over the steps (slab steps are issued from the host: one "
                    "boundary-row pair and one interior launch per slab and step, four halo "
                    "copies per slab and step)"}


def bench_small(args, L, torch):
    """A sweep of small lattices (config 4's sampling with areas 32^2 - 56^2,
    `--lattices` of them, FP32 deviation storage, 500 steps per call): MLUPS
    with the members held in shared memory for all the steps of a call
    (k_batch_resident) and with the per-step launches alone
    (LBM_RESIDENT_BYTES=0), the same handles re-initialised in between."""
    n = args.lattices
    specs = inp.batch_specs(n, seed=1107 + 6, amin=32 * 32, amax=56 * 56, steps=500)
    stream = torch.cuda.current_stream()
    hs, fields = setup_batch(L, torch, specs, "f32", stream)
    nodes = sum(sp["nx"] * sp["ny"] for sp in specs)
    out = {}
    try:
        for mode in ("resident", "per_step"):
            if mode == "per_step":
                os.environ["LBM_RESIDENT_BYTES"] = "0"
            for h, f in zip(hs, fields):
                L.lbm_init_field(h, *f)
            b = L.lbm_batch_create(hs)
            try:
                nres = int(L.lbm_batch_resident(b).sum())
                L.lbm_batch_step(b, 500)  # warm-up (and tuning)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.steps):
                    L.lbm_batch_step(b, 500)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
            finally:
                L.lbm_batch_destroy(b)
            out[mode] = {"mlups": round(nodes * 500 * args.steps / (ms * 1e-3) / 1e6, 1),
                         "ms_per_500_steps": round(ms / args.steps, 3),
                         "resident_lattices": nres}
    finally:
        os.environ.pop("LBM_RESIDENT_BYTES", None)
        for h in hs:
            L.lbm_destroy(h)
    return {"metric": "MLUPS, a sweep of %d small FP32-deviation lattices" % n,
            "value": out["resident"]["mlups"], "unit": "MLUPS", "higher_is_better": True,
            "config": {"workload": "sweep-%d-lattices-32to56-fp32dev-500-steps" % n,
                       "nodes": nodes},
            "modes": out,
            "speedup": round(out["resident"]["mlups"] / out["per_step"]["mlups"], 2)}


def bench_vn(args, L, torch):
    """Von Neumann sweep (sections 4.1-4.2): eigenvalues of G(k) on a grid
    of 256 |k| x 64 directions x U in {0, 0.1} x 4 rate sets."""
    import oracle.vn as ovn

    kk = np.linspace(0.0, math.pi, 257)[1:]
    th = np.linspace(0.0, 2 * math.pi, 64, endpoint=False)
    K, T = np.meshgrid(kk, th, indexing="ij")
    kx, ky = (K * np.cos(T)).ravel(), (K * np.sin(T)).ravel()
    cases = []
    for U in (0.0, 0.1):
        for name in ("LL", "LL*", "OPT", "OPT-Z"):
            cases.append((U, inp.rates(name, nu=1e-3)))
    n = kx.size * len(cases)
    KX = np.tile(kx, len(cases))
    KY = np.tile(ky, len(cases))
    UU = np.repeat([c[0] for c in cases], kx.size)
    SS = np.repeat(np.array([inp.s_ll(c[1]) for c in cases]), kx.size, axis=0)
    L.lbm_vn_eigs(KX[:1000], KY[:1000], UU[:1000], 0.0, SS[:1000])  # warm-up
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        L.lbm_vn_eigs(KX, KY, UU, 0.0, SS)
        times.append(time.perf_counter() - t0)
    gpu = n / min(times)
    # CPU baseline: numpy eigvals of the oracle's matrices for one rate set
    t0 = time.perf_counter()
    G = ovn.amplification(kx, ky, 0.1, 0.0, inp.s_paper(cases[-1][1]))
    np.linalg.eigvals(G)
    cpu = kx.size / (time.perf_counter() - t0)
    return {"metric": "von Neumann eigenproblems (9x9 complex) per second",
            "value": round(gpu, 1), "unit": "problems/s", "higher_is_better": True,
            "config": {"workload": "vn-sweep-%d-cases" % n},
            "note": "host (pageable) arrays in and out per call, best of the timed calls",
            "cpu_baseline": {"value": round(cpu, 1), "unit": "problems/s", "cores": 1,
                             "kind": "oracle", "sample": "%d cases, numpy eigvals" % kx.size}}


def bench_opt(args, L, torch):
    """Free-parameter optimization (sections 3.2, 4.2): calligraphic G of
    section 3.2.3 (n = 4, flow speeds in [0, 0.2]) for a 32 x 32 grid of
    (sigma_eps, sigma_q) candidates -- 4800 quadrature points each, one
    modified-equation recursion per point -- and the full minimization that
    reproduces Table 3 group A."""
    import oracle.modified as om

    t3 = inp.TABLE3["A"]
    e = np.logspace(-5, 0, 32)
    E, Qg = np.meshgrid(e, e, indexing="ij")
    sig = np.column_stack([np.full(E.size, t3["sigma_e"]), E.ravel(), Qg.ravel(),
                           np.full(E.size, t3["sigma_nu"])])
    spec = L.cost_spec("G", 4, "all", "ns-bulk")
    L.lbm_opt_cost(spec, sig[:8])  # warm-up
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        L.lbm_opt_cost(spec, sig)
        times.append(time.perf_counter() - t0)
    rate = sig.shape[0] / min(times)
    t0 = time.perf_counter()
    r, c, ev = L.lbm_opt_minimize(spec, dict(t3, sigma_eps=0.5, sigma_q=0.5),
                                  ("sigma_eps", "sigma_q"), dict(sigma_eps=0.0, sigma_q=0.0),
                                  dict(sigma_eps=1.0, sigma_q=1.0))
    t_min = time.perf_counter() - t0
    # CPU baseline: the oracle's cost (numpy, vectorized over the points)
    t0 = time.perf_counter()
    nc = 4
    for k in range(nc):
        om.cost(sig[k * 97], 4, "G", "all", 0.2, "ns-bulk")
    cpu = nc / (time.perf_counter() - t0)
    return {"metric": "section 3.2 cost evaluations (calligraphic G, n = 4) per second",
            "value": round(rate, 2), "unit": "costs/s", "higher_is_better": True,
            "config": {"workload": "opt-G-n4-%d-candidates" % sig.shape[0],
                       "points_per_cost": 4800},
            "minimize": {"seconds": round(t_min, 3), "evals": ev, "cost": c,
                         "sigma_eps": r["sigma_eps"], "sigma_q": r["sigma_q"],
                         "printed": {"sigma_eps": t3["sigma_eps"], "sigma_q": t3["sigma_q"],
                                     "cost": 14.453655614637361}},
            "note": "host arrays in and out, device allocation per call included",
            "cpu_baseline": {"value": round(cpu, 3), "unit": "costs/s", "cores": 1,
                             "kind": "oracle", "sample": "%d candidates, numpy" % nc}}


def bench_source(args, L, torch):
    """The point-source experiment of section 5.1: a 101 x 101 periodic
    lattice with the node at its centre forced to rho0 + rho_s sin(2 pi t/T)
    (rho_s = 0.01, T = 20), for the three schemes compared there -- BGK, the
    original MRT and the optimized one (Table 4 group A) -- in FP64 and
    FP32 deviation storage.  A lattice this small is bound by launch
    latency: the forced steps run as graphs of 64 (forced node, step)
    pairs."""
    import oracle as orc

    stream = torch.cuda.current_stream()
    n, rs, period, steps = 101, 0.01, 20.0, 64 * 64
    t4 = inp.TABLE4["A"]
    schemes = {"BGK": dict(s_e=t4["s_nu"], s_eps=t4["s_nu"], s_q=t4["s_nu"], s_nu=t4["s_nu"]),
               "original": dict(s_e=t4["s_e"], s_eps=inp.LL["s_eps"], s_q=inp.LL["s_q"],
                                s_nu=t4["s_nu"]),
               "optimized": inp.rates("OPT-Z")}
    per = {}
    for dtype in ("f64", "f32"):
        for name, r in schemes.items():
            h = L.lbm_create(n, n, inp.s_ll(r), 1.0, (0.0, 0.0), L.DTYPES[dtype])
            try:
                L.lbm_set_stream(h, stream)
                L.lbm_set_source(h, n // 2, n // 2, rs, period)
                L.lbm_step(h, 64 * max(args.warmup, 1))
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                L.lbm_step(h, steps)
                e1.record()
                torch.cuda.synchronize()
                per["%s-%s" % (name, dtype)] = round(n * n * steps / (e0.elapsed_time(e1) * 1e3), 1)
            finally:
                L.lbm_destroy(h)
    # CPU baseline: the oracle's forced run of the optimized scheme
    f0 = orc.init_eq(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    cpu_steps = 2000
    t0 = time.perf_counter()
    orc.run_source(f0, inp.s_paper(schemes["optimized"]), cpu_steps, (n // 2, n // 2, rs, period))
    cpu = n * n * cpu_steps / (time.perf_counter() - t0) / 1e6
    return {"metric": "MLUPS, section 5.1 point source, 101x101, forced steps",
            "value": per["optimized-f32"], "unit": "MLUPS", "higher_is_better": True,
            "config": {"workload": "point-source-101x101-%d-steps" % steps, "period": period,
                       "rho_s": rs},
            "per_scheme": per,
            "note": "launch-latency bound: 10,201 nodes per step",
            "cpu_baseline": {"value": round(cpu, 1), "unit": "MLUPS", "cores": orc.threads(),
                             "kind": "oracle", "sample": "optimized scheme, %d steps" % cpu_steps}}


def oracle_timing(args):
    """The FP64 CPU oracle as it stands on the host cores: config 1 in full
    with one thread and with all cores, and config 3 (8192^2) timed over 20
    steps with all cores, extrapolated to its 1000 steps.  CPU only."""
    import oracle as orc

    cores = os.cpu_count() or 1
    out = {"metric": "FP64 CPU oracle MLUPS", "unit": "MLUPS", "cores": cores,
           "kind": "oracle"}
    n, steps = 64, 200
    fields = inp.gaussian_pulse(n, n, 1e-3, 4.0)
    s = inp.s_paper(inp.rates("LL", nu=1e-3))
    for threads in (1, cores):
        orc.set_threads(threads)
        f = orc.init_eq(*fields)
        orc.run(f, s, 5)
        t0 = time.perf_counter()
        orc.run(f, s, steps)
        dt = time.perf_counter() - t0
        out["config1_64x64_200_steps_%d_threads" % threads] = round(n * n * steps / dt / 1e6, 2)
    n, steps = 8192, 20
    orc.set_threads(cores)
    rho, ux, uy = inp.pulse_with_vortices(n, n, seed=1107 + 3)
    f = orc.init_eq(rho, ux, uy)
    del rho, ux, uy
    s = inp.s_paper(inp.rates("OPT"))
    orc.run(f, s, 1)
    t0 = time.perf_counter()
    orc.run(f, s, steps)
    dt = time.perf_counter() - t0
    out["config3_8192x8192"] = {"mlups": round(n * n * steps / dt / 1e6, 2),
                                "seconds_per_step": round(dt / steps, 3),
                                "extrapolated_1000_steps_s": round(1000 * dt / steps, 1)}
    return out


def reference_arm(args):
    """The CPU oracle timed as the reference implementation."""
    specs = inp.batch_specs(args.lattices, seed=1107 + 4, steps=args.lbm_steps)
    vals = []
    for k in range(args.warmup + args.steps):
        mlups, cores, sample = cpu_oracle_mlups(specs, target_s=12.0)
        if k >= args.warmup:
            vals.append(mlups)
    v = float(np.mean(vals))
    return {"impl": "reference", "metric": "MLUPS (lattice updates/s, millions), batched "
            "FP32-deviation D2Q9 MRT", "value": round(v, 2), "unit": "MLUPS",
            "higher_is_better": True, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched-512-lattices-fp32dev-500-steps"},
            "cpu_baseline": {"value": round(v, 2), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 2), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return
    if args.workload == "oracle":
        if rank == 0:
            print(json.dumps(oracle_timing(args)))
        return
    import torch

    from paper_1107_4543_gb300 import build, lbm as L

    if rank == 0 or not os.path.exists(L.LIB_PATH):
        build.build()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
        torch.distributed.barrier()
    else:
        torch.cuda.set_device(0)
    # all work on one non-default stream: the library launches on it (the
    # handle of the legacy default stream is 0, which lbm_set_stream reads as
    # "the handle's own stream"), and the CUDA events record on it
    torch.cuda.set_stream(torch.cuda.Stream())
    L.load()
    if args.workload == "large":
        if rank == 0:
            for line in bench_large(args, L, torch, rank, ws):
                print(json.dumps(line))
        return
    if args.workload == "serving":
        if rank == 0:
            print(json.dumps(bench_serving(args, L, torch)))
        return
    if args.workload == "vn":
        if rank == 0:
            print(json.dumps(bench_vn(args, L, torch)))
        return
    if args.workload == "slabs":
        if rank == 0:
            print(json.dumps(bench_slabs(args, L, torch)))
        return
    if args.workload == "small":
        if rank == 0:
            print(json.dumps(bench_small(args, L, torch)))
        return
    if args.workload == "opt":
        if rank == 0:
            print(json.dumps(bench_opt(args, L, torch)))
        return
    if args.workload == "source":
        if rank == 0:
            print(json.dumps(bench_source(args, L, torch)))
        return
    line, specs = bench_batched(args, L, torch, rank, ws)
    if rank == 0 and ws == 1 and not args.no_extras:
        # the other workloads at their stated sizes, as extra keys of the one
        # line: the batch in FP16 deviation storage, config 3 per storage
        # type, a sweep of small lattices, config 5 serving
        sub = parse(["--batch-dtype", "f16", "--steps", str(max(3, min(args.steps, 5))),
                     "--warmup", "3", "--no-fp64"])
        f16, _ = bench_batched(sub, L, torch, rank, ws)
        line["batch_fp16"] = {k: f16[k] for k in ("value", "unit", "ms_per_step", "roofline",
                                                  "e2e", "clocks")}
        line["batch_fp16"]["workload"] = f16["config"]["workload"]
        line["config3_large"] = config3_record(L, torch)
        # small lattices held in shared memory for all the steps of a call,
        # against per-step launches of the same sweep
        line["small_sweep"] = bench_small(parse(["--workload", "small", "--lattices", "4096",
                                                 "--steps", "3"]), L, torch)
        srv = parse(["--workload", "serving", "--policy", "shortest",
                     "--max-nodes", str(1 << 27), "--requests", str(args.requests)])
        line["config5_serving"] = bench_serving(srv, L, torch)
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            mlups, cores, sample = cpu_oracle_mlups(specs)
            line["cpu_baseline"] = {"value": round(mlups, 2), "unit": "MLUPS", "cores": cores,
                                    "kind": "oracle", "sample": sample}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
