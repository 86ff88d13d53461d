#!/usr/bin/env python
"""Benchmark of the hot path: Lanczos steps on the 4x8 Heisenberg S^z=0 sector.

Workload: spin-1/2 Heisenberg J1 model on the 4x8 periodic square lattice
(N=32, site = x + 8y), S^z=0 sector, D = C(32,16) = 601,080,390 rows.  One
step is one Lanczos iteration through hphi_lanczos: the fused H*x kernel
(u = H w_k / beta_k - beta_k/beta_{k-1} w_{k-1} with <w_k, u>), the vector
pass (w_{k+1} = u - alpha_k/beta_k w_k with |w_{k+1}|^2), and the device-side
alpha/beta bookkeeping.  The timed region is one hphi_lanczos call of K steps
(its start-vector copy and norm, and the final host tridiagonal solve,
included).

metric: H*x GB/s = steps * (algorithmic H*x bytes: read x + write y, 8 B/row
per FP32 vector / 16 B/row FP64) / time, summed over ranks.  Vectors are FP32
by default (FP64 alpha/beta and reductions); --dtype f64 runs FP64 vectors,
and the default run also measures the FP64 path and reports it under "fp64".

--impl reference times the CPU oracle (plain C, OpenMP row loop) on a bounded
row sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

D_4X8 = 601080390
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(seconds: float = 15.0):
    """The CPU oracle's H*x over a bounded contiguous row sample of the 4x8
    S^z=0 workload; returns (GB/s H*x-equivalent, threads, sample text)."""
    import numpy as np
    import oracle as O
    from workloads import configs
    O.build()
    cfg = configs.heisenberg_square4x8()
    m = O.Model("SPIN_HALF", 32, 16, 0, cfg["terms"])
    x = np.zeros(m.dim)  # lazily mapped; the values do not change the oracle's work
    y = np.zeros(m.dim)
    r0 = m.dim // 3
    n = 20000
    t0 = time.perf_counter()
    m.apply(x, y=y, rows=(r0, r0 + n))
    dt = time.perf_counter() - t0
    n = int(min(m.dim - r0, max(n, n * seconds / max(dt, 1e-6))))
    return m, x, y, r0, n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    m, x, y, r0, n = oracle_sample(seconds=max(2.0, 20.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        m.apply(x, y=y, rows=(r0, r0 + n))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m.apply(x, y=y, rows=(r0, r0 + n))
    dt = (time.perf_counter() - t0) / args.steps
    gbs = 16.0 * n / dt / 1e9
    sample = f"oracle H*x (pull form, FP64) over rows [{r0}, {r0 + n}) of the 4x8 S^z=0 sector per step"
    line = {"impl": "reference", "metric": "hv_gbps", "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "heisenberg_square_4x8_Sz0", "n_sites": 32, "dim": D_4X8,
                       "sample_rows": n, "l2": "host run"},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(ms, dist, device="cuda"):
    """The job's time is its slowest replica's: MAX of the per-rank times."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbps(world, bytes_per_rank, ms):
    """Whole-job throughput: every replica moves the same bytes in parallel."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def lanczos_steps(ham, v0, steps):
    from paper_2307_13222_gb300 import hphi
    return hphi.hphi_lanczos(ham, v0, steps, 0.0, check_every=steps)


def measure_dtype(ctx, ham, dim, dtype_name, K, W, dist, world):
    import torch
    from paper_2307_13222_gb300 import hphi
    tdt = torch.float32 if dtype_name == "f32" else torch.float64
    es = 4 if dtype_name == "f32" else 8
    v0 = torch.empty(dim, dtype=tdt, device="cuda")
    hphi.hphi_random_vector(ctx, v0, 2)
    lanczos_steps(ham, v0, max(W, 1))
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(0)
    ctx.profile_read(1)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    r = lanczos_steps(ham, v0, K)
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    hv_n, hv_ms = ctx.profile_read(0)
    vec_n, vec_ms = ctx.profile_read(1)
    ctx.profile(False)
    ms = max_over_ranks(ms, dist)
    del v0
    torch.cuda.empty_cache()
    return dict(ms=ms, wall_s=wall, value=job_gbps(world, K * 2.0 * es * dim, ms), hv_launches=hv_n, hv_ms=hv_ms,
                vec_launches=vec_n, vec_ms=vec_ms, e0=r["e0"], steps=r["steps"], es=es)


def issue_roofline(path, kernel_name, rows, avg_ms, sms, mhz):
    """Issue-rate bound of the single-column kernel: warp instructions per row
    (from a committed ncu summary of the same kernel family and source hash on
    the 6x5 sector) x rows / (SMs x 4 schedulers x SM clock); null unless the
    summary's kernel shares the running kernel's family and hash."""
    if not os.path.exists(path) or "@" not in kernel_name:
        return None
    rec = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.split(":")[0] in ("kernel", "warp_inst_per_row"):
                k, v = ln.split(":", 1)
                rec[k] = v.strip()
    if "kernel" not in rec or "warp_inst_per_row" not in rec:
        return None
    fam = lambda n: (n.split("<")[0] + "<" + ",".join(n.split("<")[1].split(",")[:2]), n.split("@")[-1])
    if fam(rec["kernel"]) != fam(kernel_name):
        return None
    wipr = float(rec["warp_inst_per_row"])
    bound_ms = rows * wipr / (sms * 4 * mhz * 1e6) * 1e3
    return {"bound": "issue", "warp_inst_per_row": wipr, "bound_ms": bound_ms, "achieved_ms": avg_ms,
            "frac": bound_ms / avg_ms, "clock_mhz": mhz, "source": "hv_single_column_square6x5_ncu.md"}


def measure_precision(ham, dim, K):
    """Energy of the FP32-storage path against the FP64 path on the same
    workload and start vector (untimed): K Lanczos steps plus the ground-state
    pass in each precision; the Ritz value and the FP64 Rayleigh quotient of
    the returned vector (the refined energy) of the FP32 run, each relative to
    the FP64 run's Rayleigh quotient."""
    import torch
    from paper_2307_13222_gb300 import hphi
    out = {}
    for name, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        v0 = torch.empty(dim, dtype=tdt, device="cuda")
        hphi.hphi_random_vector(ham.ctx, v0, 2)
        gs = torch.empty_like(v0)
        r = hphi.hphi_lanczos(ham, v0, K, 0.0, check_every=K, gs_out=gs)
        out[name] = (r["e0"], r["e0_rq"])
        del v0, gs
        torch.cuda.empty_cache()
    ref = out["f64"][1]
    return {"steps": K, "e0_f64_rq": ref, "e0_f64_ritz": out["f64"][0], "e0_f32_ritz": out["f32"][0],
            "ritz_rel_err_f32": abs(out["f32"][0] - ref) / abs(ref),
            "rq_rel_err_f32": abs(out["f32"][1] - ref) / abs(ref), "ritz_rel_err_f64": abs(out["f64"][0] - ref) / abs(ref)}


def measure_block_leg(ctx, steps=2, autotune=True):
    """The cTPQ benchmark's block H*V at its own size: 16 complex FP32 columns
    over the 2^26 states of the 26-site random 3-regular graph; `steps` TPQ
    steps (6 Horner stages each) after one warm-up step, the stage kernel timed
    by the library's CUDA events.  Algorithmic bytes per stage: read V, gather
    W, write W' = 3 x 8 B per row and complex column."""
    import numpy as np
    import torch
    from paper_2307_13222_gb300 import hphi
    from workloads import configs
    cfg = configs.ctpq_random_regular()
    b = hphi.Basis(ctx, "SPIN_HALF_GC", cfg["n_sites"])
    h = hphi.Hamiltonian(ctx, b, cfg["terms"])
    tuned = h.autotune(torch.complex64, cfg["n_vec"], reps=2) if autotune else None
    V = torch.empty((b.dim, cfg["n_vec"]), dtype=torch.complex64, device="cuda")
    hphi.hphi_random_vector(ctx, V, cfg["seed"])
    n2 = np.zeros(cfg["n_vec"])
    hphi.hphi_tpq_step(h, V, cfg["dtau"], cfg["nmax"], n2)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(0)
    for _ in range(steps):
        hphi.hphi_tpq_step(h, V, cfg["dtau"], cfg["nmax"], n2)
    n, ms = ctx.profile_read(0)
    ctx.profile(False)
    kernel = ctx.last_kernel()
    del V, h, b
    torch.cuda.empty_cache()
    stage_bytes = 3.0 * 8 * cfg["n_vec"] * (1 << cfg["n_sites"])
    avg = ms / max(n, 1)
    peak, kind = peaks()
    ach = stage_bytes / (avg * 1e-3) / 1e9
    # DRAM bytes per stage from the committed ncu summary of the same kernel
    # pair and sources (the stages differ only in their reductions)
    traffic = traffic_for(os.path.join(ROOT, "profiles", "hv_tiled_block_rrg26_c64_traffic.md"), kernel,
                          key="bytes_per_stage", same_family=True)
    return {"workload": "ctpq_rrg3_N26_B16_c64", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": "of measured" if kind == "measured" else "of fallback",
            "traffic": traffic, "avg_stage_ms": avg, "stages": n, "bytes_per_stage": stage_bytes, "kernel": kernel,
            "autotuned_ms": tuned[0] if tuned else None}


def traffic_for(path, kernel_name, key="bytes_per_launch", same_family=False):
    """DRAM bytes per launch from a committed ncu summary, or None unless the
    summary's `kernel:` line names exactly the kernel instance that ran (its
    template arguments and the hash of the sources it was built from); with
    same_family, the kernel name before its template arguments and the hash
    must agree."""
    if not os.path.exists(path) or not kernel_name:
        return None
    rec = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.split(":")[0] in ("kernel", key):
                k, v = ln.split(":", 1)
                rec.setdefault(k, v.strip())
    if key not in rec or "kernel" not in rec:
        return None
    if same_family:
        fam = lambda n: (n.split("<")[0], n.split("@")[-1] if "@" in n else None)
        ok = "@" in rec["kernel"] and fam(rec["kernel"]) == fam(kernel_name)
    else:
        ok = rec["kernel"] == kernel_name
    return float(rec[key]) if ok else None


def gpu_local_cpus(dev):
    """The host CPUs next to GPU `dev` (its PCI device's local_cpulist), or None."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        dom, bus, d = p.pci_domain_id, p.pci_bus_id, p.pci_device_id
        with open(f"/sys/bus/pci/devices/{dom:04x}:{bus:02x}:{d:02x}.0/local_cpulist") as f:
            txt = f.read().strip()
    except Exception:  # no PCI ids in this torch, no sysfs entry, no GPU
        return None
    return parse_cpulist(txt)


def parse_cpulist(txt):
    """CPU set of a sysfs cpulist ("0-71,144-215"), or None when empty."""
    cpus = set()
    for part in txt.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.update(range(int(a), int(b or a) + 1))
    return cpus or None


def measure_e2e(ctx, ham, dim, dtype_name, K, world=1):
    """H*x through the public API with HOST buffers: one hphi_apply_H_host call
    over a batch of pinned host vectors.  The timed call (wall clock) includes,
    for every vector, its copy to the device, the product and the copy of the
    result back; inside the library the copies of one vector overlap the
    product of its neighbours.  Per-step figures are per vector."""
    import torch
    from paper_2307_13222_gb300 import hphi
    tdt = torch.float32 if dtype_name == "f32" else torch.float64
    es = 4 if dtype_name == "f32" else 8
    # vectors per call: up to 8, with the pinned buffers of all ranks of the node
    # (2 x nb vectors each) kept under a quarter of its memory
    try:
        host_bytes = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        host_bytes = 64 << 30
    fit = int(0.25 * host_bytes / max(world, 1) / (2.0 * es * dim))
    if fit < 1:
        return dict(skipped=f"one host vector pair ({2 * es * dim} bytes) exceeds a quarter of the node's memory "
                            f"shared among {world} ranks")
    nb = min(max(K, 1), 8, fit)
    # pinned buffers on the GPU's own host memory node: allocated (and first
    # touched) from the CPUs next to the GPU; a remote node's memory halves or
    # worse the device's reads over the host link
    local = gpu_local_cpus(torch.cuda.current_device())
    saved = os.sched_getaffinity(0) if local else None
    if local:
        try:
            os.sched_setaffinity(0, local & saved or local)
        except OSError:
            local = None
    try:
        xh = torch.empty((nb, dim), dtype=tdt, pin_memory=True)
        yh = torch.empty((nb, dim), dtype=tdt, pin_memory=True)
        xh.zero_()
        yh.zero_()
    finally:
        if saved:
            os.sched_setaffinity(0, saved)
    xd = torch.empty(dim, dtype=tdt, device="cuda")
    for k in range(nb):
        hphi.hphi_random_vector(ctx, xd, 3 + k)
        xh[k].copy_(xd)
    del xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    hphi.hphi_apply_H_host(ham, xh, yh)  # warm-up: device buffers, streams, first DMA of every page (untimed)
    torch.cuda.synchronize()
    calls = []
    for _ in range(3):  # three timed calls, the median reported
        t0 = time.perf_counter()
        hphi.hphi_apply_H_host(ham, xh, yh)
        calls.append((time.perf_counter() - t0) * 1e3 / nb)
    ms = statistics.median(calls)
    # this machine's host link, for reading the number: one plain copy each way
    xd = torch.empty(dim, dtype=tdt, device="cuda")
    link = {}
    for name, fn in (("h2d_gbps", lambda: xd.copy_(xh[0], non_blocking=True)),
                     ("d2h_gbps", lambda: yh[0].copy_(xd, non_blocking=True))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        link[name] = es * dim / (time.perf_counter() - t0) / 1e9
    del xh, yh, xd
    torch.cuda.empty_cache()
    link["buffers_on"] = f"GPU-local CPUs ({len(local)})" if local else "default placement"
    return dict(value=2.0 * es * dim / (ms * 1e-3) / 1e9, ms=ms, h2d=es * dim, d2h=es * dim, batch=nb, calls=calls,
                link=link)


def run_native(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    import paper_2307_13222_gb300 as P
    from paper_2307_13222_gb300 import hphi
    from workloads import configs
    if rank == 0 or not os.path.exists(P.LIBRARY_PATH):
        P.build()
    if dist:
        dist.barrier()
    ctx = hphi.Context(local)
    cfg = configs.heisenberg_square4x8()
    basis = hphi.Basis(ctx, "SPIN_HALF", 32, 16)
    ham = hphi.Hamiltonian(ctx, basis, cfg["terms"])
    dim = basis.dim
    tuned = None
    if not args.no_autotune:  # launch settings chosen by the library's autotuner (untimed set-up)
        import torch as _t
        tuned = ham.autotune(_t.float32 if args.dtype == "f32" else _t.float64, 1, reps=2)
    K, W = args.steps, args.warmup
    clocks = ClockSampler(local)
    clocks.start()
    main = measure_dtype(ctx, ham, dim, args.dtype, K, W, dist, world)
    ck = clocks.stop()
    kernel_name = ctx.last_kernel()  # the fused H*x kernel of the timed Lanczos steps
    # ranks sharing this node's host memory (torchrun sets LOCAL_WORLD_SIZE)
    node_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
    e2e = measure_e2e(ctx, ham, dim, args.dtype, K, node_ranks) if not args.no_e2e else None
    other = None
    if args.dtype == "f32" and not args.no_fp64:
        other = measure_dtype(ctx, ham, dim, "f64", max(2, K // 4), 1, dist, world)
    prec = measure_precision(ham, dim, K) if args.dtype == "f32" and not args.no_fp64 else None
    # the oracle's 20-step FP64 run from the same start vector (when the golden is present)
    gold20 = None
    gpath = os.path.join(ROOT, "tests", "golden", "lanczos_square4x8_20steps.json")
    if os.path.exists(gpath) and K == 20:
        with open(gpath) as fh:
            gold20 = json.load(fh)["e0"]
    block = measure_block_leg(ctx, autotune=not args.no_autotune) if not args.no_block else None
    peak, peak_kind = peaks()
    # dominant kernel: the fused H*x of the Lanczos step; algorithmic bytes per
    # launch = gather x + read w_{k-1} + write u = 3 vectors (24 B/row FP64, 12 B/row FP32)
    hv_avg_ms = main["hv_ms"] / max(main["hv_launches"], 1)
    kern_bytes = 3.0 * main["es"] * dim
    achieved = kern_bytes / (hv_avg_ms * 1e-3) / 1e9
    # DRAM bytes per launch of this kernel from the committed ncu summary: null
    # unless the summary names exactly the kernel instance that ran here
    traffic = traffic_for(os.path.join(ROOT, "profiles", f"hv_fused_square4x8_{args.dtype}_traffic.md"),
                          kernel_name)
    mhz = (ck or {}).get("sm_mhz") or 2070.0
    issue = issue_roofline(os.path.join(ROOT, "profiles", "hv_single_column_square6x5_ncu.md"), kernel_name, dim,
                           hv_avg_ms, ctx.sm_count, mhz)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        m, x, y, r0, n = oracle_sample(seconds=15.0)
        t0 = time.perf_counter()
        m.apply(x, y=y, rows=(r0, r0 + n))
        dt = time.perf_counter() - t0
        cpu = {"value": 16.0 * n / dt / 1e9, "unit": "GB/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"oracle H*x (pull form, FP64) over rows [{r0}, {r0 + n}) of the same sector, "
                         f"{dt:.1f} s"}
    gpu_launches = 7 * K + 4
    line = {
        "metric": "hv_gbps", "value": main["value"], "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": main["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": "heisenberg_square_4x8_Sz0", "n_sites": 32, "dim": dim, "step": "lanczos_iteration",
                   "launch": ham.get_tuning(), "autotuned_ms": tuned[0] if tuned else None,
                   "vectors": args.dtype, "scalars": "f64", "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (one vector = %.1f GB)" % (main["es"] * dim / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel_name,
                     "peak_kind": peak_kind, "avg_launch_ms": hv_avg_ms, "issue": issue},
        "gpu_launches": gpu_launches,
        "kernel_ms": {"hv": main["hv_ms"], "vector": main["vec_ms"], "hv_launches": main["hv_launches"],
                      "vector_launches": main["vec_launches"]},
        "lanczos_e0_after_steps": main["e0"],
    }
    if ck:
        line["clocks"] = ck
    if e2e and "skipped" in e2e:
        line["e2e"] = {"value": None, "unit": "GB/s", "skipped": e2e["skipped"]}
    elif e2e:
        line["e2e"] = {"value": e2e["value"], "unit": "GB/s", "h2d_bytes_per_step": e2e["h2d"],
                       "d2h_bytes_per_step": e2e["d2h"], "ms_per_step": e2e["ms"], "step": "hphi_apply_H_host",
                       "vectors_per_call": e2e["batch"], "calls_ms_per_vector": e2e["calls"],
                       "host_link": e2e["link"]}
    if other:
        a64 = 3.0 * 8 * dim / ((other["hv_ms"] / max(other["hv_launches"], 1)) * 1e-3) / 1e9
        line["fp64"] = {"value": other["value"], "ms_per_step": other["ms"] / max(2, K // 4),
                        "hv_kernel_gbps": a64, "frac": a64 / peak}
    if cpu:
        line["cpu_baseline"] = cpu
    if prec:
        if gold20 is not None:
            # the Ritz values after the same 20 steps against the oracle's FP64 run
            prec["e0_oracle_golden_20_steps"] = gold20
            prec["ritz_rel_err_vs_oracle"] = {"f32": abs(prec["e0_f32_ritz"] - gold20) / abs(gold20),
                                              "f64": abs(prec["e0_f64_ritz"] - gold20) / abs(gold20)}
        line["precision"] = prec
    if block:
        line["block"] = block
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.profile(False)
    del ham, basis
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---- further workloads (one JSON line each, same contract keys) ----------------------------


def _setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    import paper_2307_13222_gb300 as P
    from paper_2307_13222_gb300 import hphi
    if rank == 0 or not os.path.exists(P.LIBRARY_PATH):
        P.build()
    if dist:
        dist.barrier()
    return world, rank, local, dist, hphi.Context(local)


def _finish(line, rank, dist, ctx):
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.profile(False)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _roofline(ctx, bytes_per_launch, kernel):
    n, ms = ctx.profile_read(0)
    peak, kind = peaks()
    avg = ms / max(n, 1)
    ach = bytes_per_launch / (avg * 1e-3) / 1e9 if n else 0.0
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "kernel": kernel, "peak_kind": peak_kind_text(kind), "avg_launch_ms": avg, "launches": n}


def peak_kind_text(kind):
    return "of measured" if kind == "measured" else "of fallback"


def _base(args, world, metric, value, unit, ms_step, dtype, config, hib=True):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": hib, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}


def run_chain16(args):
    """Lanczos solves of the N=16 chain S^z=0 sector (12,870 rows) to 1e-12.
    value: solves/s of the batched form (one thread block per solve, as many
    solves as fill the GPU per call, distinct seeded start vectors); p50/p99:
    latency of single solves through the same entry point; grid_path: the
    grid-wide hphi_lanczos for comparison.  One step = one batched call."""
    import torch
    import numpy as np
    from paper_2307_13222_gb300 import hphi
    from workloads import configs
    world, rank, local, dist, ctx = _setup(args)
    cfg = configs.heisenberg_chain16()
    b = hphi.Basis(ctx, "SPIN_HALF", 16, 8)
    h = hphi.Hamiltonian(ctx, b, cfg["terms"])
    nb = 4 * ctx.sm_count
    vs = []
    for i in range(nb):
        v = torch.empty(b.dim, dtype=torch.float64, device="cuda")
        hphi.hphi_random_vector(ctx, v, cfg["seed"] + i)
        vs.append(v)
    gss = [torch.empty_like(v) for v in vs]
    chunk = 16

    # requests ask for the energy (the configuration's result); the ground-state
    # vector pass is measured by the tests
    def solve_batch(n):
        return hphi.hphi_lanczos_batch([h] * n, vs[:n], cfg["max_steps"], cfg["tol"], check_every=chunk)

    for _ in range(max(args.warmup, 1)):
        solve_batch(nb)
        solve_batch(1)
    torch.cuda.synchronize()
    # single-solve latency
    lat = []
    for _ in range(max(args.steps, 20)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r1 = solve_batch(1)[0]
        e1.record()
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
    # batched throughput (the timed region)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        rb = solve_batch(nb)
    t1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), dist)
    assert all(r["converged"] for r in rb) and r1["converged"]
    # the grid-wide driver on the same problem
    g_lat = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        hphi.hphi_lanczos(h, vs[0], cfg["max_steps"], cfg["tol"])
        e1.record()
        torch.cuda.synchronize()
        g_lat.append(e0.elapsed_time(e1))
    # roofline of the batched kernel: algorithmic bytes of one Lanczos step per problem
    # (gather x + read w_{k-1} + write u, then read u, w_k + write w_{k+1}: 6 vectors of 8 B) x steps
    steps_total = sum(r["steps"] for r in rb)
    peak, pk = peaks()
    alg = 6.0 * 8 * b.dim * steps_total / (ms / args.steps * 1e-3) / 1e9
    # end to end: start vectors from pinned host memory, ground states back to it
    vh = [torch.empty(b.dim, dtype=torch.float64, pin_memory=True) for _ in range(nb)]
    for i in range(nb):
        vh[i].copy_(vs[i])
    torch.cuda.synchronize()
    t0.record()
    for _ in range(args.steps):
        for i in range(nb):
            vs[i].copy_(vh[i], non_blocking=True)
        rr = solve_batch(nb)
        eh = torch.tensor([r["e0"] for r in rr], dtype=torch.float64)  # the results on the host
    t1.record()
    torch.cuda.synchronize()
    e2e_ms = t0.elapsed_time(t1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        m = O.Model("SPIN_HALF", 16, 8, 0, cfg["terms"])
        vv = vs[0].cpu().numpy()
        n, t_start = 0, time.perf_counter()
        while time.perf_counter() - t_start < 10.0 or n == 0:
            m.lanczos(vv, cfg["max_steps"], cfg["tol"], want_gs=True)
            n += 1
        dt = time.perf_counter() - t_start
        cpu = {"value": n / dt, "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"{n} oracle Lanczos solves (textbook recurrence, Sturm bisection each step, second pass) "
                         f"of the same problem in {dt:.1f} s"}
    line = _base(args, world, "lanczos_solves_per_s", world * nb * args.steps / (ms * 1e-3), "solves/s",
                 ms / args.steps, "f64",
                 {"workload": "heisenberg_chain_N16_Sz0", "dim": b.dim, "tol": cfg["tol"],
                  "solves_per_step": nb, "steps_per_solve": rb[0]["steps"], "form": "batched, one block per solve",
                  "l2": "working set of a batch 0.3 MB x %d, L2-resident (no flush)" % nb,
                  "parallelism": f"replicas{world}"})
    line.update({"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                 "single_solve_per_s": 1e3 / float(np.mean(lat)),
                 "grid_path": {"p50_ms": float(np.percentile(g_lat, 50)), "solves_per_s": 1e3 / float(np.mean(g_lat))},
                 "e0": r1["e0"],
                 "roofline": {"bound": "hbm", "achieved": alg, "peak": peak, "unit": "GB/s", "frac": alg / peak,
                              "traffic": None, "kernel": "k_lzb (batched Lanczos, L2-resident)",
                              "peak_kind": peak_kind_text(pk)},
                 "gpu_launches": args.steps * ((rb[0]["steps"] + chunk - 1) // chunk + 1),
                 "e2e": {"value": world * nb * args.steps / (e2e_ms * 1e-3), "unit": "solves/s",
                         "h2d_bytes_per_step": 8 * b.dim * nb, "d2h_bytes_per_step": 8 * nb}})
    if ck:
        line["clocks"] = ck
    if cpu:
        line["cpu_baseline"] = cpu
    return _finish(line, rank, dist, ctx)


def run_hubbard4x4(args):
    """Lanczos with full reorthogonalisation on the 4x4 Hubbard model at half
    filling (165,636,900 rows), FP32 vectors with FP64 scalars, to 1e-10
    relative residual; the FP64 run's energy is the error reference."""
    import torch
    from paper_2307_13222_gb300 import hphi
    from workloads import configs
    world, rank, local, dist, ctx = _setup(args)
    cfg = configs.hubbard_square4x4()
    b = hphi.Basis(ctx, "HUBBARD", 16, 8, 8)
    h = hphi.Hamiltonian(ctx, b, cfg["terms"])
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    for dt_name, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        v0 = torch.empty(b.dim, dtype=tdt, device="cuda")
        hphi.hphi_random_vector(ctx, v0, cfg["seed"])
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(0)
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gs = torch.empty_like(v0)
        r = hphi.hphi_lanczos(h, v0, cfg["max_steps"], cfg["tol"], check_every=5, reorth=True, gs_out=gs)
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist)
        es = 4 if tdt == torch.float32 else 8
        roof = _roofline(ctx, 3.0 * es * b.dim, None)
        ctx.profile(False)
        # the name of the steps' H*x kernel (the last launch inside the solve is the
        # FP64 H*x of the Rayleigh quotient, counted in `launches` above): one
        # untimed product of the same precision
        hphi.hphi_apply_H(h, v0, gs)
        torch.cuda.synchronize()
        roof["kernel"] = ctx.last_kernel()
        roof["launches_note"] = "the Lanczos steps' H*x plus one FP64 H*x of the Rayleigh quotient"
        out[dt_name] = dict(ms=ms, r=r, roof=roof)
        del v0, gs
        torch.cuda.empty_cache()
    ck = clocks.stop()
    f32, f64 = out["f32"], out["f64"]
    gold = None
    gpath = os.path.join(ROOT, "tests", "golden", "lanczos_hubbard4x4_U8.json")
    if os.path.exists(gpath):
        with open(gpath) as fh:
            gold = json.load(fh)["e0"]
    es = 4
    line = _base(args, world, "hv_gbps", job_gbps(world, f32["r"]["steps"] * 2.0 * es * b.dim, f32["ms"]), "GB/s",
                 f32["ms"] / max(f32["r"]["steps"], 1), "f32",
                 {"workload": "hubbard_square_4x4_half_U8", "dim": b.dim, "step": "lanczos_iteration_with_cgs2",
                  "tol": cfg["tol"], "vectors": "f32", "scalars": "f64", "parallelism": f"replicas{world}",
                  "l2": "inputs larger than L2 (one vector = %.2f GB)" % (4 * b.dim / 1e9)})
    line["steps"] = f32["r"]["steps"]
    line.update({"roofline": f32["roof"], "e0_f32": f32["r"]["e0"], "e0_f64": f64["r"]["e0"],
                 "e0_rel_err_f32": abs(f32["r"]["e0"] - f64["r"]["e0"]) / abs(f64["r"]["e0"]),
                 "e0_rq_f32": f32["r"]["e0_rq"], "e0_rq_f64": f64["r"]["e0_rq"], "e0_oracle_golden": gold,
                 "rel_err_vs_oracle": None if gold is None else {
                     "f32_ritz": abs(f32["r"]["e0"] - gold) / abs(gold),
                     "f32_rayleigh_fp64": abs(f32["r"]["e0_rq"] - gold) / abs(gold),
                     "f64_ritz": abs(f64["r"]["e0"] - gold) / abs(gold)},
                 "time_to_solution_s": {"f32": f32["ms"] / 1e3, "f64": f64["ms"] / 1e3},
                 "lanczos_steps": {"f32": f32["r"]["steps"], "f64": f64["r"]["steps"]},
                 "gpu_launches": None})
    if ck:
        line["clocks"] = ck
    return _finish(line, rank, dist, ctx)


def run_ctpq26(args):
    """cTPQ steps on the full 2^26 space of the Heisenberg model on a seeded
    random 3-regular graph, 16 complex vectors, nmax=6, dtau=0.02."""
    import torch
    import numpy as np
    from paper_2307_13222_gb300 import hphi
    from workloads import configs
    world, rank, local, dist, ctx = _setup(args)
    cfg = configs.ctpq_random_regular()
    b = hphi.Basis(ctx, "SPIN_HALF_GC", 26)
    h = hphi.Hamiltonian(ctx, b, cfg["terms"])
    tdt = torch.complex64 if args.dtype == "f32" else torch.complex128
    tuned = None if args.no_autotune else h.autotune(tdt, cfg["n_vec"], reps=2)
    V = torch.empty((b.dim, cfg["n_vec"]), dtype=tdt, device="cuda")
    hphi.hphi_random_vector(ctx, V, cfg["seed"])
    n2 = np.zeros(cfg["n_vec"])
    for _ in range(max(args.warmup, 1)):
        hphi.hphi_tpq_step(h, V, cfg["dtau"], cfg["nmax"], n2)
    if args.curve:  # the run starts at beta = 0 from the seeded vectors
        hphi.hphi_random_vector(ctx, V, cfg["seed"])
        n2[:] = 0.0
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(0)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    rec_e, rec_h2, rec_ln, acc = [], [], [], np.zeros(cfg["n_vec"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        e, h2, logd = hphi.hphi_tpq_step(h, V, cfg["dtau"], cfg["nmax"], n2)
        if args.curve:
            rec_e.append(e)
            rec_h2.append(h2)
            rec_ln.append(acc.copy())
            acc = acc + logd
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    curve = None
    if args.curve:
        # E(T) and C(T) per site from the paper's bootstrap (16 samples, 8 resamplings)
        betas = cfg["dtau"] * np.arange(args.steps)
        bs = hphi.hphi_tpq_bootstrap(np.array(rec_e).T, np.array(rec_h2).T, np.array(rec_ln).T, P=16, M=8,
                                     beta=betas, seed=1)
        curve = []
        for T in (8.0, 4.0, 2.0, 1.0, 0.5, 0.25, 0.1, 0.05, 0.025):
            k = int(round(1.0 / T / cfg["dtau"]))
            if 0 < k < args.steps:
                curve.append({"T": 1.0 / betas[k], "E_per_site": bs["e_mean"][k] / 26, "E_sd": bs["e_sd"][k] / 26,
                              "C_per_site": bs["c_mean"][k] / 26, "C_sd": bs["c_sd"][k] / 26})
    es = 8 if tdt == torch.complex64 else 16
    # algorithmic bytes of one Horner stage: read V + gather W + write W' per complex column
    stage_bytes = 3.0 * es * cfg["n_vec"] * b.dim
    roof = _roofline(ctx, stage_bytes, ctx.last_kernel())
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        m = O.Model("SPIN_HALF_GC", 26, 0, 0, cfg["terms"])
        col = V[:, :1].cpu().numpy().astype(np.complex128).copy()
        t0 = time.perf_counter()
        m.tpq_step(col, cfg["dtau"], cfg["nmax"])
        dt = time.perf_counter() - t0
        cpu = {"value": 3.0 * 16 * b.dim * cfg["nmax"] / dt / 1e9, "unit": "GB/s", "cores": O.num_threads(),
               "kind": "oracle", "sample": f"one oracle TPQ step (literal Taylor sum, FP64) of one complex column "
                                           f"of the same model, {dt:.1f} s"}
    line = _base(args, world, "hv_gbps", job_gbps(world, args.steps * cfg["nmax"] * stage_bytes, ms), "GB/s",
                 ms / args.steps, args.dtype,
                 {"workload": "ctpq_rrg3_N26_B16", "dim": b.dim, "n_vec": cfg["n_vec"], "nmax": cfg["nmax"],
                  "dtau": cfg["dtau"], "vectors": "c64" if args.dtype == "f32" else "c128",
                  "launch": h.get_tuning(), "autotuned_ms": tuned[0] if tuned else None,
                  "parallelism": f"replicas{world}",
                  "l2": "inputs larger than L2 (block = %.1f GB)" % (es * 16 * b.dim / 1e9)})
    if curve is not None:
        line["thermo"] = curve
    line.update({"tpq_steps_per_s": world * args.steps / (ms * 1e-3), "roofline": roof,
                 "gpu_launches": args.steps * (cfg["nmax"] + 2), "e_last": float(np.mean(e))})
    if ck:
        line["clocks"] = ck
    if cpu:
        line["cpu_baseline"] = cpu
    return _finish(line, rank, dist, ctx)


def run_szz(args):
    """S^zz(q, w) of the L=24 Heisenberg chain (S^z=0, 2,704,156 rows): FP64
    ground state, then every q at once through one shifted-Krylov run with
    200 shifts at eta = 0.05 to residual 1e-8."""
    import torch
    import numpy as np
    from paper_2307_13222_gb300 import hphi
    from workloads import chain, heisenberg_terms
    world, rank, local, dist, ctx = _setup(args)
    L = 24
    b = hphi.Basis(ctx, "SPIN_HALF", L, L // 2)
    h = hphi.Hamiltonian(ctx, b, heisenberg_terms(chain(L), 1.0))
    tdt = torch.float32 if args.dtype == "f32" else torch.float64
    v0 = torch.empty(b.dim, dtype=torch.float64, device="cuda")
    hphi.hphi_random_vector(ctx, v0, 1)
    gs = torch.empty_like(v0)
    lz = hphi.hphi_lanczos(h, v0, 400, 1e-12, check_every=5, gs_out=gs)
    gsd = gs.to(tdt)
    qs = 2 * np.pi * np.arange(L // 2 + 1) / L
    z = lz["e0"] + np.linspace(0.0, 4.0, 200) + 0.05j
    tol = 1e-8 if tdt == torch.float64 else 1e-6
    hphi.hphi_szz_spectrum(h, gsd, qs, z, 3000, tol, check_every=10)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(0)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        Sq, Dq, r = hphi.hphi_szz_spectrum(h, gsd, qs, z, 3000, tol, check_every=10)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    es = 4 if tdt == torch.float32 else 8
    ncol = sum(2 if np.abs(np.sin(q * np.arange(L))).max() > 1e-12 else 1 for q in qs)
    line = _base(args, world, "spectra_per_s", world * args.steps / (ms * 1e-3), "spectra/s", ms / args.steps,
                 args.dtype, {"workload": "szz_chain_L24", "dim": b.dim, "q_points": len(qs), "shifts": len(z),
                              "eta": 0.05, "tol": tol, "rhs_columns": ncol, "parallelism": f"replicas{world}",
                              "l2": "block of 32 columns = %.2f GB > L2" % (es * 32 * b.dim / 1e9)})
    line.update({"krylov_steps": r["steps"], "roofline": _roofline(ctx, 3.0 * es * 32 * b.dim,
                                                                    "block H*x of the Krylov step (32 columns)"),
                 "gpu_launches": args.steps * (r["steps"] * 7 + len(qs) + 4), "max_resid": r["max_resid"]})
    if ck:
        line["clocks"] = ck
    return _finish(line, rank, dist, ctx)


def run_serve(args):
    """Serving mix (the fifth workload): seeded Poisson arrivals of requests,
    half ground states (residual 1e-10) and half S^zz(q, w) spectra (200 shifts
    w in [0, 4] above E0, eta = 0.05, every shift's relative residual <= 1e-6,
    q = 2 pi m / L with seeded m); models drawn uniformly from Heisenberg chains
    and 2-leg ladders with N in {18, 20, ..., 30} and J_b ~ U[0.5, 1.5], and
    half-filled Hubbard 2 x L clusters with L in {4, 5, 6, 7} and U ~ U[4, 10].
    Problems up to 2^17 rows run on the batched block lane (FP64), larger ones
    on the grid lane (two workers).  The same trace is served twice, with the
    grid lane's vectors in FP64 and in FP32 (FP64 scalars; ground-state
    energies from the FP64 Rayleigh quotient); each time the service rate is
    measured first (the whole trace submitted at once) and the trace then
    arrives at 80 % of it, so p50/p99 measure service, not a growing queue.
    The line reports the --dtype run; the other is in `other`, and the energy
    difference of every ground state between the two is stated.
    One step = 2 requests of the trace; value = completed requests / s."""
    import torch
    import numpy as np
    from paper_2307_13222_gb300 import hphi
    from workloads import chain, ladder, heisenberg_terms, hubbard_terms, uniform_couplings
    world, rank, local, dist, ctx = _setup(args)
    rng = np.random.default_rng(5)
    R = 2 * args.steps
    hams = {}

    def draw(i):
        fam = int(rng.integers(0, 3))
        if fam < 2:
            N = int(rng.choice(np.arange(18, 31, 2)))
            var = int(rng.integers(0, 4))
            if fam == 0:
                key = ("chain", N, var)
                terms = heisenberg_terms(chain(N), uniform_couplings(N, 0.5, 1.5, 100 + var))
                L = N
            else:
                key = ("ladder", N, var)
                bonds = ladder(N // 2)
                terms = heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 200 + var))
                L = N // 2
            model, nu, nd = "SPIN_HALF", N // 2, 0
        else:
            Lh = int(rng.choice([4, 5, 6, 7]))
            U = float(rng.uniform(4.0, 10.0))
            key = ("hubbard", Lh, round(U, 6))
            N = 2 * Lh
            terms = hubbard_terms(N, ladder(Lh), t=1.0, U=U)
            model, nu, nd, L = "HUBBARD", Lh, Lh, Lh
        if key not in hams:
            b = hphi.Basis(ctx, model, N, nu, nd)
            hams[key] = (b, hphi.Hamiltonian(ctx, b, terms), L)
        kind = int(rng.integers(0, 2))
        q = 2 * np.pi * int(rng.integers(1, hams[key][2] // 2 + 1)) / hams[key][2]
        return (key, kind, int(1000 + i), q)

    trace = [draw(i) for i in range(R)]
    omega = np.linspace(0.0, 4.0, 200)
    MAX_STEPS = 8000

    def serve(dtype):
        srv = hphi.Server(ctx, 60e9, chunk=16, grid_dtype=dtype)

        def submit(item):
            key, kind, seed, q = item
            return srv.submit(hams[key][1], kind=kind, seed=seed, max_steps=MAX_STEPS,
                              tol=1e-10 if kind == 0 else 1e-6, q=q, eta=0.05, omega=omega)

        def drive(arrivals):
            t_start = srv.clock()
            ids, nsub, busy, last = [], 0, 0.0, 0.0
            while True:
                now = srv.clock() - t_start
                while nsub < R and arrivals[nsub] <= now:
                    ids.append(submit(trace[nsub]))
                    nsub += 1
                running, queued = srv.step()
                now2 = srv.clock() - t_start
                st = srv.stats()
                if st["block_running"] + st["grid_running"] + st["queued"] > 0:
                    busy += now2 - last
                last = now2
                if nsub == R and running == 0 and queued == 0 and st["grid_running"] == 0:
                    break
                if st["block_running"] == 0 and st["queued"] == 0:
                    nxt = arrivals[nsub] - now2 if nsub < R else 0.0005
                    time.sleep(max(0.0, min(0.0005, nxt)))
            return ids, srv.clock() - t_start, busy, t_start

        small = min(trace, key=lambda it: int(hams[it[0]][1].dim))
        srv.run_until_done([submit((small[0], k, 7, small[3])) for k in (0, 1)])  # warm-up
        torch.cuda.synchronize()
        _, t_cal, _, _ = drive(np.zeros(R))          # service rate: the whole trace at once
        mu = R / t_cal
        rate = 0.8 * mu
        arrivals = np.cumsum(np.random.default_rng(55).exponential(1.0 / rate, R))
        clocks = ClockSampler(local)
        clocks.start()
        ids, t_end, busy, t0 = drive(arrivals)
        ck = clocks.stop()
        res = [srv.result(i) for i in ids]
        sst = srv.stats()
        srv.close()
        lat = [r["t_done"] - t0 - a for r, a in zip(res, arrivals)]
        fails = [{"request": j, "kind": "spectrum" if trace[j][1] else "ground", "model": list(trace[j][0]),
                  "dim": int(hams[trace[j][0]][1].dim), "status": int(r["status"]), "max_resid": r["max_resid"],
                  "krylov_steps": r["krylov_steps"], "lanczos_steps": r["steps"]}
                 for j, r in enumerate(res) if r["status"] != 0]
        return {"dtype": dtype, "requests_per_s": R / t_end, "t_end": t_end, "service_rate_per_s": mu,
                "arrival_rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e3, "utilization": busy / t_end,
                "completed_ok": sum(r["status"] == 0 for r in res), "failures": fails,
                "grid_lane_requests": int(sum(r["lane"] for r in res)), "block_launches": int(sst["block_launches"]),
                "arena_peak_gb": sst["arena_peak"] / 1e9, "clocks": ck, "e0": [r["e0"] for r in res]}

    runs = {dt: serve(dt) for dt in ("f64", "f32")}
    main, other = runs[args.dtype], runs["f32" if args.dtype == "f64" else "f64"]
    ground = [j for j, it in enumerate(trace) if it[1] == 0]
    errs = [abs(runs["f32"]["e0"][j] - runs["f64"]["e0"][j]) / abs(runs["f64"]["e0"][j]) for j in ground
            if runs["f64"]["e0"][j] != 0.0]
    ms = max_over_ranks(main["t_end"] * 1e3, dist)
    kinds = [it[1] for it in trace]
    line = _base(args, world, "served_requests_per_s", world * R / (ms * 1e-3), "requests/s", ms / args.steps,
                 args.dtype, {"workload": "serving_mix_poisson", "requests": R,
                              "arrival_rate_per_s": main["arrival_rate_per_s"],
                              "service_rate_per_s": main["service_rate_per_s"],
                              "ground_fraction": 1.0 - float(np.mean(kinds)), "shifts": 200, "eta": 0.05,
                              "models": "chains/ladders N in {18..30} even, Hubbard 2xL L in {4..7}",
                              "form": "continuous batching: block lane (D <= 2^17, FP64, one block per recurrence) + "
                                      "grid lane (2 workers)",
                              "grid_lane_vectors": args.dtype, "scalars": "f64",
                              "parallelism": f"replicas{world}",
                              "l2": "per-request working sets 0.4 MB - 7 GB, distinct per request (no flush)"})
    line.update({"p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "utilization": main["utilization"],
                 "offered_load": 0.8, "completed_ok": main["completed_ok"], "failures": main["failures"],
                 "grid_lane_requests": main["grid_lane_requests"],
                 "max_dim": int(max(h[1].dim for h in hams.values())), "roofline": None,
                 # block-lane launches counted by the server; the grid lane's drivers launch
                 # about 7 kernels per Lanczos step besides
                 "gpu_launches": main["block_launches"], "arena_peak_gb": main["arena_peak_gb"],
                 "other": {k: v for k, v in other.items() if k not in ("e0", "clocks")},
                 "ground_e0_rel_diff_f32_vs_f64": {"max": max(errs) if errs else None,
                                                   "median": float(np.median(errs)) if errs else None,
                                                   "count": len(errs)},
                 "e2e": {"value": world * R / (ms * 1e-3), "unit": "requests/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 200 * 16}})
    if main["clocks"]:
        line["clocks"] = main["clocks"]
    return _finish(line, rank, dist, ctx)


_FMA_SRC = r"""
#include <torch/extension.h>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_chain(T *out, int iters, T a, T b) {
    T x[8];
    #pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
        #pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] * a + b;
    }
    T s = 0;
    #pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == (T)12345.678) out[0] = s;  // keeps the chain live
}
double run(int64_t blocks, int64_t threads, int64_t iters, bool dbl) {
    void *out = nullptr;
    cudaMalloc(&out, 16);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0);
        if (dbl) fma_chain<double><<<blocks, threads>>>((double *)out, (int)iters, 0.999999, 1e-7);
        else fma_chain<float><<<blocks, threads>>>((float *)out, (int)iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaFree(out);
    return (double)ms;
}
PYBIND11_MODULE(TORCH_EXTENSION_NAME, m) { m.def("run", &run); }
"""


def run_fp64peak(args):
    """FMA throughput of the FP64 and FP32 pipes (the bound of the FP64 H*x):
    a chain of 8 independent multiply-adds per thread over `iters` rounds,
    SMs x 8 blocks of 256 threads, timed with CUDA events (second launch);
    and cuBLAS DGEMM 8192^3 through torch.matmul for comparison.
    value = FP64 FMA per second."""
    import torch
    from torch.utils.cpp_extension import load_inline
    world, rank, local, dist, ctx = _setup(args)
    mod = load_inline("hphi_fma_probe", cpp_sources="", cuda_sources=_FMA_SRC, functions=None,
                      extra_cuda_cflags=["-O3", "-gencode", "arch=compute_103a,code=sm_103a"], verbose=False)
    sms = ctx.sm_count
    blocks, threads, iters = sms * 8, 256, 20000
    clocks = ClockSampler(local)
    clocks.start()
    ms64 = mod.run(blocks, threads, iters, True)
    ms32 = mod.run(blocks, threads, iters * 8, False)
    n = 4096 * 2
    A = torch.randn(n, n, dtype=torch.float64, device="cuda")
    B = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(A, B)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    torch.matmul(A, B)
    e1.record()
    torch.cuda.synchronize()
    msg = e0.elapsed_time(e1)
    ck = clocks.stop()
    fma64 = blocks * threads * 8.0 * iters / (ms64 * 1e-3)
    fma32 = blocks * threads * 8.0 * iters * 8 / (ms32 * 1e-3)
    line = _base(args, world, "fp64_fma_per_s", fma64, "FMA/s", ms64, "f64",
                 {"workload": "fma_chain_probe", "blocks": blocks, "threads": threads, "iters": iters,
                  "parallelism": f"replicas{world}", "l2": "register-only loop"})
    line.update({"fp64_tflops": 2 * fma64 / 1e12, "fp32_fma_per_s": fma32, "fp32_tflops": 2 * fma32 / 1e12,
                 "fp64_over_fp32": fma64 / fma32, "dgemm_tflops": 2.0 * n ** 3 / (msg * 1e-3) / 1e12,
                 "per_sm_per_clock_fp64_fma": None, "roofline": None, "gpu_launches": 2})
    if ck:
        line["clocks"] = ck
        mhz = ck.get("sm_mhz")
        if mhz:
            line["per_sm_per_clock_fp64_fma"] = fma64 / (sms * mhz * 1e6)
    return _finish(line, rank, dist, ctx)


def run_apply(args):
    """Plain H*x (hphi_apply_H, x -> y) on the S^z=0 sector of a periodic
    square lattice Lx x Ly (--lattice, e.g. 6x5 or 8x4), one column: the case
    used for kernel captures.  value = algorithmic GB/s (read x + write y)."""
    import torch
    from paper_2307_13222_gb300 import hphi
    from workloads import square, heisenberg_terms
    from workloads import random_regular_graph, uniform_couplings
    world, rank, local, dist, ctx = _setup(args)
    if args.lattice.lower().startswith("rrg"):
        # full space of a random 3-regular graph, 16 complex columns (the cTPQ block shape)
        N = int(args.lattice[3:])
        bonds = random_regular_graph(N, 3, 4)
        b = hphi.Basis(ctx, "SPIN_HALF_GC", N)
        h = hphi.Hamiltonian(ctx, b, heisenberg_terms(bonds, uniform_couplings(len(bonds), 0.5, 1.5, 1004)))
        shape, ncol, Lx, Ly = (b.dim, 16), 32, N, 0
        tdt = torch.complex64 if args.dtype == "f32" else torch.complex128
    else:
        Lx, Ly = (int(v) for v in args.lattice.lower().split("x"))
        N = Lx * Ly
        b = hphi.Basis(ctx, "SPIN_HALF", N, N // 2)
        h = hphi.Hamiltonian(ctx, b, heisenberg_terms(square(Lx, Ly), 1.0))
        shape, ncol = (b.dim,), 1
        tdt = torch.float32 if args.dtype == "f32" else torch.float64
    if args.variant is not None:
        h.set_tuning(variant=args.variant)
    x = torch.empty(shape, dtype=tdt, device="cuda")
    hphi.hphi_random_vector(ctx, x, 1)
    y = torch.empty_like(x)
    for _ in range(max(args.warmup, 1)):
        hphi.hphi_apply_H(h, x, y)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        hphi.hphi_apply_H(h, x, y)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    es = (4 if args.dtype == "f32" else 8) * ncol
    name = f"heisenberg_square_{Lx}x{Ly}_Sz0_apply" if Ly else f"heisenberg_rrg3_N{Lx}_block16c_apply"
    line = _base(args, world, "hv_gbps", job_gbps(world, args.steps * 2.0 * es * b.dim, ms), "GB/s", ms / args.steps,
                 args.dtype, {"workload": name, "dim": b.dim, "columns": ncol,
                              "variant": h.get_tuning()["variant"], "parallelism": f"replicas{world}",
                              "l2": "vector of %.2f GB > L2" % (es * b.dim / 1e9)})
    line.update({"roofline": _roofline(ctx, 2.0 * es * b.dim, "H*x (x + y)"), "gpu_launches": args.steps})
    return _finish(line, rank, dist, ctx)


WORKLOADS = {"chain16": run_chain16, "hubbard4x4": run_hubbard4x4, "ctpq26": run_ctpq26, "szz": run_szz,
             "serve": run_serve, "apply": run_apply, "fp64peak": run_fp64peak}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the extra FP64 measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the automatic launch settings")
    ap.add_argument("--no-block", action="store_true", help="skip the cTPQ block H*V leg of the default line")
    ap.add_argument("--curve", action="store_true",
                    help="ctpq26: run from beta = 0 and report E(T), C(T) per site (bootstrap)")
    ap.add_argument("--lattice", default="6x5",
                    help="apply workload: Lx x Ly of the square lattice, or rrgN (full space, 16 complex columns)")
    ap.add_argument("--variant", type=int, default=None, help="apply workload: H*x kernel variant (-1, 0, 1, 2)")
    ap.add_argument("--workload", choices=["square4x8"] + sorted(WORKLOADS), default="square4x8",
                    help="square4x8 (default): Lanczos steps on the 4x8 sector; the others measure the "
                         "remaining workloads (one JSON line each)")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("steps >= 1, warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "square4x8":
        return WORKLOADS[args.workload](args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
