"""Benchmark of the C*-boundary Wilson-clover Dirac operator on GB300.

Workload: physical lattice L = 48, T = 96 with C* boundaries in x, y, z,
simulated as the doubled 96 x 96 x 48 x 48 lattice (21,233,664 sites);
seeded SU(3) links exp(i 0.3 H), U(1) angles 0.3 * N(0,1), Gaussian source.
One step = one application of D in FP32 (SU(3) links as two rows plus the
U(1) angle, clover as two Hermitian 6x6 blocks per site) at charge qhat = 2,
on native-layout buffers resident in HBM. The metric is Dw GB/s: the
compulsory bytes of one application (688 B per site: spinor in 96 + out 96,
links 4 x 48, angles 16, clover 288) divided by its time. The working set
(14.6 GB per application) is far larger than L2, so no flush is needed.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of sites
of the same workload (the oracle is a deliberately plain program; the ratio
to it says nothing about kernel quality).

Multi-GPU (torchrun, N > 1): independent replicas, one per GPU; the value is
the bytes of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import os
import subprocess
import sys
import time

# the oracle runs one process per core (or on one core): keep host BLAS
# single-threaded in every process
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the throughput workload: physical L = 48, T = 96, doubled 96x96x48x48
    "full": dict(T=96, L1=48, L2=48, L3=48, mask=0b1110, eps=0.3, sigma=0.3,
                 m0=0.1, csw=1.0, cswqed=1.0, qhat=2),
    # a smaller case of the same kernel for profiling (48x48x24x24, 0.9 GB/step)
    "medium": dict(T=48, L1=24, L2=24, L3=24, mask=0b1110, eps=0.3, sigma=0.3,
                   m0=0.1, csw=1.0, cswqed=1.0, qhat=2),
    # the solver lattice (64x64x32x32) and a small one (32x32x16x16, 0.18 GB/step)
    "solve": dict(T=64, L1=32, L2=32, L3=32, mask=0b1110, eps=0.3, sigma=0.3,
                  m0=0.01, csw=1.0, cswqed=1.0, qhat=2),
    "small": dict(T=32, L1=16, L2=16, L3=16, mask=0b1110, eps=0.3, sigma=0.3,
                  m0=0.01, csw=1.0, cswqed=1.0, qhat=2),
}
WORKLOAD = WORKLOADS["full"]
# the solver workload: physical L = 32, T = 64 with C*, doubled 64x64x32x32;
# FGCR (nkv 16) with FP32 SAP (4^4 blocks, ncy 5, nmr 5) against FP64-only GCR
SOLVE_WORKLOAD = dict(T=64, L1=32, L2=32, L3=32, mask=0b1110, eps=0.3, sigma=0.3, csw=1.0, cswqed=1.0,
                      points=[(0.05, -1), (0.05, 2), (0.01, -1), (0.01, 2)], tol=1e-10)
BYTES_PER_SITE_FP32 = {True: 688, False: 672}   # qhat != 0 -> angles read
BYTES_PER_SITE_FP64 = {True: 1568, False: 1536}
METRIC = "Dw GB/s"
FALLBACK_HBM = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def reduce_max(value: float) -> float:
    """Max of `value` over all ranks (the slowest rank's time); the value
    itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(per_rank_units: float, max_seconds: float, world_size: int) -> float:
    """Whole-job rate: the units every rank processed (weak scaling: the same
    per rank) over the slowest rank's time."""
    return per_rank_units * world_size / max_seconds


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons of the samples taken
        between wall-clock times t0 and t1 (all samples if not given)."""
        import datetime
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if t0 is not None and ts is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                continue
            f = f[1:]
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_record(kernel_files):
    """Per-launch DRAM traffic of the timed kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "dirac_fp32_q2_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    h = hashlib.sha256()
    for f in kernel_files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec


TRAFFIC_SOURCES = ["paper_1710_08839_gb300/csrc/dirac.cu", "paper_1710_08839_gb300/csrc/dirac_common.cuh"]


def write_traffic_record(csv_path):
    """Per-launch DRAM traffic of the timed kernel from an ncu CSV (metrics
    gpu__time_duration.sum, dram__bytes_read.sum, dram__bytes_write.sum of
    k_dirac launches on the full workload) into profiles/, with the hash of
    the kernel sources it was measured on."""
    import csv
    import statistics
    import re
    hdr, per, kernel_names = None, {}, set()
    for r in csv.reader(open(csv_path)):
        if r and r[0] == "ID":
            hdr = r
            continue
        if hdr and len(r) == len(hdr):
            d = dict(zip(hdr, r))
            if "k_dirac" in d["Kernel Name"]:
                per.setdefault(d["ID"], {})[d["Metric Name"]] = float(d["Metric Value"])
                m = re.search(r"(k_dirac\w*)<(\d+)>", d["Kernel Name"])
                kernel_names.add(f"{m.group(1)}<{'true' if m.group(2) == '1' else 'false'}>" if m
                                 else d["Kernel Name"][:60])
    tr = [v["dram__bytes_read.sum"] + v["dram__bytes_write.sum"] for v in per.values()]
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    w = WORKLOAD
    V = w["T"] * 2 * w["L1"] * w["L2"] * w["L3"]
    names = sorted({n for n in kernel_names})
    rec = {"kernel": ", ".join(names) + " (FP32 D, the launch shape chosen by the autotuner)", "workload": f"doubled {w['T']}x{2 * w['L1']}x"
           f"{w['L2']}x{w['L3']} C* lattice, {V} sites", "launches": len(tr),
           "bytes_per_launch": statistics.mean(tr),
           "read_bytes_per_launch": statistics.mean(v["dram__bytes_read.sum"] for v in per.values()),
           "write_bytes_per_launch": statistics.mean(v["dram__bytes_write.sum"] for v in per.values()),
           "algorithmic_bytes_per_launch": BYTES_PER_SITE_FP32[True] * V,
           "duration_ns_under_ncu": statistics.mean(v["gpu__time_duration.sum"] for v in per.values()),
           "command": "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                      "--clock-control none -k regex:k_dirac -s 52 -c 5 --csv --log-file dirac_full_dram.csv "
                      "python bench.py --steps 20 --warmup 3 --no-cpu-baseline --no-solve --no-batch --no-serve "
                      "--no-variants --no-e2e (the first 49 launches are the autotuner's candidates)",
           "source_sha256": h.hexdigest(),
           "note": "full benchmark size, 1-pass metrics; stale once the kernel sources change"}
    out = os.path.join(ROOT, "profiles", "dirac_fp32_q2_traffic.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    return rec


# --kernel-times: device time per kernel of selected regions (torch.profiler,
# CUPTI activity records of every kernel on the device, the library's
# included); timings taken under it carry the profiler's overhead
KERNEL_TIMES = {"on": False}


@contextlib.contextmanager
def kernel_times(out, top=16):
    if not KERNEL_TIMES["on"]:
        yield
        return
    import re
    import torch
    from torch.profiler import profile, ProfilerActivity
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        yield
        torch.cuda.synchronize()
    tot = {}
    for e in prof.events():
        if e.device_type != torch.autograd.DeviceType.CUDA:
            continue
        m = re.search(r"(k_\w+)(<[^(]*>)?", e.name)
        k = (m.group(1) + (m.group(2) or "")) if m else e.name[:48]
        t = tot.setdefault(k, [0, 0.0])
        t[0] += 1
        t[1] += getattr(e, "device_time_total", 0.0) or getattr(e, "cuda_time_total", 0.0)
    busy = sum(v[1] for v in tot.values())
    rows = sorted(tot.items(), key=lambda kv: -kv[1][1])[:top]
    out["kernel_times"] = {"device_ms": busy / 1e3,
                           "kernels": [{"kernel": k, "launches": n, "ms": us / 1e3,
                                        "share": us / busy if busy else 0.0} for k, (n, us) in rows]}


def _start_kernel_times():
    """The first profiler session of a process records no device activity:
    open and close one before the measured regions."""
    KERNEL_TIMES["on"] = True
    import torch
    from torch.profiler import profile, ProfilerActivity
    with profile(activities=[ProfilerActivity.CUDA]):
        torch.zeros(1, device="cuda").add_(1)
        torch.cuda.synchronize()


def make_inputs(device, w=None):
    import synth
    w = w or WORKLOAD
    su3 = synth.su3_field(w["T"], w["L1"], w["L2"], w["L3"], w["eps"], synth.SEED_GAUGE + 1,
                          device=device)
    ang = synth.u1_field(w["T"], w["L1"], w["L2"], w["L3"], w["sigma"], synth.SEED_GAUGE + 501,
                         device=device)
    N1 = 2 * w["L1"]
    V = w["T"] * N1 * w["L2"] * w["L3"]
    psi = synth.spinor_field(w["T"], N1, w["L2"], w["L3"], synth.SEED_SOURCE + 1).reshape(V, 4, 3)
    return su3, ang, psi, V


def solve_benchmark(qxd, torch, solvers=("mixed", "fp64_eo", "fp64_full")):
    """Solves of D x = b at every (m0, qhat) point of the solver workload with
    each solver; wall time of the qxd_solve call (which synchronises)."""
    w = SOLVE_WORKLOAD
    su3, ang, psi, V = make_inputs("cuda", dict(w, T=w["T"]))
    b = psi.cuda()
    del psi
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    del su3, ang
    kinds = {
        "mixed": dict(precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32),
        "fp64_sap": dict(precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP64, delta=0.0),
        "fp64_eo": dict(system=qxd.QXD_SOLVE_EO, inner_prec=qxd.QXD_FP64, max_iter=20000, delta=0.0),
        "fp64_full": dict(system=qxd.QXD_SOLVE_FULL, inner_prec=qxd.QXD_FP64, max_iter=20000, delta=0.0),
    }
    rows = []
    totals = {k: 0.0 for k in solvers}
    first = True
    for m0, q in w["points"]:
        lat.set_params(m0, w["csw"], w["cswqed"], q)
        lat.sw_build()
        xs = {}
        row = {"m0": m0, "qhat": q}
        for k in solvers:
            x = torch.zeros_like(b)
            if first:  # work vectors are allocated by the first solve
                lat.solve(x, b, tol=w["tol"], **kinds[k])
                first = False
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = lat.solve(x, b, tol=w["tol"], **kinds[k])
            dt = time.perf_counter() - t0
            totals[k] += dt
            xs[k] = x
            row[k] = {"status": rc, "ms": dt * 1e3, "iterations": info["iterations"],
                      "restarts": info["restarts"], "true_relres": info["true_relres"],
                      "dw64_calls": info["dw64_calls"]}
        ref = "fp64_eo" if "fp64_eo" in xs else None
        if ref:
            for k in xs:
                if k != ref:
                    row[k]["rel_diff_vs_" + ref] = float((xs[k] - xs[ref]).norm() / xs[ref].norm())
        rows.append(row)
        del xs
    lat.close()
    n = len(w["points"])
    out = {"workload": "doubled 64x64x32x32 C* lattice (L=32, T=64), eps 0.3, csw=cswqed=1, "
                       "tol 1e-10 (true FP64 residual), FGCR nkv 16; mixed = FP32 SAP 4^4 ncy 5 nmr 5",
           "points": rows, "solves_per_s": {k: n / totals[k] for k in solvers}}
    if "mixed" in solvers:
        for k in solvers:
            if k != "mixed":
                out["speedup_mixed_vs_" + k] = totals[k] / totals["mixed"]
    return out


# multi-right-hand-side workload: two lattices, point sources (3 colours x 4
# spins at a seeded site) for several quarks each, solved together
BATCH_WORKLOAD = dict(
    lattices=[dict(T=48, L1=24, L2=24, L3=24, mask=0b1110, seed=3,
                   quarks=[(m0, q) for m0 in (0.05, 0.1) for q in (-1, 0, 2)]),
              dict(T=32, L1=16, L2=16, L3=16, mask=0b1110, seed=4, quarks=[(0.05, -1), (0.1, 2)])],
    eps=0.3, sigma=0.3, csw=1.0, cswqed=1.0, tol=1e-10, budget_gb=120)

# serving workload: Poisson arrivals, sizes (L, T) with probabilities, one
# resident ensemble per size, m0 ~ U[0.02, 0.2], qhat from {-1, 0, 2}
SERVE_WORKLOAD = dict(sizes=[(8, 16), (16, 32), (24, 48), (32, 64)], probs=[0.4, 0.3, 0.2, 0.1], n=512,
                      eps=0.3, sigma=0.3, csw=1.0, cswqed=1.0, m0=(0.02, 0.2), qs=(-1, 0, 2), tol=1e-10,
                      seed=3000, budget_gb=80, load=0.8,
                      # serving runtime: one engine lane per size class (bounds on the simulated sites)
                      lane_sites=[100000, 1000000, 2000000], lane_budget_gb=[4, 12, 24, 40])


def _fp64_params(qxd):
    return dict(system=qxd.QXD_SOLVE_EO, inner_prec=qxd.QXD_FP64, max_iter=20000, delta=0.0)


def _mixed_params(qxd):
    return dict(precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)


def batch_benchmark(qxd, torch):
    """All point-source solves of the multi-RHS workload through the engine
    (one batched launch set per step) against sequential FP64-only solves."""
    import synth
    w = BATCH_WORKLOAD
    lats, ops = [], []
    for lw in w["lattices"]:
        su3 = synth.su3_field(lw["T"], lw["L1"], lw["L2"], lw["L3"], w["eps"], synth.SEED_GAUGE + lw["seed"],
                              device="cuda")
        ang = synth.u1_field(lw["T"], lw["L1"], lw["L2"], lw["L3"], w["sigma"], synth.SEED_GAUGE + 500 + lw["seed"],
                             device="cuda")
        lat = qxd.Lattice(lw["T"], lw["L1"], lw["L2"], lw["L3"], lw["mask"])
        lat.set_gauge(su3, ang)
        del su3, ang
        lats.append(lat)
        N1 = 2 * lw["L1"]
        site, src = synth.point_source(lw["T"], N1, lw["L2"], lw["L3"], synth.SEED_SOURCE + lw["seed"])
        V = lw["T"] * N1 * lw["L2"] * lw["L3"]
        for m0, q in lw["quarks"]:
            v = lat.view()
            v.set_params(m0, w["csw"], w["cswqed"], q)
            v.sw_build()
            ops.append((lw, v, m0, q, src.reshape(12, V, 4, 3)))
    reqs = []  # (op, b)
    for lw, v, m0, q, src in ops:
        for k in range(12):
            reqs.append((v, src[k].cuda()))
    nreq = len(reqs)
    # batched D throughput over all right-hand sides (FP32, native layout)
    handles, ins, outs = [], [], []
    for v, b in reqs:
        xn = torch.empty(v.spinor_bytes(qxd.QXD_FP32), dtype=torch.uint8, device="cuda")
        v.pack(xn, b.to(torch.complex64), qxd.QXD_FP32)
        handles.append(v.handle)
        ins.append(xn)
        outs.append(torch.empty_like(xn))
    st = torch.cuda.current_stream().cuda_stream
    args = (handles, [o.data_ptr() for o in outs], [i.data_ptr() for i in ins], qxd.QXD_FP32, 0, st)
    qxd.qxd_Dw_batch(*args)  # autotunes
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        qxd.qxd_Dw_batch(*args)
    e1.record()
    torch.cuda.synchronize()
    dms = e0.elapsed_time(e1) / 5
    sites_rhs = sum(v.V for v, _ in reqs)
    single_bytes = 688 * sites_rhs  # what nreq separate applications would move
    del ins, outs
    # engine: every request submitted at once, admitted by budget; the first
    # pass warms the engine's allocator and the autotuned kernels, the
    # second is timed
    eng = qxd.Engine(hbm_budget_bytes=w["budget_gb"] << 30, max_active=nreq)
    xs = [torch.zeros_like(b) for _, b in reqs]
    kt_eng = {}
    for timed in (False, True):
        torch.cuda.synchronize()
        with kernel_times(kt_eng) if timed else contextlib.nullcontext():
            t0 = time.perf_counter()
            ids = [eng.submit(v, x, b, tol=w["tol"]) for (v, b), x in zip(reqs, xs)]
            eng.run()
            t_eng = time.perf_counter() - t0
        infos = [eng.poll(i)[1] for i in ids]
        for i in ids:
            eng.forget(i)
    stats = eng.stats()
    eng.close()
    ok = all(i["status"] == qxd.QXD_OK for i in infos)
    # sequential references on one request per quark, extrapolated to all
    seq64, seqmix, diffs = 0.0, 0.0, []
    for lw, v, m0, q, src in ops:
        b = src[0].cuda()
        x64 = torch.zeros_like(b)
        v.solve(x64, b, tol=w["tol"], **_mixed_params(qxd))  # allocates the view's solver work
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v.solve(x64, b, tol=w["tol"], **_fp64_params(qxd))
        seq64 += (time.perf_counter() - t0) * 12
        xm = torch.zeros_like(b)
        t0 = time.perf_counter()
        v.solve(xm, b, tol=w["tol"], **_mixed_params(qxd))
        seqmix += (time.perf_counter() - t0) * 12
        k = next(i for i, (vv, bb) in enumerate(reqs) if vv is v)
        diffs.append(float((xs[k] - x64).norm() / x64.norm()))
    for _, v, _, _, _ in ops:
        v.close()
    for lat in lats:
        lat.close()
    return {
        "workload": "point sources (12 spin-colour) on 48x48x24x24 (L=24, T=48; 2 masses x 3 charges = 72) and "
                    "32x32x16x16 (L=16, T=32; 24) C* lattices, eps 0.3, tol 1e-10; engine: FGCR + FP32 SAP "
                    "(4^4, ncy 5, nmr 5) in lockstep, batched launches",
        "requests": nreq, "all_converged": ok,
        "max_true_relres": max(i["true_relres"] for i in infos),
        "engine_s": t_eng, "engine_solves_per_s": nreq / t_eng, "engine_steps": stats["steps"], **kt_eng,
        "sequential_fp64_s_est": seq64, "sequential_fp64_solves_per_s_est": nreq / seq64,
        "sequential_mixed_s_est": seqmix,
        "speedup_vs_sequential_fp64": seq64 / t_eng, "speedup_vs_sequential_mixed": seqmix / t_eng,
        "max_rel_diff_vs_fp64": max(diffs),
        "note": "sequential times: one solve per quark timed, times 12",
        "batched_dw": {"rhs": nreq, "ms": dms, "effective_GB_per_s": single_bytes / dms / 1e6,
                       "note": "688 B per site and right-hand side (the single-RHS byte model) / time"},
    }


def serve_benchmark(qxd, torch):
    """Continuous batching of a Poisson request stream: through the serving
    runtime (one engine lane per size class, each with its own stream and
    worker thread), and for comparison through one lockstep engine at the
    same arrival rate."""
    import numpy as np

    import synth
    w = SERVE_WORKLOAD
    rng = np.random.default_rng(w["seed"])
    n = w["n"]
    size_idx = rng.choice(len(w["sizes"]), size=n, p=w["probs"])
    m0s = rng.uniform(*w["m0"], size=n)
    qs = rng.choice(w["qs"], size=n)
    ens = []
    for i, (L, T) in enumerate(w["sizes"]):
        su3 = synth.su3_field(T, L, L, L, w["eps"], synth.SEED_GAUGE + 10 + i, device="cuda")
        ang = synth.u1_field(T, L, L, L, w["sigma"], synth.SEED_GAUGE + 510 + i, device="cuda")
        lat = qxd.Lattice(T, L, L, L, 0b1110)
        lat.set_gauge(su3, ang)
        del su3, ang
        ens.append(lat)
    pools = [[] for _ in ens]
    import queue
    import threading
    pool_lock = threading.Lock()
    prep_stream = torch.cuda.Stream()

    def acquire(i, m0, q):
        with pool_lock:
            v = pools[i].pop() if pools[i] else None
        if v is None:
            v = ens[i].view(stream=prep_stream)
        v.set_params(float(m0), w["csw"], w["cswqed"], int(q))
        v.sw_build()
        return v

    def release(i, v):
        with pool_lock:
            pools[i].append(v)

    def source(r):
        L, T = w["sizes"][size_idx[r]]
        return synth.spinor_field_device(T, 2 * L, L, L, synth.SEED_SOURCE + 100 + r).reshape(-1, 4, 3)

    # requests in flight per size (each holds a view with its clover term and
    # its source and solution fields); arrived requests beyond this wait in
    # a host queue, their latency counted from arrival
    cap = w.get("inflight_cap", [64, 32, 12, 6])
    eng = qxd.Engine(hbm_budget_bytes=w["budget_gb"] << 30, max_active=256)
    srv = qxd.Server(w["lane_sites"], [g << 30 for g in w["lane_budget_gb"]], max_active=256)

    def run(arrivals, server=None):
        """Serve the requests with arrival times `arrivals` (s). A preparation
        thread builds each admitted request's operator (view + clover term) and
        source on its own stream while the main thread submits and polls
        (server: the lanes step themselves) or steps the lockstep engine."""
        be = server if server is not None else eng
        from collections import deque
        todo, ready = queue.Queue(), queue.Queue()

        def prep():
            with torch.cuda.stream(prep_stream):
                while True:
                    r = todo.get()
                    if r is None:
                        return
                    v = acquire(size_idx[r], m0s[r], qs[r])
                    b = source(r)
                    x = torch.zeros_like(b)
                    prep_stream.synchronize()
                    ready.put((r, v, x, b))

        worker = threading.Thread(target=prep, daemon=True)
        worker.start()
        inflight = {}
        waiting = [deque() for _ in ens]
        busy = [0] * len(ens)
        lat_ms = []
        nxt = 0
        done = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                waiting[size_idx[nxt]].append(nxt)
                nxt += 1
            for i in range(len(ens)):
                while waiting[i] and busy[i] < cap[i]:
                    todo.put(waiting[i].popleft())
                    busy[i] += 1
            while True:
                try:
                    r, v, x, b = ready.get_nowait()
                except queue.Empty:
                    break
                rid = be.submit(v, x, b, tol=w["tol"])
                inflight[rid] = (r, v, x, b, arrivals[r])
            if server is None:
                a, p, d = eng.step()
                check, idle = d or (a == 0 and p == 0), a == 0 and p == 0
            else:
                time.sleep(0.0002)
                check, idle = True, not inflight
            if check:
                for rid in list(inflight):
                    fin, info = be.poll(rid)
                    if fin:
                        r, v, x, b, t_arr = inflight.pop(rid)
                        if info["status"] != qxd.QXD_OK:
                            raise RuntimeError(f"request {r} failed: {info}")
                        lat_ms.append((time.perf_counter() - t0 - t_arr) * 1e3)
                        release(size_idx[r], v)
                        busy[size_idx[r]] -= 1
                        be.forget(rid)
                        done += 1
            if idle:
                if ready.empty() and any(busy):
                    time.sleep(0.0005)  # the preparation thread is working
                elif not any(busy) and nxt < n:
                    time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
        total = time.perf_counter() - t0
        todo.put(None)
        worker.join()
        lat_ms.sort()
        return total, lat_ms

    # saturated throughput (all requests at t = 0; a first pass warms the
    # view pools, allocator and autotuned kernels), then Poisson arrivals at
    # `load` times that rate
    run(np.zeros(n), srv)
    t_sat, _ = run(np.zeros(n), srv)
    rate = w["load"] * n / t_sat
    arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
    arr -= arr[0]
    t_poi, lat_ms = run(arr, srv)
    lane_stats = [srv.stats(i) for i in range(srv.nlanes)]
    srv.close()
    # the same stream through one lockstep engine
    t_sat_e, _ = run(np.zeros(n))
    t_poi_e, lat_e = run(arr)
    eng.close()
    # one-at-a-time references: the first six requests of each size timed
    # alone (operator build + solve), averaged per size
    per_size_fp64, per_size_mix = [], []
    for i in range(len(ens)):
        rs = [int(r) for r in np.nonzero(size_idx == i)[0][:6]]
        v = acquire(i, m0s[rs[0]], qs[rs[0]])
        b0 = source(rs[0])
        v.solve(torch.zeros_like(b0), b0, tol=w["tol"], **_mixed_params(qxd))  # solver work allocated
        for kind, store in ((_fp64_params(qxd), per_size_fp64), (_mixed_params(qxd), per_size_mix)):
            tsum = 0.0
            for r in rs:
                b = source(r)
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                v.set_params(float(m0s[r]), w["csw"], w["cswqed"], int(qs[r]))  # the request's operator
                v.sw_build()
                v.solve(x, b, tol=w["tol"], **kind)
                tsum += time.perf_counter() - t0
            store.append(tsum / len(rs))
        release(i, v)
    counts = np.bincount(size_idx, minlength=len(ens))
    seq64 = float(np.dot(counts, per_size_fp64))
    seqmix = float(np.dot(counts, per_size_mix))
    for pl in pools:
        for v in pl:
            v.close()
    for e in ens:
        e.close()
    def pct(v, f):
        return v[min(len(v) - 1, int(f * len(v)))]

    return {
        "workload": f"{n} requests, Poisson arrivals, sizes (L,T) {w['sizes']} with p {w['probs']} (C*, doubled), "
                    "m0 ~ U[0.02,0.2], qhat in {-1,0,2}, Gaussian sources, tol 1e-10",
        "runtime": f"qxd_server: {len(w['lane_budget_gb'])} engine lanes by simulated sites {w['lane_sites']}, "
                   f"budgets {w['lane_budget_gb']} GB, each with its own stream and worker thread",
        "saturated_solves_per_s": n / t_sat, "arrival_rate_per_s": rate,
        "poisson_solves_per_s": n / t_poi, "p50_latency_ms": pct(lat_ms, 0.5), "p99_latency_ms": pct(lat_ms, 0.99),
        "lanes": lane_stats,
        "lockstep_engine": {"saturated_solves_per_s": n / t_sat_e, "poisson_solves_per_s": n / t_poi_e,
                            "p50_latency_ms": pct(lat_e, 0.5), "p99_latency_ms": pct(lat_e, 0.99),
                            "note": "one qxd_engine stepping every request in lockstep, same arrivals"},
        "one_at_a_time_fp64_solves_per_s_est": n / seq64, "one_at_a_time_mixed_solves_per_s_est": n / seqmix,
        "speedup_saturated_vs_fp64_one_at_a_time": seq64 / t_sat,
        "counts_per_size": counts.tolist(),
        "note": "one-at-a-time rates: the first six requests of each size timed alone (operator build + "
                "solve), mean per size weighted by the size counts",
    }


# pseudofermion action: the factor P_1 of the paper's rational approximation
# (Table 2, seven zero/pole pairs, solved by multi-shift CG) on the solver
# workload's lattice
RATIONAL_WORKLOAD = dict(points=[(0.05, -1), (0.05, 2)], factor=1, tol=1e-10, reps=2)


def table2_factor(k):
    """(nu, mu) of factor P_k from the Table 2 fixture (zeros, poles, factor)."""
    nu, mu = [], []
    with open(os.path.join(ROOT, "tests", "golden", "table2_rational.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                _, n_j, m_j, fac = ln.split()
                if int(fac) == k:
                    nu.append(float(n_j))
                    mu.append(float(m_j))
    return nu, mu


# algorithmic bytes per even site of one multi-shift CG step (FP64): two
# applications of Q = gamma5 D_hat, each an M_oo^-1 H_oe kernel (spinor in and
# out 192 + 192, the 8 links of the site 8 x 144, their U(1) factors 8 x 16,
# clover inverse 576) and a M_ee - H_eo kernel (the same plus the aux spinor
# 192); |Q p|^2 (192); r -= alpha (w + s p) (4 x 192); and per active shift
# x += a p, p = z r + b p (4 x 192, plus r once)
MSCG_BYTES_Q = (192 + 192 + 8 * 144 + 8 * 16 + 576) + (3 * 192 + 8 * 144 + 8 * 16 + 576)
MSCG_BYTES_FIXED = 2 * MSCG_BYTES_Q + 192 + 4 * 192 + 192
MSCG_BYTES_PER_SHIFT = 4 * 192


def rational_benchmark(qxd, torch):
    """P_1 phi by one multi-shift CG over its seven poles, against the same
    seven systems solved one at a time; wall time of the synchronous calls."""
    w = SOLVE_WORKLOAD
    R = RATIONAL_WORKLOAD
    su3, ang, psi, V = make_inputs("cuda", w)
    phi = psi.cuda()
    del psi
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    del su3, ang
    nu, mu = table2_factor(R["factor"])
    out = torch.empty_like(phi)
    x1 = [torch.empty_like(phi)]
    Vh = V // 2
    rows = []
    t_multi = t_single = t_mixed = 0.0
    for m0, q in R["points"]:
        lat.set_params(m0, w["csw"], w["cswqed"], q)
        lat.sw_build()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        logdet = lat.sw_logdet(qxd.QXD_SITES_ODD)
        t_ld = time.perf_counter() - t0
        lat.rational_apply(out, phi, nu, mu, tol=R["tol"])  # allocates the work vectors
        ms = []
        for _ in range(R["reps"]):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = lat.rational_apply(out, phi, nu, mu, tol=R["tol"])
            ms.append((time.perf_counter() - t0) * 1e3)
        t_multi += min(ms) / 1e3
        # the GB300 path: FP32 operator, FP64 reliable updates and refinement
        out32 = torch.empty_like(phi)
        ms32 = []
        for _ in range(R["reps"]):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc32, info32 = lat.rational_apply(out32, phi, nu, mu, tol=R["tol"], prec=qxd.QXD_FP32)
            ms32.append((time.perf_counter() - t0) * 1e3)
        t_mixed += min(ms32) / 1e3
        mixed = {"status": rc32, "ms": min(ms32), "iterations": info32["iterations"],
                 "true_relres": info32["true_relres"], "dhat_calls": info32["dhat_calls"],
                 "rel_diff_vs_fp64": float((out32 - out).norm() / out.norm()),
                 "action_rel_diff": abs(info32["action"] - info["action"]) / abs(info["action"])}
        it = info["iterations"]
        # the seven systems one at a time (plain CG each)
        single = []
        for m_j in mu:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc1, info1, rel1 = lat.mscg(x1, phi, [m_j * m_j], tol=R["tol"])
            single.append({"ms": (time.perf_counter() - t0) * 1e3, "iterations": info1["iterations"],
                           "status": rc1})
        t_single += sum(s["ms"] for s in single) / 1e3
        # bytes of the CG steps: every shift is active until it converges;
        # counted here as if all stayed active (an upper bound on the work)
        bytes_it = Vh * (MSCG_BYTES_FIXED + len(mu) * MSCG_BYTES_PER_SHIFT)
        rows.append({"m0": m0, "qhat": q, "status": rc, "ms": min(ms), "iterations": it,
                     "ms_per_iteration": min(ms) / max(it, 1), "true_relres": info["true_relres"],
                     "action": info["action"], "ln_abs_det_Doo": logdet, "logdet_ms": t_ld * 1e3,
                     "GBs_per_iteration_model": bytes_it / (min(ms) / 1e3 / max(it, 1)) / 1e9,
                     "mixed_fp32_operator": mixed, "single_shift_cg": single})
    lat.close()
    n = len(R["points"])
    return {"workload": "P_1 of Table 2 (7 zero/pole pairs) by FP64 multi-shift CG on D_hat^dag D_hat, "
                        "doubled 64x64x32x32 C* lattice (L=32, T=64), eps 0.3, csw=cswqed=1, tol 1e-10 "
                        "per shift (true FP64 residual)",
            "points": rows, "rational_applies_per_s": n / t_multi,
            "rational_applies_per_s_mixed": n / t_mixed,
            "speedup_mixed_vs_fp64_multishift": t_multi / t_mixed,
            "speedup_multishift_vs_7_single_cg": t_single / t_multi,
            "bytes_per_even_site_per_iteration": MSCG_BYTES_FIXED + len(mu) * MSCG_BYTES_PER_SHIFT}


# Wilson flow of the solver workload's gauge field: FP64 work per RK3 stage
# and integrated link: the staple sum (12 complex 3x3 products of 198 flops),
# W = U S and exp(X) U (2 more), the exponential by Cayley-Hamilton (X^2: one
# product; det X ~ 60; 24 terms of the scalar recurrence ~ 26 each; the
# combination A + B X + C X^2 ~ 144), plus the U(1) angle update (~ 60); the
# links integrated are the physical ones (half the simulated lattice with C*
# boundaries)
FLOW_WORKLOAD = dict(eps=0.02, steps=(5, 5, 10), q_el=1.0 / 6.0)
FLOW_FLOPS_PER_LINK_STAGE = 15 * 198 + 60 + 24 * 26 + 144 + 60


def flow_benchmark(qxd, torch):
    """Wilson flow to t = 0.4 in stages, timing each call; observables at
    every stage."""
    w = SOLVE_WORKLOAD
    F = FLOW_WORKLOAD
    su3, ang, psi, V = make_inputs("cuda", w)
    del psi
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    del su3, ang
    lat.wflow(F["eps"], 1)  # warm-up (and t = eps)
    t = F["eps"]
    rows = [{"t": t, "obs": lat.gauge_observables(F["q_el"])}]
    ms_per_step = []
    for n in F["steps"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.wflow(F["eps"], n)
        dt = time.perf_counter() - t0
        t += n * F["eps"]
        ms_per_step.append(dt * 1e3 / n)
        rows.append({"t": round(t, 6), "ms_per_step": dt * 1e3 / n, "obs": lat.gauge_observables(F["q_el"])})
    lat.close()
    links = 4 * V // 2
    flops_step = 3 * links * FLOW_FLOPS_PER_LINK_STAGE
    best = min(ms_per_step)
    return {"workload": "Wilson flow (Luscher RK3, SU(3) and compact U(1)), doubled 64x64x32x32 C* lattice "
                        "(L=32, T=64), eps 0.02, FP64; obs = (E_SU(3), E_U(1) at q_el=1/6, Q_top)",
            "stages": rows, "ms_per_rk3_step": best,
            "fp64_tflops_model": flops_step / (best / 1e3) / 1e12,
            "flops_per_rk3_step_model": flops_step}


# local deflation: the solver workload's lattice near its critical mass
# (m0 = -0.62 on the eps = 0.3 field, where the SAP solver needs ~40 steps);
# the subspace is built once per operator and serves every solve with it
DFL_WORKLOAD = dict(m0=-0.62, qhat=2, ns=16, niter=20, ncy=4, seed=3, tol=1e-10)


def dfl_benchmark(qxd, torch):
    """SAP-preconditioned FGCR against the deflated solver on the same
    system; wall time of the synchronous solves, subspace build timed apart."""
    w = SOLVE_WORKLOAD
    D = DFL_WORKLOAD
    su3, ang, psi, V = make_inputs("cuda", w)
    b = psi.cuda()
    del psi
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    del su3, ang
    lat.set_params(D["m0"], w["csw"], w["cswqed"], D["qhat"])
    lat.sw_build()
    out = {"workload": "doubled 64x64x32x32 C* lattice, eps 0.3, csw=cswqed=1, qhat 2, m0 -0.62, tol 1e-10; "
                       f"deflation: ns {D['ns']} fields on the 4^4 SAP blocks, {D['niter']} SAP-smoothing passes "
                       f"(ncy {D['ncy']}), little system on its even blocks"}
    x = torch.zeros_like(b)
    lat.solve(x, b, tol=D["tol"], precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)  # warm-up
    torch.cuda.synchronize()
    kt_sap = {}
    with kernel_times(kt_sap):
        t0 = time.perf_counter()
        rc, info = lat.solve(x, b, tol=D["tol"], precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
        t_sap = time.perf_counter() - t0
    out["sap"] = {"status": rc, "s": t_sap, "iterations": info["iterations"],
                  "true_relres": info["true_relres"], **kt_sap}
    t0 = time.perf_counter()
    lat.dfl_subspace(D["ns"], niter=D["niter"], ncy=D["ncy"], seed=D["seed"])
    out["subspace_build_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    lat.dfl_refresh()
    out["little_operator_s"] = time.perf_counter() - t0
    x2 = torch.zeros_like(b)
    kt_dfl = {}
    with kernel_times(kt_dfl):
        t0 = time.perf_counter()
        rc, info = lat.solve(x2, b, tol=D["tol"], precond=qxd.QXD_PRECOND_DFL_SAP, inner_prec=qxd.QXD_FP32)
        t_dfl = time.perf_counter() - t0
    out["dfl_sap"] = {"status": rc, "s": t_dfl, "iterations": info["iterations"],
                      "little_iters": info["little_iters"], "true_relres": info["true_relres"],
                      "rel_diff_vs_sap": float((x2 - x).norm() / x.norm()), **kt_dfl}
    lat.close()
    return out


def alu_benchmark(qxd, torch):
    """FP64 and FP32 fused multiply-add throughput of this GPU (qxd_fma_rate):
    the denominators of the ALU-bound rooflines, with the SM clock seen."""
    props = torch.cuda.get_device_properties(0)
    kinds = (("fp64_fma", qxd.QXD_PROBE_FMA64, 5000), ("fp32_fma", qxd.QXD_PROBE_FMA32, 400000),
             ("fp32x2_fma", qxd.QXD_PROBE_FMA32X2, 200000))
    out = {"gpu": props.name, "sms": props.multi_processor_count,
           "probe": "16 independent FMA chains per thread, 8 blocks of 256 threads per SM, "
                    "best of 3 launches (CUDA events); 2 flops per FMA"}
    for name, kind, iters in kinds:
        qxd.fma_rate(kind, max(1, iters // 10))  # clocks up, module loaded
        with ClockSampler(torch.cuda.current_device()) as clk:
            t0 = time.time()
            rate = qxd.fma_rate(kind, iters)
            t1 = time.time()
        c = clk.summary(t0, t1)
        row = {"TFLOP/s": rate / 1e12, "clocks": c}
        if c.get("sm_mhz"):
            row["flop_per_clk_per_sm"] = rate / (props.multi_processor_count * c["sm_mhz"] * 1e6)
        out[name] = row
    return out


def oracle_benchmark(qxd, torch):
    """The FP64 oracle on this machine's host cores: the small workload's
    plain GCR solve to 1e-12 (one core), and the oracle's D at sampled sites
    of the throughput and solver workloads on one core and on all cores, from
    which the time of one FP64 D application and of a plain FP64 GCR solve of
    the solver workload are estimated (the oracle cannot finish that solve in
    a bench run)."""
    import numpy as np

    import oracle as O
    import synth
    out = {}
    # small workload: doubled 8x8x4x4 (L=4, T=8), q=-1, m0=0.2, eps 0.4, sigma 0.5
    T, L = 8, 4
    lat = O.Lattice(T, L, L, L, 0b1110)
    su3 = synth.su3_field(T, L, L, L, 0.4, synth.SEED_GAUGE).numpy()
    ang = synth.u1_field(T, L, L, L, 0.5, synth.SEED_GAUGE + 500).numpy()
    b = synth.spinor_field(T, 2 * L, L, L, synth.SEED_SOURCE).reshape(-1, 4, 3).numpy()
    op = O.Dirac(lat, O.GaugeField.from_physical(lat, su3, ang), 0.2, 1.0, 1.0, -1)
    op.apply(b)  # clover matrices of the small lattice built once
    t0 = time.perf_counter()
    _, it, res = O.gcr(op.apply, b, tol=1e-12)
    out["small_gcr_1e-12"] = {"seconds": time.perf_counter() - t0, "iterations": it, "relres": res, "cores": 1,
                              "workload": "doubled 8x8x4x4 C* lattice (L=4, T=8), qhat=-1, m0=0.2, nkv 16"}
    for name, w in (("throughput", WORKLOAD), ("solver", dict(WORKLOADS["solve"], m0=0.05, qhat=-1))):
        su3, ang, psi, V = make_inputs("cuda", w)
        su3h, angh, psih = su3.cpu().numpy(), ang.cpu().numpy(), psi.numpy()
        del su3, ang
        r1, n1, t1 = oracle_sample_rate(su3h, angh, psih, V, w, target_s=8.0)
        ra, na, ta, cores = oracle_sample_rate_all_cores(su3h, angh, psih, V, w, target_s=10.0)
        row = {"sites": V, "one_core_sites_per_s": r1, "all_cores_sites_per_s": ra, "cores": cores,
               "one_core_apply_s": V / r1, "all_cores_apply_s": V / ra,
               "fp64_GB_per_s_one_core": r1 * BYTES_PER_SITE_FP64[True] / 1e9,
               "fp64_GB_per_s_all_cores": ra * BYTES_PER_SITE_FP64[True] / 1e9}
        if name == "solver":
            # the plain FP64 GCR (nkv 16) of the GPU needs 119 steps and 8 restarts
            # at this point (m0 = 0.05, qhat = -1): one D per step and per restart
            applies = 119 + 8
            row["plain_gcr_1e-10_estimate_s_all_cores"] = applies * V / ra
            row["estimate_note"] = (f"{applies} applications of D (the GPU's plain FP64 GCR to 1e-10 at "
                                    "m0=0.05, qhat=-1: 119 steps, 8 restarts) x the all-cores time of one")
        out[name] = row
        del su3h, angh, psih
    return out


def sap_benchmark(qxd, torch, steps, w):
    """Time one FP32 SAP application (ncy 5, nmr 5) on the lattice of workload w."""
    su3, ang, psi, V = make_inputs("cuda", w)
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    lat.set_params(w["m0"], w["csw"], w["cswqed"], w["qhat"])
    lat.sw_build()
    x = psi.to(torch.complex64).cuda()
    xn = torch.empty(lat.spinor_bytes(qxd.QXD_FP32), dtype=torch.uint8, device="cuda")
    lat.pack(xn, x, qxd.QXD_FP32)
    yn = torch.empty_like(xn)
    for _ in range(3):
        lat.sap(yn, xn, 5, 5, native=True, prec=qxd.QXD_FP32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        lat.sap(yn, xn, 5, 5, native=True, prec=qxd.QXD_FP32)
    e1.record()
    torch.cuda.synchronize()
    single = e0.elapsed_time(e1) / steps
    # 12 right-hand sides of the operator in one pass (qxd_sap_multi)
    R = 12
    ins = [xn] + [torch.roll(xn, 4096 * k) for k in range(1, R)]
    outs = [torch.empty_like(xn) for _ in range(R)]
    lat.sap_multi(outs, ins, 5, 5)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        lat.sap_multi(outs, ins, 5, 5)
    e1.record()
    torch.cuda.synchronize()
    multi = e0.elapsed_time(e1) / steps / R
    lat.close()
    return {"sap_ms": single, "sites": V, "ncy": 5, "nmr": 5,
            "lattice": f"{w['T']}x{2 * w['L1']}x{w['L2']}x{w['L3']}",
            "multi_rhs": {"rhs": R, "ms_per_rhs": multi, "speedup_vs_single": single / multi,
                          "note": "qxd_sap_multi: links staged once per block for all right-hand sides"}}


# --- the oracle on all host cores ------------------------------------------
# The oracle is plain numpy; its many small array operations hold the GIL, so
# threads do not scale. All cores are used by a process pool started with
# "spawn" (a fresh interpreter: no CUDA state is inherited). The workers map
# the gauge field and the spinor read-only from .npy files written once to
# /dev/shm (or to a temporary directory when /dev/shm is too small).

_W_OP = None
_W_PSI = None


def _oracle_worker_init(paths, w):
    global _W_OP, _W_PSI
    import numpy as np

    import oracle as O
    su3 = np.load(paths["su3"], mmap_mode="r")
    ang = np.load(paths["ang"], mmap_mode="r")
    _W_PSI = np.load(paths["psi"], mmap_mode="r")
    lat = O.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    _W_OP = O.Dirac(lat, O.GaugeField.from_physical(lat, su3, ang), w["m0"], w["csw"], w["cswqed"], w["qhat"])


def _oracle_worker_apply(idx):
    _W_OP.apply_at(_W_PSI, idx)
    return len(idx)


class OraclePool:
    """The FP64 oracle's D on sampled sites of a workload, on `nproc` processes."""

    def __init__(self, su3_host, ang_host, psi_host, w, nproc=None):
        import multiprocessing as mp
        import shutil
        import tempfile

        import numpy as np
        self.nproc = nproc or len(os.sched_getaffinity(0))
        need = su3_host.nbytes + ang_host.nbytes + psi_host.nbytes + (1 << 28)
        base = None
        for d in ("/dev/shm", tempfile.gettempdir()):
            try:
                if os.path.isdir(d) and shutil.disk_usage(d).free > need:
                    base = d
                    break
            except OSError:
                continue
        if base is None:
            raise RuntimeError("no room to share the fields with the oracle's worker processes")
        self.dir = tempfile.mkdtemp(prefix="qxd_oracle_", dir=base)
        try:
            self.paths = {}
            for k, a in (("su3", su3_host), ("ang", ang_host), ("psi", psi_host)):
                self.paths[k] = os.path.join(self.dir, k + ".npy")
                np.save(self.paths[k], np.ascontiguousarray(a))
            ctx = mp.get_context("spawn")
            self.pool = ctx.Pool(self.nproc, initializer=_oracle_worker_init, initargs=(self.paths, dict(w)))
        except BaseException:
            shutil.rmtree(self.dir, ignore_errors=True)
            raise
        self.where = base

    def apply(self, idx):
        """Wall seconds of the oracle's D at sites idx, split over the workers."""
        import numpy as np
        parts = [p for p in np.array_split(np.asarray(idx), 4 * self.nproc) if len(p)]
        t0 = time.perf_counter()
        n = sum(self.pool.map(_oracle_worker_apply, parts, chunksize=1))
        dt = time.perf_counter() - t0
        assert n == len(idx)
        return dt

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def oracle_sample_rate_all_cores(su3_host, ang_host, psi_host, V, w, target_s=15.0):
    """FP64 oracle on a sample of sites on all host cores: (sites/s, sites, seconds, cores)."""
    import numpy as np
    pool = OraclePool(su3_host, ang_host, psi_host, w)
    try:
        rng = np.random.default_rng(8)
        n = 2048 * pool.nproc
        pool.apply(rng.choice(V, size=n, replace=False))          # workers start, pages mapped
        dt = pool.apply(rng.choice(V, size=n, replace=False))
        n2 = int(min(4_000_000, max(n, n * target_s / max(dt, 1e-3))))
        idx = rng.choice(V, size=n2, replace=False)
        dt = pool.apply(idx)
        return n2 / dt, n2, dt, pool.nproc
    finally:
        pool.close()


def oracle_sample_rate(su3_host, ang_host, psi_host, V, w, target_s=12.0):
    """FP64 oracle on a sample of sites of the workload: (sites/s, sites, seconds)."""
    import numpy as np

    import oracle as O
    lat = O.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    op = O.Dirac(lat, O.GaugeField.from_physical(lat, su3_host, ang_host), w["m0"], w["csw"],
                 w["cswqed"], w["qhat"])
    rng = np.random.default_rng(7)
    n = 2048
    idx = rng.choice(V, size=n, replace=False)
    t0 = time.perf_counter()
    op.apply_at(psi_host, idx)
    dt = time.perf_counter() - t0
    n2 = int(min(200000, max(n, n * target_s / max(dt, 1e-3))))
    idx = rng.choice(V, size=n2, replace=False)
    t0 = time.perf_counter()
    op.apply_at(psi_host, idx)
    dt = time.perf_counter() - t0
    return n2 / dt, n2, dt


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (one process per
    core), on a bounded random sample of sites of the workload per step."""
    import numpy as np
    import torch

    import oracle as O
    ws, rank, _ = _dist()
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    su3, ang, psi, V = make_inputs(dev)
    su3h, angh, psih = su3.cpu().numpy(), ang.cpu().numpy(), psi.numpy()
    del su3, ang
    w = WORKLOAD
    rng = np.random.default_rng(11)
    try:
        pool = OraclePool(su3h, angh, psih, w)
        cores = pool.nproc
        run = pool.apply
        how = f"{cores} processes, one per host core"
    except Exception as e:  # no room to share the fields: one core in this process
        pool, cores = None, 1
        lat = O.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
        op = O.Dirac(lat, O.GaugeField.from_physical(lat, su3h, angh), w["m0"], w["csw"],
                     w["cswqed"], w["qhat"])

        def run(idx):
            t0 = time.perf_counter()
            op.apply_at(psih, idx)
            return time.perf_counter() - t0
        how = f"one core (all-cores run unavailable: {e})"
    # size each step so that warm-up + timed steps take about 90 s in total
    cal = 512 * cores
    run(rng.choice(V, size=cal, replace=False))
    rate = cal / run(rng.choice(V, size=cal, replace=False))
    S = int(min(8192 * cores, max(64 * cores, rate * 90.0 / (args.steps + args.warmup))))
    samples = [rng.choice(V, size=S, replace=False) for _ in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        run(samples[i])
    dt = 0.0
    for i in range(args.steps):
        dt += run(samples[args.warmup + i])
    if pool:
        pool.close()
    sites_s = S * args.steps / dt
    # the metric's byte model (688 B per site), so the ratio of the two arms
    # is the ratio of sites per second
    b = BYTES_PER_SITE_FP32[True]
    value = sites_s * b / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Dw apply FP32 (2-row SU(3) + U(1) angle), doubled 96x96x48x48 "
                               "C* lattice (L=48, T=96), qhat=2, csw=cswqed=1",
                   "sites": V, "bytes_per_site": b,
                   "sample": f"FP64 oracle at {S} random sites per step ({how})"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{S} random sites per step x {args.steps} steps on {how} "
                                   f"({sites_s:.0f} sites/s)"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="full", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="dw",
                    choices=["dw", "solve", "sap", "batch", "serve", "rational", "flow", "dfl", "alu", "oracle"],
                    help="dw: the Dw throughput line (plus a solver summary unless --no-solve); "
                         "solve: solver comparison only; sap: time the SAP preconditioner only; "
                         "batch / serve: multi-RHS and serving workloads; rational: pseudofermion action; "
                         "flow: Wilson flow and gauge observables; dfl: deflated vs SAP solver; "
                         "alu: FP64/FP32 FMA throughput (the ALU roofline denominators); "
                         "oracle: the FP64 oracle timed on the host cores")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the multi-RHS summary of the default line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving summary of the default line")
    ap.add_argument("--kernel-times", action="store_true",
                    help="with --mode dfl or batch: device time per kernel of the timed solves (torch.profiler; "
                         "the timings then include its overhead)")
    ap.add_argument("--write-traffic", metavar="NCU_CSV",
                    help="write profiles/dirac_fp32_q2_traffic.json from an ncu CSV of k_dirac launches and exit")
    args = ap.parse_args()
    if args.write_traffic:
        print(json.dumps(write_traffic_record(args.write_traffic)))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    ge.build()
    from paper_1710_08839_gb300 import qxd

    if args.mode in ("solve", "sap", "batch", "serve", "rational", "flow", "dfl", "alu", "oracle"):
        if args.kernel_times:
            _start_kernel_times()
        if args.mode == "oracle":
            res = oracle_benchmark(qxd, torch)
        elif args.mode == "alu":
            res = alu_benchmark(qxd, torch)
        elif args.mode == "dfl":
            res = dfl_benchmark(qxd, torch)
        elif args.mode == "flow":
            res = flow_benchmark(qxd, torch)
        elif args.mode == "solve":
            res = solve_benchmark(qxd, torch)
        elif args.mode == "rational":
            res = rational_benchmark(qxd, torch)
        elif args.mode == "batch":
            res = batch_benchmark(qxd, torch)
        elif args.mode == "serve":
            res = serve_benchmark(qxd, torch)
        else:
            res = sap_benchmark(qxd, torch, args.steps, WORKLOADS[args.workload])
        if rank == 0:
            print(json.dumps({"mode": args.mode, **res}), flush=True)
        return

    w = WORKLOADS[args.workload]
    su3, ang, psi, V = make_inputs("cuda", w)
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    lat.set_params(w["m0"], w["csw"], w["cswqed"], w["qhat"])
    lat.sw_build()
    stream = torch.cuda.current_stream()

    def native_pair(prec, dtype):
        x = psi.to(dtype).cuda()
        xn = torch.empty(lat.spinor_bytes(prec), dtype=torch.uint8, device="cuda")
        lat.pack(xn, x, prec)
        del x
        return xn, torch.empty_like(xn)

    window = {}

    def time_applies(prec, xn, yn, steps, warmup, min_warm_s=0.0):
        t_w = time.perf_counter()
        n = 0
        while n < warmup or time.perf_counter() - t_w < min_warm_s:
            lat.Dw(yn, xn, prec=prec, native=True)
            n += 1
            if n % 50 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        window["t0"] = time.time()
        e0.record(stream)
        for _ in range(steps):
            lat.Dw(yn, xn, prec=prec, native=True)
        e1.record(stream)
        torch.cuda.synchronize()
        window["t1"] = time.time()
        return reduce_max(e0.elapsed_time(e1) / steps)

    # headline: FP32, qhat = 2
    xn, yn = native_pair(qxd.QXD_FP32, torch.complex64)
    with ClockSampler(local) as clk:
        # warm up for >= 1 s so the sampler is running when the timed region starts
        ms = time_applies(qxd.QXD_FP32, xn, yn, args.steps, args.warmup, min_warm_s=1.0)
    clocks = clk.summary(window["t0"], window["t1"])
    shape = lat.dw_shape(qxd.QXD_FP32)  # chosen by the autotuner on the first application
    bps = BYTES_PER_SITE_FP32[True]
    gbs_rank = bps * V / (ms * 1e-3) / 1e9
    value = aggregate_value(bps * V / 1e9, ms * 1e-3, ws)
    peak, peak_kind = _peaks()

    variants = {}
    if not args.no_variants:
        vsteps = max(3, min(args.steps, 10))
        lat.set_params(w["m0"], w["csw"], w["cswqed"], 0)
        lat.sw_build()
        ms0 = time_applies(qxd.QXD_FP32, xn, yn, vsteps, 3)
        variants["fp32_q0"] = {"ms": ms0, "GB/s": BYTES_PER_SITE_FP32[False] * V / ms0 / 1e6,
                               "bytes_per_site": BYTES_PER_SITE_FP32[False]}
        lat.set_params(w["m0"], w["csw"], w["cswqed"], w["qhat"])
        lat.sw_build()
        del xn, yn
        xd, yd = native_pair(qxd.QXD_FP64, torch.complex128)
        ms64 = time_applies(qxd.QXD_FP64, xd, yd, max(3, min(args.steps, 5)), 3)
        variants["fp64_q2"] = {"ms": ms64, "GB/s": BYTES_PER_SITE_FP64[True] * V / ms64 / 1e6,
                               "bytes_per_site": BYTES_PER_SITE_FP64[True],
                               "note": "FP64 Dw is bound by the FP64 ALUs, not HBM"}
        del xd, yd

    # end to end: host (pinned) lexicographic buffers through the C ABI; the
    # call copies the input in, packs, applies D, unpacks and copies the
    # result out, then synchronises.
    e2e = None
    if not args.no_e2e:
        xh = psi.to(torch.complex64).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        e2e_steps = max(3, min(args.steps, 5))
        lat.Dw(yh, xh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            lat.Dw(yh, xh)
        e2e_ms = reduce_max((time.perf_counter() - t0) / e2e_steps * 1e3)
        _ = float(yh[0, 0, 0].real)  # the step's result is on the host
        e2e = {"value": aggregate_value(bps * V / 1e9, e2e_ms * 1e-3, ws), "unit": "GB/s",
               "h2d_bytes_per_step": V * 96, "d2h_bytes_per_step": V * 96, "ms_per_step": e2e_ms}
        del xh, yh

    cpu = cpu1 = None
    if rank == 0 and not args.no_cpu_baseline:
        su3h, angh = su3.cpu().numpy(), ang.cpu().numpy()
        rate, n, dt = oracle_sample_rate(su3h, angh, psi.numpy(), V, w, target_s=8.0)
        cpu1 = {"value": rate * bps / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": f"FP64 oracle D at {n} random sites of the workload in {dt:.1f} s on one core "
                          f"({rate:.0f} sites/s x {bps} B/site, the metric's byte model)"}
        try:
            rate, n, dt, cores = oracle_sample_rate_all_cores(su3h, angh, psi.numpy(), V, w)
            cpu = {"value": rate * bps / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
                   "sample": f"FP64 oracle D at {n} random sites of the workload in {dt:.1f} s on "
                             f"{cores} processes, one per host core ({rate:.0f} sites/s x {bps} B/site, "
                             "the metric's byte model)"}
        except Exception as e:  # no room to share the fields: the one-core figure stands
            cpu = dict(cpu1, note=f"all-cores run unavailable: {e}")
        del su3h, angh

    solve = batch = serve = None
    if not (args.no_solve and args.no_batch and args.no_serve):
        lat.close()
        xn = yn = None
        del su3, ang
        torch.cuda.empty_cache()
    if not args.no_solve:
        solve = solve_benchmark(qxd, torch)
        torch.cuda.empty_cache()
    if not args.no_batch:
        batch = batch_benchmark(qxd, torch)
        torch.cuda.empty_cache()
    if not args.no_serve:
        serve = serve_benchmark(qxd, torch)
        torch.cuda.empty_cache()

    rec = _traffic_record(TRAFFIC_SOURCES)
    traffic = rec["bytes_per_launch"] if rec else None
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Dw apply FP32 (2-row SU(3) + U(1) angle), doubled "
                               f"{w['T']}x{2 * w['L1']}x{w['L2']}x{w['L3']} C* lattice "
                               f"(L={w['L1']}, T={w['T']}), qhat={w['qhat']}, csw=cswqed=1",
                   "sites": V, "bytes_per_site": bps, "l2": "inputs larger than L2 "
                   f"({bps * V / 1e9:.1f} GB per step), no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": gbs_rank, "peak": peak, "unit": "GB/s",
                     "frac": gbs_rank / peak, "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes": bps * V},
        "cpu_baseline": cpu,
        "cpu_baseline_1core": cpu1,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "variants": variants,
        "autotune": {"timed_shape": shape, "choices": [l for l in qxd.tune_report().splitlines() if l]},
        "solve": solve,
        "batch": batch,
        "serve": serve,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if args.no_solve and args.no_batch and args.no_serve:
        lat.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
