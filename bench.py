"""Benchmark of the multi-RHS Dirac mat-vec on GB300.

Default workload (one step = one sweep): Wilson D_W, 32^4 periodic lattice,
Nc = 3, Nv = 12, FP32, kappa = 0.125, links exp(0.3 i H), Gaussian source,
internal blocked layout, inputs resident in HBM.  Each step reads and
writes 2.7 GB, far more than the 129 MB L2, so no flush is needed between
steps.  The JSON line reports model Gflop/s (1368 flop per site and
right-hand side), the HBM roofline of the kernel, the end-to-end rate through
the C ABI with host buffers, the FP64 CPU oracle timed on a bounded sample,
and the clocks seen during the timed region.  Extra lines in "extra" time the
staggered and Brillouin sweeps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extra]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica of
the workload (the sweeps do not shard without a halo exchange); the value is
the sum over ranks divided by the slowest rank's time.
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

import synth  # noqa: E402

METRIC = "Dirac-apply Gflop/s & HBM GB/s (Nc=3,Nv=12); mixed-vs-FP32 solve time @1e-10"
WORKLOAD = {"op": "wilson", "L": (32, 32, 32, 32), "Nv": 12, "mass": 0.125, "prec": "f32",
            "links": "near_identity", "eps": 0.3, "seed_links": 1002, "seed_source": 2002}
PAPER_CONTEXT = {"wilson_sp_knl_gflops": 345, "staggered_sp_knl_gflops": 475,
                 "brillouin_sp_knl_gflops": 790, "note": "one 68-core KNL node, Nc=3, Nv=12 (abstract)"}
KERNEL_SOURCES = ["paper_1808_05506_gb300/csrc/dirac_kernels.cuh",
                  "paper_1808_05506_gb300/csrc/dirac_common.cuh",
                  "paper_1808_05506_gb300/csrc/apply_wilson_impl.cuh",
                  "paper_1808_05506_gb300/csrc/apply_wilson_f32.cu",
                  "paper_1808_05506_gb300/csrc/apply_wilson.cu"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "wilson_apply_traffic.json")
NOMINAL_HBM_GBS = 7900.0   # HBM3e nominal bandwidth of one GB300 (the measured copy peak is lower)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def gen_inputs(w):
    L, Nv = w["L"], w["Nv"]
    ns = 1 if w["op"] == "staggered" else 4
    V = synth.gauge_links(L, 3, w["links"], w["seed_links"], eps=w.get("eps", 0.3))
    psi = synth.spinor(L, Nv, ns, 3, w["seed_source"], dtype=np.complex64)
    return V.astype(np.complex64), psi


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for_smi(torch) -> str:
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[torch.cuda.current_device()] if vis else str(torch.cuda.current_device())


def time_kernel(torch, fn, steps, warmup):
    """Per-launch CUDA-event timing on the current stream; returns (total_ms, [per-launch ms])."""
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for a, b in ev:
        a.record(st)
        fn()
        b.record(st)
    t1.record(st)
    t1.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev]


def sweep_rate(dg, torch, w, steps, warmup, kernel=None, compare_formats=False):
    """Time one sweep workload on the internal layout; returns a dict of rates.
    kernel = (R, block, variant): that launch shape instead of the autotuner.
    compare_formats: also time the link format the tuner did not keep."""
    V, psi = gen_inputs(w)
    D = dg.Dirac(w["op"], w["L"], w["Nv"], w["mass"], w["prec"])
    D.set_links(torch.from_numpy(V).cuda())
    if kernel:
        D.set_kernel_config(*kernel)
    else:
        D.autotune()
    x = D.pack(torch.from_numpy(psi).cuda())
    y = D.new_internal()
    total, per = time_kernel(torch, lambda: D.apply(x, out=y), steps, warmup)
    vol = int(np.prod(w["L"]))
    t = statistics.mean(per) * 1e-3
    flops = dg.flops_per_site_rhs(w["op"]) * vol * w["Nv"]
    byts = dg.bytes_per_site(w["op"], w["Nv"], w["prec"]) * vol
    cfg = D.kernel_config()
    order = D.site_order()
    fmt = D.link_format()
    byts = dg.bytes_per_site(w["op"], w["Nv"], w["prec"], link_format=fmt) * vol
    out = {"gflops": flops / t / 1e9, "gbs": byts / t / 1e9, "ms": t * 1e3, "R": cfg[0], "block": cfg[1],
           "variant": cfg[2], "site_order_tchunk": order, "link_format": fmt}
    if compare_formats:
        out["other_link_format"] = other_format_time(dg, torch, D, x, y, w, steps, warmup, fmt)
    D.close()
    return out


def other_format_time(dg, torch, D, x, y, w, steps, warmup, fmt):
    """The sweep in the link format the tuner did not keep (two-row links vs
    nine entries for Wilson / staggered, 80 vs 40 stored W for Brillouin), in
    the tuned launch shape if that shape reads both formats, else in variant 1
    with two right-hand sides per thread, 64 sites per block, t-chunks of 8."""
    other = 1 - fmt
    try:
        D.set_link_format(other)
    except dg.DiracError as e:
        return {"fmt": other, "unavailable": str(e)}
    R, B, variant = D.kernel_config()
    if not (variant == 1 or (w["op"] != "brillouin" and variant == 6) or (w["op"] == "brillouin" and variant == 0)):
        D.set_kernel_config(2, 64, 1)
        D.set_site_order(min(8, w["L"][3]))
    _, per = time_kernel(torch, lambda: D.apply(x, out=y), steps, warmup)
    t = statistics.mean(per) * 1e-3
    byts = dg.bytes_per_site(w["op"], w["Nv"], w["prec"], link_format=other) * int(np.prod(w["L"]))
    res = {"fmt": other, "ms": t * 1e3, "gbs": byts / t / 1e9, "kernel": list(D.kernel_config()),
           "site_order_tchunk": D.site_order()}
    D.set_link_format(fmt)
    return res


class OracleSample:
    """The FP64 oracle (as it stands) on a bounded random sample of output sites."""

    def __init__(self, w, inputs=None):
        import oracle
        self.oracle = oracle
        V, psi = inputs if inputs is not None else gen_inputs(w)
        self.V = np.ascontiguousarray(V, dtype=np.complex128)
        self.psi = np.ascontiguousarray(psi, dtype=np.complex128)
        self.w = w
        self.m0 = oracle.kappa_to_m0(w["mass"]) if w["op"] == "wilson" else w["mass"]
        self.vol = int(np.prod(w["L"]))
        self.rng = np.random.default_rng(0)
        self.cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def run(self, n):
        sites = self.rng.integers(0, self.vol, n)
        t = time.perf_counter()
        self.oracle.apply(self.w["op"], self.V, self.psi, self.m0, sites=sites)
        return time.perf_counter() - t

    def calibrate(self, seconds):
        n = 64
        while True:
            dt = self.run(n)
            if dt > seconds / 2 or n >= self.vol:
                break
            n = min(self.vol, int(n * min(16.0, max(2.0, seconds / max(dt, 1e-4)))))
        return max(1, min(self.vol, int(n * seconds / max(dt, 1e-6))))

    def rate(self, n, dt):
        from paper_1808_05506_gb300 import flops_per_site_rhs   # flop model only; no library load
        return flops_per_site_rhs(self.w["op"]) * n * self.w["Nv"] / dt / 1e9

    def describe(self, n, dt):
        return (f"{n} random output sites of the {self.w['op']} {'x'.join(map(str, self.w['L']))} "
                f"Nv={self.w['Nv']} workload (FP64 gather oracle, OpenMP), {dt:.2f} s")


def solve_times(dg, torch, L=(24, 24, 24, 48), Nv=12, m0=0.05, precs=("f32", "bf16", "f16")):
    """Brillouin D_B x = b to a true FP64 relative residual of 1e-10, Nv = 12,
    by defect correction (FP64 outer residual) with the inner CGLS stored in
    each precision: the mixed-vs-FP32 solve-time part of the metric."""
    w = dict(WORKLOAD, op="brillouin", L=L, mass=m0, seed_links=1003, seed_source=2003)
    V, psi = gen_inputs(w)
    b = torch.from_numpy(psi.astype(np.complex128)).cuda()
    out = {}
    for prec in precs:
        D = dg.Dirac("brillouin", L, Nv, m0, prec)
        D.set_links(torch.from_numpy(V).cuda())
        D.autotune()
        # untimed warm-up: one short solve loads the solver's kernels and
        # captures its graphs, so that no precision pays them in its timing
        D.solve(b, tol=1e-10, max_outer=1, max_inner=16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, res, st, status = D.solve(b, tol=1e-10, max_outer=40, max_inner=6000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[prec] = {"seconds": dt, "status": int(status), "max_rel_residual": float(res.max()),
                     "outer": st["outer_iterations"], "inner": st["inner_iterations"],
                     "sweeps": st["sweeps"], "fp64_sweeps": st["fp64_sweeps"], "kernel": list(D.kernel_config()),
                     "df_residual": st.get("df_residual"), "split_fields": st.get("split_fields"),
                     "even_odd": st.get("even_odd")}
        D.close()
        del x
        torch.cuda.empty_cache()
    if "f32" in out:
        for p in precs:
            if p != "f32":
                out[p]["speedup_vs_f32"] = out["f32"]["seconds"] / out[p]["seconds"]
    out["workload"] = "brillouin_solve_{}_nv{}_m0_{}".format("x".join(map(str, L)), Nv, m0)
    return out


def batched_solve_times(dg, torch, L=(32, 32, 32, 64), nsys=4, slots=24, precs=("f32", "bf16", "f16"),
                        rank=0, ws=1, dist=None, precond=1, autotune=True, inner_fields=1):
    """Wilson systems D(kappa_i) x_i = b_i on one gauge field, Nv_i ~ U{1..24},
    kappa_i ~ U[0.120, 0.124], through dirac_solve_batched with `slots` resident
    right-hand-side columns, each precision to a true FP64 residual of 1e-10:
    the batched form of the mixed-vs-FP32 solve time (fewer systems than the
    48 of the full configuration, so that the benchmark stays within minutes).
    With N ranks the systems are shared out (sharding.assign_systems, 4 * N
    systems in all: weak scaling) and each rank solves its own; the time is
    the slowest rank's.  precond: 1 even-odd inner solves (the library's
    default), 0 whole-lattice ones; inner_fields: 1 split fields for 16-bit
    storage (the default: FP32 solution, residual and products, 16-bit search
    directions), 0 every inner field in 16 bits."""
    from paper_1808_05506_gb300 import sharding
    nsys = nsys * ws
    key = (tuple(L), nsys, ws, rank)
    if key not in _BATCHED_INPUTS:
        rng = np.random.default_rng(7)
        nvs = [int(v) for v in rng.integers(1, 25, nsys)]
        kap = [float(v) for v in rng.uniform(0.120, 0.124, nsys)]
        V = batched_links(L)
        # this rank's right-hand sides, generated before any timing (and kept for
        # the next call on the same systems)
        local_b = {i: torch.from_numpy(synth.spinor(L, nvs[i], 4, 3, 2100 + i)).cuda()
                   for i in sharding.assign_systems(nvs, ws)[rank]}
        _BATCHED_INPUTS[key] = (nvs, kap, V, local_b)
    nvs, kap, V, local_b = _BATCHED_INPUTS[key]

    def make_b(i):
        return local_b[i]

    out = {}
    for prec in precs:
        D = dg.Dirac("wilson", L, slots, 0.122, prec)
        D.set_preconditioner(precond)
        D.set_inner_fields(inner_fields)
        D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
        if autotune:
            D.autotune()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        local, xs, status, stats, tot = sharding.solve_batched_sharded(
            D.solve_batched, nvs, kap, make_b, rank, ws,
            gather=(lambda o: [o]) if dist is None else None, tol=1e-10)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            tt = torch.tensor([dt], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt = float(tt.item())
        out[prec] = {"seconds": dt, "status": int(status),
                     "max_rel_residual": max(s["residual_max"] for s in stats),
                     "outer_max": max(s["outer_iterations"] for s in stats),
                     "all_converged": all(s["converged"] for s in stats), "kernel": list(D.kernel_config()),
                     "rank0_totals": {k: tot.get(k) for k in ("outer_iterations", "inner_iterations", "sweeps",
                                                                "fp64_sweeps", "even_odd", "split_fields")}}
        D.close()
        del xs
        torch.cuda.empty_cache()
    if "f32" in out:
        for p in precs:
            if p != "f32":
                out[p]["speedup_vs_f32"] = out["f32"]["seconds"] / out[p]["seconds"]
    out["workload"] = "wilson_batched_solve_{}_{}sys_nv{}_{}slots".format("x".join(map(str, L)), nsys,
                                                                        "-".join(map(str, nvs)), slots)
    out["sharding"] = f"{ws} rank(s), systems per rank by assign_systems"
    out["inner_solver"] = ("even-odd: CGLS on the Schur complement of the odd sites" if precond
                           else "whole lattice: CGLS on D")
    if inner_fields and precond:
        out["inner_solver"] += "; 16-bit storage: split fields (FP32 e, r, t and links, 16-bit p, s)"
    return out


# inputs of batched_solve_times, shared by its calls on the same systems
_BATCHED_INPUTS = {}
_LINKS = {}


def batched_links(L):
    """The gauge field of the batched Wilson systems (exp(0.3 i H), seed 1005),
    generated once per lattice and shared by the batched lines."""
    key = tuple(L)
    if key not in _LINKS:
        _LINKS[key] = synth.gauge_links(L, 3, "near_identity", 1005, eps=0.3).astype(np.complex64)
    return _LINKS[key]


def c5_batched_times(dg, torch, precs=("f32", "bf16", "f16"), rank=0, ws=1, dist=None, L=(32, 32, 32, 64),
                     nsys=48, slots=64, wave_cols=128):
    """The full batched configuration: 48 Wilson systems D(kappa_i) x_i = b_i
    on 32^3 x 64 sharing one gauge field, Nv_i ~ U{1..24}, kappa_i ~
    U[0.120, 0.124] (the draw of the GPU test of this configuration), each
    storage precision to a true FP64 residual of 1e-10 through
    dirac_solve_batched with `slots` resident columns and the library's
    defaults (even-odd inner solves, split inner fields for 16-bit storage,
    double-float outer residual).  The sources are complex Gaussian fields
    drawn on the device (one seeded generator per system) before each solve
    call.  The FP64 b and x of all systems (about 440 GB) exceed one GPU, so
    the systems go through the solver in waves of at most `wave_cols`
    columns; the time is the sum of the solve calls.  With N ranks the
    systems are shared out by sharding.assign_systems (strong scaling: the
    48 systems in all) and the time is the slowest rank's."""
    from paper_1808_05506_gb300 import sharding
    rng = synth.rng(1005, synth.STREAM_MISC)
    nvs = [int(v) for v in rng.integers(1, 25, nsys)]
    kap = [float(v) for v in rng.uniform(0.120, 0.124, nsys)]
    V = batched_links(L)
    local = sharding.assign_systems(nvs, ws)[rank]
    waves, cur, cols = [], [], 0
    for i in local:
        if cur and cols + nvs[i] > wave_cols:
            waves.append(cur)
            cur, cols = [], 0
        cur.append(i)
        cols += nvs[i]
    if cur:
        waves.append(cur)
    Nx, Ny, Nz, Nt = L

    def make_b(i):
        g = torch.Generator(device="cuda")
        g.manual_seed(2005 + i)
        z = torch.randn((Nt, Nz, Ny, Nx, nvs[i], 4, 3, 2), dtype=torch.float64, device="cuda", generator=g)
        return torch.view_as_complex(z.mul_(0.5 ** 0.5))

    out = {}
    for prec in precs:
        D = dg.Dirac("wilson", L, slots, kap[0], prec)
        D.set_links(torch.from_numpy(V).cuda())
        D.autotune()
        # untimed warm-up: a short solve of one system loads the solver's kernels and captures its graphs
        wb = make_b(waves[0][0]) if waves else None
        if wb is not None:
            D.solve_batched([wb], [kap[waves[0][0]]], tol=1e-10, max_outer=1, max_inner=16)
            del wb
        seconds, worst, outer, inner, sweeps, fp64_sweeps, ok = 0.0, 0.0, 0, 0, 0, 0, True
        even_odd = split = df = None
        for wave in waves:
            bs = [make_b(i) for i in wave]
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            xs, res, sst, tot, status = D.solve_batched(bs, [kap[i] for i in wave], tol=1e-10, max_outer=60,
                                                        max_inner=8000)
            torch.cuda.synchronize()
            seconds += time.perf_counter() - t0
            worst = max(worst, float(res.max()))
            ok = ok and status == dg.OK and all(s["converged"] for s in sst)
            outer = max(outer, tot["outer_iterations"])
            inner += tot["inner_iterations"]
            sweeps += tot["sweeps"]
            fp64_sweeps += tot["fp64_sweeps"]
            even_odd, split, df = tot["even_odd"], tot["split_fields"], tot["df_residual"]
            del bs, xs
            torch.cuda.empty_cache()   # the next wave's fields have other sizes
        if dist:
            tt = torch.tensor([seconds], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            seconds = float(tt.item())
        out[prec] = {"seconds": seconds, "all_converged": ok, "max_rel_residual": worst,
                     "outer_max": outer, "inner_iterations": inner, "sweeps": sweeps, "fp64_sweeps": fp64_sweeps,
                     "even_odd": even_odd, "split_fields": split, "df_residual": df,
                     "kernel": list(D.kernel_config())}
        D.close()
        torch.cuda.empty_cache()
    if "f32" in out:
        for p in precs:
            if p != "f32":
                out[p]["speedup_vs_f32"] = out["f32"]["seconds"] / out[p]["seconds"]
    out["workload"] = "wilson_batched_solve_{}_{}sys_{}cols_{}slots".format("x".join(map(str, L)), nsys,
                                                                          sum(nvs), slots)
    out["systems"] = {"nv": nvs, "kappa": kap}
    out["waves"] = [[int(i) for i in w] for w in waves]
    out["sharding"] = f"{ws} rank(s), systems per rank by assign_systems (strong scaling)"
    out["inner_solver"] = ("even-odd CGLS on the Schur complement; 16-bit storage with split fields "
                           "(FP32 e, r, t and links, 16-bit p, s); double-float outer residual")
    return out


def cpu_oracle_rate(w, inputs=None, seconds=15.0, seconds_1thread=5.0):
    """The FP64 oracle on all host cores (the line's cpu_baseline) and on one
    thread (single_thread), each on a bounded random sample of output sites."""
    s = OracleSample(w, inputs)
    n = s.calibrate(seconds)
    dt = s.run(n)
    out = {"value": s.rate(n, dt), "unit": "Gflop/s", "cores": s.cores, "kind": "oracle",
           "sample": s.describe(n, dt)}
    s.cores = s.oracle.set_threads(1)
    n1 = s.calibrate(seconds_1thread)
    dt1 = s.run(n1)
    out["single_thread"] = {"value": s.rate(n1, dt1), "unit": "Gflop/s", "cores": 1, "sample": s.describe(n1, dt1)}
    s.oracle.set_threads(0)
    return out


CPU_TABLE = [
    ("C1", dict(op="staggered", L=(8, 8, 8, 8), Nv=4, mass=0.0, links="haar")),
    ("C2", dict(op="wilson", L=(32, 32, 32, 32), Nv=12, mass=0.125, links="near_identity")),
    ("C3", dict(op="brillouin", L=(24, 24, 24, 48), Nv=12, mass=0.05, links="near_identity")),
    ("H", dict(op="staggered", L=(34, 34, 34, 68), Nv=12, mass=0.0, links="gaussian")),
    ("H", dict(op="wilson", L=(34, 34, 34, 68), Nv=12, mass=0.125, links="gaussian")),
    ("H", dict(op="brillouin", L=(34, 34, 34, 68), Nv=12, mass=0.05, links="gaussian")),
]


def cpu_table(seconds=2.0):
    """The oracle (as it stands: the FP64 build and its FP32 instance) on the
    host cores, on 1 thread and on all of them, for the configurations of the
    CPU-baseline protocol: staggered 8^4 Nv=4, Wilson 32^4 Nv=12, Brillouin
    24^3x48 Nv=12 and the paper's 34^3x68 lattice (Nv=12, all three
    operators).  Each entry times a random sample of output sites sized to
    take about `seconds`, and extrapolates to one whole-lattice apply.  The
    34^3x68 inputs are complex Gaussian links and sources (the oracle's time
    does not depend on the values); the others use the configurations' own
    generators."""
    import oracle
    rows = []
    nproc = os.cpu_count() or 1
    for name, c in CPU_TABLE:
        L, Nv, op = c["L"], c["Nv"], c["op"]
        ns = 1 if op == "staggered" else 4
        if c["links"] == "gaussian":
            V = synth.complex_gaussian(synth.lattice_shape(L) + (4, 3, 3), 1100)
        else:
            V = synth.gauge_links(L, 3, c["links"], 1000 + int(name[1]) if name != "H" else 1100)
        psi = synth.spinor(L, Nv, ns, 3, 2000 + (int(name[1]) if name != "H" else 100), dtype=np.complex64)
        m0 = oracle.kappa_to_m0(c["mass"]) if op == "wilson" else c["mass"]
        vol = int(np.prod(L))
        flops_site = {"staggered": 570, "wilson": 1368, "brillouin": 29208}[op] * Nv
        for prec in ("f64", "f32"):
            fp32 = prec == "f32"
            Vp = V.astype(np.complex64 if fp32 else np.complex128)
            pp = psi.astype(np.complex64 if fp32 else np.complex128)
            for threads in (1, nproc):
                used = oracle.set_threads(threads, fp32=fp32)
                rng = np.random.default_rng(0)
                n = 16
                while True:
                    sites = rng.integers(0, vol, n)
                    t0 = time.perf_counter()
                    oracle.apply(op, Vp, pp, m0, sites=sites, fp32=fp32)
                    dt = time.perf_counter() - t0
                    if dt >= seconds or n >= vol:
                        break
                    n = min(vol, max(2 * n, int(n * seconds * 1.2 / max(dt, 1e-4))))
                rows.append({"config": name, "op": op, "lattice": list(L), "Nv": Nv, "prec": prec,
                             "threads": used, "sites_sampled": int(n), "seconds": dt,
                             "gflops": flops_site * n / dt / 1e9,
                             "seconds_per_apply": dt * vol / n})
            oracle.set_threads(0, fp32=fp32)
        del V, psi
    return {"cpu_table": rows, "host_cores": nproc,
            "note": "model flops (570 / 1368 / 29208 per site and right-hand side); oracle built with gcc -O2 "
                    "-fopenmp, FP64 and its -DORACLE_FP32 instance"}


def dist_init(torch):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, dist


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (host cores, bounded sample per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    s = OracleSample(w)
    per_step = max(0.05, min(5.0, 150.0 / (args.steps + args.warmup)))
    n = s.calibrate(per_step)
    for _ in range(args.warmup):
        s.run(n)
    dts = [s.run(n) for _ in range(args.steps)]
    dt = statistics.mean(dts)
    v = s.rate(n, dt)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gflop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "wilson_apply_32x32x32x32_nv12_f32", "lattice": list(w["L"]), "Nc": 3,
                       "Nv": w["Nv"], "kappa": w["mass"]},
            "cpu_baseline": {"value": v, "unit": "Gflop/s", "cores": s.cores, "kind": "oracle",
                             "sample": s.describe(n, dt) + " per step"},
            "e2e": {"value": v, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solve-variants", action="store_true",
                    help="also the 4-system batched solve with every inner field in 16 bits and with "
                         "whole-lattice inner solves (comparisons; not in the default run)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="only the CPU-baseline table: the oracle on 1 and all host threads, FP64 and FP32, "
                         "for the staggered 8^4, Wilson 32^4, Brillouin 24^3x48 and 34^3x68 configurations")
    ap.add_argument("--full-batched-only", action="store_true",
                    help="only the full 48-system batched solve (--prec for one precision)")
    ap.add_argument("--lattice", default=None, help="Nx,Ny,Nz,Nt (a smaller case for profiling)")
    ap.add_argument("--prec", default=None, choices=["f32", "bf16", "f16", "f64"])
    ap.add_argument("--kernel", default=None,
                    help="R,block,variant[,tchunk]: fixed launch shape (and site order) instead of the autotuner")
    ap.add_argument("--link-format", type=int, default=None, choices=[0, 1],
                    help="with --kernel: the link format (dirac_set_link_format) instead of the default 0")
    ap.add_argument("--op", default="wilson", choices=["wilson", "staggered", "brillouin"],
                    help="operator of the timed sweep (the default workload is Wilson; the others are for profiling)")
    ap.add_argument("--batched-solve-only", action="store_true",
                    help="only the batched Wilson solve (for profiling; --lattice, --prec, --precond, --no-autotune)")
    ap.add_argument("--precond", type=int, default=1, choices=[0, 1], help="with --batched-solve-only")
    ap.add_argument("--no-autotune", action="store_true", help="with --batched-solve-only: default launch shapes")
    ap.add_argument("--inner-fields", type=int, default=1, choices=[0, 1],
                    help="with --batched-solve-only: 1 split inner fields for 16-bit storage (default), 0 all 16-bit")
    args = ap.parse_args()
    global WORKLOAD
    if args.lattice:
        WORKLOAD = dict(WORKLOAD, L=tuple(int(v) for v in args.lattice.split(",")))
    if args.prec:
        WORKLOAD = dict(WORKLOAD, prec=args.prec)
    if args.op != "wilson":
        WORKLOAD = dict(WORKLOAD, op=args.op, mass=0.05 if args.op == "brillouin" else 0.0)
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_table:
        print(json.dumps(cpu_table()), flush=True)
        return
    args.warmup = max(3, args.warmup)

    import torch
    rank, ws, dist = dist_init(torch)
    if ws == 1:
        torch.cuda.set_device(0)
    import paper_1808_05506_gb300 as dg

    if args.full_batched_only:
        out = c5_batched_times(dg, torch, precs=(args.prec,) if args.prec else ("f32", "bf16", "f16"), rank=rank,
                               ws=ws, dist=dist)
        if rank == 0:
            print(json.dumps({"batched_solve_full": out}), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.batched_solve_only:
        out = batched_solve_times(dg, torch, L=WORKLOAD["L"] if args.lattice else (32, 32, 32, 64),
                                  precs=(args.prec,) if args.prec else ("f32", "bf16", "f16"), rank=rank, ws=ws,
                                  dist=dist, precond=args.precond, autotune=not args.no_autotune,
                                  inner_fields=args.inner_fields)
        if rank == 0:
            print(json.dumps({"batched_solve": out}), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    w = WORKLOAD
    V, psi = gen_inputs(w)
    op = w["op"]
    D = dg.Dirac(op, w["L"], w["Nv"], w["mass"], w["prec"])
    D.set_links(torch.from_numpy(V).cuda())
    if args.kernel:
        k = [int(v) for v in args.kernel.split(",")]
        D.set_kernel_config(*k[:3])
        if len(k) > 3:
            D.set_site_order(k[3])
        if args.link_format is not None:
            D.set_link_format(args.link_format)
    else:
        D.autotune()                   # best of the built launch shapes on this GPU
    xin = torch.from_numpy(psi).cuda()
    x = D.pack(xin)
    y = D.new_internal()
    vol = int(np.prod(w["L"]))
    workload = "{}_apply_{}_nv{}_{}".format(op, "x".join(map(str, w["L"])), w["Nv"], w["prec"])
    flops_step = dg.flops_per_site_rhs(op) * vol * w["Nv"]
    link_fmt = D.link_format()
    # the bytes the chosen link format moves (two-row links: two thirds of the link bytes)
    bytes_step = dg.bytes_per_site(op, w["Nv"], w["prec"], link_format=link_fmt) * vol
    if bytes_step < 4 * 129e6:
        raise SystemExit("the timed step must stream more than the L2 (use a larger --lattice)")

    step = lambda: D.apply(x, out=y)   # noqa: E731  one launch of the sweep kernel
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id_for_smi(torch)) as clk:
        total_ms, per = time_kernel(torch, step, args.steps, 0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = total_ms / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = flops_step * ws / (ms * 1e-3) / 1e9
    kern_ms = statistics.mean(per)
    hbm_peak, peak_kind = peaks()
    achieved = bytes_step / (kern_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: dirac_apply_host takes the
    # canonical source from pinned host memory and writes the result there (the
    # H2D copy, pack, sweep, unpack and D2H copy of t-slabs overlap); every step
    # moves the whole field in and out
    host_in = torch.from_numpy(psi).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def e2e_step():
        D.apply_host(host_in, out=host_out, sync=False)

    e2e_steps = max(3, min(50, args.steps // 20))
    e2e_total, _ = time_kernel(torch, e2e_step, e2e_steps, 2)
    e2e_ms = e2e_total / e2e_steps
    h2d = host_in.numel() * host_in.element_size()
    d2h = host_out.numel() * host_out.element_size()

    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        tf = json.load(open(TRAFFIC_FILE))
        if tf.get("kernel_hash") == kernel_hash() and tf.get("workload") == workload:
            traffic = tf.get("dram_bytes_per_launch")
    cfg = D.kernel_config()
    site_order = D.site_order()
    other_fmt = other_format_time(dg, torch, D, x, y, w, 200, 5, link_fmt) if not args.no_extra else None
    D.set_kernel_config(*cfg)
    D.set_site_order(site_order)
    line = {
        "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if w["prec"] != "f64" else "f64", "data": "synthetic",
        "config": {"workload": workload, "op": op, "storage": w["prec"], "lattice": list(w["L"]),
                   "Nc": 3, "Nv": w["Nv"], "kappa": w["mass"], "links": "exp(0.3 i H), H traceless Gaussian",
                   "source": "complex Gaussian N(0,1)", "layout": "internal blocked SoA (blocks of 32 sites)",
                   "l2": "no flush: each step streams {:.2f} GB > 129 MB L2".format(bytes_step / 1e9),
                   "kernel": {"rhs_per_thread": cfg[0], "block": cfg[1], "variant": cfg[2],
                              "site_order_tchunk": site_order, "link_format": link_fmt},
                   "parallelism": f"replicas x{ws}"},
        "hbm_gbs": achieved,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": "k_{}{}<{},R={}>".format(op, {0: "", 1: "_groups", 2: "_march", 3: "_pipe", 5: "_xrow", 6: "_xlast", 7: "_tc"}[cfg[2]],
                                                      w["prec"], cfg[0]),
                     "algorithmic_bytes_per_launch": bytes_step,
                     "link_format": link_fmt,
                     "bytes_per_launch_nine_entry_links": dg.bytes_per_site(op, w["Nv"], w["prec"]) * vol},
        "clocks": clk.summary(),
        "e2e": {"value": flops_step / (e2e_ms * 1e-3) / 1e9, "unit": "Gflop/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "dirac_apply_host: pinned host field in, pinned host field out, "
                        "t-slab copies overlapped with pack / sweep / unpack"},
        "gpu_launches": args.steps,
        "other_link_format": other_fmt,
        "paper_context": PAPER_CONTEXT,
    }
    D.close()
    del x, y, xin
    torch.cuda.empty_cache()
    if not args.no_extra:
        extra = {}
        sw = dict(WORKLOAD, op="staggered", mass=0.0)
        extra["staggered_32x32x32x32_nv12_f32"] = sweep_rate(dg, torch, sw, 200, 5, compare_formats=True)
        bw = dict(WORKLOAD, op="brillouin", L=(24, 24, 24, 48), mass=0.05, seed_links=1003, seed_source=2003)
        extra["brillouin_24x24x24x48_nv12_f32"] = sweep_rate(dg, torch, bw, 20, 3, compare_formats=True)
        extra["brillouin_24x24x24x48_nv12_bf16"] = sweep_rate(dg, torch, dict(bw, prec="bf16"), 20, 3,
                                                              compare_formats=True)
        # the same BF16 sweep on the tensor cores (launch variant 7), which the tuner times but does not keep
        extra["brillouin_24x24x24x48_nv12_bf16_tensor_cores"] = sweep_rate(dg, torch, dict(bw, prec="bf16"), 20, 3,
                                                                           kernel=(1, 128, 7))
        extra["wilson_32x32x32x32_nv12_bf16"] = sweep_rate(dg, torch, dict(WORKLOAD, prec="bf16"), 200, 5,
                                                           compare_formats=True)
        # the paper's own lattice (non-power-of-two extents) and the FP64 sweeps
        extra["wilson_34x34x34x68_nv12_f32"] = sweep_rate(dg, torch, dict(WORKLOAD, L=(34, 34, 34, 68)), 50, 3)
        extra["staggered_34x34x34x68_nv12_f32"] = sweep_rate(dg, torch, dict(sw, L=(34, 34, 34, 68)), 50, 3)
        extra["brillouin_34x34x34x68_nv12_f32"] = sweep_rate(dg, torch, dict(bw, L=(34, 34, 34, 68)), 10, 2)
        # the staggered 8^4, Nv = 4 configuration: 2 MB, resident in L2 (latency-bound; no HBM grading)
        c1 = dict(sw, L=(8, 8, 8, 8), Nv=4, links="haar", seed_links=1001, seed_source=2001)
        extra["staggered_8x8x8x8_nv4_f32_l2_resident"] = sweep_rate(dg, torch, c1, 500, 20)
        extra["wilson_32x32x32x32_nv12_f64"] = sweep_rate(dg, torch, dict(WORKLOAD, prec="f64"), 20, 3)
        extra["staggered_32x32x32x32_nv12_f64"] = sweep_rate(dg, torch, dict(sw, prec="f64"), 20, 3)
        extra["brillouin_24x24x24x48_nv12_f64"] = sweep_rate(dg, torch, dict(bw, prec="f64"), 3, 1,
                                                             kernel=(2, 128, 0))
        line["extra"] = extra
    if not args.no_solve and not args.no_extra:
        line["solve"] = solve_times(dg, torch)
        # the full batched configuration: 48 systems, every column to 1e-10
        line["batched_solve_full"] = c5_batched_times(dg, torch, rank=rank, ws=ws, dist=dist)
        sp = {}
        for p in ("bf16", "f16"):
            sp["brillouin_solve_" + p] = line["solve"][p].get("speedup_vs_f32")
            sp["batched_solve_full_" + p] = line["batched_solve_full"][p].get("speedup_vs_f32")
        line["speedup_vs_f32"] = sp
        if args.solve_variants:
            line["batched_solve"] = batched_solve_times(dg, torch, rank=rank, ws=ws, dist=dist)
            # 16-bit storage with every inner field in 16 bits, for comparison
            uni = batched_solve_times(dg, torch, precs=("bf16", "f16"), rank=rank, ws=ws, dist=dist,
                                      inner_fields=0)
            for p in ("bf16", "f16"):
                uni[p]["speedup_vs_f32"] = line["batched_solve"]["f32"]["seconds"] / uni[p]["seconds"]
            uni["inner_solver"] += "; every inner field in 16 bits"
            line["batched_solve_all16"] = uni
            # the same systems with the whole-lattice inner solver, for comparison
            line["batched_solve_whole_lattice"] = batched_solve_times(dg, torch, rank=rank, ws=ws, dist=dist,
                                                                      precond=0)
        _BATCHED_INPUTS.clear()
        _LINKS.clear()
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(w, inputs=(V, psi))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
