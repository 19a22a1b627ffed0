#!/usr/bin/env python
"""Benchmark of the overlap hot path on GB300.

Workload (the overlap-apply configuration): D(mu) v = 1/2 (1 + mu + (1 - mu) gamma5 sign(K)) v
on a 16^3 x 32 lattice with smooth random SU(3) links (eps = 0.3, seed 1002), m0 = 1.4,
mu = 0.05, 20 Zolotarev poles with Delta <= 1e-10, applied to 16 Gaussian vectors per
step with the sign function evaluated to eta = 1e-10. An FP32 sign cannot reach 1e-10; the
step runs the multi-shift CG and the Wilson kernel in double-float (two floats per value,
~47-bit significand, on the FP32 pipes, since GB300 issues FP64 at 1/60 of FP32), with the
Zolotarev sum evaluated by Lanczos on K^2 whose basis is kept in HBM (one vector per step,
every pole's solution from a tridiagonal solve and one pass over the basis); the same step
with native FP64 is reported beside it. Inputs are resident in HBM when the timed region
starts; 16 input vectors and the 16 x ~120 stored basis vectors (~48 GB) exceed the 126 MB L2.

One JSON line on rank 0:
  value      applies/s over all ranks (device-resident inputs, CUDA events around the
             timed steps; the library's production path: multi-shift iterations replayed
             as cached CUDA graphs, no per-launch events)
  e2e        the same through the C ABI with host buffers (copies inside the timed region)
  roofline   the dominant kernel of the step, from a second, profiled pass of the same
             step (CUDA events recorded by the library around every launch, on the
             launching stream): algorithmic bytes per launch (per site and system: K mode
             2 spinors, r-update mode 4 spinors, plus 576 B of 18-real FP64 links per site
             shared by the launch's systems) over its mean launch time, against the
             measured HBM copy bandwidth; the FP32-issue view of the same kernel beside it
             against a measured FMA rate
  cpu_baseline  the oracle (plain NumPy/SciPy, every pole of every vector by its own CG)
             on this host: complete applies on 8^4 timed on all cores and on one core,
             extrapolated to 16^3 x 32 by the measured cost of one oracle K application
  extras     FP32 / FP16-storage applies with their error against the FP64 result,
             Wilson-kernel bandwidth on 24^3 x 48, and one right-hand-side solve to 1e-10
             (mixed GMRESR(relSUMR) and plain FP64)

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU (the path
shards by right-hand sides; weak scaling, no collective on the data path).
"""
import argparse
import contextlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

DIMS = (16, 16, 16, 32)
M0, MU, NPOLES, EPS = 1.4, 0.05, 20, 1e-10
NVEC = 16
LINK_SEED, SRC_SEED = 1002, 2002
WILSON_FLOPS_PER_SITE = 1320          # conventional count of the hopping term
FP64_NOMINAL_TFLOPS = 1.25            # GB300 FP64 (nominal; the ALU roofline of the FP64 kernel)
# FP32 operations one double-float site application needs by construction: per neighbour
# 12 lazy double-float sums for the projection (8 each), 12 link-product components as
# 6-term Dot2 sums (4 + 5 x 12 each) and 24 lazy sums into the accumulator (8 each) =
# 1056; x 8 neighbours, plus the diagonal term in - kappa hop (24 x (7 + 11)). Loads,
# index arithmetic, phase selects and the epilogue reductions are not counted.
DF64_FP32_OPS_PER_SITE = 8 * (12 * 8 + 12 * (4 + 5 * 12) + 24 * 8) + 24 * (7 + 11)
# DRAM bytes (read + write) per launch of the double-float Wilson kernel in this step: the
# mean of the first six timed launches (three of each Lanczos mode) in one ncu capture of
# this command (profiles/launches_overlap_apply_lanczos_df64_16x16x16x32.md); each mode moves
# 1.18-1.19 x its algorithmic bytes.
TRAFFIC_WILSON_DF64 = 1.44e9
# Algorithmic bytes of one Wilson launch, per site: every system reads its input spinor
# and writes its output (K mode) or also reads p and r and writes r (r-update mode); the
# four 18-real FP64 links of the site (576 B) are read once per launch.
LINK_BYTES_18REAL = 576


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class Clocks:
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
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_lines(f)
        os.unlink(self.path)
        return out


def parse_clock_lines(lines):
    """Median SM clock, maximum clock and the throttle reasons seen, from nvidia-smi
    csv lines (noheader, nounits) of Clocks.FIELDS."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline
ORACLE_DIMS = (8, 8, 8, 8)
ORACLE_BOUNDS = (0.2, 2.6)     # [a, b] of the oracle's rational (the library estimates its own)
ORACLE_POLE_TOL = 1e-11        # per-pole CG residual: the sum of Sec. 3 then errs by ~1e-10


def _oracle_setup():
    import synth
    from oracle import zolotarev as zo
    U8 = synth.gauge_links(ORACLE_DIMS, 0.3, LINK_SEED)
    om, sg, _ = zo.zolotarev(NPOLES, *ORACLE_BOUNDS)
    return U8, om, sg


def _k_cost_ratio():
    """Measured cost of one oracle K application (apply_K) on 16^3x32 over 8^4."""
    import synth
    from oracle import wilson
    out = []
    for dims in (ORACLE_DIMS, DIMS):
        U = synth.gauge_links(dims, 0.3, LINK_SEED)
        v = synth.gaussian_source(dims, SRC_SEED)
        wilson.apply_K(U, v, M0)
        t0 = time.perf_counter()
        reps = 6 if dims == ORACLE_DIMS else 2
        for _ in range(reps):
            wilson.apply_K(U, v, M0)
        out.append((time.perf_counter() - t0) / reps)
    return out[1] / out[0]


class OraclePool:
    """A spawn-context pool of oracle workers, each holding K of the 8^4 field as a sparse
    matrix; one apply = every pole of every vector by its own CG (the oracle's
    shifted_solves), then K sum_i omega_i x_i on this process."""

    def __init__(self, workers):
        import multiprocessing as mp
        from oracle import overlap, wilson
        self.U8, self.om, self.sg = _oracle_setup()
        self.workers = workers
        self.K = wilson.sparse_K(self.U8, M0)
        self.pool = None
        if workers > 1:
            keep = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
            for k in keep:
                os.environ[k] = "1"
            self.pool = mp.get_context("spawn").Pool(workers, initializer=overlap._worker_init,
                                                     initargs=(self.U8, M0, False))
            for k, v in keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        else:
            overlap._worker_init(self.U8, M0, False)

    def apply(self, vs):
        from oracle import overlap, wilson
        tasks = [(v.ravel(), float(s), ORACLE_POLE_TOL) for v in vs for s in self.sg]
        if self.pool is not None:
            res = self.pool.map(overlap._worker_pole_solve, tasks, chunksize=1)
        else:
            res = [overlap._worker_pole_solve(t) for t in tasks]
        n = len(self.sg)
        its, outs = 0, []
        for j, v in enumerate(vs):
            y = sum(om * res[j * n + i][0] for i, om in enumerate(self.om))
            its += sum(res[j * n + i][1] for i in range(n))
            outs.append(0.5 * (1 + MU) * v + 0.5 * (1 - MU) * wilson.apply_gamma5((self.K @ y).reshape(v.shape)))
        return its, outs

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_baseline():
    """The oracle timed on this host: complete applies D(mu) v at eta = 1e-10 on 8^4 (m0,
    mu and 20 poles as in the benchmark, the oracle's own rational on [0.2, 2.6]), once
    with every core (as many vectors as cores, in a process pool) and once with one
    core (one vector); the 16^3 x 32 figure is extrapolated from them by the measured
    cost ratio of one oracle K application (same iteration counts assumed)."""
    import synth
    cores = _cores()
    vs = synth.gaussian_source(ORACLE_DIMS, SRC_SEED, nvec=cores)
    op = OraclePool(cores)
    t0 = time.perf_counter()
    op.apply(vs)
    t_all = time.perf_counter() - t0
    op.close()
    one = OraclePool(1)
    t0 = time.perf_counter()
    its1, _ = one.apply(vs[:1])
    t_one = time.perf_counter() - t0
    ratio = _k_cost_ratio()
    rate8 = cores / t_all
    return {"value": rate8 / ratio, "unit": "applies/s", "cores": cores, "kind": "oracle",
            "sample": "complete oracle applies on 8^4 (%d vectors on %d cores in %.1f s; 1 vector on 1 core in "
                      "%.1f s; %d per-pole CG iterations per vector), extrapolated to 16^3x32 by the measured "
                      "cost ratio %.1f of one oracle K application" % (cores, cores, t_all, t_one, its1, ratio),
            "extrapolated_to_16x16x16x32": True,
            "measured_8x8x8x8": {"applies_per_s_all_cores": rate8, "cores": cores,
                                 "applies_per_s_1_core": 1.0 / t_one, "cg_iterations_per_vector": its1}}


# ------------------------------------------------------------------ ours
def run_ours(args, ws, rank, local):
    import torch
    import synth
    from paper_1501_01855_gb300 import build, binding as B

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    U = synth.gauge_links(DIMS, 0.3, LINK_SEED)
    vecs = synth.gaussian_source(DIMS, SRC_SEED + rank, nvec=NVEC)
    p = B.ovl_params_default()
    p.stream = stream.cuda_stream
    ctx = B.Overlap(DIMS, U, M0, MU, NPOLES, EPS, params=p)
    om, sg, delta, a, b = ctx.zolotarev()
    dv = torch.from_numpy(vecs).to(dev)
    dout = torch.empty_like(dv)
    step = lambda: ctx.apply(dv, dout, eta=EPS, prec=B.OVL_PREC_F64E)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")    # lets a profiler select the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_total = e0.elapsed_time(e1)
    barrier(ws)
    ms_total = max_over_ranks(ms_total, ws)
    value = ws * NVEC * args.steps / (ms_total * 1e-3)

    # per-kernel breakdown: the same step again with the library's profiler on (events
    # around every launch on the context stream; the multi-shift iterations are then
    # launched one by one instead of as graphs), outside the timed region
    prof_steps = 2
    ctx.profile_reset()
    ctx.profile_enable(True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    prof = ctx.profile_get()
    prof_ms_total = sum(v["ms"] for v in prof.values())

    # end to end through the C ABI with host buffers (page-locked, so the copies are DMA)
    hv = torch.from_numpy(np.ascontiguousarray(vecs)).pin_memory().numpy()
    hout = torch.empty(hv.shape, dtype=torch.complex128).pin_memory().numpy()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.apply(hv, hout, eta=EPS, prec=B.OVL_PREC_F64E)
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - t0, ws)
    nbytes = hv.nbytes
    e2e = {"value": ws * NVEC * args.steps / te, "unit": "applies/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    # roofline of the dominant kernel class (by time in the profiled pass)
    hbm, hbm_src = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    avg_ms = d["ms"] / max(1, d["launches"])
    ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    names = {"wilson_f64e": "wilson_kernel (double-float; the Lanczos K and three-term-recurrence launches + "
                            "the final overlap epilogue)",
             "mscg_update": "lz_combine_df_kernel (y from the stored Lanczos basis)"}
    roof = {"kernel": names.get(dom, dom), "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": TRAFFIC_WILSON_DF64 if dom == "wilson_f64e" else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s copy bandwidth)" % hbm_src,
            "launches": d["launches"], "avg_launch_ms": avg_ms,
            "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
            "share_of_profiled_step": d["ms"] / prof_ms_total if prof_ms_total > 0 else None}
    if dom == "wilson_f64e":
        fma = ctx.bench_fp32()
        ops = d["units"] * DF64_FP32_OPS_PER_SITE
        roof["fp32_issue_view"] = {"achieved_T_ops_per_s": ops / (d["ms"] * 1e-3) / 1e12,
                                   "peak_T_fma_per_s_measured": fma / 1e12,
                                   "frac": ops / (d["ms"] * 1e-3) / fma,
                                   "ops_per_site": DF64_FP32_OPS_PER_SITE,
                                   "note": "the kernel issues FP32 error-free transformations; this "
                                           "counts them (not loads, index arithmetic or selects) against "
                                           "a measured FMA issue rate"}
    launches_per_step = sum(v["launches"] for v in prof.values()) / prof_steps
    launches = int(round(launches_per_step * args.steps))

    line = {
        "metric": "overlap D applies/s & RHS solves/s at 1e-10; Dslash HBM GB/s vs plain FP64",
        "value": value, "unit": "applies/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "df64", "data": "synthetic",
        "config": {"workload": "overlap D(mu) apply, 16^3x32, m0=1.4, mu=0.05, 20 Zolotarev poles, eta=1e-10, "
                               "16 Gaussian vectors per step",
                   "lattice": "16x16x16x32", "links": "proj_SU3(exp(i 0.3 H)), seed 1002", "n_poles": NPOLES,
                   "zolotarev_delta": delta, "bounds": [a, b],
                   "sign_precision": "double-float (hi+lo FP32 pairs) Wilson kernel and stored-basis Lanczos "
                                     "evaluation of the Zolotarev sum", "nvec": NVEC,
                   "l2": "inputs larger than L2 (16 x 25 MB vectors, ~48 GB of stored Lanczos basis per step)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": e2e, "roofline": roof, "gpu_launches": launches, "clocks": clocks,
        "profile": {"steps": prof_steps, "note": "profiled pass outside the timed region (per-launch events, "
                                                 "no graphs); ms and GB/s per kernel class over the pass",
                    "classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                    "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None}
                                for k, v in prof.items() if v["launches"]}},
    }
    ref_out = dout.cpu().numpy()
    ctx.trim()     # the extras create contexts of their own

    if rank == 0 and not args.no_extras:
        with _section(line, "extras"):
            line["extras"] = extras(args, ctx, dv, dout, ref_out, B, torch, stream, hbm)
    ctx.close()
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            line["cpu_baseline"] = oracle_baseline()
        except Exception as e:   # the oracle's timing must not cost the GPU line
            line["cpu_baseline"] = {"kind": "oracle", "error": "%s: %s" % (type(e).__name__, e)}
    return line


@contextlib.contextmanager
def _section(out, key):
    """One block of the extras: an exception is recorded under key instead of costing the
    benchmark line."""
    try:
        yield
    except Exception as e:
        out[key] = {"error": "%s: %s" % (type(e).__name__, e)}


def extras(args, ctx, dv, dout, ref_out, B, torch, stream, hbm):
    import synth
    out = {}
    with _section(out, "precision_applies"):
        # the same apply in native FP64 (the plain path), and the mixed-precision applies:
        # FP32 sign at eta=1e-6, FP16 storage at eta=1e-2; errors against the double-float result
        for name, prec, eta in (("native_fp64_eta1e-10", B.OVL_PREC_F64, 1e-10), ("fp32_eta1e-6", B.OVL_PREC_F32, 1e-6),
                                ("fp16_eta1e-2", B.OVL_PREC_F16, 1e-2)):
            ctx.apply(dv, dout, eta=eta, prec=prec)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps = 3
            for _ in range(reps):
                ctx.apply(dv, dout, eta=eta, prec=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            got = dout.cpu().numpy()
            err = max(np.linalg.norm(got[j] - ref_out[j]) / np.linalg.norm(ref_out[j]) for j in range(NVEC))
            out[name] = {"applies_per_s": NVEC / (ms * 1e-3), "max_rel_error_vs_df64": err}
    ctx.trim()
    with _section(out, "wilson_24x24x24x48"):
        # Wilson kernel bandwidth on 24^3x48 (working set larger than L2)
        dims = (24, 24, 24, 48)
        p = B.ovl_params_default()
        p.a_override, p.b_override = 0.2, 2.6
        p.stream = stream.cuda_stream
        cw = B.Overlap(dims, synth.unit_links(dims), M0, MU, 8, 1e-3, params=p)
        ds = {}
        for prec, nm in ((0, "f64"), (3, "df64"), (1, "f32"), (2, "f16")):
            for n in (1, 12):
                ms, by = cw.bench_wilson(prec, n, 40 if n == 1 else 8)
                gbs = by / (ms * 1e-3) / 1e9
                ds["%s_n%d" % (nm, n)] = {"ms": ms, "GB/s": gbs, "frac_hbm": gbs / hbm,
                                         "Gsites/s": 663552 * n / (ms * 1e-3) / 1e9}
        cw.close()
        out["wilson_24x24x24x48"] = ds
    with _section(out, "solve_16x16x16x32_mu0.05"):
        # one RHS solve to 1e-10: mixed GMRESR(relSUMR) vs plain FP64
        U = synth.gauge_links(DIMS, 0.3, LINK_SEED)
        b = synth.gaussian_source(DIMS, 3002)
        sol = {}
        for nm, mixed, emul in (("mixed_relSUMR", 1, 1), ("mixed_relSUMR_native_fp64_outer", 1, 0),
                                ("plain_fp64_relSUMR", 0, 0)):
            p = B.ovl_params_default()
            p.mixed = mixed
            p.emulate_fp64 = emul
            p.stream = stream.cuda_stream
            cs = B.Overlap(DIMS, U, M0, MU, NPOLES, EPS, params=p)
            x = np.zeros_like(b)
            cs.solve(b, x, 1e-10)             # warm-up (allocations)
            t0 = time.perf_counter()
            info = cs.solve(b, x, 1e-10)[0]
            dt = time.perf_counter() - t0
            cs.profile_reset()
            cs.profile_enable(True)
            cs.solve(b, x, 1e-10)
            cs.profile_enable(False)
            prof = {k: round(v["ms"], 2) for k, v in cs.profile_get().items() if v["launches"]}
            sol[nm] = {"seconds": dt, "solves_per_s": 1.0 / dt, "true_residual": info["true_residual"],
                       "outer": info["outer_iters"], "inner": info["inner_iters"],
                       "wilson_calls_dp2": info["wilson_calls"], "profile_ms": prof}
            cs.close()
        out["solve_16x16x16x32_mu0.05"] = sol
    with _section(out, "deflated_batched_16x16x16x32_mu0.02"):
        out["deflated_batched_16x16x16x32_mu0.02"] = deflated_batched(B, stream)
    with _section(out, "host_eigh_ms"):
        # the m x m Hermitian eigendecomposition of a Ritz step on the host (m = 192: the basis
        # of the 24^3 x 48 deflated solves; Householder + implicit QR), through the C ABI
        rng = np.random.default_rng(5)
        res = {}
        for m in (64, 192):
            Qm, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
            A = (Qm * np.sort(rng.uniform(1e-4, 3.0, m))) @ Qm.conj().T
            B.ovl_host_eigh(A)
            t0 = time.perf_counter()
            for _ in range(3):
                B.ovl_host_eigh(A)
            res["m%d" % m] = (time.perf_counter() - t0) / 3 * 1e3
        # a whole Ritz restart on the host (Alg. 6 with the locally optimal restart) at the
        # 24^3 x 48 accumulation's sizes: basis 192, 64 kept, on Gram blocks of random data
        V = rng.normal(size=(2048, 192)) + 1j * rng.normal(size=(2048, 192))
        VD = rng.uniform(0.05, 1.0, size=(2048, 1)) * V
        E, M, G = V.conj().T @ V, VD.conj().T @ VD, V.conj().T @ VD
        B.ovl_host_ritz(E, M, G, 0.05, 0.01, 64, restart=True)
        t0 = time.perf_counter()
        B.ovl_host_ritz(E, M, G, 0.05, 0.01, 64, restart=True)
        res["ritz_restart_k192_keep64"] = (time.perf_counter() - t0) * 1e3
        out["host_eigh_ms"] = res
    # Gram block of the Ritz step (128 x 128 spinors on 16^3 x 32): tensor cores at FP64 level
    # against the CUDA-core kernel with FP32 products
    try:
        p = B.ovl_params_default()
        p.a_override, p.b_override = 0.2, 2.6
        p.stream = stream.cuda_stream
        cg = B.Overlap(DIMS, synth.unit_links(DIMS), M0, MU, 8, 1e-3, params=p)
        v = int(np.prod(DIMS))
        g = {}
        for name, prec, method in (("f64_tensor_cores", B.OVL_PREC_F64, 0), ("f32_tensor_cores", B.OVL_PREC_F32, 0),
                                   ("f64_cuda_cores_fp32_products", B.OVL_PREC_F64, 1)):
            ms = cg.bench_gram(prec, 128, 128, method, 3)
            g[name] = {"ms": ms, "T_complex_mac_per_s": 128.0 * 128 * 12 * v / (ms * 1e-3) / 1e12}
            if method == 0:
                # 2 K-steps x 26 digit-pair MMAs of 128 x 64 x 16 per 16 complex elements and tile
                g[name]["bf16_TFLOP_per_s_tensor_pipe"] = 4 * (12.0 * v / 16) * 2 * 26 * (128 * 64 * 16) * 2 / (ms * 1e-3) / 1e12
        cg.close()
        out["gram_128x128_16x16x16x32"] = g
    except Exception as e:   # the extras must not cost the benchmark line
        out["gram_128x128_16x16x16x32"] = {"error": str(e)}
    return out


def deflated_batched(B, stream):
    """Deflated, batched right-hand sides (the shape of the paper's use case): eigSUMR
    solves of three Gaussian sources accumulate and refine 32 low modes of D^dag D
    (basis 2 n + 64 = 128), then the 12 spin-colour point sources at one site are solved in one
    lock-step batch, undeflated and deflated, with relSUMR (deflated start) and relCG
    (spectral preconditioner; the space is handed over through ovl_defl_save/load),
    against one plain-FP64 (no mixed precision, no deflation) solve. mu = 0.02, 1e-10."""
    import tempfile
    import synth
    mu, tol = 0.02, 1e-10
    U = synth.gauge_links(DIMS, 0.3, 1003)
    srcs = np.stack([synth.point_source(DIMS, s, c) for s in range(4) for c in range(3)])
    res = {}
    p = B.ovl_params_default()
    p.stream = stream.cuda_stream
    ctx = B.Overlap(DIMS, U, M0, mu, NPOLES, EPS, params=p)
    defl = None
    t0 = time.perf_counter()
    for k in range(3):
        b0 = synth.gaussian_source(DIMS, 2003 + k)
        x0 = np.zeros_like(b0)
        if k == 2:
            ctx.profile_reset()
            ctx.profile_enable(True)
        defl, info0 = ctx.eigsumr_accumulate(b0, x0, tol, 32, 128, defl=defl)
    ctx.profile_enable(False)
    res["eigsumr_3_accumulation_solves_s"] = time.perf_counter() - t0
    prof = ctx.profile_get()
    tot = sum(v["ms"] for v in prof.values())
    # the dense contractions (Gram blocks of the Ritz steps, basis rotations) against the
    # whole third accumulation solve, as timed by the profiler
    res["gram_combine_share_of_accumulation_solve"] = prof["gram"]["ms"] / tot if tot > 0 else None
    ritz, rres = defl.info()
    res["ritz_values_lowest4"] = [float(v) for v in ritz[:4]]
    res["ritz_residual_lowest8_max"] = float(np.max(rres[:8]))
    res["ritz_residual_median"] = float(np.median(rres))

    def batch(c, d):
        xs = np.zeros_like(srcs)
        t0 = time.perf_counter()
        infos = c.solve(srcs, xs, tol, defl=d)
        dt = time.perf_counter() - t0
        return {"seconds": dt, "rhs_solves_per_s": len(srcs) / dt,
                "max_true_residual": max(i["true_residual"] for i in infos),
                "inner_iters_mean": float(np.mean([i["inner_iters"] for i in infos])),
                "wilson_calls_dp2_total": int(sum(i["wilson_calls"] for i in infos))}

    res["relSUMR_undeflated"] = batch(ctx, None)
    res["relSUMR_deflated"] = batch(ctx, defl)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "defl.bin")
        defl.save(path)
        defl.close()
        ctx.close()
        p = B.ovl_params_default()
        p.solver = B.OVL_SOLVER_CG
        p.stream = stream.cuda_stream
        cc = B.Overlap(DIMS, U, M0, mu, NPOLES, EPS, params=p)
        dc = B.Deflation.load_file(cc, path)
        res["relCG_undeflated"] = batch(cc, None)
        res["relCG_deflated"] = batch(cc, dc)
        dc.close()
        cc.close()
    p = B.ovl_params_default()
    p.mixed = 0
    p.emulate_fp64 = 0
    p.stream = stream.cuda_stream
    cp = B.Overlap(DIMS, U, M0, mu, NPOLES, EPS, params=p)
    x1 = np.zeros_like(srcs[:1])
    t0 = time.perf_counter()
    info = cp.solve(srcs[:1], x1, tol)[0]
    dt = time.perf_counter() - t0
    res["plain_fp64_single_rhs"] = {"seconds": dt, "rhs_solves_per_s": 1.0 / dt,
                                    "true_residual": info["true_residual"], "inner_iters": info["inner_iters"],
                                    "wilson_calls_dp2": info["wilson_calls"]}
    cp.close()
    best = max(res[k]["rhs_solves_per_s"] for k in ("relSUMR_deflated", "relCG_deflated"))
    res["best_deflated_batched_over_plain_fp64"] = best / res["plain_fp64_single_rhs"]["rhs_solves_per_s"]
    return res


def config_c4(B, stream):
    """Batched multi-mass deflated solves on 24^3 x 48 (the largest configuration of the
    benchmark set): 12 spin-colour point sources x 3 masses mu in {0.01, 0.02, 0.04} = 36
    systems in one lock-step batch, 64 eigenvectors of D^dag D (accumulated by eigSUMR at
    mu = 0.01 over three Gaussian-source solves, basis 2 n + 64 = 192) shared by all masses, 24
    Zolotarev poles, autotuned Wilson kernel, CUDA-graph multi-shift iterations, relative
    residual 1e-10; against one plain-FP64 solve of one source at mu = 0.01."""
    import synth
    dims = (24, 24, 24, 48)
    tol, npoles = 1e-10, 24
    mus = [0.01, 0.02, 0.04]
    U = synth.gauge_links(dims, 0.3, 1004)
    srcs = np.stack([synth.point_source(dims, s, c) for s in range(4) for c in range(3)])
    out = {"workload": "24^3x48, eps 0.3 links seed 1004, m0 1.4, 24 poles, 12 point sources x 3 masses, "
                       "64 eigenvectors, tol 1e-10"}
    p = B.ovl_params_default()
    p.stream = stream.cuda_stream
    ctx = B.Overlap(dims, U, M0, mus[0], npoles, EPS, params=p)
    out["zolotarev"] = dict(zip(("delta", "a", "b"), ctx.zolotarev()[2:]))
    defl = None
    t0 = time.perf_counter()
    for k in range(3):
        b0 = synth.gaussian_source(dims, 2004 + k)
        x0 = np.zeros_like(b0)
        defl, _ = ctx.eigsumr_accumulate(b0, x0, tol, 64, 192, defl=defl)
    out["eigsumr_3_solves_s"] = time.perf_counter() - t0
    ritz, rres = defl.info()
    out["ritz_residual_lowest8_max"] = float(np.max(rres[:8]))
    for name, d in (("undeflated", None), ("deflated", defl)):
        xs = np.zeros((len(srcs) * len(mus),) + srcs.shape[1:], dtype=srcs.dtype)
        t0 = time.perf_counter()
        infos = ctx.solve(srcs, xs, tol, mus=mus, defl=d)
        dt = time.perf_counter() - t0
        out["batched_" + name] = {"seconds": dt, "rhs_solves_per_s": len(infos) / dt,
                                  "max_true_residual": max(i["true_residual"] for i in infos),
                                  "inner_iters_by_mass": [float(np.mean([i["inner_iters"] for i in
                                                                         infos[m * len(srcs):(m + 1) * len(srcs)]]))
                                                          for m in range(len(mus))]}
    defl.close()
    ctx.close()
    p = B.ovl_params_default()
    p.mixed = 0
    p.emulate_fp64 = 0
    p.stream = stream.cuda_stream
    cp = B.Overlap(dims, U, M0, mus[0], npoles, EPS, params=p)
    x1 = np.zeros_like(srcs[:1])
    t0 = time.perf_counter()
    info = cp.solve(srcs[:1], x1, tol)[0]
    dt = time.perf_counter() - t0
    out["plain_fp64_single_rhs_mu0.01"] = {"seconds": dt, "rhs_solves_per_s": 1.0 / dt,
                                           "true_residual": info["true_residual"]}
    cp.close()
    out["deflated_batched_over_plain_fp64"] = (out["batched_deflated"]["rhs_solves_per_s"]
                                               / out["plain_fp64_single_rhs_mu0.01"]["rhs_solves_per_s"])
    return out


def deflation_gain(B, stream):
    """The deflation-gain experiment of Sec. 6 (Figs. 7 and 9) on the synthetic 16^3 x 32
    ensemble at mu = 0.02: spaces of 15, 30 and 45 vectors, (a) accumulated by eigSUMR
    during three solves and (b) from the standalone eigensolver, then 4 point sources
    solved in one batch with relSUMR and relCG, undeflated and deflated. The gain in
    middle-solver iterations is set against the bound the paper uses,
    |lambda_{n+1}(gamma5 D)| / |lambda_1(gamma5 D)|, here from the Ritz values of a
    46-vector space (|lambda(H)|^2 ~ lambda(D^dag D))."""
    import tempfile
    import synth
    mu, tol = 0.02, 1e-10
    U = synth.gauge_links(DIMS, 0.3, 1003)
    srcs = np.stack([synth.point_source(DIMS, 0, c) for c in range(3)] + [synth.point_source(DIMS, 1, 0)])
    out = {"workload": "16^3x32, eps 0.3 links seed 1003, m0 1.4, mu 0.02, 20 poles, 4 point sources, tol 1e-10"}

    def solve(c, d):
        xs = np.zeros_like(srcs)
        t0 = time.perf_counter()
        infos = c.solve(srcs, xs, tol, defl=d)
        dt = time.perf_counter() - t0
        return {"inner_iters_mean": float(np.mean([i["inner_iters"] for i in infos])),
                "wilson_calls_dp2_mean": float(np.mean([i["wilson_calls"] for i in infos])),
                "seconds": dt, "max_true_residual": max(i["true_residual"] for i in infos)}

    def make(solver):
        p = B.ovl_params_default()
        p.stream = stream.cuda_stream
        p.solver = solver
        return B.Overlap(DIMS, U, M0, mu, NPOLES, EPS, params=p)

    cs = make(B.OVL_SOLVER_SUMR)
    ccg = make(B.OVL_SOLVER_CG)
    out["undeflated"] = {"relSUMR": solve(cs, None), "relCG": solve(ccg, None)}

    def evaluate(defl, key, n, seconds):
        ritz, res = defl.info()
        row = {"build_s": seconds, "ritz_residual_median": float(np.median(res)),
               "ritz_residual_max": float(np.max(res)), "ritz": [float(x) for x in ritz],
               "relSUMR": solve(cs, defl)}
        with tempfile.TemporaryDirectory() as dd:
            path = os.path.join(dd, "defl.bin")
            defl.save(path)
            dc = B.Deflation.load_file(ccg, path)
            row["relCG"] = solve(ccg, dc)
            dc.close()
        out.setdefault(key, {})["n%d" % n] = row

    for n in (15, 30, 45):
        # (a) the accumulation during three solves (eigSUMR), basis 2 n + 64
        defl = None
        t0 = time.perf_counter()
        for k in range(3):
            b0 = synth.gaussian_source(DIMS, 2003 + k)
            defl, _ = cs.eigsumr_accumulate(b0, np.zeros_like(b0), tol, n, 2 * n + 64, defl=defl)
        evaluate(defl, "eigsumr_3_solves", n, time.perf_counter() - t0)
        defl.close()
        # (b) the standalone eigensolver, 2500 sign applications at most
        t0 = time.perf_counter()
        defl, used = cs.eigensolve(n, 2 * n + 64, 2500, res_tol=1e-3)
        evaluate(defl, "standalone", n, time.perf_counter() - t0)
        out["standalone"]["n%d" % n]["sign_applications"] = used
        if n == 45:
            ritz_all = defl.info()[0]
        defl.close()
    # the bound of Sec. 6: |lambda_{n+1}(H)| / |lambda_1(H)| from the best 45-vector space
    # (Ritz values of D^dag D + 2 mu delta H ~ lambda(H)^2); lambda_46 from a 46th vector
    d46, _ = cs.eigensolve(46, 2 * 46 + 64, 2500, res_tol=1e-3)
    ritz_all = d46.info()[0]
    d46.close()
    lam = np.sqrt(np.maximum(np.asarray(ritz_all), 0.0))    # |lambda(H)| estimates, ascending
    for key in ("eigsumr_3_solves", "standalone"):
        for n in (15, 30, 45):
            row = out[key]["n%d" % n]
            row["bound"] = float(lam[n] / lam[0])
            for sv in ("relSUMR", "relCG"):
                row[sv]["gain_inner_iters"] = out["undeflated"][sv]["inner_iters_mean"] / row[sv]["inner_iters_mean"]
                row[sv]["gain_wilson_calls"] = (out["undeflated"][sv]["wilson_calls_dp2_mean"]
                                                / row[sv]["wilson_calls_dp2_mean"])
    out["lambda_H_lowest_from_ritz"] = [float(x) for x in lam[:4]]
    cs.close()
    ccg.close()
    return out


def config_c5(B, stream):
    """Gradient of S = phi^dag (D^dag D)^-1 phi with respect to every gauge link (the fermion
    force) on 8^4 and 16^3 x 32, mu = 0.05, 16 Zolotarev poles on [0.2, 2.6]: the FP32 adjoint
    (FP32 outer products, FP64 accumulation) timed against the FP64 one, the recompute path
    (shifted solutions in groups of 4 poles instead of all stored) against the stored one,
    and central finite differences of the action along 4 random Lie-algebra directions
    (2 at 16^3 x 32) against the gradient."""
    import synth
    out = {"workload": "fermion force, eps 0.3 links seed 1005, m0 1.4, mu 0.05, 16 poles on [0.2, 2.6], "
                       "one Gaussian phi, solves to 1e-11"}
    lam = synth._gell_mann()

    def make(dims, U, **kw):
        p = B.ovl_params_default()
        p.stream = stream.cuda_stream
        p.a_override, p.b_override = 0.2, 2.6
        for k, v in kw.items():
            setattr(p, k, v)
        return B.Overlap(dims, U, M0, 0.05, 16, 1e-8, params=p)

    for dims, ndir in (((8, 8, 8, 8), 4), ((16, 16, 16, 32), 2)):
        key = "x".join(map(str, dims))
        U = synth.gauge_links(dims, 0.3, 1005)
        phi = synth.gaussian_source(dims, 2005)
        row = {}
        grads = {}
        for name, kw in (("fp32_adjoint", {"mixed": 1}), ("fp64_adjoint", {"mixed": 0}),
                         ("fp32_adjoint_pole_groups_of_4", {"mixed": 1, "force_pole_group": 4})):
            c = make(dims, U, **kw)
            c.force(phi, tol=1e-11)                      # warm-up: graphs, workspaces
            t0 = time.perf_counter()
            G, S = c.force(phi, tol=1e-11)
            dt = time.perf_counter() - t0
            c.close()
            grads[name] = G
            row[name] = {"seconds": dt, "action": S, "gradient_norm": float(np.linalg.norm(G))}
        g0 = grads["fp64_adjoint"]
        for name in ("fp32_adjoint", "fp32_adjoint_pole_groups_of_4"):
            row[name]["rel_diff_vs_fp64_adjoint"] = float(np.linalg.norm(grads[name] - g0) / np.linalg.norm(g0))
        # central finite differences of the action (FP64 path) along random directions
        rng = np.random.Generator(np.random.PCG64(33))
        h = 1e-4
        G = grads["fp32_adjoint"]
        fd_rows = []
        for _ in range(ndir):
            X = np.einsum("...a,aij->...ij", rng.standard_normal(U.shape[:5] + (8,)), lam) * 0.5
            w, v = np.linalg.eigh(X)
            ex = lambda t: np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * t * w), np.conj(v))
            S2 = []
            for t in (h, -h):
                c = make(dims, ex(t) @ U, mixed=1)
                S2.append(c.force(phi, tol=1e-11)[1])
                c.close()
            fd = (S2[0] - S2[1]) / (2 * h)
            an = float(2 * np.real(np.sum(np.conj(G) * (1j * X @ U))))
            fd_rows.append({"finite_difference": fd, "gradient": an, "rel_diff": abs(fd - an) / abs(an)})
        row["finite_differences"] = fd_rows
        out[key] = row
        del grads, U
    return out


def kernel_deflation(B, stream):
    """Kernel low-mode deflation of the sign function (Sec. 1) on rough synthetic links
    (eps 0.7, where the smallest |lambda(K)| are small and spread, so b/a is large) at
    8^4: the overlap apply of 16 Gaussian vectors at eta = 1e-10 (double-float,
    stored-basis Lanczos), undeflated with the fewest poles that reach Delta <= 1e-10 on the
    library's [a, b], and with 8, 16 and 32 eigenvectors of K deflated (the rational
    rebuilt on the narrowed interval with the fewest poles); the cost of finding the
    eigenvectors, the Lanczos steps per apply, and the difference between the results."""
    import torch
    import synth
    dims = (8, 8, 8, 8)
    U = synth.gauge_links(dims, 0.7, 1006)
    vecs = synth.gaussian_source(dims, 2006, nvec=NVEC)
    out = {"workload": "8^4, eps 0.7 links seed 1006, m0 1.4, mu 0.05, 16 Gaussian vectors, eta 1e-10"}
    p = B.ovl_params_default()
    p.stream = stream.cuda_stream
    probe = B.Overlap(dims, U, M0, MU, 64, 1.0, params=p)     # spectral bounds only
    _, _, _, a, b = probe.zolotarev()
    probe.close()
    npoles = next(n for n in range(4, 65) if B.ovl_zolotarev_coeffs(n, a, b)[2] <= EPS)
    p.a_override, p.b_override = a, b
    ctx = B.Overlap(dims, U, M0, MU, npoles, EPS, params=p)
    dv = torch.from_numpy(vecs).cuda()
    ref = torch.empty_like(dv)
    out_t = torch.empty_like(dv)

    def timed(dst):
        ctx.apply(dv, dst, eta=EPS, prec=B.OVL_PREC_F64E)        # warm-up (caps, graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            ctx.apply(dv, dst, eta=EPS, prec=B.OVL_PREC_F64E)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 2
        ctx.profile_reset()
        ctx.profile_enable(True)
        ctx.apply(dv, dst, eta=EPS, prec=B.OVL_PREC_F64E)
        ctx.profile_enable(False)
        launches = ctx.profile_get()["wilson_f64e"]["launches"]
        return {"applies_per_s": NVEC / dt, "ms_per_apply_of_16": dt * 1e3, "wilson_launches_per_apply": launches}

    out["undeflated"] = dict(timed(ref), a=a, b=b, n_poles=npoles)
    r = ref.cpu().numpy()
    for n_ev in (8, 16, 32):
        t0 = time.perf_counter()
        lam, res, a2, np2, its = ctx.kernel_deflate(n_ev, tol=1e-10, max_iter=400)
        tk = time.perf_counter() - t0
        row = dict(timed(out_t), find_eigenvectors_s=tk, filter_steps=its, a=a2, n_poles=np2,
                   lambda_abs_range=[float(np.min(np.abs(lam))), float(np.max(np.abs(lam)))],
                   max_residual=float(np.max(res)))
        g = out_t.cpu().numpy()
        row["max_rel_diff_vs_undeflated"] = float(max(np.linalg.norm(g[j] - r[j]) / np.linalg.norm(r[j])
                                                      for j in range(NVEC)))
        out["deflated_%d" % n_ev] = row
    ctx.kernel_deflate(0)
    ctx.close()
    return out


def run_reference(args, ws, rank):
    """The oracle on this host's cores as the reference arm: every step is a complete
    oracle apply of as many 8^4 vectors as there are cores (a pool of that many
    workers), reported as applies/s extrapolated to the benchmark's 16^3 x 32 lattice
    by the measured cost ratio of one oracle K application."""
    if rank != 0:
        return None
    import synth
    cores = _cores()
    nv = args.oracle_vectors if args.oracle_vectors > 0 else cores
    op = OraclePool(cores)
    vs = synth.gaussian_source(ORACLE_DIMS, SRC_SEED, nvec=nv)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        its, _ = op.apply(vs)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    op.close()
    ratio = _k_cost_ratio()
    t = sum(times) / len(times)
    value = nv / t / ratio
    cpu = {"value": value, "unit": "applies/s", "cores": cores, "kind": "oracle",
           "sample": "per step a complete oracle apply of %d Gaussian vectors on 8^4 (every pole by its own CG, "
                     "%d workers; %.2f s per step), extrapolated to 16^3x32 by the measured K-cost ratio %.1f"
                     % (nv, cores, t, ratio)}
    return {"metric": "overlap D applies/s & RHS solves/s at 1e-10; Dslash HBM GB/s vs plain FP64",
            "impl": "reference", "value": value, "unit": "applies/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "overlap D(mu) apply, 16^3x32, m0=1.4, mu=0.05, 20 Zolotarev poles, eta=1e-10",
                       "implementation": "oracle (NumPy/SciPy, per-pole plain CG, sparse K) on the host cores: "
                                         "complete applies on 8^4 per step, extrapolated to 16^3x32",
                       "measured_lattice": "8x8x8x8"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--oracle-vectors", type=int, default=0,
                    help="reference arm: 8^4 vectors per step (default: one per core)")
    ap.add_argument("--config-c4", action="store_true",
                    help="run only the 24^3x48 batched multi-mass deflated solves and print their JSON")
    ap.add_argument("--config-c5", action="store_true",
                    help="run only the fermion-force measurements (8^4 and 16^3x32) and print their JSON")
    ap.add_argument("--kernel-deflation", action="store_true",
                    help="run only the kernel low-mode deflation measurements (rough links) and print their JSON")
    ap.add_argument("--deflation-gain", action="store_true",
                    help="run only the deflation-gain experiment (15/30/45 vectors) and print its JSON")
    args = ap.parse_args()
    if args.config_c4 or args.config_c5 or args.deflation_gain or args.kernel_deflation:
        import torch
        from paper_1501_01855_gb300 import build, binding as B
        build.build()
        fn = (config_c4 if args.config_c4 else config_c5 if args.config_c5 else
              kernel_deflation if args.kernel_deflation else deflation_gain)
        print(json.dumps(fn(B, torch.cuda.current_stream())), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
    else:
        line = run_ours(args, ws, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
