"""Benchmark: fast directional matrix-vector products per second on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision tc|fp64]

A step is one full product y = A x (S2M, M2M, M2L, L2L, L2T, nearfield) of
the named workload (default: 2^22 uniform targets and sources in [0, 1]^3,
kappa = 128, tree depth 7, Chebyshev order 6) with 1 right-hand side, on
inputs already resident in HBM.  The plan (trees, partition, operators) is
built once before the timed region.  Prints one JSON line.

--impl reference times the CPU oracle instead: the exact FP64 direct sum of
Eq. (1) (plain C, OpenMP over the host cores) on a bounded sample of target
rows per step, scaled to the whole product.

With --gpus N > 1 every rank (one process per GPU: started by torchrun, or by
bench.py itself through torch.distributed.run when no launcher set WORLD_SIZE)
runs an independent replica of the workload (the product is not sharded); the
value is the total over all ranks.

--batch P times the batched form instead: P independent problems (N
log-uniform in [1e4, 1e6], kappa log-uniform in [8, 256], uniform / Gaussian /
shell points, Chebyshev order 5, tree depth ceil(log8(N / 64))), each with 16
complex64 right-hand sides, applied together from one CUDA graph; the value is
right-hand-side products per second.
"""
import argparse
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

from paper_2004_14229_gb300.workloads import WORKLOADS, sample_rows, workload  # noqa: E402

METRIC = "matvecs/s at N=4M, kappa=128, rel.err<=1e-6: tensor-core form vs plain FP64"
UNIT = "matvecs/s"
DEFAULT_WORKLOAD = "uniform-4M-k128-d7-o6"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for name, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _config(args, w, world):
    return {"workload": args.workload, "n_targets": w["n"], "n_sources": w["n"], "kappa": w["kappa"],
            "max_depth": w["depth"], "n_max": w.get("n_max", 0), "order": w["order"],
            "root_side": w["root"][1], "precision": args.precision, "nrhs": 1,
            "parallelism": "replicas" if world > 1 else "1gpu",
            "l2": "inputs larger than L2 (coupling operators streamed every step)"}


def max_over_ranks(seconds, world, device="cuda"):
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if world <= 1:
        return float(seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed / the slowest time."""
    return world * units_per_rank / seconds


def _m2l_source_sha1():
    """sha1 of the M2L kernel's source: csrc/tc.cu from its "M2L (TC)"
    section marker to the "L2T" one (arguments, shared-memory plan, operator
    image writer, k_m2l_pair), plus the PTX helper header it uses."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2004_14229_gb300", "csrc")
    text = open(os.path.join(csrc, "tc.cu")).read()
    a = text.index("// ------------------------------------------------------------- M2L (TC)")
    b = text.index("// ----------------------------------------------------------------- L2T")
    h = hashlib.sha1(text[a:b].encode())
    h.update(open(os.path.join(csrc, "sm100_ptx.cuh"), "rb").read())
    return h.hexdigest()


def _traffic(workload_name):
    """HBM bytes (read + write) of all M2L launches of one product, from the
    ncu summary under profiles/ for this workload -- None when there is none
    or when the M2L kernel's source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "m2l_pair_%s_dram.md" % workload_name)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("k_m2l_pair source sha1") != _m2l_source_sha1() or "dram bytes per product" not in fields:
        return None
    return float(fields["dram bytes per product"])


def _fp64_comparator(workload_name):
    """The plain FP64 form's products/s on this workload, from its measured
    summary under profiles/ (one product takes minutes, so it is measured
    once, not every run) -- None when there is none."""
    path = os.path.join(ROOT, "profiles", "fp64_comparator_%s.md" % workload_name)
    if not os.path.exists(path):
        return None
    out = {"source": os.path.relpath(path, ROOT)}
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) != 2:
            continue
        if cells[0] == "time per product":
            out["s_per_product"] = float(cells[1].split()[0])
            out["value"] = 1.0 / out["s_per_product"]
            out["unit"] = UNIT
        elif cells[0] == "clocks":
            out["clocks"] = cells[1]
        elif cells[0].startswith("rel-l2 against"):
            out["rel_err_vs_oracle_rows"] = float(cells[1].split()[0])
    return out if "value" in out else None


def _blas_threads():
    """Threads numpy's BLAS may use (the O_fdm oracle's only parallelism)."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except ImportError:
        pass
    return len(os.sched_getaffinity(0))


def _oracle_fdm_rate(targets, sources, kappa, order, depth, x, nrows):
    """O_fdm (Alg. 4, FP64 numpy oracle) on the host: plan setup, then the
    whole upward pass and the downward pass restricted to nrows sampled rows.
    A full product costs at least this, so 1 / time bounds its rate from above."""
    from oracle.fdm import FDMOracle
    rows = sample_rows(targets.shape[0], nrows, seed=5)
    t0 = time.perf_counter()
    o = FDMOracle(targets, sources, kappa, order, [0, 0, 0], 1.0, depth)
    t1 = time.perf_counter()
    o.apply(x, rows=rows)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def _oracle_rows_per_sec(targets, sources, kappa, x, nrows):
    from oracle.direct import direct_rows, direct_threads
    rows = sample_rows(targets.shape[0], nrows, seed=5)
    t0 = time.perf_counter()
    direct_rows(targets, sources, kappa, x, rows)
    dt = time.perf_counter() - t0
    return nrows / dt, dt, direct_threads()


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    t, s, x, w = workload(args.workload)
    nrows = args.ref_rows
    for _ in range(args.warmup):
        _oracle_rows_per_sec(t, s, w["kappa"], x, max(8, nrows // 8))
    times = []
    cores = 1
    for _ in range(args.steps):
        _, dt, cores = _oracle_rows_per_sec(t, s, w["kappa"], x, nrows)
        times.append(dt)
    per_step = sum(times) / len(times)
    value = (nrows / w["n"]) / per_step
    sample = ("O_direct (FP64 C double loop, OpenMP) on %d of %d target rows x all %d sources per step, "
              "scaled to the full product" % (nrows, w["n"], w["n"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args, w, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_2004_14229_gb300 as pkg

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    t, s, x, w = workload(args.workload)
    prec = pkg.TC_FP16X3 if args.precision == "tc" else pkg.FP64
    cdt = np.complex64 if prec == pkg.TC_FP16X3 else np.complex128
    tdt = torch.complex64 if prec == pkg.TC_FP16X3 else torch.complex128
    t_setup = time.perf_counter()
    plan = pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"], n_max=w.get("n_max", 0),
                    root=w["root"], precision=prec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    st = plan.stats()
    xd = torch.from_numpy(x.astype(cdt)).cuda()
    yd = torch.empty(w["n"], dtype=tdt, device="cuda")
    stream = torch.cuda.current_stream()
    tuning = None
    if args.autotune and prec == pkg.TC_FP16X3:
        # measured launch shapes, chosen before the timed region (set-up)
        t_tune = time.perf_counter()
        tuning = plan.autotune(xd, cache=args.tune_cache)
        tuning["seconds"] = time.perf_counter() - t_tune

    for _ in range(args.warmup):
        plan.apply(xd, yd)
    torch.cuda.synchronize()
    plan.check()

    # ---------------------------------------------------------- timed region
    plan.set_timing(True)
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0.record(stream)
    # no host synchronisation inside: the library's per-phase events of all
    # steps accumulate and are read once afterwards
    for i in range(args.steps):
        step_ev[i].record(stream)
        plan.apply(xd, yd)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    tm = plan.timing()
    plan.set_timing(False)
    plan.check()
    assert tm["applies"] == args.steps
    m2l_ms = list(tm["m2l_ms"])
    phases = {k: tm[k] for k in ("s2m_ms", "m2m_ms", "split_ms", "l2l_ms", "l2t_ms", "near_ms", "total_ms")}
    launches = tm["launches"]
    ends = step_ev[1:] + [ev1]
    step_ms = sorted(a.elapsed_time(b) for a, b in zip(step_ev, ends))
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    value = job_rate(args.steps, world, elapsed)

    # accuracy against the FP64 oracle on stored rows (written by the oracle)
    err = None
    gold = os.path.join(ROOT, "tests", "golden", "%s_rows.npz" % args.workload)
    if os.path.exists(gold):
        g = np.load(gold)
        yv = yd.cpu().numpy()[g["rows"]]
        err = float(np.linalg.norm(yv - g["y_fdm"]) / np.linalg.norm(g["y_fdm"]))

    # workloads without stored oracle rows: the approximation error against
    # exact rows of Eq. (1) (the library's FP64 direct-sum kernel, 64 rows)
    err_direct = None
    if err is None:
        rows = sample_rows(w["n"], 64, seed=4)
        td = torch.from_numpy(t).cuda()
        sd = td if s is t else torch.from_numpy(s).cuda()
        want = pkg.direct_rows(td, sd, w["kappa"], torch.from_numpy(x).cuda(), torch.from_numpy(rows).cuda())
        got = yd.cpu().numpy()[rows].astype(np.complex128)
        want = want.cpu().numpy()
        err_direct = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        del td, sd

    # ------------------------------------------------------------ end to end
    e2e = None
    if args.e2e_steps > 0:
        xh = torch.from_numpy(x.astype(cdt)).pin_memory()
        yh = torch.empty(w["n"], dtype=tdt).pin_memory()
        plan.apply_host(xh.numpy(), yh.numpy())
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.apply_host(xh.numpy(), yh.numpy())
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": xh.numel() * xh.element_size(),
               "d2h_bytes_per_step": yh.numel() * yh.element_size()}

    # -------------------------------------------------------------- roofline
    # dominant kernel: M2L (tensor cores) or, with large leaves, the nearfield
    n = w["order"] ** 3
    peaks, src = _peaks()
    m2l_s = sum(m2l_ms) / 1e3 / args.steps
    near_s = phases["near_ms"] / 1e3 / args.steps
    if m2l_s >= near_s:
        flops_step = 8.0 * n * n * st["n_coupling"]          # complex n x n MAC = 8 real flops
        peak = peaks.get("bf16_tflops_sustained", 1700.0) if prec == pkg.TC_FP16X3 else 1.25
        achieved = flops_step / m2l_s / 1e12
        roofline = {"bound": "tensor" if prec == pkg.TC_FP16X3 else "alu", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": _traffic(args.workload) if prec == pkg.TC_FP16X3 else None,
                    "traffic_unit": "HBM bytes of all M2L launches of one product (ncu)",
                    "kernel": "k_m2l_pair" if prec == pkg.TC_FP16X3 else "k_m2l_fp64",
                    "peak_source": ("%s sustained bf16 (fp16 has the same nominal rate)" % src)
                    if prec == pkg.TC_FP16X3 else "nominal GB300 FP64",
                    "algorithmic_flops_per_step": flops_step, "m2l_ms_per_step": m2l_s * 1e3}
        if prec == pkg.TC_FP16X3:
            # tensor work the split form executes per algorithmic flop: three
            # FP16 products per K step (every MMA row a target), operands
            # padded from 2n to KP
            kp = {2: 64, 3: 64, 4: 128, 5: 256, 6: 448}[w["order"]]
            ratio = 3.0 * (kp / (2.0 * n)) ** 2
            roofline["executed_per_algorithmic"] = ratio
            roofline["executed_tflops"] = achieved * ratio
            roofline["executed_frac"] = achieved * ratio / peak
    else:
        # 20 FP32 flops per pair (differences, |r|, kappa r, scale, complex
        # multiply-add) + rsqrt, sin, cos; peak: 152 SMs x 128 FP32 lanes x 2
        # flops at the sampled SM clock
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        pairs = float(st["nf_entries"])
        achieved = 20.0 * pairs / near_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "k_p2p_f32" if prec == pkg.TC_FP16X3 else "k_p2p_fp64",
                    "peak_source": "FP32 FMA pipe, 152 SMs x 128 lanes x 2 flops x sampled SM clock",
                    "pairs_per_step": pairs, "near_ms_per_step": near_s * 1e3}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "ms_per_step_median": step_ms[len(step_ms) // 2], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x3+f32" if prec == pkg.TC_FP16X3 else "f64", "data": "synthetic",
            "config": _config(args, w, world),
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": launches,
            "phase_ms_per_step": {k: v / args.steps for k, v in phases.items()},
            "m2l_ms_per_level": [v / args.steps for v in m2l_ms[:w["depth"] + 1]],
            "setup_s": setup_s, "n_coupling": st["n_coupling"], "n_stored_coupling": st["n_stored_coupling"],
            "n_coupling_per_level": st["level_coupling"][:w["depth"] + 1],
            "rel_err_vs_oracle_rows": err, "rel_err_vs_direct_rows": err_direct, "clocks": clocks,
            "autotune": tuning}
    if prec == pkg.TC_FP16X3:
        cmp64 = _fp64_comparator(args.workload)
        if cmp64 is not None:
            cmp64["tc_over_fp64"] = value / world / cmp64["value"]
        line["fp64_comparator"] = cmp64
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rps, dt, cores = _oracle_rows_per_sec(t, s, w["kappa"], x, args.ref_rows)
        line["cpu_baseline"] = {"value": rps / w["n"], "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "O_direct (FP64 C double loop, OpenMP) on %d target rows x all %d "
                                          "sources (%.1f s), scaled to the full product"
                                          % (args.ref_rows, w["n"], dt)}
    if rank == 0 and world == 1 and args.fdm_baseline > 0:
        setup, apply_s = _oracle_fdm_rate(t, s, w["kappa"], w["order"], w["depth"], x, args.fdm_baseline)
        line["cpu_baseline_fdm"] = {"value": 1.0 / apply_s, "unit": UNIT, "bound": "upper",
                                    "cores": _blas_threads(),
                                    "kind": "oracle", "setup_s": setup,
                                    "sample": "O_fdm (Alg. 4, FP64 numpy) on the host: full upward pass, "
                                              "downward pass to %d sampled rows (%.1f s; plan %.1f s); a "
                                              "full product takes at least this long" % (args.fdm_baseline,
                                                                                        apply_s, setup)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    import torch

    import paper_2004_14229_gb300 as pkg
    from paper_2004_14229_gb300.workloads import batch_problems

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    nrhs, order = 16, 5
    probs = batch_problems(args.batch, nrhs=nrhs)
    t_setup = time.perf_counter()
    batch = pkg.Batch(probs, order=order, root="bounding", precision=pkg.TC_FP16X3, nrhs_max=nrhs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    stats = [pl.stats() for pl in batch.plans]
    xs = [torch.from_numpy(p["x"].astype(np.complex64)).cuda() for p in probs]
    ys = [torch.empty((nrhs, p["targets"].shape[0]), dtype=torch.complex64, device="cuda") for p in probs]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.apply(xs, ys)
    torch.cuda.synchronize()
    batch.check()
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batch.apply(xs, ys)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    batch.check()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    units = len(probs) * nrhs
    value = job_rate(units * args.steps, world, elapsed)
    _, _, launches = batch.info()

    # error of three problems against exact direct-sum rows (approximation error)
    from paper_2004_14229_gb300 import direct_rows
    errs = []
    for i in range(min(3, len(probs))):
        p = probs[i]
        rows = sample_rows(p["targets"].shape[0], 64, seed=11 + i)
        want = direct_rows(torch.from_numpy(p["targets"]).cuda(), torch.from_numpy(p["sources"]).cuda(),
                           p["kappa"], torch.from_numpy(p["x"][0]).cuda(), torch.from_numpy(rows).cuda())
        got = ys[i][0].cpu().numpy()[rows]
        w = want.cpu().numpy()
        errs.append(float(np.linalg.norm(got - w) / np.linalg.norm(w)))

    # end to end: pinned host x in, y out, every step
    xh = [torch.from_numpy(p["x"].astype(np.complex64)).pin_memory() for p in probs]
    yh = [torch.empty(y.shape, dtype=y.dtype).pin_memory() for y in ys]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for a, b in zip(xs, xh):
            a.copy_(b, non_blocking=True)
        batch.apply(xs, ys)
        for a, b in zip(yh, ys):
            a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = sum(v.numel() * v.element_size() for v in xh)
    d2h = sum(v.numel() * v.element_size() for v in yh)

    n = order ** 3
    flops = sum(8.0 * n * n * st["n_coupling"] for st in stats) * nrhs
    peaks, src = _peaks()
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = flops / (elapsed / args.steps) / 1e12
    line = {"metric": "RHS-matvecs/s, %d independent problems x %d complex64 RHS (batched form)"
                      % (len(probs), nrhs),
            "value": value, "unit": "RHS-matvecs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x3+f32", "data": "synthetic",
            "config": {"workload": "batch-%d-o5-nrhs16" % len(probs), "problems": len(probs), "nrhs": nrhs,
                       "order": order, "n_points_total": int(sum(p["targets"].shape[0] for p in probs)),
                       "root": "bounding dyadic cube", "precision": "tc",
                       "parallelism": "replicas" if world > 1 else "1gpu",
                       "l2": "inputs larger than L2 (operators of all problems streamed every step)"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_m2l_pair",
                         "peak_source": "%s sustained bf16; achieved = M2L algorithmic flops / whole step"
                                        % src},
            "e2e": {"value": world * units / e2e_s, "unit": "RHS-matvecs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches * args.steps,
            "setup_s": setup_s, "device_bytes": int(sum(st["device_bytes"] for st in stats)),
            "rel_err_vs_direct_rows": errs, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


SEL_KAPPAS = (32.0, 128.0, 256.0)
SEL_TOLS = (1e-3, 1e-5, 1e-7)
SEL_N, SEL_DEPTH = 1 << 21, 6
FP64_M2L_TFLOPS = 0.62        # measured rate of k_m2l_fp64 (4M workload, one product)


def selector_record_json(rec):
    """A measured selector record (selector_data.measure) as plain JSON."""
    out = {k: v for k, v in rec.items() if k != "err"}
    out["orders"] = list(rec.get("orders", ()))
    out["err"] = [[int(o), int(sh), float(e)] for (o, sh), e in sorted(rec["err"].items())]
    return out


def run_selector_study(args):
    """The learned selector against the fixed rule at 2^21 points.

    Training (args.sel_recipe "mixed"): depth-3 problems (selector_problems,
    kappa 2..96, orders 2..7) alternating with depth-4 problems of 8k-32k
    points (kappa 8..300, tensor-core orders 2..6), problems without
    admissible blocks skipped ("depth3": the depth-3 problems only, none
    skipped); each measured at two l_hf (selector_data.measure), in order
    until args.sel_budget seconds are spent; samples at 57 tolerances
    1e-1..1e-8 per level; full-batch Adam for 2000 epochs on the GPU.  Fixed rule: per tolerance the smallest order whose error stays
    below tol / 3 on every training problem, with the default l_hf.  Test:
    2^21 uniform targets and sources (seeds 1, 2), depth 6, x seed 3, kappa in
    {32, 128, 256}, tol in {1e-3, 1e-5, 1e-7}; each choice is applied once
    after a warm-up (tensor-core form for tol >= 1e-6 and order <= 6, FP64
    otherwise; FP64 cells after all tensor-core cells, skipped when their M2L
    is estimated above args.sel_fp64_cap seconds) and scored on 2048 exact
    rows of Eq. (1).  One JSON line per cell, then a summary line."""
    import torch

    import paper_2004_14229_gb300 as pkg
    from paper_2004_14229_gb300 import selector_data as D
    from paper_2004_14229_gb300.workloads import (complex_normal, selector_init, selector_problems,
                                                  uniform_points)

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    if args.sel_recipe == "depth3":
        queue = [(p, {}) for p in selector_problems(args.sel_train, seed0=200, kappa_range=(2.0, 96.0))]
    else:
        # depth-3 problems (orders 2..7) alternating with depth-4 problems of
        # 8k-32k points up to kappa 300 (tensor-core orders 2..6), both only
        # when they have admissible blocks
        d3 = selector_problems(args.sel_train // 2, seed0=200, kappa_range=(2.0, 96.0))
        d4 = selector_problems(args.sel_train - args.sel_train // 2, seed0=400, kappa_range=(8.0, 300.0),
                               n_range=(1000, 4000), depths=(4,))
        # van der Corput order, so that any prefix the time budget allows
        # spans the whole kappa range
        def spread(v):
            def vdc(i):
                x, f = 0.0, 0.5
                while i:
                    x += f * (i & 1)
                    i >>= 1
                    f /= 2
                return x
            return [v[i] for i in sorted(range(len(v)), key=vdc)]
        d3, d4 = spread(d3), spread(d4)
        queue = []
        for i in range(max(len(d3), len(d4))):
            if i < len(d3):
                queue.append((d3[i], dict(require_far=True)))
            if i < len(d4):
                queue.append((d4[i], dict(orders=(2, 3, 4, 5, 6), tc_max=6, require_far=True)))
    train = []
    for p, opt in queue:
        if time.perf_counter() - t0 > args.sel_budget:
            break
        train += D.measure([p], **opt)
        print("measured %d problems, %.0f s" % (len(train), time.perf_counter() - t0), file=sys.stderr, flush=True)
    t_measure = time.perf_counter() - t0
    if args.sel_save:
        # the measured errors, for offline work on the network and its labels
        with open(args.sel_save, "w") as f:
            json.dump([selector_record_json(r) for r in train], f)
    tols = np.logspace(-1, -8, 57)
    X, T = D.make_samples(train, tols)
    sel, losses = pkg.Selector.train(selector_init(), X, T, epochs=2000, lr=3e-3)
    fixed = {}
    for tol in SEL_TOLS:
        fixed[tol] = max(D.labels(r, tol)[0] for r in train)
    print(json.dumps({"selector_training": {"recipe": args.sel_recipe, "problems": len(train),
                                            "depths": sorted(set(r["depth"] for r in train)),
                                            "samples": int(X.shape[0]),
                                            "measure_s": t_measure, "loss_first": float(losses[0]),
                                            "loss_last": float(losses[-1]),
                                            "fixed_rule_order": {str(k): v for k, v in fixed.items()}}}),
          flush=True)

    t = uniform_points(SEL_N, 1)
    s = uniform_points(SEL_N, 2)
    x = complex_normal(SEL_N, 3)
    xd64 = torch.from_numpy(x).cuda()
    xd32 = xd64.to(torch.complex64)
    rows = sample_rows(SEL_N, 2048, seed=4)
    td, sd = torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda()
    summary = []
    refs, lhf0 = {}, {}
    for kappa in SEL_KAPPAS:
        refs[kappa] = pkg.direct_rows(td, sd, kappa, xd64, torch.from_numpy(rows).cuda()).cpu().numpy()
        with pkg.Plan(t, s, kappa, order=2, max_depth=SEL_DEPTH, precision=pkg.FP64) as probe:
            lhf0[kappa] = probe.stats()["l_hf"]
    cells = [(k, tol) for tol in SEL_TOLS for k in SEL_KAPPAS]
    # tensor-core cells first, FP64 cells while the time budget lasts
    for kappa, tol in cells:
        ref = refs[kappa]
        o_sel, lhf_sel = sel.select(kappa, tol, SEL_N, SEL_DEPTH)
        cell = {"kappa": kappa, "tol": tol}
        for who, order, lhf in (("selector", o_sel, lhf_sel), ("fixed", fixed[tol], lhf0[kappa])):
            order = min(max(order, 2), 10)
            tc = tol >= 1e-6 and order <= 6
            prec = pkg.TC_FP16X3 if tc else pkg.FP64
            r = {"order": order, "l_hf": lhf, "form": "tc" if tc else "fp64", "nodes_per_box": order ** 3}
            # the planner's counts for the fully occupied tree (host only)
            n_c, n_sc, _ = pkg.uniform_counts(kappa, SEL_DEPTH, l_hf=lhf)
            est = 8.0 * order ** 6 * n_c / (FP64_M2L_TFLOPS * 1e12)
            op_gb = 16.0 * order ** 6 * n_sc / 1e9
            r["n_coupling"] = n_c
            if not tc and (est > args.sel_fp64_cap or op_gb > 60.0):
                r["skipped"] = ("FP64 M2L estimated at %.0f s (cap %.0f s), FP64 operators %.0f GB"
                                % (est, args.sel_fp64_cap, op_gb))
            elif not tc and time.perf_counter() - t0 > args.sel_total:
                r["skipped"] = "study time budget (%.0f s) spent" % args.sel_total
            else:
                with pkg.Plan(t, s, kappa, order=order, max_depth=SEL_DEPTH, l_hf=lhf, precision=prec) as pl:
                    xin = xd32 if tc else xd64
                    # tensor-core products after one warm-up; an FP64 product
                    # (tens of seconds) is timed cold, once
                    y = pl.apply(xin) if tc else torch.empty(SEL_N, dtype=torch.complex128, device="cuda")
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    pl.apply(xin, y)
                    e1.record()
                    torch.cuda.synchronize()
                    pl.check()
                    r["n_coupling"] = pl.stats()["n_coupling"]
                yr = y.cpu().numpy()[rows].astype(np.complex128)
                r["err"] = float(np.linalg.norm(yr - ref) / np.linalg.norm(ref))
                r["meets_tol"] = r["err"] <= tol
                r["ms"] = e0.elapsed_time(e1)
            cell[who] = r
        print(json.dumps({"selector_study_cell": cell}), flush=True)
        summary.append(cell)
    print(json.dumps({"selector_study": {"n": SEL_N, "depth": SEL_DEPTH, "direct_rows": int(rows.size),
                                         "cells": len(summary), "total_s": time.perf_counter() - t0}}),
          flush=True)
    return 0


def _free_port():
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def launch_replicas(nproc, argv):
    """`--gpus N` without a launcher: run this script as N ranks (one per GPU,
    torch.distributed.run on 127.0.0.1) and return the launcher's exit code;
    rank 0 prints the JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(nproc),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.abspath(__file__), *argv]
    return subprocess.run(cmd).returncode


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="tc", choices=["tc", "fp64"])
    ap.add_argument("--ref-rows", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fdm-baseline", type=int, default=0,
                    help="also time the O_fdm oracle on the host, downward pass to this many rows")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="products timed end to end through dfdm_apply_host (0: none)")
    ap.add_argument("--batch", type=int, default=0, help="time the batched form on this many problems")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="time candidate launch shapes before the timed region and keep the fastest")
    ap.add_argument("--tune-cache", default=None, help="JSON-lines cache of the launch-shape tuner")
    ap.add_argument("--selector-study", action="store_true",
                    help="train the parameter selector and compare it with the fixed rule at 2^21 points")
    ap.add_argument("--sel-train", type=int, default=64, help="training problems of the selector study")
    ap.add_argument("--sel-recipe", default="mixed", choices=["mixed", "depth3"],
                    help="training problems: depth 3 and 4 with admissible blocks, or depth 3 only")
    ap.add_argument("--sel-budget", type=float, default=300.0,
                    help="seconds the selector study may spend measuring training problems")
    ap.add_argument("--sel-total", type=float, default=540.0,
                    help="no FP64 cell of the selector study starts after this many seconds")
    ap.add_argument("--sel-save", default=None, help="write the measured training records to this JSON file")
    ap.add_argument("--sel-fp64-cap", type=float, default=110.0,
                    help="skip FP64 products of the selector study whose M2L is estimated above this (s)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return launch_replicas(args.gpus, sys.argv[1:])
    world, _, _ = _dist()
    if args.gpus != world:
        raise SystemExit("--gpus %d but %d ranks were launched" % (args.gpus, world))
    if args.impl == "reference":
        return run_reference(args)
    if args.selector_study:
        return run_selector_study(args)
    if args.batch > 0:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
