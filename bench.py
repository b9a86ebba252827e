"""Benchmark: sparsity-aware batched assembly of FETI dual Schur complements.

Workload (default): 3D heat transfer, unit cube split 4x4x4 into 64 subdomains
of 16^3 hex8 elements (4913 dofs each), every subdomain floating with one
fixed node, non-redundant gluing (817..1634 multipliers per subdomain), FP64.

One step = one pass of the whole hot path over the batch: sc_assemble_batch
(reciprocal diagonal + F padding, sparse TRSM, pruned SYRK with the back
permutation fused) followed by one sc_apply (q = sum_i F_i lambda_i).

value     -- SC assemblies/s = subdomains / device time of a step, inputs
             resident in HBM; L2 is flushed (256 MB write) before every timed step.
e2e       -- the same through the public API from pinned host buffers: the
             step's L values and lambda are copied host->device, q is read back.
roofline  -- the dominant kernel (pruned SYRK), timed live with CUDA events
             recorded by the library on the launching stream; it is bound by
             the FP64 pipe.
cpu_baseline / --impl reference -- the FP64 oracle on the host cores.
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

import synth  # noqa: E402

METRIC = "SC assemblies/s and effective TFLOP/s vs dense TRSM+SYRK path on 1 GB300"
UNIT = "assemblies/s"
# FP64 peak of the GPU: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def _measured_hbm_gbps() -> float:
    """HBM copy bandwidth measured on this GPU model (MEASURED_PEAKS.json),
    else 6.8 TB/s, an earlier copy-bandwidth measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBPS = _measured_hbm_gbps()


def _measured_bf16_tflops() -> float:
    """Dense BF16 tensor rate measured on this GPU model (cuBLAS burst,
    MEASURED_PEAKS.json), else 1.9 PFLOP/s, an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


BF16_PEAK_TFLOPS = _measured_bf16_tflops()


def _json_default(o):
    """numpy scalars and arrays in the JSON line (a type the encoder does not know must not end the run)."""
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    if isinstance(o, np.ndarray):
        return o.tolist()
    return str(o)


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _max_over_ranks(ms: float, dev=None) -> float:
    """The slowest rank's time (every rank gets it): value = all ranks' units / this."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload_config(args):
    return {"workload": "heat3d_cube_4x4x4_subdomains_16^3_hex8", "subdomains": 64, "dofs_per_subdomain": 4913,
            "multipliers_total": 39807, "precision": "fp64", "seed": args.seed,
            "l2": "flushed before every timed step (256 MB write); inputs 0.33 GB L + 0.44 GB F also exceed L2"}


class ClockSampler:
    """nvidia-smi sampling (200 ms) while the timed region runs."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples (the JSON line carries their summary); SC_BENCH_CLOCKS_DIR keeps them
        d = os.environ.get("SC_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"sc_bench_clocks_rank{index}.csv")
        self.window = None

    def mark(self, t0: float, t1: float):
        """Keep only samples taken between host times t0 and t1 (seconds)."""
        self.window = (t0, t1)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.window and not (self.window[0] - 0.25 <= ts <= self.window[1] + 0.25):
                    continue
                sm.append(float(p[2]))
                smax = float(p[3])
            except ValueError:
                continue
            for nm, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# the source file of each profiled kernel
_KERNEL_SOURCE = {"apply_digits_kernel": "sc_apply_digits.cu", "apply_fixed_kernel": "sc_apply_fixed.cu",
                  "implicit_kernel": "sc_implicit.cu"}


def _kernel_source_hash(kernel: str = "syrk_kernel"):
    src = os.path.join(ROOT, "paper_2509_21037_gb300", "csrc", _KERNEL_SOURCE.get(kernel, "sc_kernels.cu"))
    return hashlib.sha256(open(src, "rb").read()).hexdigest()


def _traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, only while the
    kernel source is the one that was profiled."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(kernel)
        if e and e.get("source_sha256") == _kernel_source_hash(kernel):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def _oracle_sample(prob, idx):
    import oracle
    t0 = time.perf_counter()
    oracle.dual_operators([prob.subdomains[i] for i in idx], refine=1)
    return time.perf_counter() - t0


def _oracle_unmemoised(prob):
    """The oracle's cost per subdomain with nothing shared: one subdomain of
    each distinct size (config 2: one size), fresh memo, so its dense
    Cholesky is paid in full; with the batch's count it projects the
    un-memoised oracle time of the whole batch."""
    sizes = {}
    for i, sd in enumerate(prob.subdomains):
        sizes.setdefault(sd.K.shape[0], []).append(i)
    per = {n: _oracle_sample(prob, [idx[0]]) for n, idx in sizes.items()}
    total = sum(per[n] * len(idx) for n, idx in sizes.items())
    return {"s_per_subdomain": {str(n): t for n, t in per.items()}, "projected_batch_s": total,
            "assemblies_per_s": len(prob.subdomains) / total}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    """The oracle (FP64, host cores) timed as the reference arm."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    prob = synth.make_config(2, seed=args.seed)
    S = args.ref_sample
    nsub = len(prob.subdomains)
    times = []
    for k in range(args.warmup + args.steps):
        idx = [(k * S + j) % nsub for j in range(S)]
        t = _oracle_sample(prob, idx)
        if k >= args.warmup:
            times.append(t)
    tot = sum(times)
    val = S * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload_config(args),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                             "sample": f"{S} of 64 subdomains per step, fresh memo (dense Cholesky of K_reg once per "
                                       f"distinct K, then forward/backward substitution on the B^T dofs)",
                             "unmemoised": _oracle_unmemoised(prob)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_json_default))
    return 0


def _gpu_implicit(fs, n_dual, Lv, lam, q_expl, stream, reps=20):
    """The GPU implicit application (include/sc_implicit.h) on the same L and
    lambda: mean ms over `reps` calls, its FP64 roofline, and its relative
    difference from the explicit q."""
    import torch

    from paper_2509_21037_gb300 import implicit
    ip = implicit.ImplicitPlan(fs, n_dual).upload(lam.device)
    q = torch.empty_like(lam)
    ip.apply(Lv, lam, q, stream)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        ip.apply(Lv, lam, q, stream)
    a1.record(stream)
    a1.synchronize()
    if ip.device_status(stream) != 0:
        raise RuntimeError("device status not OK after the implicit apply")
    ms = a0.elapsed_time(a1) / reps
    tf = ip.sizes.flops / (ms / 1e3) / 1e12
    diff = (torch.linalg.vector_norm(q - q_expl) / torch.linalg.vector_norm(q_expl)).item()
    # the same with each subdomain's subtrees on a pair of CTAs (sci_options.pairs), for the comparison
    one = implicit.ImplicitPlan(fs, n_dual, pairs=1).upload(lam.device)
    one.apply(Lv, lam, q, stream)
    a0.record(stream)
    for _ in range(reps):
        one.apply(Lv, lam, q, stream)
    a1.record(stream)
    a1.synchronize()
    ms_one = a0.elapsed_time(a1) / reps
    del one
    return ms, {"ms": ms, "flops": ip.sizes.flops, "nnz_visited": int(ip.sizes.nnz_visited),
                "max_levels": int(ip.sizes.max_levels), "tflops": tf, "frac_fp64_peak_nominal": tf / FP64_PEAK_TFLOPS,
                "rel_diff_vs_explicit": diff, "ms_cta_pairs": ms_one}


def _fp64_fma_peak(dev, stream):
    """The FP64 fused multiply-add rate of this GPU, measured (include/sc_probe.h):
    8 independent chains per thread, 8 blocks of 256 threads per SM; CUDA
    events on the launching stream, 3 warm-up launches, the best of 5."""
    import ctypes

    import torch

    from paper_2509_21037_gb300 import _native
    lib = _native.sc_lib()
    flops, n = ctypes.c_double(), ctypes.c_int64()
    iters, bps = 4096, 8
    if lib.sc_probe_fp64_fma(iters, bps, None, ctypes.byref(flops), ctypes.byref(n), None) != 0:
        raise RuntimeError("sc_probe_fp64_fma size query failed")
    out = torch.empty(n.value, dtype=torch.float64, device=dev)
    sp = _stream_ptr(stream)
    for _ in range(3):
        if lib.sc_probe_fp64_fma(iters, bps, out.data_ptr(), ctypes.byref(flops), ctypes.byref(n), sp) != 0:
            raise RuntimeError("sc_probe_fp64_fma launch failed")
    rates = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lib.sc_probe_fp64_fma(iters, bps, out.data_ptr(), ctypes.byref(flops), ctypes.byref(n), sp)
        b.record(stream)
        b.synchronize()
        rates.append(flops.value / (a.elapsed_time(b) / 1e3) / 1e12)
    if not bool(torch.isfinite(out).all()):
        raise RuntimeError("FP64 probe produced non-finite values")
    return max(rates), {"tflops_best": max(rates), "tflops_median": statistics.median(rates),
                        "flops_per_launch": flops.value, "launches": 8}


def _stream_ptr(stream):
    return None if stream is None else int(stream.cuda_stream)


def _secondary(section):
    """A secondary section of the line (measured after the headline numbers):
    its failure is reported in the line instead of ending the run."""
    try:
        return section()
    except Exception as e:  # report, do not hide
        return {"error": f"{type(e).__name__}: {str(e)[:300]}"}


def _pipeline_section(args, prob, fs, dev, stream):
    """The whole numeric stage (include/sc_pipeline.h): every subdomain's host
    Cholesky (all host cores) overlapped chunk by chunk with the H2D copy of
    L and the GPU assembly; best of three runs against the same work done one
    step after another."""
    from paper_2509_21037_gb300 import pipeline
    pipe = pipeline.Pipeline(prob.subdomains, fs, prob.n_dual, nchunks=args.pipeline_chunks, device=dev)
    pipe.run(stream)
    runs = [pipe.run(stream) for _ in range(3)]
    best = min(runs, key=lambda r: r["wall_ms"])
    out = dict(best)
    out.update({"chunks": args.pipeline_chunks, "host_threads": os.cpu_count(),
                "subdomains_per_s": len(fs) / (best["wall_ms"] / 1e3),
                "speedup_vs_serial": best["serial_ms"] / best["wall_ms"],
                "note": "host numeric factorisation of every subdomain + H2D of L + GPU assembly"})
    return out


def _feti_section(prob, fs, dev, t_asm, t_expl, t_gimpl, t_himpl):
    """FETI-1 PCPG on the bench batch (feti.py): iterations to a 1e-10
    projected residual with the Dirichlet and lumped preconditioners (both
    scaled by (B B^T)^+) and without one, and what a solve of that many
    iterations costs with the explicit operator (assembly + applications)
    against the GPU and host implicit applications.  Each solver solves once
    untimed first: the first solve after set-up also pays the first use of
    the loop's device kernels (seconds once, against ~20-50 ms a solve)."""
    import torch
    from paper_2509_21037_gb300 import feti
    loads = feti.compatible_loads(prob, seed=1)
    out = {}
    for pc in ("dirichlet", "lumped", "none"):
        first_setup = None
        if pc == "dirichlet":
            # the first set-up in a process also pays the first use of the device
            # operations it launches (module loading, allocations): reported
            # beside the steady-state set-up of a second solver
            first = feti.FETISolver(prob, fs, device=dev, precond=pc)
            first_setup = first.precond_setup_s
            del first
            torch.cuda.empty_cache()
        solver = feti.FETISolver(prob, fs, device=dev, precond=pc)
        solver.solve(loads, tol=1e-10, recover=False)
        res = solver.solve(loads, tol=1e-10)
        n = res.iterations
        out[pc] = {"iterations": n, "pcpg_ms": res.solve_ms, "F_apply_ms": res.apply_ms,
                   "ms_per_iteration": res.solve_ms / max(n, 1),
                   "precond_setup_s": solver.precond_setup_s, "precond_setup_first_in_process_s": first_setup,
                   "precond_setup_breakdown": getattr(feti.dirichlet_operator_gpu, "last_breakdown", None)
                   if pc == "dirichlet" else None,
                   "continuity": res.continuity, "equilibrium": res.equilibrium,
                   "explicit_total_ms": t_asm + n * t_expl, "implicit_gpu_total_ms": n * t_gimpl,
                   "implicit_host_total_ms": n * t_himpl}
    return out


def run_sc(args):
    import torch
    import torch.distributed as dist

    from paper_2509_21037_gb300 import host, sc

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    prob = synth.make_config(2, seed=args.seed)
    fs = host.factorize_problem(prob.subdomains)
    if args.profile and args.profile_slices:
        from paper_2509_21037_gb300 import abi
        plan = sc.Plan(fs, prob.n_dual, precision=abi.SC_SPLIT_BF16, n_slices=args.profile_slices,
                       tile=args.profile_tile).upload(dev)
    else:
        plan = sc.Plan(fs, prob.n_dual).upload(dev)
    Lh = sc.concat_L_values(fs)
    Lv = torch.from_numpy(Lh).to(dev)
    F = plan.new_F(dev)
    lam = torch.from_numpy(np.random.default_rng(args.seed).standard_normal(prob.n_dual)).to(dev)
    q = torch.empty_like(lam)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = plan.stats_dict()

    def step():
        plan.assemble(Lv, F, stream)
        plan.apply(F, lam, q, stream)

    clocks = ClockSampler(local).__enter__()
    time.sleep(1.0)                               # nvidia-smi start-up
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if plan.device_status(stream) != 0:
        raise RuntimeError("device status not OK after warm-up")
    plan.enable_stage_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    syrk_ms, trsm_ms, prep_ms = [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_host0 = time.time()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        p, t, s = plan.stage_times()        # waits for this step's syrk
        prep_ms.append(p); trsm_ms.append(t); syrk_ms.append(s)
    torch.cuda.synchronize(dev)
    clocks.mark(t_host0, time.time())
    time.sleep(0.3)
    clocks.__exit__()
    plan.enable_stage_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        ms = _max_over_ranks(ms, dev)
        dist.barrier()
    nsub = len(fs)
    value = world * nsub / (ms / 1e3)

    if args.profile:
        for _ in range(args.warmup + args.steps):
            plan.apply_fixed(F, lam, q, stream)
        for _ in range(args.warmup + args.steps):
            plan.apply_mixed(F, lam, q, args.profile_mixed, stream)
        Fd = plan.prepare_digits(F, stream=stream)
        for _ in range(args.warmup + args.steps):
            plan.apply_digits(Fd, lam, q, stream)
        torch.cuda.synchronize(dev)
        del Fd
        if args.profile_implicit:
            from paper_2509_21037_gb300 import implicit
            ip = implicit.ImplicitPlan(fs, prob.n_dual).upload(dev)
            for _ in range(args.warmup + args.steps):
                ip.apply(Lv, lam, q, stream)
            torch.cuda.synchronize(dev)
            if ip.device_status(stream) != 0:
                raise RuntimeError("device status not OK after the implicit apply")
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms, "stage_ms": {
                "trsm": sum(trsm_ms) / len(trsm_ms), "syrk": sum(syrk_ms) / len(syrk_ms)}}))
        return 0

    # end to end through the public API from pinned host buffers
    Lpin = torch.from_numpy(Lh).pin_memory()
    lam_pin = lam.cpu().pin_memory()
    q_pin = torch.empty_like(lam_pin).pin_memory()
    Ld = torch.empty_like(Lv)
    lamd = torch.empty_like(lam)

    def e2e_step():
        Ld.copy_(Lpin, non_blocking=True)
        lamd.copy_(lam_pin, non_blocking=True)
        plan.assemble(Ld, F, stream)
        plan.apply(F, lamd, q, stream)
        q_pin.copy_(q, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    e2e_serial_ms = sum(e_ms) / len(e_ms)
    # the same steps back to back as a pipeline: step k+1's L goes up on a
    # copy stream into the other device buffer while step k assembles; every
    # step's inputs are still copied and its result read back inside the
    # timed region (inputs exceed L2, so no flush between steps)
    Lbuf = [Ld, torch.empty_like(Lv)]
    cs = torch.cuda.Stream(dev)
    K = max(3, args.steps)
    copied = [torch.cuda.Event() for _ in range(K)]
    used = [torch.cuda.Event() for _ in range(K)]
    torch.cuda.synchronize(dev)
    e0.record(stream)
    cs.wait_event(e0)
    with torch.cuda.stream(cs):
        Lbuf[0].copy_(Lpin, non_blocking=True)
        copied[0].record(cs)
    for k in range(K):
        if k + 1 < K:
            with torch.cuda.stream(cs):
                if k >= 1:
                    cs.wait_event(used[k - 1])          # the buffer step k-1 read is free again
                Lbuf[(k + 1) % 2].copy_(Lpin, non_blocking=True)
                copied[k + 1].record(cs)
        stream.wait_event(copied[k])
        with torch.cuda.stream(stream):
            lamd.copy_(lam_pin, non_blocking=True)
        plan.assemble(Lbuf[k % 2], F, stream)
        used[k].record(stream)
        plan.apply(F, lamd, q, stream)
        with torch.cuda.stream(stream):
            q_pin.copy_(q, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1) / K
    if plan.device_status(stream) != 0:
        raise RuntimeError("device status not OK after the timed steps")

    # amortisation point (paper Sec. 1 and Sec. 5): iterations after which the
    # explicit operator (assembly + cheap applies) beats the implicit one (no
    # assembly, sparse triangular solves every iteration); the numeric
    # factorisation is common to both and cancels
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(20):
        plan.apply(F, lam, q, stream)
    a1.record(stream)
    a1.synchronize()
    t_expl = a0.elapsed_time(a1) / 20
    # the same product on the integer pipes (sc_apply_fixed)
    qf = torch.empty_like(q)
    plan.apply_fixed(F, lam, qf, stream)
    a0.record(stream)
    for _ in range(20):
        plan.apply_fixed(F, lam, qf, stream)
    a1.record(stream)
    a1.synchronize()
    t_fixed = a0.elapsed_time(a1) / 20
    # the tiles split between the FP64 pipe and the integer pipes (sc_apply_mixed): every share
    mixed = {}
    qm = torch.empty_like(q)
    for quarters in (1, 2, 3):
        plan.apply_mixed(F, lam, qm, quarters, stream)
        a0.record(stream)
        for _ in range(20):
            plan.apply_mixed(F, lam, qm, quarters, stream)
        a1.record(stream)
        a1.synchronize()
        tm = a0.elapsed_time(a1) / 20
        mixed[str(quarters)] = {"ms": tm, "GBps": st["bytes_apply"] / (tm / 1e3) / 1e9,
                                "frac_hbm": st["bytes_apply"] / (tm / 1e3) / 1e9 / HBM_PEAK_GBPS,
                                "rel_diff_vs_fp64": (torch.linalg.vector_norm(qm - q) /
                                                     torch.linalg.vector_norm(q)).item()}
    best_q = min(mixed, key=lambda k: mixed[k]["ms"])
    # the digit form on the tensor cores (sc_apply_digits): prepared once per assembly, then streamed
    Fd = plan.prepare_digits(F, stream=stream)
    a0.record(stream)
    plan.prepare_digits(F, Fd, stream=stream)
    a1.record(stream)
    a1.synchronize()
    t_prep = a0.elapsed_time(a1)
    qd = torch.empty_like(q)
    plan.apply_digits(Fd, lam, qd, stream)
    a0.record(stream)
    for _ in range(20):
        plan.apply_digits(Fd, lam, qd, stream)
    a1.record(stream)
    a1.synchronize()
    t_dig = a0.elapsed_time(a1) / 20
    n_tiles = plan.sizes.F_doubles // 1024
    # streamed per call: the digit tiles, lambda gathered once per row block and q
    dig_bytes = n_tiles * 7184 + 16.0 * sum(plan.m)
    apply_sec_digits = {
        "ms": t_dig, "bytes": dig_bytes, "GBps": dig_bytes / (t_dig / 1e3) / 1e9,
        "frac_hbm": dig_bytes / (t_dig / 1e3) / 1e9 / HBM_PEAK_GBPS,
        "fp64_form_GBps": st["bytes_apply"] / (t_dig / 1e3) / 1e9,
        "speedup_vs_fp64": t_expl / t_dig, "prepare_ms": t_prep,
        "traffic": _traffic_for("apply_digits_kernel"),
        "rel_diff_vs_fp64": (torch.linalg.vector_norm(qd - q) / torch.linalg.vector_norm(q)).item()}
    del Fd
    apply_sec = {
        "digits": apply_sec_digits,
        "bytes": st["bytes_apply"],
        "mixed": {"best_fp64_quarters": int(best_q), **mixed[best_q], "by_fp64_quarters": mixed},
        "fp64": {"ms": t_expl, "GBps": st["bytes_apply"] / (t_expl / 1e3) / 1e9,
                 "frac_hbm": st["bytes_apply"] / (t_expl / 1e3) / 1e9 / HBM_PEAK_GBPS},
        "fixed": {"ms": t_fixed, "GBps": st["bytes_apply"] / (t_fixed / 1e3) / 1e9,
                  "frac_hbm": st["bytes_apply"] / (t_fixed / 1e3) / 1e9 / HBM_PEAK_GBPS,
                  "rel_diff_vs_fp64": (torch.linalg.vector_norm(qf - q) / torch.linalg.vector_norm(q)).item()},
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    t_gimpl, gimpl = _gpu_implicit(fs, prob.n_dual, Lv, lam, q, stream)
    impl = host.ImplicitApply(fs, prob.n_dual)
    lam_h = lam.cpu().numpy()
    q_host = impl(lam_h)
    q_dev = q.cpu().numpy()
    host_rel_diff = float(np.linalg.norm(q_host - q_dev) / np.linalg.norm(q_dev))
    t_impl = []
    for _ in range(5):
        t0 = time.perf_counter()
        impl(lam_h)
        t_impl.append(1e3 * (time.perf_counter() - t0))
    t_impl = statistics.median(t_impl)
    # the column-by-column host form, for reference (the planned form above is the comparator)
    impl_col = host.ImplicitApply(fs, prob.n_dual, planned=False)
    impl_col(lam_h)
    t_col = []
    for _ in range(3):
        t0 = time.perf_counter()
        impl_col(lam_h)
        t_col.append(1e3 * (time.perf_counter() - t0))
    t_col = statistics.median(t_col)
    t_asm = sum(prep_ms) / len(prep_ms) + sum(trsm_ms) / len(trsm_ms) + sum(syrk_ms) / len(syrk_ms)

    # the FP64 peak the roofline divides by: measured on this GPU, after the timed region
    # The probe (independent FMA chains) is measured in every run; it stays below what the
    # FP64 SYRK itself sustains, so it is a lower bound of the pipe's ceiling, not the ceiling:
    # the roofline divides by the larger of the probe and the nominal rate.
    try:
        probe, fp64_probe = _fp64_fma_peak(dev, stream)
    except Exception as e:  # report, fall back to the nominal figure
        probe, fp64_probe = 0.0, {"error": f"{type(e).__name__}: {str(e)[:200]}"}
    fp64_peak = max(probe, FP64_PEAK_TFLOPS)
    peak_source = (f"nominal FP64 pipe rate 152 SMs x 4 flop/clk x 2.07 GHz = {FP64_PEAK_TFLOPS:.3f} TFLOP/s "
                   f"(measured at 2070 MHz during the run); the FMA probe measured {probe:.3f} TFLOP/s in this run "
                   f"(sc_probe_fp64_fma, best of 5 launches, CUDA events), below the SYRK's own rate, so the "
                   f"larger of the two is the ceiling")
    gimpl["frac_fp64_peak"] = gimpl["tflops"] / fp64_peak
    # dominant kernel roofline (FP64 pipe)
    syrk_avg = sum(syrk_ms) / len(syrk_ms)
    trsm_avg = sum(trsm_ms) / len(trsm_ms)
    dom, dom_ms, dom_flops = ("syrk_kernel", syrk_avg, st["flops_syrk"]) if syrk_avg >= trsm_avg else \
        ("trsm_kernel", trsm_avg, st["flops_trsm"])
    achieved = dom_flops / (dom_ms / 1e3) / 1e12
    useful = st["flops_trsm"] + st["flops_syrk"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _workload_config(args),
        "effective_tflops": st["flops_dense"] / (ms / 1e3) / 1e12,
        "executed_tflops": useful / (ms / 1e3) / 1e12,
        "stage_ms": {"prep": sum(prep_ms) / len(prep_ms), "trsm": trsm_avg, "syrk": syrk_avg},
        "flops": {"useful_trsm": st["flops_trsm"], "useful_syrk": st["flops_syrk"],
                  "dense_equivalent": st["flops_dense"]},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "traffic": _traffic_for(dom),
                     "peak_source": peak_source, "peak_nominal": FP64_PEAK_TFLOPS,
                     "frac_of_probe": achieved / probe if probe > 0 else None, "fp64_probe": fp64_probe,
                     "other_kernel": {"kernel": "trsm_kernel" if dom == "syrk_kernel" else "syrk_kernel",
                                      "frac": (st["flops_trsm"] / (trsm_avg / 1e3) / 1e12 if dom == "syrk_kernel"
                                               else st["flops_syrk"] / (syrk_avg / 1e3) / 1e12) / fp64_peak}},
        "e2e": {"value": world * nsub / (e2e_serial_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(Lpin.numel() * 8 + lam_pin.numel() * 8),
                "d2h_bytes_per_step": int(q_pin.numel() * 8),
                "note": "each step timed alone: copy of L and lambda, assemble, apply, read back q"},
        "e2e_pipelined": {"value": world * nsub / (e2e_ms / 1e3), "unit": UNIT,
                          "note": "steps back to back; step k+1's L copy overlaps step k's assembly"},
        "amortization": {"iterations": t_asm / (t_impl - t_expl) if t_impl > t_expl else None,
                         "iterations_incl_L_h2d": (t_asm + (e2e_serial_ms - ms)) / (t_impl - t_expl)
                         if t_impl > t_expl else None,
                         "t_assembly_ms": t_asm, "t_apply_explicit_gpu_ms": t_expl,
                         "t_apply_implicit_host_ms": t_impl, "implicit_host_threads": os.cpu_count(),
                         "implicit_host_form": "planned: per supernode, symbolic work once",
                         "implicit_host_rel_diff_vs_explicit": host_rel_diff,
                         "t_apply_implicit_host_column_ms": t_col,
                         "iterations_vs_gpu_implicit": t_asm / (t_gimpl - t_expl) if t_gimpl > t_expl else None,
                         "t_apply_implicit_gpu_ms": t_gimpl,
                         "iterations_vs_gpu_implicit_fixed_apply": t_asm / (t_gimpl - t_fixed) if t_gimpl > t_fixed else None},
        "sc_apply": apply_sec,
        "gpu_implicit_apply": gimpl,
        "gpu_launches": args.steps * 5,
        "clocks": clocks.summary(),
    }
    if args.feti and rank == 0:
        line["feti_pcpg"] = _secondary(lambda: _feti_section(prob, fs, dev, t_asm, t_expl, t_gimpl, t_impl))
    if args.pipeline_chunks > 0 and rank == 0:
        line["assembly_pipeline"] = _secondary(lambda: _pipeline_section(args, prob, fs, dev, stream))
    if args.split and rank == 0:
        line["split_precision"] = _secondary(lambda: _split_section(args, fs, prob, Lv, lam, flush, stream, dev, ms))
    if args.dense and rank == 0:
        from paper_2509_21037_gb300 import dense
        del flush
        torch.cuda.empty_cache()
        res = {}
        for emu in (0, 1):
            try:
                r = dense.DenseRunner(fs, dev, emulation=emu)
                r.run()
                torch.cuda.synchronize(dev)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r.run()
                b.record(stream)
                b.synchronize()
                dms = a.elapsed_time(b)
                res["fp64_emulation" if emu else "native_fp64"] = {
                    "ms_per_batch": dms, "assemblies_per_s": nsub / (dms / 1e3),
                    "effective_tflops": st["flops_dense"] / (dms / 1e3) / 1e12,
                    "speedup_of_sparse_path": dms / ms}
                del r
                torch.cuda.empty_cache()
            except Exception as e:  # report, do not hide
                res["fp64_emulation" if emu else "native_fp64"] = {"error": str(e)[:200]}
        line["dense_comparator"] = res
    if args.cpu_baseline and rank == 0:
        S = args.ref_sample
        t = _oracle_sample(prob, list(range(S)))
        line["cpu_baseline"] = {"value": S / t, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                                "sample": f"first {S} of 64 subdomains, fresh memo, FP64 dense Cholesky + solves + one refinement step",
                                "unmemoised": _oracle_unmemoised(prob)}
    if rank == 0:
        print(json.dumps(line, default=_json_default))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _split_section(args, fs, prob, Lv, lam, flush, stream, dev, fp64_ms):
    """The same workload with the off-diagonal GEMM work on the tensor cores
    (SC_SPLIT_BF16), per number of 8-bit digit slices: throughput and the
    per-subdomain relative Frobenius error against the refined FP64 oracle."""
    import torch

    import oracle
    from paper_2509_21037_gb300 import abi, sc
    Fo = oracle.dual_operators(prob.subdomains, refine=1) if args.split_error else None
    out = {}
    for S, tile in [(S, t) for S in args.split_slices for t in (abi.SC_TILE_32, abi.SC_TILE_TC128)]:
        plan = sc.Plan(fs, prob.n_dual, precision=abi.SC_SPLIT_BF16, n_slices=S, tile=tile).upload(dev)
        F = plan.new_F(dev)
        q = torch.empty_like(lam)
        for _ in range(args.warmup):
            plan.assemble(Lv, F, stream)
            plan.apply(F, lam, q, stream)
        torch.cuda.synchronize(dev)
        if plan.device_status(stream) != 0:
            raise RuntimeError("device status not OK (split)")
        plan.enable_stage_timing(True)
        tot, trsm, syrk = [], [], []
        for _ in range(args.steps):
            flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.assemble(Lv, F, stream)
            plan.apply(F, lam, q, stream)
            b.record(stream)
            _, tm, sy = plan.stage_times()
            b.synchronize()
            tot.append(a.elapsed_time(b)); trsm.append(tm); syrk.append(sy)
        plan.enable_stage_timing(False)
        ms = sum(tot) / len(tot)
        st = plan.stats_dict()
        rec = {"ms_per_step": ms, "assemblies_per_s": len(fs) / (ms / 1e3),
               "speedup_vs_fp64_path": fp64_ms / ms,
               "stage_ms": {"trsm": sum(trsm) / len(trsm), "syrk": sum(syrk) / len(syrk)},
               "tensor_products_per_fp64_product": S * (S + 1) // 2,
               "useful_fp64_equivalent_tflops": (st["flops_trsm"] + st["flops_syrk"]) / (ms / 1e3) / 1e12}
        # tensor roofline: useful FP64 flops x digit products per FP64 product = the BF16 work done
        P = S * (S + 1) // 2
        syrk_stage = rec["stage_ms"]["syrk"]
        step_tf = (st["flops_trsm"] + st["flops_syrk"]) * P / (ms / 1e3) / 1e12
        syrk_tf = st["flops_syrk"] * P / (syrk_stage / 1e3) / 1e12
        rec["roofline"] = {"bound": "tensor", "unit": "TFLOP/s", "peak": BF16_PEAK_TFLOPS,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst, of measured)",
                           "step": {"achieved": step_tf, "frac": step_tf / BF16_PEAK_TFLOPS},
                           "syrk_stage": {"achieved": syrk_tf, "frac": syrk_tf / BF16_PEAK_TFLOPS}}
        if Fo is not None:
            errs = [oracle.relative_frobenius(plan.export(F, i).cpu().numpy(), Fo[i]) for i in range(len(fs))]
            rec["rel_frobenius_error"] = {"max": max(errs), "median": float(np.median(errs)), "min": min(errs)}
        rec["syrk_tile"] = "128x32 tcgen05.mma (TMEM accumulators)" if tile else "32x32 mma.sync"
        out[f"slices_{S}" + ("_tc128" if tile else "")] = rec
        del plan, F
    return out


def _apply_suite(plan, F, lam, q, steps):
    """Every form of the explicit product on one assembled F: the FP64 apply,
    the integer-pipe fixed point and the tensor-core digit form (prepared
    once), each timed back to back over `steps` calls (F is larger than L2);
    bytes are the stored triangle in FP64 (fp64, fixed) or the streamed digit
    tiles (digits), against the measured HBM peak."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    by = plan.stats.bytes_apply

    def time_it(fn):
        fn()
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / steps

    out = {}
    t = time_it(lambda: plan.apply(F, lam, q))
    out["fp64"] = {"ms": t, "GBps": by / (t / 1e3) / 1e9, "frac_hbm": by / (t / 1e3) / 1e9 / HBM_PEAK_GBPS}
    qx = torch.empty_like(q)
    t = time_it(lambda: plan.apply_fixed(F, lam, qx))
    out["fixed"] = {"ms": t, "GBps": by / (t / 1e3) / 1e9, "frac_hbm": by / (t / 1e3) / 1e9 / HBM_PEAK_GBPS,
                    "rel_diff_vs_fp64": (torch.linalg.vector_norm(qx - q) / torch.linalg.vector_norm(q)).item()}
    Fd = plan.prepare_digits(F)
    a.record()
    plan.prepare_digits(F, Fd)
    b.record()
    b.synchronize()
    t_prep = a.elapsed_time(b)
    t = time_it(lambda: plan.apply_digits(Fd, lam, qx))
    dby = plan.sizes.F_doubles // 1024 * 7184 + 16.0 * sum(plan.m)
    out["digits"] = {"ms": t, "bytes": dby, "GBps": dby / (t / 1e3) / 1e9,
                     "frac_hbm": dby / (t / 1e3) / 1e9 / HBM_PEAK_GBPS, "prepare_ms": t_prep,
                     "speedup_vs_fp64": out["fp64"]["ms"] / t,
                     "rel_diff_vs_fp64": (torch.linalg.vector_norm(qx - q) / torch.linalg.vector_norm(q)).item()}
    if plan.digits_status(Fd) != 0:
        raise RuntimeError("sc_apply_digits reported a timeout")
    del Fd
    out["bytes_fp64"] = by
    out["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return out


def run_config3(args):
    """512 elasticity cubes (edge 8..16), FP64 path: assembly and every form of
    the explicit product (the apply roofline at a second size)."""
    import torch

    from paper_2509_21037_gb300 import host, sc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prob = synth.make_config(3, seed=args.seed)
    fs = host.factorize_problem(prob.subdomains, threads=0)
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    lam = torch.from_numpy(np.random.default_rng(args.seed).standard_normal(prob.n_dual)).to(dev)
    plan = sc.Plan(fs, prob.n_dual).upload(dev)
    F = plan.new_F(dev)
    q = torch.empty_like(lam)
    for _ in range(args.warmup):
        plan.assemble(Lv, F)
    torch.cuda.synchronize(dev)
    if plan.device_status() != 0:
        raise RuntimeError("device status not OK (config 3)")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(args.steps):
        a.record()
        plan.assemble(Lv, F)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    plan.apply(F, lam, q)
    t = sum(ms) / len(ms)
    line = {"metric": METRIC, "value": len(fs) / (t / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "elasticity3d_hex8_512_cubes_k8-16", "subdomains": len(fs),
                       "multipliers_total": int(prob.n_dual), "seed": args.seed},
            "sc_apply": _apply_suite(plan, F, lam, q, 20)}
    print(json.dumps(line, default=_json_default))
    return 0


def run_config5(args):
    """Mixed batch: 1024 2D heat squares (edge 32..96) + 1024 3D elasticity cubes
    (edge 8..20), learned per-subdomain variant selection (autotuner on a third
    of the subdomain classes as fallback and as the yardstick of the learned choice),
    workspace in waves."""
    import torch

    from paper_2509_21037_gb300 import host, sc, tune
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    prob = synth.make_config(5, seed=args.seed)
    fs = host.factorize_problem(prob.subdomains, threads=0)
    t_prep = time.time() - t0
    Lv = torch.from_numpy(sc.concat_L_values(fs)).to(dev)
    lam = torch.from_numpy(np.random.default_rng(args.seed).standard_normal(prob.n_dual)).to(dev)
    V = tune.VARIANTS
    keys = sorted({tune.class_key(f) for f in fs}, key=lambda k: (k[0], k[2], k[1]))
    train = keys[::3]
    t1 = time.time()
    recs = tune.autotune(fs, dev, variants=V, classes=train, reps=1)
    t_tune = time.time() - t1
    sel = tune.LearnedSelector(variants=V, device=dev)
    sel.fit(list(recs.values()), epochs=3000)
    var = tune.select(fs, args.tol, sel, measured=recs)

    def timed(var_codes, ws_limit, keep_F=False):
        plan = sc.Plan(fs, prob.n_dual, ws_limit=ws_limit, **tune.plan_options(var_codes)).upload(dev)
        F = plan.new_F(dev)
        q = torch.empty_like(lam)
        plan.assemble(Lv, F)
        plan.apply(F, lam, q)
        torch.cuda.synchronize(dev)
        if plan.device_status() != 0:
            raise RuntimeError("device status not OK (config 5)")
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        asm, app = [], []
        for _ in range(args.steps):
            a.record()
            plan.assemble(Lv, F)
            b.record()
            plan.apply(F, lam, q)
            c.record()
            c.synchronize()
            asm.append(a.elapsed_time(b))
            app.append(b.elapsed_time(c))
        out = {"assembly_ms": sum(asm) / len(asm), "apply_ms": sum(app) / len(app),
               "waves": int(plan.stats.n_waves), "ws_GB": plan.sizes.ws_bytes / 1e9,
               "apply_GBps": plan.stats.bytes_apply / (sum(app) / len(app) / 1e3) / 1e9,
               "sc_apply": _apply_suite(plan, F, lam, q, 20)}
        F_off = plan.F_offsets.copy()
        st = plan.stats_dict()
        out["q"] = q
        del plan
        torch.cuda.empty_cache()
        return out, (F if keep_F else None), F_off, st

    lim = int(args.ws_limit_gb * 1e9)
    r64, F64, F_off, st = timed([0] * len(fs), lim, keep_F=True)
    rsel, Fsel, _, _ = timed(var, lim, keep_F=True)
    errs = []
    for i in range(len(fs)):
        a, b = F_off[i], F_off[i + 1]
        nr = torch.linalg.vector_norm(F64[a:b]).item()
        errs.append(torch.linalg.vector_norm(Fsel[a:b] - F64[a:b]).item() / max(nr, 1e-300))
    del Fsel
    q_expl = r64.pop("q")
    rsel.pop("q")
    del F64
    torch.cuda.empty_cache()
    t_gimpl, gimpl = _gpu_implicit(fs, prob.n_dual, Lv, lam, q_expl, None, reps=3)
    impl = host.ImplicitApply(fs, prob.n_dual)
    lam_h = lam.cpu().numpy()
    impl(lam_h)
    t_impl = []
    for _ in range(3):
        t2 = time.perf_counter()
        impl(lam_h)
        t_impl.append(1e3 * (time.perf_counter() - t2))
    t_impl = statistics.median(t_impl)
    counts = {str(v): int(c) for v, c in zip(*np.unique(var, return_counts=True))}
    best = rsel["assembly_ms"]
    line = {
        "metric": METRIC, "value": len(fs) / (best / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": 1, "ms_per_step": best + rsel["apply_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+split", "data": "synthetic",
        "config": {"workload": "mixed_1024_heat2d_q1_k32-96_1024_elasticity3d_hex8_k8-20", "subdomains": len(fs),
                   "multipliers_total": int(prob.n_dual), "error_target": args.tol, "seed": args.seed},
        "fp64_only": r64, "selected": rsel, "selection_counts": counts,
        "selected_rel_error_vs_fp64": {"max": max(errs), "median": float(np.median(errs))},
        "speedup_selected_vs_fp64": r64["assembly_ms"] / rsel["assembly_ms"],
        "effective_tflops_selected": st["flops_dense"] / (rsel["assembly_ms"] / 1e3) / 1e12,
        "amortization": {"iterations": rsel["assembly_ms"] / (t_impl - rsel["apply_ms"]),
                         "iterations_fp64_only": r64["assembly_ms"] / (t_impl - r64["apply_ms"]),
                         "t_apply_implicit_host_ms": t_impl, "implicit_host_threads": os.cpu_count(),
                         "iterations_vs_gpu_implicit": rsel["assembly_ms"] / (t_gimpl - rsel["apply_ms"])
                         if t_gimpl > rsel["apply_ms"] else None,
                         "t_apply_implicit_gpu_ms": t_gimpl},
        "gpu_implicit_apply": gimpl,
        "autotune": {"classes_measured": len(recs), "classes_total": len(keys), "seconds": t_tune},
        "host_factorisation_s": t_prep,
    }
    print(json.dumps(line, default=_json_default))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sc", choices=["sc", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ref-sample", type=int, default=8)
    ap.add_argument("--no-dense", dest="dense", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-feti", dest="feti", action="store_false",
                    help="skip the FETI-1 PCPG section (iteration counts against the amortisation point)")
    ap.add_argument("--pipeline-chunks", type=int, default=4,
                    help="chunks of the CPU/GPU numeric-stage pipeline section (0: skip it)")
    ap.add_argument("--no-split", dest="split", action="store_false",
                    help="skip the split-precision (tensor-core) variant of the workload")
    ap.add_argument("--split-slices", type=int, nargs="+", default=[7, 5])
    ap.add_argument("--no-split-error", dest="split_error", action="store_false")
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 5],
                    help="2: the 64-subdomain heat cube (default); 3: 512 elasticity cubes (FP64 path and "
                         "the product forms); 5: the mixed 2048-subdomain batch")
    ap.add_argument("--tol", type=float, default=1e-8, help="config 5: error target of the variant selection")
    ap.add_argument("--ws-limit-gb", type=float, default=48.0, help="config 5: workspace bound per wave")
    ap.add_argument("--profile-slices", type=int, default=0,
                    help="with --profile: run the split-precision variant with this many slices")
    ap.add_argument("--profile-tile", type=int, default=0, choices=[0, 1],
                    help="with --profile-slices: SYRK tile (0 = 32x32 mma.sync, 1 = 128x32 tcgen05)")
    ap.add_argument("--profile-mixed", type=int, default=2, choices=[0, 1, 2, 3, 4],
                    help="with --profile: sc_apply_mixed's FP64 share (quarters of the tiles)")
    ap.add_argument("--profile-implicit", action="store_true",
                    help="with --profile: also run the GPU implicit apply warmup + steps times")
    ap.add_argument("--profile", action="store_true",
                    help="device steps only (no e2e, comparator or CPU baseline): for ncu captures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 5:
        return run_config5(args)
    if args.config == 3:
        return run_config3(args)
    return run_sc(args)


if __name__ == "__main__":
    sys.exit(main())
