"""Benchmark: ELM trainings per second on one GB300 (sparse-pixel workload:
X 60000 x 784 with 80% zeros, L = 2000 sigmoid neurons, 10 one-hot classes,
full column rank), beta checked against the FP64 CPU oracle's accuracy bar.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl native|reference] [--workload W] [--fp64-steps K64]
                  [--no-oracle-check]

One step = one complete training (hidden layer, Gram, pivoted rank
decision, solves, refinement) of the workload, inputs resident in HBM.
Every training streams more than the 129 MB L2 (X is 188 MB, H 0.96 GB),
so no L2 flush is inserted.  The e2e figure repeats the step through the C
ABI with pinned host buffers: the host->device copy of X, W, b, T and the
device->host copy of beta are inside the timed region.

With --gpus N > 1 (torchrun, one process per GPU) every rank trains its own
replica of the workload (independent problems, no collective); the value is
the trainings of all ranks divided by the slowest rank's time.

Before timing, a verified run checks every problem: status OK (or
NOT_CONVERGED with beta written), the planted rank, and beta against the
FP64 CPU oracle's (within 1e-6 relative Frobenius for the mixed form, 1e-9
for the FP64 form).  The oracle trains the sparse-pixel workload in full on
the host cores (that run is also the line's cpu_baseline); the other
workloads are checked against the oracle's stored results in tests/golden
where they exist.  A line that fails a check carries "valid": false and the
script exits 1.  The default line also times the plain FP64 GPU form of the
same workload (fp64_form) and reports the mixed form's speedup over it.

--impl reference times the FP64 CPU oracle (the method's plain definition)
on the host cores: each step trains a bounded sample of the workload (the
first rows of X; N-proportional phases scaled to the full N), and one full
training of the workload, timed once, gives the line's value.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ELM trainings/sec (beta at rel err <=1e-6) mixed+batched vs plain FP64, 1 GB300"
WORKLOAD = dict(workload="sparse-pixel ELM: X 60000x784 (80% zeros, U[0,1], FP32), L=2000 "
                         "sigmoid, 10 one-hot classes, full column rank",
                N=60000, n=784, L=2000, m=10)


def flops_model(N, n, L, m):
    """Algorithmic work per training (symmetric Gram counted once)."""
    return dict(hidden=2.0 * N * n * L, gram=float(N) * L * (L + 1) + 2.0 * N * L * m,
                factor=L ** 3 / 3.0, refine_iter=4.0 * N * L * m)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = {}
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
    return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), bf16=d.get("bf16_tflops", 1900.0),
                bf16_sus=d.get("bf16_tflops_sustained", 1700.0),
                source="measured" if d else "fallback",
                # FP64 has no measured entry: nominal GB300 rate (1.25 TFLOP/s)
                fp64=1.25)


GOLDEN = os.path.join(ROOT, "tests", "golden")


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx,
                    reasons=sorted(reasons), samples=len(sm))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """Largest `value` over all ranks (the slowest rank's time); `value`
    itself when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(count, rank, world):
    """Indices of `count` independent problems handled by `rank` of `world`
    (contiguous blocks, sizes differing by at most one; no collective)."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def oracle_full(p):
    """One full training of problem p by the oracle (Alg. 1), timed:
    (beta, rank, seconds)."""
    import oracle
    t0 = time.perf_counter()
    beta, r, _ = oracle.train(p["X"], p["W"], p["b"], p.get("a"), int(p["act"]), p["T"])
    return beta, r, time.perf_counter() - t0


def cores_used():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(full, sample_rows=2000, threads=None):
    """Time the oracle, as it stands, on the first `sample_rows` rows of the
    workload and scale its N-proportional phases to the full N."""
    import oracle
    p = synth.workload_sparse_pixels(N=sample_rows)
    X, W, b, T = p["X"], p["W"], p["b"], p["T"]
    N, L, m = full["N"], full["L"], full["m"]
    t0 = time.perf_counter()
    H = oracle.hidden(X, W, b, None, 0)
    t1 = time.perf_counter()
    S, Z = oracle.gram(H, T)
    t2 = time.perf_counter()
    r, perm, R = oracle.pivchol(S)
    beta = oracle.frsolve(R, r, perm, Z)
    t3 = time.perf_counter()
    for _ in range(2):             # the oracle's two refinement steps, as orc_train runs them
        Res = T - oracle.matmul_hb(H, beta)
        G = oracle.gram(H, Res)[1]
        beta = beta + oracle.frsolve(R, r, perm, G)
    t4 = time.perf_counter()
    scale = N / float(sample_rows)
    t_full = (t1 - t0 + t2 - t1 + t4 - t3) * scale + (t3 - t2)
    cores = cores_used()
    return dict(value=1.0 / t_full, unit="trainings/s", cores=cores, kind="oracle",
                sample="first %d of %d rows of the workload; hidden/Gram/refinement times "
                       "scaled by N, factorisation+solve (L=%d) timed in full "
                       "(%.1f s of CPU time: hidden %.1f, Gram %.1f, factor %.1f, refine %.1f)"
                       % (sample_rows, N, L, t4 - t0, t1 - t0, t2 - t1, t3 - t2, t4 - t3),
                projected_s_per_training=t_full, step_s=t4 - t0)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    full = dict(WORKLOAD)
    steps, proj = [], []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(full, sample_rows=args.ref_rows)
        if i >= args.warmup:
            steps.append(cb["step_s"])
            proj.append(cb["projected_s_per_training"])
    # one full training of the workload, timed once: the line's value
    # (--ref-full-rows < N only to test the arm quickly)
    nfull = args.ref_full_rows
    _, _, t_full = oracle_full(synth.workload_sparse_pixels(N=nfull))
    val = nfull / float(full["N"]) / t_full
    line = dict(metric=METRIC, value=val, unit="trainings/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=statistics.median(steps) * 1e3,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config=dict(WORKLOAD, inputs="host memory; oracle on the host cores"),
                impl="reference",
                cpu_baseline=dict(value=val, unit="trainings/s", kind="oracle", cores=cores_used(),
                                  sample="value: one training of the workload on %d of "
                                         "its %d rows, %.1f s; each timed step: the first %d "
                                         "rows (%s); median projection of the steps to the "
                                         "full N: %.4f trainings/s"
                                         % (nfull, full["N"], t_full, args.ref_rows,
                                            cb["sample"], 1.0 / statistics.median(proj)),
                                  full_training_s=t_full),
                e2e=dict(value=val, unit="trainings/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


WORKLOADS = {
    "sparse_pixels": (lambda rows: [synth.workload_sparse_pixels(N=rows or WORKLOAD["N"])],
                      WORKLOAD["workload"]),
    "small": (lambda rows: [synth.workload_small_fp64()],
              "small ELM: X 2000x16 U[0,1] FP64, L=200 sigmoid (180 unique + 20 duplicates, "
              "rank 180), 4 one-hot classes"),
    "rank_deficient": (lambda rows: [synth.workload_rank_deficient()],
                       "rank-deficient ELM: X 100000x64 N(0,1) FP32, L=6000 sigmoid (5100 unique "
                       "+ 600 duplicates + 300 scaled copies, rank 5100), 3 regression targets"),
    "batched": (lambda rows: synth.workload_batched(),
                "batched uneven ELMs: 128 problems, N in [5000,50000], d in {16,54,128}, "
                "L in [100,3000], sigmoid/tanh, 2-26 one-hot classes"),
    "large": (lambda rows: [synth.workload_large(**({"N": rows} if rows else {}))],
              "large ELM: X 500000x128 U[-1,1] FP32, L=8000 sigmoid, 20 one-hot classes"),
    # the shape of the paper's Table 1 experiment; L from --hidden
    "gina_shaped": (lambda rows: [synth.workload_gina_shaped(L=ARGS_HIDDEN[0])],
                    "Table-1-shaped ELM: X 3468x971 (80% zeros, U[0,1], FP32), L={L} sigmoid, "
                    "2 one-hot classes"),
}
ARGS_HIDDEN = [2000]


def reference_results(workload, plist, time_first=False):
    """The oracle's (beta, rank) per problem, or None where unavailable:
    trained live for the workloads the oracle finishes in seconds to
    minutes on the host cores, else read from the results the oracle stored
    in tests/golden (written by tests/golden/make_full_goldens.py).
    Returns (list, seconds of the first live training or None)."""
    if workload in ("sparse_pixels", "small", "gina_shaped"):
        out, t_first = [], None
        for p in plist:
            beta, r, t = oracle_full(p)
            out.append((beta, r))
            if t_first is None:
                t_first = t
        return out, t_first
    path = os.path.join(GOLDEN, "full_%s.npz" % workload)
    if not os.path.exists(path):
        return [None] * len(plist), None
    g = np.load(path)
    return [(g["beta_%03d" % i], int(g["rank"][i]), error_scale(g, i))
            for i in range(len(plist))], None


def error_scale(g, i, steps=2):
    """Forward error scale of problem i's beta computed in FP64 through the
    normal equations with `steps` refinement steps, from the conditioning
    the oracle recorded: u (kappa + kappa^2 eta) + (kappa^2 u)^(steps+1)
    (Wedin's bound, plus what the steps leave of the first solve's error).
    The parity tests use the same scale."""
    u = 2.0 ** -53
    kappa = float(g["kappa"][i])
    L = g["beta_%03d" % i].shape[0]
    h2 = np.sqrt(float(g["ev_max"][i])) * float(g["h_fro"][i]) / np.sqrt(L)
    eta = float(g["res_norm"][i]) / (h2 * float(g["beta_norm"][i]))
    return u * (kappa + kappa * kappa * eta) + (kappa * kappa * u) ** (steps + 1)


def check_results(res, betas, refs, planted, tol):
    """Per problem: status OK (or NOT_CONVERGED, beta written), the planted
    rank, the oracle's rank, beta within tol (relative Frobenius) of the
    oracle's.  Returns (worst error, list of failure descriptions)."""
    worst, bad = 0.0, []
    widened = 0
    for i, (r, beta, ref, pr) in enumerate(zip(res, betas, refs, planted)):
        if r["status"] not in (0, 5):
            bad.append("problem %d: status %d" % (i, r["status"]))
            continue
        if pr is not None and r["rank"] != pr:
            bad.append("problem %d: rank %d, planted %d" % (i, r["rank"], pr))
        if ref is None:
            continue
        bref, rref = ref[0], ref[1]
        if r["rank"] != rref:
            bad.append("problem %d: rank %d, oracle %d" % (i, r["rank"], rref))
        err = float(np.linalg.norm(beta - bref) / np.linalg.norm(bref))
        # where FP64 arithmetic cannot fix beta to the bar (the recorded
        # scale above 1/100 of it), 8 times the problem's scale
        bar = tol
        if len(ref) > 2 and ref[2] > tol / 100.0:
            bar = max(tol, 8.0 * ref[2])
            widened += 1
        else:
            worst = max(worst, err)
        if not err <= bar:
            bad.append("problem %d: beta error %.3g > %.3g" % (i, err, bar))
    return worst, bad, widened


def run_native(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_02436_gb300 as elm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = dict(mixed=elm.PREC_MIXED, fp64=elm.PREC_FP64, fp64_tc=elm.PREC_FP64_TC)[args.precision]
    tol = 1e-6 if prec == elm.PREC_MIXED else 1e-9

    gen, desc = WORKLOADS[args.workload]
    desc = desc.replace("{L}", str(args.hidden))
    plist = gen(args.rows)
    probs, hosts = [], []
    for p in plist:
        L, m = p["W"].shape[1], p["T"].shape[1]
        probs.append(dict(X=torch.from_numpy(p["X"]).to(dev), W=torch.from_numpy(p["W"]).to(dev),
                          b=torch.from_numpy(p["b"]).to(dev),
                          a=None if p.get("a") is None else torch.from_numpy(p["a"]).to(dev),
                          act=int(p.get("act", 0)), T=torch.from_numpy(p["T"]).to(dev),
                          beta=torch.empty((L, m), dtype=torch.float64, device=dev)))
        hosts.append(p)
    count = len(probs)
    stream = torch.cuda.current_stream(dev)
    ctx = elm.elm_create(local, stream)
    # launch choices picked by the library's autotuner on this workload,
    # before anything is timed (the tuning runs train the problems too)
    tune = None
    if not args.no_autotune:
        t_tune = time.time()
        tune = elm.elm_autotune(ctx, probs if len(probs) > 1 else probs[0], precision=prec)
        tune["seconds"] = round(time.time() - t_tune, 2)
    planted = [int(p["rank"]) if p.get("rank") is not None else None for p in hosts]
    full_rows = args.rows is None or args.workload not in ("sparse_pixels", "large")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    invalid = []

    def timed_ok(res, what):
        for i, r in enumerate(res):
            if r["status"] not in (0, 5) or (planted[i] is not None and r["rank"] != planted[i]):
                invalid.append("%s problem %d: status %d rank %d" % (what, i, r["status"], r["rank"]))

    # verified run: statuses, ranks and beta against the oracle (rank 0)
    bs = dict(block_split=args.block_split) if args.block_split > 0 else {}
    if args.lanes > 0:
        bs["lanes"] = args.lanes
    res = elm.elm_train(ctx, probs, precision=prec, check=False, **bs)
    betas = [pr["beta"].cpu().numpy() for pr in probs]
    check = dict(rank=[r["rank"] for r in res] if count > 1 else res[0]["rank"],
                 refine_iters=max(r["refine_iters"] for r in res),
                 statuses=sorted(set(r["status"] for r in res)),
                 forms={str(f): sum(r["form"] == f for r in res) for f in (0, 1, 2, 3, 4)})
    t_oracle, refs = None, None
    if rank == 0 and full_rows and not args.no_oracle_check:
        refs, t_oracle = reference_results(args.workload, hosts)
        if any(x is not None for x in refs):
            worst, bad, widened = check_results(res, betas, refs, planted, tol)
            check["rel_err_vs_oracle"] = worst
            if widened:
                check["bar_widened_to_fp64_scale"] = widened
            check["oracle_checked"] = sum(x is not None for x in refs)
            invalid += bad
        else:
            check["oracle_checked"] = 0
            timed_ok(res, "verified")
    else:
        timed_ok(res, "verified")

    for _ in range(args.warmup):
        timed_ok(elm.elm_train(ctx, probs, precision=prec, check=False, **bs), "warm-up")
    elm.elm_phase_times(ctx)                       # reset
    barrier()
    l0 = elm.elm_launch_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_res = []
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step_res.append(elm.elm_train(ctx, probs, precision=prec,
                                          flags=elm.FLAG_PHASE_TIMING, check=False, **bs))
        e1.record(stream)
        barrier()
    launches = elm.elm_launch_counter() - l0
    phases = elm.elm_phase_times(ctx)
    for r in step_res:
        timed_ok(r, "timed")
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    value = ws * count * 1000.0 / ms_max

    # the plain FP64 GPU form of the same workload, for the metric's ratio
    fp64 = None
    if prec == elm.PREC_MIXED and args.fp64_steps > 0 and not bs:
        p64 = [dict(pr, beta=torch.empty_like(pr["beta"])) for pr in probs]
        r64 = elm.elm_train(ctx, p64, precision=elm.PREC_FP64, check=False)     # warm-up
        if refs is not None and any(x is not None for x in refs):
            w64, bad64, _ = check_results(r64, [q["beta"].cpu().numpy() for q in p64], refs,
                                          planted, 1e-9)
            check["fp64_form_rel_err_vs_oracle"] = w64
            if bad64:
                check["fp64_form_failures"] = bad64[:8]
        barrier()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.fp64_steps):
            timed_ok(elm.elm_train(ctx, p64, precision=elm.PREC_FP64, check=False), "fp64")
        g1.record(stream)
        barrier()
        ms64 = max_over_ranks(g0.elapsed_time(g1) / args.fp64_steps, dev)
        fp64 = dict(value=ws * count * 1000.0 / ms64, unit="trainings/s", ms_per_step=ms64,
                    steps=args.fp64_steps)

    # e2e through the C ABI with pinned host buffers
    hprobs = []
    h2d = 0
    for p in hosts:
        hp = dict(X=torch.from_numpy(p["X"]).pin_memory(), W=torch.from_numpy(p["W"]).pin_memory(),
                  b=torch.from_numpy(p["b"]).pin_memory(),
                  a=None if p.get("a") is None else torch.from_numpy(p["a"]).pin_memory(),
                  act=int(p.get("act", 0)), T=torch.from_numpy(p["T"]).pin_memory(),
                  beta=torch.empty((p["W"].shape[1], p["T"].shape[1]),
                                   dtype=torch.float64).pin_memory())
        h2d += sum(hp[k].numel() * hp[k].element_size() for k in ("X", "W", "b", "a", "T")
                   if hp[k] is not None)
        hprobs.append(hp)
    d2h = sum(hp["beta"].numel() * 8 for hp in hprobs)
    timed_ok(elm.elm_train(ctx, hprobs, precision=prec, check=False, **bs), "e2e warm-up")
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        timed_ok(elm.elm_train(ctx, hprobs, precision=prec, check=False, **bs), "e2e")
    f1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / e2e_steps, dev)

    if rank == 0:
        pk = peaks()
        ph_ms = {k: v / args.steps for k, v in phases.items()}
        gram_fl, issued = 0.0, 0.0
        for p in hosts:
            N, n = p["X"].shape
            L, m = p["W"].shape[1], p["T"].shape[1]
            gram_fl += flops_model(N, n, L, m)["gram"]
            Lp, Np = -(-(L + m) // 128) * 128, -(-N // 64) * 64
            nJ = Lp // 128
            pairs = 36 if prec == elm.PREC_FP64_TC else 15
            issued += pairs * 2.0 * (nJ * (nJ + 1)) * 128 * 64 * Np
        if prec == elm.PREC_FP64:
            # Gram on the FP64 pipe (nominal rate; the measured peaks have no FP64 entry)
            achieved = gram_fl / (ph_ms["gram"] * 1e-3) / 1e12
            roof = dict(bound="alu", achieved=achieved, peak=pk["fp64"], unit="TFLOP/s",
                        frac=achieved / pk["fp64"], traffic=None, kernel="gram_f64_kernel",
                        peak_source="nominal GB300 FP64 1.25 TFLOP/s (no measured FP64 entry)")
        else:
            # Gram on the tensor cores: algorithmic FLOPs (symmetric Gram counted
            # once, as in the contract) over the Gram phase (that kernel alone),
            # against the measured bf16 burst peak; the digit emulation issues 15
            # digit-pair products of the lower-triangle tiles, reported beside it
            achieved = gram_fl / (ph_ms["gram"] * 1e-3) / 1e12
            tc = prec == elm.PREC_FP64_TC
            # DRAM counters are reported only for the kernel they were taken
            # on; the Gram kernel's plane layout (blocks of 65536 samples,
            # 3-D tensor maps) changed after its last capture
            roof = dict(bound="tensor", achieved=achieved, peak=pk["bf16"], unit="TFLOP/s",
                        frac=achieved / pk["bf16"], traffic=None,
                        traffic_source="no DRAM capture of the current Gram kernel",
                        kernel=("ozaki_kernel (FP64-accurate Gram, 8 digits x 7 bits, 36 pairs "
                                "in two launches)") if tc
                        else "ozaki_kernel (Gram, 5 digits x 7 bits, 15 pairs)",
                        peak_source="%s bf16 dense burst" % pk["source"],
                        issued_tflops=issued / (ph_ms["gram"] * 1e-3) / 1e12,
                        issued_frac=issued / (ph_ms["gram"] * 1e-3) / 1e12 / pk["bf16"])
        roof["phase_ms"] = ph_ms
        first = hosts[0]
        cfg = dict(workload=desc, autotune=tune,
                   precision=args.precision if args.block_split <= 0 else "fp64 (block route)",
                   parallelism="replicas" if ws > 1 else "single",
                   l2="inputs larger than L2 (X and the digit planes stream from HBM): no flush")
        if args.block_split > 0:
            cfg.update(route="the paper's block formulae (Eqs. 19-23), H1 = first %d columns"
                       % args.block_split)
        if count == 1:
            cfg.update(N=first["X"].shape[0], n=first["X"].shape[1], L=first["W"].shape[1],
                       m=first["T"].shape[1])
        else:
            cfg.update(problems=count, lanes=args.lanes or 4,
                       phases="factor, solve and refine summed over the lanes")
        line = dict(metric=METRIC, value=value, unit="trainings/s", n_gpus=ws, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_max, higher_is_better=True,
                    scaling="weak", vs_baseline=None,
                    dtype="f64" if (prec == elm.PREC_FP64 or bs) else "bf16-slices+f64",
                    data="synthetic", config=cfg,
                    e2e=dict(value=ws * count * 1000.0 / e2e_ms, unit="trainings/s",
                             h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    gpu_launches=launches, roofline=roof, clocks=clk.summary(), check=check)
        if fp64 is not None:
            line["fp64_form"] = fp64
            line["speedup_vs_fp64_form"] = value / fp64["value"]
        # the oracle on the host cores (rank 0 of a single-GPU run): the
        # verified run's full training of the default workload
        if args.workload == "sparse_pixels" and ws == 1 and t_oracle is not None:
            line["cpu_baseline"] = dict(value=1.0 / t_oracle, unit="trainings/s",
                                        cores=cores_used(), kind="oracle",
                                        sample="one full training of the workload (%d rows), "
                                               "%.1f s" % (WORKLOAD["N"], t_oracle))
        line["valid"] = not invalid
        if invalid:
            line["invalid_reasons"] = invalid[:16]
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 1 if invalid else 0


def run_sharded(args):
    """--shard rows: one training of the workload with its rows split over
    the ranks (paper_2011_02436_gb300.sharded): every rank forms its block's
    Gram blocks, one exchange sums them in rank order, every rank factorises
    the same sum, refinement residuals are summed the same way.  Strong
    scaling: the work per step is one whole training however many ranks."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_02436_gb300 as elm
    from paper_2011_02436_gb300.sharded import LibraryOps, train_row_blocks

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = elm.PREC_MIXED if args.precision == "mixed" else elm.PREC_FP64
    gen, desc = WORKLOADS[args.workload]
    plist = gen(args.rows)
    if len(plist) != 1:
        raise SystemExit("--shard rows takes a single-problem workload")
    p = plist[0]
    rows = shard(p["X"].shape[0], rank, ws)
    r0, r1 = rows[0], rows[-1] + 1

    def dev_block(src):
        return (torch.from_numpy(src["X"][r0:r1]).to(dev), torch.from_numpy(src["W"]).to(dev),
                torch.from_numpy(src["b"]).to(dev),
                None if src.get("a") is None else torch.from_numpy(src["a"]).to(dev),
                int(src.get("act", 0)), torch.from_numpy(src["T"][r0:r1]).to(dev))

    blk = dev_block(p)
    ctx = elm.elm_create(local, torch.cuda.current_stream(dev))
    ops = LibraryOps(ctx, prec)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    invalid = []
    beta, r, info = train_row_blocks(ops, [blk], precision=prec)
    check = dict(rank=r, refine_iters=info["refine_iters"], converged=info["converged"])
    if r != p["rank"]:
        invalid.append("rank %d, planted %d" % (r, p["rank"]))
    if rank == 0 and not args.no_oracle_check and args.workload in ("sparse_pixels", "small",
                                                                    "gina_shaped"):
        refs, _ = reference_results(args.workload, [p])
        bref, rref = refs[0]
        err = float(np.linalg.norm(beta.cpu().numpy() - bref) / np.linalg.norm(bref))
        check["rel_err_vs_oracle"] = err
        if rref != r or not err <= (1e-6 if prec == elm.PREC_MIXED else 1e-9):
            invalid.append("beta error %.3g or rank %d against the oracle's %d" % (err, r, rref))
    for _ in range(args.warmup):
        train_row_blocks(ops, [blk], precision=prec)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            _, rr, inf = train_row_blocks(ops, [blk], precision=prec)
            if rr != p["rank"] or not inf["converged"]:
                invalid.append("timed step: rank %d converged %s" % (rr, inf["converged"]))
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    # e2e: this rank's rows from pinned host memory each step, beta to the host
    hp = {k: (None if p.get(k) is None else torch.from_numpy(
        np.ascontiguousarray(p[k][r0:r1] if k in ("X", "T") else p[k])).pin_memory())
        for k in ("X", "W", "b", "a", "T")}
    h2d = sum(v.numel() * v.element_size() for v in hp.values() if v is not None)
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        hb = tuple(None if hp[k] is None else hp[k].to(dev, non_blocking=True)
                   for k in ("X", "W", "b", "a"))
        b2 = (hb[0], hb[1], hb[2], hb[3], int(p.get("act", 0)), hp["T"].to(dev, non_blocking=True))
        bh, _, _ = train_row_blocks(ops, [b2], precision=prec)
        bh = bh.cpu()
    f1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / e2e_steps, dev)
    if rank == 0:
        cfg = dict(workload=desc.replace("{L}", str(args.hidden)), precision=args.precision,
                   parallelism="rows sharded over %d rank(s), one exchange per sum" % ws,
                   l2="inputs larger than L2: no flush", N=p["X"].shape[0], L=p["W"].shape[1],
                   m=p["T"].shape[1], rows_per_rank=r1 - r0)
        line = dict(metric=METRIC, value=1000.0 / ms, unit="trainings/s", n_gpus=ws,
                    steps=args.steps, warmup=args.warmup, ms_per_step=ms,
                    higher_is_better=True, scaling="strong", vs_baseline=None,
                    dtype="f64" if prec == elm.PREC_FP64 else "bf16-slices+f64",
                    data="synthetic", config=cfg,
                    e2e=dict(value=1000.0 / e2e_ms, unit="trainings/s", h2d_bytes_per_step=h2d,
                             d2h_bytes_per_step=int(beta.numel() * 8)),
                    clocks=clk.summary(), check=check, valid=not invalid)
        if invalid:
            line["invalid_reasons"] = invalid[:16]
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 1 if invalid else 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp64_tc"], default="mixed",
                    help="fp64_tc: the FP64 form with its Gram on the tensor cores")
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the check of beta against the oracle (and so the CPU baseline)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed trainings of the plain FP64 GPU form (0: skip)")
    ap.add_argument("--ref-rows", type=int, default=6000,
                    help="rows of the oracle's sample per step of --impl reference")
    ap.add_argument("--ref-full-rows", type=int, default=WORKLOAD["N"],
                    help="rows of the one timed full training of --impl reference "
                         "(the workload's N; smaller only to test the arm)")
    ap.add_argument("--rows", type=int, default=None,
                    help="rows of the sparse-pixel or large workload (fewer only for profiling "
                         "captures; the oracle check needs the full size)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sparse_pixels",
                    help="the timed workload (the default is the headline configuration)")
    ap.add_argument("--shard", choices=["none", "rows"], default="none",
                    help="rows: one training with the rows of H split over the ranks")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch choices instead of tuning them first")
    ap.add_argument("--lanes", type=int, default=0,
                    help="batched mixed trainings: problems whose factorisation, solves and "
                         "refinement run at once (0: the library's default, 4)")
    ap.add_argument("--block-split", type=int, default=0,
                    help="> 0: train by the paper's block formulae (Eqs. 19-23) with H1 the "
                         "first BLOCK_SPLIT columns instead of the rank-based route")
    ap.add_argument("--hidden", type=int, default=2000,
                    help="hidden width L of the gina_shaped workload (the paper's Table 1 "
                         "uses 500, 1000, 1500, 2000)")
    args = ap.parse_args()
    ARGS_HIDDEN[0] = args.hidden
    if args.impl == "reference":
        return run_reference(args)
    if args.shard == "rows":
        return run_sharded(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
