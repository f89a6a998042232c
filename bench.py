#!/usr/bin/env python
"""Throughput of the batched DD NM-ROM-HR SQP solve (arXiv 2305.15163, Sec. 4.1) on GB300.

Workload (default): 128x128 interior Burgers grid on [-1,1]^2, 4x4 equal subdomains, latent
(n^O, n^G) = (6, 3), width 256, three-band masks with 8 nonzeros per band, collocation HR on 5 %
of each subdomain's residual rows, Gaussian test matrix with n_C = 24, random-init decoders,
64 parameter instances mu ~ U[0.9,1.1]^2 in one launch; FP32 evaluation, FP64 KKT / merit.
One step = one ddnm_solve_batch of the 64 instances to the paper's stopping rule
(||F||_2 < 1e-4 or 15 SQP iterations, Sec. 7.1).  metric = solves/s (instances per second).

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--config c2]
N > 1: launched by torchrun, one rank per GPU, each rank solving its own 64 instances
(weak scaling, no collective on the data path; a barrier and a max-reduction of the time only).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "DD NM-ROM-HR SQP solves/s at 1 GB300 (rel err ≤1e-4 vs FOM); % HBM roofline"
UNIT = "solves/s"
FLUSH_BYTES = 512 << 20          # > 129 MB L2
SMS, FP32_LANES, FP64_PER_CLK = 152, 128, 2   # GB300: SMs, FP32 lanes / SM, DFMA / clk / SM
SM_MAX_MHZ = 2070.0


def eval_traffic_profile():
    """DRAM bytes per launch of the evaluation kernel on this workload from the committed ncu summary, if it
    was taken on the current kernel source (same SHA-256), else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_eval_c2.md")
    src = os.path.join(ROOT, "paper_2305_15163_gb300", "csrc", "ddnm_kernels.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"kernel source sha256: ([0-9a-f]{64})", text)
    m_b = re.search(r"dram bytes per launch: ([0-9]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return int(m_b.group(1))


def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except OSError:
        pass
    mhz = float(p.get("sm_max_mhz", SM_MAX_MHZ))
    return dict(hbm_gbs=float(p.get("hbm_gbs", 6800.0)), hbm_src="measured" if "hbm_gbs" in p else "fallback",
                fp32_tflops=SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12,
                fp64_tflops=SMS * FP64_PER_CLK * 2 * mhz * 1e6 / 1e12)


# ------------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        self.t0 = self.t1 = None

    def mark(self, start: bool):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm, mx, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                ts = time.mktime(time.strptime(r[0].strip().split(".")[0], "%Y/%m/%d %H:%M:%S"))
            except ValueError:
                ts = None
            if ts is not None and self.t0 is not None and not (self.t0 - 1.0 <= ts <= (self.t1 or ts) + 1.0):
                continue
            n += 1
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                pass
            for k, nm in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


def gpu_id_for(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ------------------------------------------------------------------------ oracle (CPU) leg

def _oracle_worker(args):
    name, idx = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import setup as osetup
    wl = inputs.workload(name)
    _, _, rom, _ = osetup.build(wl)
    mu = inputs.mu_batch(wl.batch)
    t0 = time.perf_counter()
    res = [rom.solve(mu[i % wl.batch]) for i in idx]
    return time.perf_counter() - t0, len(res), [r.n_evals for r in res]


def oracle_sample(name: str, per_worker: int = 1, workers: int | None = None):
    """Oracle solves of the same workload on the host cores: one spawn process per core, each
    single-threaded (BLAS threads pinned to 1), each solving ``per_worker`` instances."""
    workers = workers or max(1, min(os.cpu_count() or 1, 16))
    env = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        ctx = mp.get_context("spawn")
        jobs = [(name, [w * per_worker + k for k in range(per_worker)]) for w in range(workers)]
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            out = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    solved = sum(o[1] for o in out)
    busy = max(o[0] for o in out)          # solve phase (after each worker's own set-up)
    return dict(value=solved / busy, unit=UNIT, cores=workers, kind="oracle",
                sample=f"{solved} instances of workload {name} (first {solved} mu), one spawn process per core, "
                       f"single-threaded numpy/scipy FP64, paper's stopping rule; {busy:.1f} s solve phase, "
                       f"{wall:.1f} s wall with set-up")


# ------------------------------------------------------------------------ replicas over ranks

def shard(mu_all: np.ndarray, rank: int, world: int) -> np.ndarray:
    """This rank's instances: the global batch cut into `world` equal consecutive pieces (replicas, weak
    scaling: every rank solves its own piece, no collective on the data path)."""
    B = len(mu_all) // world
    return mu_all[rank * B:(rank + 1) * B]


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the job's time), by an all-reduce MAX; the value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job units per second: the units all ranks processed over the slowest rank's time."""
    return per_rank * world * steps / seconds


# ------------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = args.config
    steps = max(1, min(args.steps, 3))
    vals = []
    base = None
    for _ in range(steps):
        base = oracle_sample(cfg)
        vals.append(base["value"])
    v = statistics.median(vals)
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "steps_requested": args.steps, "warmup": 0, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(cfg),
            "cpu_baseline": base, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(cfg):
    wl = inputs.workload(cfg)
    return {"workload": f"{cfg}: Burgers {wl.nx}x{wl.ny} on [-1,1]^2, {wl.kx}x{wl.ky} subdomains, latent "
                        f"({wl.n_omega[0]},{wl.n_gamma[0]}), width {wl.width[0]}, mask 3x{wl.band}, HR "
                        f"{100 * wl.hr_frac[0]:.0f}% rows, n_C {wl.n_c()}, {wl.batch} mu per GPU, random-init decoders",
            "global_batch": wl.batch, "l2": "flushed (512 MiB write) before every timed step",
            "stopping": "||F||_2 < 1e-4 or 15 SQP iterations (Sec. 7.1)"}


# ------------------------------------------------------------------------ learned warm start (c4)

def run_warmstart(args, lib, torch, name="c2", n_train=4096, n_test=1024, epochs=60):
    """MLP 2 -> 256 -> 256 -> n_D trained on n_train SQP solutions of workload `name` (paper's stopping rule,
    default start), judged on n_test held-out mu: iterations the SQP needs from the learned start to reach
    the merit the default start ends with after 15 iterations, final merits, and solves/s of the
    warm-started mixed-precision solve next to the plain mixed and the plain FP64 solves on the same GPU."""
    wl = inputs.workload(name)
    B = wl.batch
    s = lib.Solver(wl)
    dec_o, dec_g = inputs.decoders_for(wl, [d["interior"] for d in s.subs], [d["interface"] for d in s.subs])
    Cm = inputs.test_matrix(wl.n_c(), s.sizes.N_A)
    s.load(dec_o, dec_g, Cm)
    s.options()
    nD = s.sizes.n_D

    def solve_all(solver, mu):
        xs, sts = [], []
        for b0 in range(0, len(mu), B):
            x, lam, st = solver.solve(mu[b0:b0 + B])
            xs.append(x)
            sts.append(st)
        return np.concatenate(xs), np.concatenate(sts)

    plan, _ = lib.ddnm_autotune(s.ctx, inputs.mu_batch(B, seed=3003), max_iter=2, reps=1)
    t0 = time.perf_counter()
    mu_tr = inputs.mu_batch(n_train, seed=1001)
    x_tr, _ = solve_all(s, mu_tr)
    t_data = time.perf_counter() - t0
    H = 256
    lib.ddnm_ws_init(s.ctx, H, inputs.mlp_init(2, H, nD))
    t0 = time.perf_counter()
    losses = lib.ddnm_ws_train(s.ctx, mu_tr, x_tr, epochs, 64, 2e-3, inputs.mlp_order(n_train, epochs))
    t_train = time.perf_counter() - t0
    mu_te = inputs.mu_batch(n_test, seed=2002)

    def timed(solver, mu):
        solve_all(solver, mu[:B])          # untimed: captures the solve graph for these options and this start
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st = solve_all(solver, mu)
        torch.cuda.synchronize()
        return len(mu) / (time.perf_counter() - t), st

    lib.ddnm_ws_enable(s.ctx, False)
    solve_all(s, mu_te[:B])
    v_plain, st_plain = timed(s, mu_te)
    lib.ddnm_ws_enable(s.ctx, True)
    v_ws, st_ws = timed(s, mu_te)
    reach = np.full(len(mu_te), -1)
    for K in (1, 2, 3, 4, 6, 8, 11, 15):
        s.options(tol=0.0, max_iter=K)
        _, st = solve_all(s, mu_te)
        newly = (st["merit"] <= st_plain["merit"]) & (reach < 0)
        reach[newly] = K
    # throughput at equal final merit: the learned start with the iteration budget that reaches the
    # default start's 15-iteration merit for every held-out instance
    k_eq = int(reach.max()) if (reach > 0).all() else 15
    s.options(tol=0.0, max_iter=k_eq)
    v_ws_eq, st_ws_eq = timed(s, mu_te)
    s.options()
    lib.ddnm_ws_enable(s.ctx, False)
    # plain FP64 solve of the same workload on the same GPU
    s64 = lib.Solver(wl, precision=lib.DDNM_FP64)
    s64.load(dec_o, dec_g, Cm)
    lib.ddnm_set_tune(s64.ctx, **plan)
    s64.options()
    solve_all(s64, mu_te[:B])
    n64 = max(B, len(mu_te) // 4)
    v_fp64, st_fp64 = timed(s64, mu_te[:n64])
    reached = reach > 0
    line = {"metric": METRIC + " [mixed + learned warm start at the plain solve's final merit]", "value": v_ws_eq,
            "unit": UNIT, "n_gpus": 1, "steps": len(mu_te) // B, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 eval / f64 KKT",
            "data": "synthetic",
            "config": {"workload": f"learned warm start on the {wl.nx}x{wl.ny} {wl.kx}x{wl.ky} setup ({name}), MLP "
                                   f"2-256-256-{nD} (bf16 weights, fp32 accumulation), {n_train} training "
                                   f"solutions, {n_test} held-out mu, batches of {B}",
                       "launch_plan": plan, "fp64_timed_on": n64},
            "warm_start": {"train_seconds": t_train, "data_seconds": t_data, "epochs": epochs,
                           "loss_first_last": [float(losses[0]), float(losses[-1])],
                           "fraction_reaching_plain_final_merit": float(reached.mean()),
                           "mean_iters_to_plain_final_merit": float(reach[reached].mean()) if reached.any() else None,
                           "plain_iters": float(st_plain["iters"].mean()),
                           "median_final_merit_plain": float(np.median(st_plain["merit"])),
                           "median_final_merit_warm": float(np.median(st_ws["merit"])),
                           "fallback_fraction": float(np.mean(st_ws["flags"] & lib.DDNM_FLAG_WS_FALLBACK > 0)),
                           "solves_per_s_plain_mixed": v_plain, "solves_per_s_warm_mixed": v_ws,
                           "equal_merit_iters": k_eq, "solves_per_s_warm_mixed_equal_merit": v_ws_eq,
                           "equal_merit_holds": bool(np.all(st_ws_eq["merit"] <= st_plain["merit"])),
                           "solves_per_s_plain_fp64": v_fp64,
                           "median_final_merit_plain_fp64": float(np.median(st_fp64["merit"]))}}
    print(json.dumps(line))
    s.close()
    s64.close()


# ------------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plan", default="auto",
                    help="launch plan: auto (autotuned on the workload), host (host-driven passes), "
                         "or chains,con_split,eval_persist for the graph-resident loop")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2305_15163_gb300 as lib

    if args.config == "c4":
        torch.cuda.set_device(0)
        return run_warmstart(args, lib, torch)
    if args.config == "c5":
        torch.cuda.set_device(0)
        return run_warmstart(args, lib, torch, name="c5", n_train=2048, n_test=1024, epochs=60)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # CPU baseline first (spawn pool, before heavy GPU work), rank 0 at N = 1 only
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.config)

    wl = inputs.workload(args.config)
    B = wl.batch
    s = lib.Solver(wl, device=local)
    dec_o, dec_g = inputs.decoders_for(wl, [d["interior"] for d in s.subs], [d["interface"] for d in s.subs])
    Cm = inputs.test_matrix(wl.n_c(), s.sizes.N_A)
    s.load(dec_o, dec_g, Cm)
    s.options()
    mu = shard(inputs.mu_batch(B * world), rank, world)
    dev = torch.device("cuda", local)
    nD, nC = s.sizes.n_D, s.sizes.n_C
    mu_d = torch.from_numpy(mu).to(dev)
    x_d = torch.zeros((B, nD), dtype=torch.float64, device=dev)
    l_d = torch.zeros((B, nC), dtype=torch.float64, device=dev)
    st_d = torch.zeros(B * 32, dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        lib.ddnm_solve_batch(s.ctx, B, mu_d, None, None, x_d, l_d, None, st_d)

    # launch plan: the autotuner times candidate plans on this very batch (untimed here)
    if args.plan == "auto":
        plan, tune_ms = lib.ddnm_autotune(s.ctx, mu, reps=3)
        plan_info = dict(plan, source="autotuned on this workload", tune_median_ms_per_solve=round(tune_ms, 4))
    elif args.plan == "host":
        lib.ddnm_set_tune(s.ctx, graph=0)
        plan_info = dict(lib.ddnm_get_tune(s.ctx), source="host-driven passes")
    else:
        ch, sp, pe = (int(v) for v in args.plan.split(","))
        lib.ddnm_set_tune(s.ctx, graph=1, chains=ch, con_split=sp, eval_persist=pe)
        plan_info = dict(lib.ddnm_get_tune(s.ctx), source="--plan")

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    st_warm = np.frombuffer(st_d.cpu().numpy().tobytes(), dtype=lib.STATS_DTYPE).copy()

    clocks = Clocks(gpu_id_for(local))
    time.sleep(0.3)
    tm0 = lib.ddnm_get_timing(s.ctx)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark(True)
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    if dist:
        dist.barrier()
    tm1 = lib.ddnm_get_timing(s.ctx)
    clk = clocks.stop()
    launch_keys = ("eval_launches", "constraint_launches", "step_launches", "other_launches")
    gpu_launches = sum(tm1[k] - tm0[k] for k in launch_keys)
    t_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_max = max_over_ranks(t_ms, dist, dev)
    st = np.frombuffer(st_d.cpu().numpy().tobytes(), dtype=lib.STATS_DTYPE).copy()
    deterministic = bool(np.array_equal(st["n_evals"], st_warm["n_evals"]))
    value = job_throughput(B, world, args.steps, t_max / 1000.0)

    # roofline of the dominant kernel: per-kernel device time from the library's CUDA events, taken in a
    # separate run of the same solves through the host-driven loop (events around every launch)
    # (non-persistent evaluation, so that every launch covers its whole grid alone on the GPU)
    kb = max(3, args.steps // 4)
    plan_now = lib.ddnm_get_tune(s.ctx)
    lib.ddnm_set_tune(s.ctx, **dict(plan_now, graph=0, eval_persist=0))
    lib.ddnm_timing_enable(s.ctx, True)
    for _ in range(kb):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    tm = lib.ddnm_get_timing(s.ctx)
    lib.ddnm_timing_enable(s.ctx, False)
    lib.ddnm_set_tune(s.ctx, **plan_now)
    work = lib.ddnm_get_work(s.ctx)
    pk = peaks()
    evals_per_step = float(st["n_evals"].sum())
    kern = {"k_eval": tm["eval_ms"], "k_constraint": tm["constraint_ms"], "k_kkt": tm["step_ms"]}
    dom = max(kern, key=kern.get)
    if dom == "k_eval":
        fl = work["eval_flops"] * evals_per_step * kb
        peak, bound, unit = pk["fp32_tflops"], "alu", "TFLOP/s"
        launches = tm["eval_launches"]
    elif dom == "k_constraint":
        fl = work["constraint_fp64_flops"] * evals_per_step * kb
        peak, bound, unit = pk["fp64_tflops"], "alu", "TFLOP/s"
        launches = tm["constraint_launches"]
    else:
        fl = work["step_fp64_flops"] * float(st["iters"].sum()) * kb
        peak, bound, unit = pk["fp64_tflops"], "alu", "TFLOP/s"
        launches = tm["step_launches"]
    achieved = fl / (kern[dom] / 1000.0) / 1e12
    roof = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": None,
            "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 x sm_max_mhz" if dom == "k_eval"
            else "derived: 152 SMs x 2 DFMA/clk x 2 x sm_max_mhz",
            "launches": launches, "flops_per_launch": fl / max(launches, 1),
            "avg_launch_us": 1000.0 * kern[dom] / max(launches, 1),
            # algorithmic bytes of the evaluation launches: shared tables once per launch, the instance
            # bytes per instance-evaluation
            "hbm_frac_of_measured": ((work["table_bytes"] * tm["eval_launches"] + work["instance_bytes"] * evals_per_step * kb)
                                     / (tm["eval_ms"] / 1000.0) / 1e9) / pk["hbm_gbs"],
            "eval_algorithmic_bytes_per_launch": (work["table_bytes"] * tm["eval_launches"]
                                                  + work["instance_bytes"] * evals_per_step * kb) / max(tm["eval_launches"], 1),
            "kernel_ms_per_step": {k: round(v / kb, 4) for k, v in kern.items()},
            "timed_in": f"{kb} extra solves, host-driven loop, one CTA per item, CUDA events around every launch"}
    prof = eval_traffic_profile()
    if dom == "k_eval" and prof is not None:
        roof["traffic"] = prof
        roof["traffic_source"] = "profiles/k_eval_c2.md (ncu dram__bytes_read.sum + dram__bytes_write.sum per launch)"

    # end to end through the public API with host (pinned) buffers, copies inside the timed region
    mu_h = torch.from_numpy(mu.copy()).pin_memory()
    x_h = torch.zeros((B, nD), dtype=torch.float64).pin_memory()
    l_h = torch.zeros((B, nC), dtype=torch.float64).pin_memory()
    st_h = np.zeros(B, dtype=lib.STATS_DTYPE)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lib.ddnm_solve_batch(s.ctx, B, mu_h.numpy(), None, None, x_h.numpy(), l_h.numpy(), None, st_h)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": job_throughput(B, world, e2e_steps, t_e2e), "unit": UNIT, "h2d_bytes_per_step": int(mu.nbytes),
           "d2h_bytes_per_step": int(x_h.numel() * 8 + l_h.numel() * 8 + st_h.nbytes)}

    cfg = workload_config(args.config)
    cfg["launch_plan"] = plan_info
    cfg.update({"converged_fraction": float(np.mean(st["status"] == lib.DDNM_CONVERGED)),
                "mean_iters": float(st["iters"].mean()), "mean_evals": float(st["n_evals"].mean()),
                "median_final_merit": float(np.median(st["merit"])), "deterministic_across_steps": deterministic,
                "parallelism": f"replicas: {world} GPU(s), {B} mu each"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 eval / f64 KKT", "data": "synthetic",
            "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(gpu_launches),
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line))
    s.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
