"""Benchmark: FMM velocity + stretching throughput on GB300.

Default workload: N = 128^3 = 2,097,152 Gaussian vortex blobs on the lattice
of the periodic cube [0, 2pi)^3 with Taylor-Green strengths, sigma = 1.2h,
p = 10, theta = 0.4, ncrit = 64, 27 explicit images + 2 lattice rings.
A step = one full fmm_eval_velocity_stretching call (tree build, upward
pass, traversal, M2L, downward pass, P2P) on inputs resident in HBM; L2 is
flushed (512 MB write) before every timed step.  `e2e` is the same metric
through fmm_eval_velocity_stretching_host with pinned host buffers (copies
in the timed region).  Multi-GPU: independent replicas (one problem per GPU,
no collective); value = total particles / max-over-ranks time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fmm|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM Biot-Savart+stretching particles/s at rel-L2<=1e-4"
UNIT = "particles/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# FP32 flops per P2P pair counted from the CUDA source of the packed pair
# kernel (per element; FMA = 2): difference 3, r^2 5, S and T' = -T/3 (near
# 20 / mid 19 / far 3: 1/r^2, 1/r^3, ex2 argument, degree-4 Horner in 1/r, S,
# T'; near adds the series test), T' (gamma_i . d) 6, the four accumulated
# sums 24; plus MUFU ops (rsqrt and ex2; far pairs rsqrt only).  The
# near-class series branch (rho^2 < 2) is not counted.
P2P_FLOPS = {"near": 56, "mid": 55, "far": 41}
# FP32-pipe instructions per pair (FMA, MUL and ADD alike), for the pipe-slot
# utilisation reported beside the flop rate.
P2P_SLOTS = {"near": 34, "mid": 33, "far": 25}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fmm", choices=["fmm", "reference"])
    ap.add_argument("--n-side", type=int, default=128)
    ap.add_argument("--m2l", default="auto", choices=["auto", "simt", "tensor"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-targets", type=int, default=48)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer runs (profiling)")
    ap.add_argument("--workload", default="taylor-green", choices=["taylor-green", "batched", "serving"],
                    help="taylor-green: the 128^3 periodic evaluation (default); batched: 512 independent "
                         "free-space problems; serving: a Poisson request stream")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving run of the default line")
    ap.add_argument("--no-config3", action="store_true", help="skip the 512^3 spectrum run of the default line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched run of the default line")
    ap.add_argument("--no-reuse", action="store_true", help="skip the tree-reuse / graph-replay run")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP32 throughput probe (profiling runs)")
    ap.add_argument("--serving-seconds", type=float, default=1.0, help="arrival horizon of the serving run")
    ap.add_argument("--serving-rate", type=float, default=200.0, help="mean arrivals per second")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
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
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def job_time(t_step_ms, dist=None):
    """Max over ranks of the per-step time (each rank runs its own replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_step_ms)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_step_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank, world, t_step_ms):
    """Whole-job throughput: all ranks' particles over the slowest rank's step time."""
    return world * n_per_rank / (t_step_ms * 1e-3)


def bf16_peak():
    """Dense BF16 tensor rate: the measured burst figure, else the recipe's fallback."""
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        try:
            return float(json.load(open(mp))["bf16_tflops"]), "measured (MEASURED_PEAKS.json, burst)"
        except Exception:
            pass
    return 1900.0, "fallback (no MEASURED_PEAKS.json)"


def p2p_roofline(st, p2p_ms, traffic=None):
    """FP32-pipe roofline of the P2P kernel from its CUDA-event time (ms per launch)."""
    p2p_t = p2p_ms * 1e-3
    flops = (P2P_FLOPS["near"] * st.p2p_pairs_near + P2P_FLOPS["mid"] * st.p2p_pairs_mid
             + P2P_FLOPS["far"] * st.p2p_pairs_far)
    slots = (P2P_SLOTS["near"] * st.p2p_pairs_near + P2P_SLOTS["mid"] * st.p2p_pairs_mid
             + P2P_SLOTS["far"] * st.p2p_pairs_far)
    clk_mhz = 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * clk_mhz * 1e6 / 1e12
    achieved = flops / p2p_t / 1e12
    return {"bound": "alu", "kernel": "k_p2p_x2", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "flops_per_pair": P2P_FLOPS, "pairs_per_launch": st.p2p_pairs,
            "pairs_by_class": {"near": st.p2p_pairs_near, "mid": st.p2p_pairs_mid, "far": st.p2p_pairs_far},
            "ms_per_launch": p2p_ms,
            "fp32_pipe_slot_frac": slots / p2p_t / (SM_COUNT * FP32_LANES_PER_SM * clk_mhz * 1e6),
            "peak_note": "152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz (derived from unit counts and the "
                         "maximum clock)"}


def m2l_roofline(st, p):
    """Tensor roofline of the M2L phase: the products issued per M2L pair are
    2 P x 3 components x (3 K3 + (P - K3)), K3 = the source coefficients that take
    all three split products (the rest take hi x hi only); peak = the dense BF16 rate.
    `issued` counts what the tensor pipe executes instead: every MMA of 128 rows x 192
    columns x 16 (BF16 path), padding rows above P and empty tile slots included."""
    P = int(p) ** 2
    if not (st.ms_m2l > 0 and st.m2l_tensor):
        return None
    peak, src = bf16_peak()
    k3 = int(st.m2l_split_coefs) or P
    ach = 2.0 * P * 3 * (3 * k3 + (P - k3)) * st.m2l_pairs / (st.ms_m2l * 1e-3) / 1e12
    out = {"bound": "tensor", "kernel": "k_m2l_tc", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
           "frac": ach / peak, "peak_source": src, "ms": st.ms_m2l, "split_coefs": k3,
           "flops": "2 P x 3 components x (3 K3 + (P - K3)) per M2L pair (useful rows only)"}
    if k3 % 16 == 0 or k3 == P:  # BF16 path: K steps of 16
        ks = (P + 15) // 16
        k3s = min(ks, (k3 + 15) // 16)
        mmas = (3 * k3s + (ks - k3s)) * ((P + 127) // 128)
        iss = 2.0 * 128 * 192 * 16 * mmas * st.m2l_steps / (st.ms_m2l * 1e-3) / 1e12
        out["issued"] = {"achieved": iss, "frac": iss / peak, "mmas_per_step": mmas,
                         "what": "2 x 128 x 192 x 16 per MMA x MMAs per step x steps"}
    return out


PHASES = ("ms_tree", "ms_upward", "ms_traverse", "ms_m2l", "ms_downward", "ms_p2p", "ms_total")
WORK = ("ncells", "nleaves", "nlevels", "p2p_cell_pairs", "p2p_pairs", "m2l_pairs", "m2l_steps", "m2l_keys",
        "m2l_split_coefs", "m2l_stage_chunks",
        "m2l_built", "m2l_tensor")


def workload(n_side):
    import workloads
    return workloads.taylor_green(n_side)


def cpu_baseline(w, vel_gpu, n_targets):
    """Oracle leg: FP64 direct sum (C, OpenMP) on sampled targets + accuracy of the GPU result."""
    import numpy as np
    from oracle import direct as od
    from oracle import periodic as op
    od.build()
    n = w["pos"].shape[0]
    rng = np.random.default_rng(7)
    tgt = rng.choice(n, size=n_targets, replace=False)
    imgs = op.image_shifts(w["box_len"], 1)
    t0 = time.perf_counter()
    od.direct(w["pos"][tgt], w["gamma"][tgt], w["pos"], w["gamma"], float(w["sigma"]), images=imgs)
    dt = time.perf_counter() - t0
    out = {"value": n_targets / dt, "unit": UNIT, "cores": od.num_threads(), "kind": "oracle",
           "sample": "FP64 direct sum of Eqs. 1-3 (plain C, OpenMP) for %d sampled targets against all %d "
                     "sources in the 27 explicit periodic images (no lattice far field); value = targets/s"
                     % (n_targets, n)}
    acc = None
    if vel_gpu is not None:
        u_ref, _ = op.taylor_green(w["pos"].astype(np.float64), w["gamma"].astype(np.float64), float(w["sigma"]))
        d = vel_gpu.astype(np.float64) - u_ref
        acc = float(np.linalg.norm(d) / np.linalg.norm(u_ref))
    return out, acc


def cpu_fmm_baseline():
    """The oracle's plain FP64 FMM (Cartesian Taylor expansions, numpy) timed on the host:
    the 4096-blob jittered lattice in full (p=6, theta 0.5, ncrit 32, free space), and a
    4096-blob Taylor-Green lattice (16^3) with the benchmark's parameters (p=10, theta 0.4,
    ncrit 64, periodic, 3 image levels) -- the 128^3 evaluation would take hours in it."""
    import workloads
    from oracle import fmm as ofmm
    out = {}
    for key, w, args, kw in (
            ("jittered_lattice_16", workloads.jittered_lattice(16), (6, 0.5, 32), {}),
            ("taylor_green_16_p10", workloads.taylor_green(16), (10, 0.4, 64), None)):
        if kw is None:
            kw = dict(periodic=True, box_min=w["box_min"], box_len=w["box_len"], images=3)
        t0 = time.perf_counter()
        ofmm.fmm(w["pos"], w["gamma"], float(w["sigma"]), *args, **kw)
        dt = time.perf_counter() - t0
        n = w["pos"].shape[0]
        out[key] = {"particles_per_s": n / dt, "seconds": dt, "n": n, "p": args[0], "theta": args[1],
                    "ncrit": args[2], "threads": "numpy (BLAS calls may use several cores)"}
    return out


def run_reference(args, rank, world):
    """Reference arm: the oracle as it stands, on the host cores, same workload/metric."""
    if rank != 0:
        return
    import numpy as np
    from oracle import direct as od
    from oracle import periodic as op
    w = workload(args.n_side)
    od.build()
    n = w["pos"].shape[0]
    imgs = op.image_shifts(w["box_len"], 1)
    rng = np.random.default_rng(11)
    per_step = max(1, args.cpu_targets // 4)
    times = []
    for it in range(args.warmup + args.steps):
        tgt = rng.choice(n, size=per_step, replace=False)
        t0 = time.perf_counter()
        od.direct(w["pos"][tgt], w["gamma"][tgt], w["pos"], w["gamma"], float(w["sigma"]), images=imgs)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "n": n, "p": 10, "theta": 0.4, "ncrit": 64, "periodic": True},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": od.num_threads(),
                             "sample": "FP64 direct sum over the 27 explicit images for %d sampled targets per "
                                       "step; value = targets/s" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVING_ORDERS = (4, 8, 12)


def serving_inputs(specs):
    """Host arrays (page-locked) of a request stream: Plummer requests take the
    first N particles of one Plummer sample (independent draws, so every prefix
    is a Plummer sample of its size), spectrum requests the random-spectrum
    lattice of their size (one per size)."""
    import numpy as np
    import torch
    import workloads
    nmax = max([r["n"] for r in specs if not r["periodic"]] + [1])
    pool = workloads.plummer(nmax, seed=workloads.BASE_SEED + 50)
    ppos = torch.from_numpy(pool["pos"]).pin_memory().numpy()
    pgam = torch.from_numpy(pool["gamma"]).pin_memory().numpy()
    spec = {}
    out = []
    for r in specs:
        n = r["n"]
        if r["periodic"]:
            m = int(round(n ** (1.0 / 3.0)))
            if m not in spec:
                w = workloads.random_spectrum(m, seed=r["seed"])
                spec[m] = (torch.from_numpy(w["pos"]).pin_memory().numpy(),
                           torch.from_numpy(w["gamma"]).pin_memory().numpy(), float(w["sigma"]))
            pos, gam, sig = spec[m]
            out.append(dict(pos=pos, gamma=gam, sigma=sig, box=(0.0, 0.0, 0.0, 2 * math.pi)))
        else:
            out.append(dict(pos=ppos[:n], gamma=pgam[:n], sigma=workloads.plummer_sigma(n), box=None))
    return out


def serve_stream(specs, inputs, workers, batching, budget, ncrit=64, keep=()):
    """Submit every request at its arrival time; per-request latency = completion - arrival.
    ncrit = 0: the server autotunes the leaf size per class on the warm-up requests.
    keep: indices of requests whose velocity is returned (for the accuracy check)."""
    import numpy as np
    from paper_1106_5273_gb300 import Server
    srv = Server(workers=workers, batching=batching, theta=0.5, ncrit=ncrit, hbm_budget_bytes=budget,
                 max_batch_particles=16 << 20)
    # warm-up (untimed): one request of every class creates the plans and operator caches
    seen = {}
    for r, x in zip(specs, inputs):
        seen.setdefault((r["p"], r["periodic"]), (r, x))
    for r, x in seen.values():
        t = srv.submit(x["pos"], x["gamma"], r["p"], x["sigma"], periodic=r["periodic"], box=x["box"])
        srv.wait(t, 600.0)
    c0 = srv.counters()
    t0 = srv.clock()
    tickets = []
    for r, x in zip(specs, inputs):
        while True:
            dt = t0 + r["t"] - srv.clock()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.001))
        tickets.append(srv.submit(x["pos"], x["gamma"], r["p"], x["sigma"], periodic=r["periodic"], box=x["box"]))
    lat, done, bsz, status, kept = [], [], [], [], {}
    for k, (r, t) in enumerate(zip(specs, tickets)):
        res, u, _ = srv.wait(t, 3600.0)
        if k in keep:
            kept[k] = u
        lat.append(res["t_done"] - (t0 + r["t"]))
        done.append(res["t_done"])
        bsz.append(res["batch_problems"])
        status.append(res["status"])
    c1 = srv.counters()
    srv.close()
    parts = sum(r["n"] for r in specs)
    span = max(done) - t0
    lat = np.array(lat) * 1e3
    return {"particles_per_s": parts / span, "makespan_s": span, "latency_ms": {
                "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "max": float(lat.max())},
            "requests": len(specs), "particles": parts, "failed": int(sum(1 for s_ in status if s_ != 0)),
            "batches": c1["batches"] - c0["batches"], "mean_batch_problems": float(np.mean(bsz)),
            "peak_device_bytes": c1["peak_bytes"], "hbm_budget_bytes": budget,
            "memory_waits": c1["memory_waits"] - c0["memory_waits"],
            "workers": workers, "batching": bool(batching), "ncrit": ncrit or "autotuned per class", "_kept": kept}


def serving_accuracy(specs, inputs, kept, ntargets=256):
    """rel-L2 of the velocity of sampled requests: Plummer requests against the FP64 direct sum
    (C, OpenMP) on sampled targets, periodic spectrum requests against the exact blob field of
    their generating modes."""
    import numpy as np
    import workloads
    from oracle import direct as od
    from oracle import periodic as op
    od.build()
    out = []
    for k, u in sorted(kept.items()):
        r, x = specs[k], inputs[k]
        n = r["n"]
        idx = np.random.default_rng(k).choice(n, size=min(ntargets, n), replace=False)
        if r["periodic"]:
            m = int(round(n ** (1.0 / 3.0)))
            w = workloads.random_spectrum(m, seed=r["seed"])
            ref, _ = op.spectral_field(w["modes"], w["uhat"], w["pos"][idx].astype(np.float64),
                                       w["gamma"][idx].astype(np.float64), float(w["sigma"]))
        else:
            # all sources, the target's own blob included: its pair adds exactly zero to u (d = 0)
            ref, _ = od.direct(x["pos"][idx], x["gamma"][idx], x["pos"], x["gamma"], float(x["sigma"]))
        e = float(np.linalg.norm(u[idx].astype(np.float64) - ref) / np.linalg.norm(ref))
        out.append({"request": k, "n": n, "p": r["p"], "kind": r["kind"], "rel_l2_u": e})
    return out


def _pick_checked(specs):
    """The smallest periodic and the two smallest free-space requests of each order."""
    keep = []
    for p in SERVING_ORDERS:
        for per, cnt in ((True, 1), (False, 2)):
            c = sorted((r["n"], k) for k, r in enumerate(specs) if r["p"] == p and r["periodic"] == per)
            keep += [k for _, k in c[:cnt]]
    return tuple(sorted(keep))


def run_serving(args, horizon=None):
    """Poisson request stream (N log-uniform in [1e4, 4e6], p in {4, 8, 12}, 30% periodic
    random-spectrum lattices, 70% Plummer clusters, theta 0.5): continuous batching against one
    request per call, both with two workers and the leaf size autotuned per class, at the
    configured rate (above what one GPU evaluates: queueing) and at 20 requests/s (below
    saturation: service time); velocity accuracy of sampled requests for both arms."""
    import workloads
    horizon = args.serving_seconds if horizon is None else horizon
    budget = 200 << 30
    out = {"hbm_budget_bytes": budget}
    for key, rate, hz in (("saturated", args.serving_rate, horizon), ("below_saturation", 20.0, 2.0)):
        specs = workloads.request_specs(rate=rate, horizon_s=hz, orders=SERVING_ORDERS)
        inputs = serving_inputs(specs)
        keep = _pick_checked(specs) if key == "saturated" else ()
        served = serve_stream(specs, inputs, 2, 1, budget, ncrit=0, keep=keep)
        plain = serve_stream(specs, inputs, 2, 0, budget, ncrit=0, keep=keep)
        ks, kp = served.pop("_kept"), plain.pop("_kept")
        entry = {"stream": "Poisson %.0f req/s for %.1f s (%d requests, %d particles), N log-uniform [1e4, 4e6], "
                           "p in {4,8,12}, 30%% periodic spectrum / 70%% Plummer, host arrays in and out"
                           % (rate, hz, len(specs), served["particles"]),
                 "continuous_batching": served, "one_request_per_call": plain,
                 "speedup_particles_per_s": served["particles_per_s"] / plain["particles_per_s"],
                 "p99_ratio": plain["latency_ms"]["p99"] / served["latency_ms"]["p99"]}
        if keep:
            entry["accuracy"] = {"continuous_batching": serving_accuracy(specs, inputs, ks),
                                 "one_request_per_call": serving_accuracy(specs, inputs, kp)}
        out[key] = entry
    out["arms"] = "both arms: 2 workers, leaf size autotuned per (p, periodic) class on the warm-up requests"
    return out


def run_batched(args, compact=False):
    """512 independent free-space problems (N log-uniform [1e3, 1e6], ball or Plummer, p in
    {4, 8, 12}, theta 0.5): one fmm_eval_batch per order, leaf size autotuned per order on a
    sample of its problems (untimed), against one fmm_eval_velocity_stretching per problem
    (ncrit 64); inputs resident in HBM.  A step evaluates all 512
    problems: the three order groups run one after the other (each group's plan is created before
    its timed evaluations and released after them, so one group's workspace is held at a time);
    the step time is the sum of the groups' mean times."""
    import numpy as np
    import torch
    import workloads
    from paper_1106_5273_gb300 import Params, Plan, autotune_ncrit, kernel_launch_count
    specs = workloads.batch_specs()
    groups = {}
    for sp in specs:
        groups.setdefault(sp["p"], []).append(sp)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    steps, warm = (2, 3) if compact else (max(1, min(args.steps, 5)), max(3, args.warmup))

    def timed(fn, nsteps, nwarm):
        for _ in range(nwarm):
            fn()
        torch.cuda.synchronize()
        ms = []
        l0 = kernel_launch_count()
        for _ in range(nsteps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms), (kernel_launch_count() - l0) // nsteps

    clocks = ClockSampler(0)
    clocks.start()
    ntot, t_b, t_p, l_b, l_p, per_group = 0, 0.0, 0.0, 0, 0, {}
    for p, lst in sorted(groups.items()):
        probs = [workloads.make_problem(sp) for sp in lst]
        off = np.zeros(len(probs) + 1, np.int64)
        for k, w in enumerate(probs):
            off[k + 1] = off[k] + w["pos"].shape[0]
        n = int(off[-1])
        pos = torch.from_numpy(np.concatenate([w["pos"] for w in probs])).cuda()
        gam = torch.from_numpy(np.concatenate([w["gamma"] for w in probs])).cuda()
        sig = np.array([w["sigma"] for w in probs], np.float32)
        del probs
        vel, dg = torch.empty_like(pos), torch.empty_like(pos)
        # leaf size measured on a sample of the group (its first 24 problems; not timed)
        ns = min(24, len(off) - 1)
        tuned, tune_ms = autotune_ncrit(Params.default(p=p, theta=0.5, ncrit=64), off[:ns + 1],
                                        pos[:int(off[ns])], gam[:int(off[ns])], sig[:ns])
        plan = Plan(n, Params.default(p=p, theta=0.5, ncrit=64))
        fb = lambda: plan.eval_batch(off, pos, gam, sigma_prob=sig, vel=vel, dgamma=dg)
        t64, _ = timed(fb, steps, warm)
        plan.close()
        plan = Plan(n, Params.default(p=p, theta=0.5, ncrit=tuned))
        tb, lb = timed(fb, steps, warm)
        st = plan.stats()
        dev_bytes = plan.device_bytes()
        plan.close()
        one = Plan(int(max(np.diff(off))), Params.default(p=p, theta=0.5, ncrit=64))

        def fp():
            for k in range(len(off) - 1):
                a, b = int(off[k]), int(off[k + 1])
                one.eval(pos[a:b], gam[a:b], sigma_uniform=float(sig[k]), vel=vel[a:b], dgamma=dg[a:b])

        tp, lp = timed(fp, 1, 1)
        one.close()
        ntot += n
        t_b += tb
        t_p += tp
        l_b += lb
        l_p += lp
        per_group[str(p)] = {"problems": len(lst), "n": n, "batched_ms": tb, "one_per_call_ms": tp,
                             "ncrit": tuned, "batched_ncrit64_ms": t64, "autotune_sample_ms": tune_ms,
                             "m2l_tensor": st.m2l_tensor, "p2p_pairs": st.p2p_pairs, "m2l_pairs": st.m2l_pairs,
                             "m2l_keys": st.m2l_keys, "device_bytes": dev_bytes}
        del pos, gam, vel, dg
        torch.cuda.empty_cache()
    clk = clocks.stop()
    return {"metric": "FMM batched evaluation particles/s (512 independent problems)", "value": ntot / (t_b * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": t_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-512-free-space", "problems": len(specs), "n_total": ntot,
                       "n_range": [1000, 1000000], "theta": 0.5,
                       "ncrit": "autotuned per order on the group's first 24 problems (one per call: 64)",
                       "l2": "flushed (512 MB write) before every timed evaluation"},
            "gpu_launches": l_b, "groups": per_group,
            "one_problem_per_call": {"value": ntot / (t_p * 1e-3), "ms_per_step": t_p, "gpu_launches": l_p},
            "speedup": t_p / t_b, "clocks": clk}


def timed_evals(fn, steps, warmup, flush, stream, stats=None):
    """CUDA-event times (ms) of fn() after warm-up, L2 flushed before each; also the phase
    stats of each step when stats (a plan) is given."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms, st = [], []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        if stats is not None:
            st.append(stats.stats())
    return ms, st


def run_tree_reuse(plan, pos, gam, sig, vel, dg, flush, stream, steps, w):
    """Strength-only re-evaluation on the kept tree (fmm_eval_strengths) and its captured CUDA
    graph (fmm_graph_launch), against the full evaluation: the vortex method puts its particles
    back on the same lattice every step and keeps the tree (Sec. 3.4)."""
    import numpy as np
    import torch
    from paper_1106_5273_gb300 import kernel_launch_count
    plan.eval(pos, gam, sigma_uniform=sig, vel=vel, dgamma=dg)
    torch.cuda.synchronize()
    ref_u = vel.clone()
    gbuf = gam.clone()
    ms_s, _ = timed_evals(lambda: plan.eval_strengths(gbuf, vel, dg), steps, 3, flush, stream)
    graph = plan.capture_graph(gbuf, vel, dg)
    l0 = kernel_launch_count()
    ms_g, _ = timed_evals(graph.launch, steps, 3, flush, stream)
    launches = (kernel_launch_count() - l0) // (steps + 3)
    torch.cuda.synchronize()
    same = bool(torch.equal(vel, ref_u)) and plan.status() == 0
    graph.close()
    n = pos.shape[0]
    t_s, t_g = sum(ms_s) / len(ms_s), sum(ms_g) / len(ms_g)
    return {"eval_strengths": {"ms_per_step": t_s, "particles_per_s": n / (t_s * 1e-3)},
            "graph_replay": {"ms_per_step": t_g, "particles_per_s": n / (t_g * 1e-3), "gpu_launches": launches,
                             "graph_launches_per_step": 1},
            "bit_identical_to_full_evaluation": same, "steps": steps,
            "note": "same positions and core widths, new strengths: tree, lists and M2L operators kept"}


def run_config3(args, steps=3, warmup=1):
    """The 512^3 random-phase spectrum workload (E(k) ~ k^4 exp(-2 (k/k0)^2), k0 = 4, u_rms = 1,
    sigma = 1.2h) in the periodic cube: p=10, theta 0.4, ncrit 64, tensor-core M2L, with its own
    clocks, phases, rooflines and rel-L2 on 4096 sampled targets against the exact blob field
    of the generating modes."""
    import numpy as np
    import torch
    import workloads
    from oracle import periodic as op
    from paper_1106_5273_gb300 import Params, Plan, kernel_launch_count
    t0 = time.perf_counter()
    w = workloads.random_spectrum(512)
    gen_s = time.perf_counter() - t0
    n = w["pos"].shape[0]
    idx = np.random.default_rng(7).choice(n, size=4096, replace=False)
    us, ss = op.spectral_field(w["modes"], w["uhat"], w["pos"][idx].astype(np.float64),
                               w["gamma"][idx].astype(np.float64), float(w["sigma"]))
    prm = Params.default(p=10, theta=0.4, ncrit=64, periodic=1, box_min=w["box_min"], box_len=w["box_len"],
                         images=5)
    plan = Plan(n, prm)
    pos = torch.from_numpy(w["pos"]).cuda()
    gam = torch.from_numpy(w["gamma"]).cuda()
    sig = float(w["sigma"])
    del w["pos"], w["gamma"]
    vel = torch.empty((n, 3), device="cuda")
    dg = torch.empty((n, 3), device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    plan.set_timing(True)
    fn = lambda: plan.eval(pos, gam, sigma_uniform=sig, vel=vel, dgamma=dg)
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = kernel_launch_count()
    ms, sts = timed_evals(fn, steps, 0, flush, stream, stats=plan)
    launches = (kernel_launch_count() - l0) // steps
    clk = clocks.stop()
    st = sts[-1]
    t = sum(ms) / len(ms)
    ti = torch.from_numpy(idx).cuda()
    u = vel[ti].cpu().numpy().astype(np.float64)
    s_ = dg[ti].cpu().numpy().astype(np.float64)
    eu = float(np.linalg.norm(u - us) / np.linalg.norm(us))
    es = float(np.linalg.norm(s_ - ss) / np.linalg.norm(ss))
    out = {"workload": "random-spectrum-512^3", "n": n, "p": 10, "theta": 0.4, "ncrit": 64, "images": 5,
           "images_note": "27 explicit images + 4 lattice levels (3^5 cells per axis): with 3 levels the truncated "
                          "lattice sum of this field leaves rel-L2(u) 1.04e-4",
           "split_tie": "source (Alg. 1 as printed)", "steps": steps, "warmup": warmup, "ms_per_step": t,
           "particles_per_s": n / (t * 1e-3), "gpu_launches": launches,
           "phases_ms": {k: float(np.mean([getattr(x, k) for x in sts])) for k in PHASES},
           "work": {k: getattr(st, k) for k in WORK},
           "roofline": p2p_roofline(st, float(np.mean([x.ms_p2p for x in sts]))),
           "roofline_m2l": m2l_roofline(st, 10),
           "accuracy": {"rel_l2_u": eu, "rel_l2_s": es, "targets": 4096,
                        "reference": "exact blob field of the generating Fourier modes (oracle)"},
           "device_bytes": plan.device_bytes(), "input_generation_s": gen_s, "clocks": clk,
           "l2": "inputs (4.3 GB) larger than L2; also flushed before every timed step"}
    plan.close()
    del pos, gam, vel, dg, flush
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.workload in ("batched", "serving") and args.impl == "fmm":
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        if int(os.environ.get("RANK", "0")) == 0:
            out = run_batched(args) if args.workload == "batched" else dict(
                metric="FMM serving particles/s (Poisson request stream)", **run_serving(args))
            print(json.dumps(out), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1106_5273_gb300 import Params, Plan, kernel_launch_count

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.n_side)
    n = w["pos"].shape[0]
    mode = {"auto": 0, "simt": 1, "tensor": 2}[args.m2l]
    prm = Params.default(p=w["p"], theta=w["theta"], ncrit=w["ncrit"], periodic=1, box_min=w["box_min"],
                         box_len=w["box_len"], images=w["images"], m2l_mode=mode)
    plan = Plan(n, prm)
    pos = torch.from_numpy(w["pos"]).cuda()
    gam = torch.from_numpy(w["gamma"]).cuda()
    vel = torch.empty((n, 3), device="cuda")
    dg = torch.empty((n, 3), device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sig = float(w["sigma"])
    for _ in range(args.warmup):
        plan.eval(pos, gam, sigma_uniform=sig, vel=vel, dgamma=dg)
    torch.cuda.synchronize()
    plan.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, p2p_ms = [], []
    launches0 = kernel_launch_count()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(pos, gam, sigma_uniform=sig, vel=vel, dgamma=dg)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        st = plan.stats()
        p2p_ms.append(st.ms_p2p)
    torch.cuda.synchronize()
    launches = (kernel_launch_count() - launches0) // args.steps
    if dist:
        dist.barrier()
    clk = clocks.stop()
    st = plan.stats()
    # the same evaluation without the stretching output (velocity-only kernels)
    vo_ms, vo_p2p = [], []
    for it in range(3 + 3):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(pos, gam, sigma_uniform=sig, vel=vel, stretching=False)
        e1.record(stream)
        e1.synchronize()
        if it >= 3:
            vo_ms.append(e0.elapsed_time(e1))
            vo_p2p.append(plan.stats().ms_p2p)
    velocity_only = {"ms_per_step": sum(vo_ms) / len(vo_ms), "ms_p2p": sum(vo_p2p) / len(vo_p2p),
                     "particles_per_s": job_value(n, world, job_time(sum(vo_ms) / len(vo_ms), dist)),
                     "steps": len(vo_ms), "note": "dgamma = NULL: P2P skips T and the stretching sums"}
    t_step = job_time(sum(ms) / len(ms), dist)
    value = job_value(n, world, t_step)
    # end to end through the host-buffer entry point (pinned memory)
    hp = torch.from_numpy(w["pos"]).pin_memory().numpy()
    hg = torch.from_numpy(w["gamma"]).pin_memory().numpy()
    hv = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
    hd = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
    plan.set_timing(False)
    e2e_ms = []
    if not args.no_e2e:
        plan.eval_host(hp, hg, sigma_uniform=sig, vel=hv, dgamma=hd)
    for _ in range(0 if args.no_e2e else max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.eval_host(hp, hg, sigma_uniform=sig, vel=hv, dgamma=hd)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_t = sum(e2e_ms) / len(e2e_ms) if e2e_ms else float("nan")
    # roofline of the dominant kernel (P2P), from its CUDA-event time inside the step
    traffic = None
    prof = os.path.join(ROOT, "profiles", "p2p_traffic.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("bytes_per_launch_full_workload")
        except Exception:
            traffic = None
    roof = p2p_roofline(st, sum(p2p_ms) / len(p2p_ms), traffic)
    if rank == 0 and not args.no_probe:
        from paper_1106_5273_gb300 import binding as _b
        pclk = ClockSampler(local)
        pclk.start()
        probe_tf, probe_ms = _b.probe_fp32_rate(1000)
        pc = pclk.stop()
        roof["peak_probe"] = {"value": probe_tf, "unit": "TFLOP/s", "frac": roof["achieved"] / probe_tf,
                              "ms_per_launch": probe_ms, "clocks": pc,
                              "what": "fmm_probe_fp32_rate: independent FFMA2 chains, 8 CTAs x 256 threads per SM, "
                                      "1000 launches timed with CUDA events"}
    roof_m2l = m2l_roofline(st, w["p"])
    reuse = None
    if rank == 0 and not args.no_reuse:
        reuse = run_tree_reuse(plan, pos, gam, sig, vel, dg, flush, stream, max(3, args.steps // 2), w)
    if rank == 0:
        cpu, acc = (None, None)
        if not args.no_cpu_baseline and world == 1:
            cpu, acc = cpu_baseline(w, vel.cpu().numpy(), args.cpu_targets)
            cpu["fmm"] = cpu_fmm_baseline()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "n": n, "p": w["p"], "theta": w["theta"], "ncrit": w["ncrit"],
                       "periodic": True, "images": w["images"], "sigma_over_h": 1.2,
                       "l2": "flushed (512 MB write) before every timed step", "m2l": args.m2l,
                       "parallelism": "replicas" if world > 1 else "single"},
            "accuracy": {"rel_l2_u_vs_closed_form": acc},
            "e2e": {"value": job_value(n, world, e2e_t), "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * n * 12), "d2h_bytes_per_step": int(2 * n * 12)},
            "gpu_launches": launches,
            "roofline": roof,
            "paper_convention_tflops": 174 * st.p2p_pairs / (roof["ms_per_launch"] * 1e-3) / 1e12,
            "roofline_m2l": roof_m2l,
            "velocity_only": velocity_only,
            "phases_ms": {k: getattr(st, k) for k in PHASES},
            "work": {k: getattr(st, k) for k in WORK},
            "clocks": clk,
            "cpu_baseline": cpu,
            "tree_reuse": reuse,
        }
        if world == 1:
            plan.close()
            del pos, gam, vel, dg
            torch.cuda.empty_cache()
            if not args.no_config3:
                line["config3"] = run_config3(args)
            if not args.no_batched:
                line["batched"] = run_batched(args, compact=True)
            if not args.no_serving:
                line["serving"] = run_serving(args)
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
