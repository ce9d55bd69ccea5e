#!/usr/bin/env python3
"""Benchmark of the wave-tank hot path on GB300.

Workload: the 2D nonlinear wave over a Gaussian bar (periodic x in [0, 32),
Nx = 1024, Nz = 24, h = 1 - 0.5 exp(-((x-16)/2)^2), second-order Stokes wave
with H/L = 0.04 and kh = 0.98 at the deep end, linear-theory velocity,
dt = 0.5 dx / sqrt(g h_max), exponential filter on, Poisson tolerance 1e-10
at every stage).  One step = one full five-stage low-storage Runge-Kutta step
(five mixed-stage Poisson solves plus the free-surface and stage updates).

Metric: RK4 DOF-updates/s = 5 stages x Nx x Ny x (Nz+1) / step time (the
headline, mixed FP32/FP64 solver) with Poisson solves/s, and the same for the
plain FP64 solver on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (numpy float64, one thread) on a
bounded sample of the same workload (one Runge-Kutta stage per step).
"""

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

METRIC = "RK4 DOF-updates/s (mixed FP32/FP64 p-MG Poisson solves at 1e-10 residual)"
# DRAM bytes (read + write) of one FP32 operator apply, summed over its
# kernels, from one ncu capture of the same build and size (the operator-apply
# traffic summary under profiles/): 2D 1024 x 24, 3 launches; 3D 256 x 256 x 16,
# 5 launches.  The writes read 0 there: each output stays dirty in L2 past the
# end of its kernel.
OP_TRAFFIC_2D = 154624 + 259840 + 256768
OP_TRAFFIC_3D = 4491008 + 4493568 + 16569344 + 8947200 + 8949504
UNIT = "DOF-updates/s"
SMOOTHERS = {0: "damped block-Jacobi", 1: "mean-depth spectral", 2: "block-Jacobi then mean-depth spectral"}
STAGES = 5


def workload():
    p = si.nonlinear_2d_tank()
    x = np.arange(p["Nx"]) * p["L"] / p["Nx"]
    h = si.bump(x, p["L"], p["bump_A"], p["bump_w"])[None, :]
    return p, x, np.ascontiguousarray(h)


def config(p, extra=None):
    c = {"workload": "2D nonlinear Stokes-2 wave over a Gaussian bar (Nx=1024, Nz=24, L=32, "
                     "H/L=0.04, kh=0.98, CFL 0.5, filter on, tol 1e-10 per stage)",
         "Nx": p["Nx"], "Ny": 1, "Nz": p["Nz"], "L": p["L"], "dt": p["dt"],
         "dof_per_stage": p["Nx"] * (p["Nz"] + 1), "stages_per_step": STAGES,
         "poisson_tol": 1e-10, "l2": "flushed between timed steps (256 MiB device write)"}
    if extra:
        c.update(extra)
    return c


def initial_state(p, x, h, sigma):
    eta = si.nonlinear_2d_initial(x, None, p)
    d = h[0] + eta
    z = sigma[:, None] * d[None, :] - h[0][None, :]
    _, u, w = si.nonlinear_2d_initial(x[None, :], z, p)
    M1 = p["Nz"] + 1
    return (np.ascontiguousarray(eta[None, :]), np.ascontiguousarray(u.reshape(M1, 1, -1)),
            np.zeros((M1, 1, p["Nx"])), np.ascontiguousarray(w.reshape(M1, 1, -1)))


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every `interval_ms` while the
    timed region runs (start() returns once the first sample is written, so
    the samples cover the region that follows)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, interval_ms=20, wait_s=3.0):
        self.idx = gpu_index
        self.interval_ms = interval_ms
        self.wait_s = wait_s
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + self.wait_s
        while time.time() < deadline:
            try:
                if self.proc.poll() is not None or os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "interval_ms": self.interval_ms}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------- our arm
def over_ranks(dist, v, op, device):
    """v reduced ("max" or "sum") over the ranks of the process group `dist`
    (the torch.distributed module, or None for a single process)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(dist, device, units, ms):
    """Whole-job throughput of independent replicas (one per rank): the units
    every rank processed divided by the slowest rank's time.  Returns
    (units per second, slowest ms)."""
    ms_max = over_ranks(dist, ms, "max", device)
    total = over_ranks(dist, units, "sum", device)
    return total / (ms_max / 1e3), ms_max


def run_ours(args):
    import torch
    import paper_2406_00991_gb300 as w

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()            # the tank launches on this stream; events time it
    torch.cuda.set_stream(stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return over_ranks(dist, v, "max", dev)

    def sum_over_ranks(v):
        return over_ranks(dist, v, "sum", dev)

    p, x, h = workload()
    T = w.Tank(p["Nx"], 1, p["Nz"], p["L"], h, mode=w.WT_MIXED, tol=1e-10, filter=1)
    T.set_stream(stream.cuda_stream)
    _, _, sigma = T.grid()
    st0 = initial_state(p, x, h, sigma)
    dof_step = STAGES * p["Nx"] * (p["Nz"] + 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed_steps(K, prof_mask=0):
        """K steps, each timed by CUDA events on the tank's stream, L2 flushed before each."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        T.profile(prof_mask)
        l0 = T.launches()
        s0, i0 = T.stats()
        barrier()
        t0 = time.perf_counter()
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            T.step(p["dt"], 1)
            evs[k][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in evs]
        s1, i1 = T.stats()
        return ms, wall, T.launches() - l0, (s1 - s0, i1 - i0)

    # ---------------- mixed (headline)
    T.set_state(*st0)
    T.step(p["dt"], 1)
    # solver settings (damping, sweeps, coarsest size, mixed variant) picked by
    # the library's autotuner on this tank's own step; the state is restored
    tuned, tuned_ms, entry_ms = T.autotune_step(p["dt"], reps=2) if not args.no_tune else (T.options(), 0.0, 0.0)
    # the first warm-up step times every kernel class to find the dominant one
    T.profile((1 << len(w.KERNEL_CLASSES)) - 1)
    T.step(p["dt"], 1)
    cls_ms = []
    for c in range(len(w.KERNEL_CLASSES)):
        cls_ms.append(T.profile_read(c))
    T.profile(0)
    dom = int(np.argmax([c["ms"] for c in cls_ms]))
    for _ in range(max(0, args.warmup - 1)):
        T.step(p["dt"], 1)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms, wall, launches, (solves, iters) = timed_steps(args.steps)          # graphs, no events
    ck = clocks.stop()
    value, step_ms = replica_throughput(dist, dev, dof_step, float(np.mean(ms)))
    solves_s = sum_over_ranks(STAGES) / (step_ms / 1e3)
    # the unit whose algorithmic traffic the roofline counts: one FP32 operator
    # apply A_{a,b} p (read p, write Ap: 8 B per DOF) on this tank's geometry,
    # and the FP32 V-cycle, each timed as one CUDA graph of many units between
    # two events (no per-launch events to inflate them)
    eta0 = np.ascontiguousarray(st0[0])
    op_ms, op_launches = T.time_kernel(eta0, eta0, w.WT_TIME_OPERATOR, w.WT_FP32, reps=400)
    vc_ms, vc_launches = T.time_kernel(eta0, eta0, w.WT_TIME_VCYCLE, w.WT_FP32, reps=50)

    # ---------------- end to end through the C ABI with pinned host buffers
    host = [torch.from_numpy(a.copy()).pin_memory().numpy() for a in st0]
    out_eta = torch.zeros(host[0].shape, dtype=torch.float64).pin_memory().numpy()
    out_u = torch.zeros(host[1].shape, dtype=torch.float64).pin_memory().numpy()
    out_w = torch.zeros(host[3].shape, dtype=torch.float64).pin_memory().numpy()
    Ke = max(1, min(args.steps, 3))
    barrier()
    e2e_ms = []
    se, ie = 0, 0
    for k in range(Ke):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w.wt_set_state(T.handle, host[0], host[1], host[2], host[3], 0.0)
        T.step(p["dt"], 1)
        w.wt_get_state(T.handle, out_eta, out_u, None, out_w)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        s_k, i_k = T.stats()                 # wt_set_state restarts the counters
        se, ie = se + s_k, ie + i_k
    e2e_step = max_over_ranks(float(np.mean(e2e_ms)))
    # the copies alone (state in and out, no step), to split the end-to-end time
    copy_ms = []
    for k in range(Ke):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w.wt_set_state(T.handle, host[0], host[1], host[2], host[3], 0.0)
        w.wt_get_state(T.handle, out_eta, out_u, None, out_w)
        copy_ms.append((time.perf_counter() - t0) * 1e3)
    bytes_io = 8 * (host[0].size + host[1].size + host[3].size)

    # ---------------- plain FP64 solver on the same GPU (FP64 arithmetic throughout)
    T.set_options(mode=w.WT_FP64, df64=0)
    T.set_state(*st0)
    T.step(p["dt"], 1)
    Kf = max(1, min(args.steps, 3))
    ms64, _, _, (s64, it64) = timed_steps(Kf)
    step64 = max_over_ranks(float(np.mean(ms64)))

    if rank != 0:
        return
    hbm, peak_src = peaks()
    dof = p["Nx"] * (p["Nz"] + 1)
    op_bytes = 8.0 * dof
    achieved = op_bytes / (op_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": config(p, {"parallelism": "replicas" if world > 1 else "single-gpu",
                             "solver": ("mixed: FP64 flexible GMRES(30) preconditioned by the FP32 p-multigrid V-cycle"
                                        if tuned["mode"] == w.WT_MIXED else
                                        "refine: FP64 iterative refinement around FP32 FGMRES + FP32 V-cycle"),
                             "smoother": SMOOTHERS.get(tuned["smoother"], "?") + (
                                 " (spectral on levels of >= %d unknowns, block-Jacobi below)" % tuned["spectral_min"]
                                 if tuned["smoother"] and tuned["spectral_min"] else ""),
                             "autotuned": {"omega": tuned["omega"], "nu1": tuned["nu1"], "nu2": tuned["nu2"],
                                           "coarsest_max": tuned["coarsest_max"], "mode": tuned["mode"],
                                           "tail_max": tuned["tail_max"], "tail_cluster": tuned["tail_cluster"],
                                           "vcycle_grid": tuned["vcycle_grid"], "smoother": tuned["smoother"],
                                           "omega_s": tuned["omega_s"], "spectral_min": tuned["spectral_min"],
                                           "cycle": tuned["cycle"], "inner_tol": tuned["inner_tol"],
                                           "pdl": tuned["pdl"],
                                           "tuned_ms_per_step": tuned_ms, "default_ms_per_step": entry_ms}}),
        "solves_per_s": solves_s,
        "krylov_iterations_per_solve": iters / max(1, solves),
        "fp64": {"value": dof_step * world / (step64 / 1e3),
                 "unit": UNIT, "ms_per_step": step64, "solves_per_s": STAGES * world / (step64 / 1e3),
                 "krylov_iterations_per_solve": it64 / max(1, s64), "steps": Kf},
        "mixed_over_fp64": step64 / step_ms,
        "e2e": {"value": dof_step * world / (e2e_step / 1e3), "unit": UNIT,
                "ms_per_step": e2e_step, "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                "krylov_iterations_per_solve": ie / max(1, se),
                "copies_ms": float(np.mean(copy_ms)),
                "gap_note": "every end-to-end step starts from the host state with the pressure warm start "
                            "cleared (wt_set_state), so its five solves start cold: more iterations per "
                            "solve than the device-timed steps; copies_ms is the state in and out alone",
                "note": "wt_set_state(host) + wt_step + wt_get_state(host), pinned buffers"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "FP32 operator apply A_{a,b} p (x-row pass, sigma columns, "
                                                "x-row pass: %d launches)" % op_launches,
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": OP_TRAFFIC_2D,
                     "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak_src == "measured"
                                     else peak_src),
                     "algorithmic_bytes_per_apply": op_bytes, "apply_us": op_ms * 1e3,
                     "timing": "one CUDA-event pair around a graph of 400 applies on the tank's stream",
                     "note": "the 1024 x 25 FP32 field (100 KB) is L2-resident; the apply is bound by "
                             "launch and per-phase latency, not by HBM"},
        "vcycle": {"ms": vc_ms, "launches": vc_launches, "precision": "fp32",
                   "timing": "one CUDA-event pair around a graph of 50 V-cycles"},
        "kernel_classes_first_warmup_step": {
            w.KERNEL_CLASSES[c]: {"ms": round(cls_ms[c]["ms"], 3), "launches": cls_ms[c]["launches"],
                                  "avg_us": round(cls_ms[c]["ms"] * 1e3 / max(1, cls_ms[c]["launches"]), 2)}
            for c in range(len(cls_ms))},
        "kernel_classes_note": "CUDA events around every launch of one warm-up step: per-launch event "
                               "overhead inflates these times; shares only (the ncu launch list in "
                               "profiles/ is the reference)",
        "clocks": ck,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, x, h, budget_s=args.cpu_budget)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_budget)
    if not args.no_extras:
        # the further workloads of the line; one that fails is reported as such
        # and does not cost the headline measurement
        sections = (("batch", lambda: bench_batch(w, torch, args)),
                    ("table1_cycles", lambda: bench_cycles(w, torch, p, h, st0)),
                    ("e2_convergence", lambda: bench_e2(w)),
                    ("adjoint", lambda: bench_adjoint(w, torch, args)),
                    ("sea3d", lambda: bench_sea3d(w, torch, args)))
        for name, fn in sections:
            try:
                line[name] = fn()
            except Exception as e:                       # noqa: BLE001
                line[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    print(json.dumps(line), flush=True)


def bench_batch(w, torch, args):
    """The batched workload: 256 uneven 2D tanks, one persistent launch per
    call, in the mixed form (FP32 V-cycle) and the plain FP64 form on the same
    GPU, each timed with CUDA events on the batch's stream."""
    tanks, redrawn = si.batch_tanks()
    st, hs = [], []
    for q in tanks:
        xq = np.arange(q["Nx"]) * q["L"] / q["Nx"]
        hq = si.bump(xq, q["L"], q["bump_A"], q["bump_w"])
        sig = (np.cos(np.pi * np.arange(q["Nz"] + 1) / q["Nz"]) + 1.0) / 2.0
        e, u, _, ww = initial_state(q, xq, hq[None], sig)
        st.append((e, u, ww))
        hs.append(hq[None])
    dts = [q["dt"] for q in tanks]
    dof = sum(STAGES * q["Nx"] * (q["Nz"] + 1) for q in tanks)
    stream = torch.cuda.current_stream()
    K = max(1, min(args.steps, 2))
    out = {"workload": "256 uneven 2D tanks (Nx 128-2048, Nz 8-32, Battjes-limited Stokes-2 waves "
                       "over Gaussian bars), one persistent launch (one CTA per tank, largest first)",
           "metric": "RK4 DOF-updates/s", "unit": UNIT, "steps": K, "tanks_redrawn": redrawn,
           "timing": "CUDA events on the batch's stream around one wt_batch_step call of K steps"}
    tuned = None
    for name, mode in (("mixed", w.WT_MIXED), ("fp64", w.WT_FP64)):
        B = w.Batch([q["Nx"] for q in tanks], [q["Nz"] for q in tanks], [q["L"] for q in tanks], hs,
                    tol=1e-10, mode=mode)
        B.set_stream(stream.cuda_stream)
        for i, s_ in enumerate(st):
            B.set_state(i, *s_)
        if tuned is None:
            # damping and sweep counts picked by the batch autotuner on one step of
            # the mixed batch (the FP64 batch runs with the same smoother settings)
            tuned, tuned_ms, entry_ms = B.autotune(dts, reps=1)
            out["autotuned"] = {"omega": tuned["omega"], "nu1": tuned["nu1"], "nu2": tuned["nu2"],
                                "tuned_ms_per_step": tuned_ms, "default_ms_per_step": entry_ms}
        else:
            B.set_options(mode=mode, tol=1e-10, omega=tuned["omega"], nu1=tuned["nu1"], nu2=tuned["nu2"])
        B.step(dts, 1)                               # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        B.step(dts, K)                               # one launch for all K steps of all tanks
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        its = [B.stats(i) for i in range(len(tanks))]
        B.close()
        out[name] = {"value": dof / (ms / 1e3), "ms_per_step": ms,
                     "solves_per_s": STAGES * len(tanks) / (ms / 1e3),
                     "krylov_iterations_per_solve": float(np.sum([a[1] for a in its]) /
                                                          max(1, np.sum([a[0] for a in its]))),
                     "max_last_rel_residual": float(max(a[2] for a in its))}
    out["value"] = out["mixed"]["value"]
    out["ms_per_step"] = out["mixed"]["ms_per_step"]
    out["solves_per_s"] = out["mixed"]["solves_per_s"]
    out["mixed_over_fp64_solves"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def bench_sea3d(w, torch, args):
    """The 3D directional sea: 256 x 256 x 16, 4096 JONSWAP components, mixed solver."""
    N, Nz, L = 256, 16, 64.0
    stream = torch.cuda.current_stream()
    sea = si.jonswap_sea(seed=3, L=L, ncomp=4096, kp=1.5, hs_over_lp=0.02)
    dt = 0.5 * (L / N) / math.sqrt(9.81)
    K = 2

    def run(**opts):
        opts.setdefault("mode", w.WT_MIXED)
        T = w.Tank(N, N, Nz, L, np.ones((N, N)), tol=1e-10, filter=1, max_it=400, **opts)
        T.set_stream(stream.cuda_stream)
        _, _, sigma = T.grid()
        eta0, u0, v0, w0 = si.jonswap_fields(sea, N, sigma)
        T.set_state(*(np.ascontiguousarray(a) for a in (eta0, u0, v0, w0)))
        T.step(dt, 1)                                # warm-up (graph capture)
        s0, i0 = T.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        T.step(dt, K)
        e1.record(stream)
        torch.cuda.synchronize()
        s1, i1 = T.stats()
        return T, e0.elapsed_time(e1) / K, (i1 - i0) / max(1, s1 - s0)

    # block-Jacobi V(2,2) (the paper's smoother family) in the mixed form, then
    # the configuration the 3D sea runs with: the mean-depth spectral smoother
    # V(1,1) inside the refinement form (FP64 residual, FP32 GMRES to 1e-4):
    # on this GPU the FP64 operator apply costs about 7 FP32 ones, so the
    # form that applies it once per refinement wins
    Tb, ms_bj, its_bj = run(omega=0.6)
    Tb.close()
    T, ms, its = run(smoother=1, nu1=1, nu2=1, mode=w.WT_REFINE, inner_tol=1e-4, spectral_min=20000)
    eta_now = np.ascontiguousarray(T.get_state()[0])
    op_ms, op_launches = T.time_kernel(eta_now, eta_now, w.WT_TIME_OPERATOR, w.WT_FP32, reps=100)
    vc_ms, vc_launches = T.time_kernel(eta_now, eta_now, w.WT_TIME_VCYCLE, w.WT_FP32, reps=10)
    T.close()
    hbm, _ = peaks()
    dof1 = N * N * (Nz + 1)
    ach = 8.0 * dof1 / (op_ms / 1e3) / 1e9
    return {"workload": "3D directional JONSWAP sea, 256 x 256 x 16, L = 64, 4096 components, filter on, "
                        "FP64 refinement (FP32 GMRES + FP32 V-cycle to 1e-4) to 1e-10, mean-depth spectral smoother V(1,1) "
                        "on the levels of >= 20,000 unknowns (block-Jacobi below), FP64 passes in double-float",
            "metric": "RK4 DOF-updates/s", "value": STAGES * dof1 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "solves_per_s": STAGES / (ms / 1e3),
            "krylov_iterations_per_solve": its, "steps": K,
            "block_jacobi": {"ms_per_step": ms_bj, "krylov_iterations_per_solve": its_bj,
                             "smoother": "damped block-Jacobi V(2,2), omega 0.6, mixed form"},
            "roofline": {"bound": "hbm", "kernel": "FP32 operator apply A_{a,b} p (%d launches)" % op_launches,
                         "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": OP_TRAFFIC_3D, "algorithmic_bytes_per_apply": 8.0 * dof1,
                         "apply_us": op_ms * 1e3,
                         "timing": "one CUDA-event pair around a graph of 100 applies"},
            "vcycle": {"ms": vc_ms, "launches": vc_launches, "precision": "fp32"},
            "timing": "CUDA events on the tank's stream around wt_step of K steps"}


def bench_cycles(w, torch, p, h, st0):
    """Table 1's comparison on the benchmark tank's geometry: iterations and
    device time per solve for V-cycle + GMRES and FMG + GMRES (Algorithms 1
    and 2 as the preconditioner) at relative residuals 1e-4, 1e-8, 1e-12, in
    the mixed and the FP64 form, on a seeded right-hand side."""
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    eta = torch.from_numpy(np.ascontiguousarray(st0[0])).to(dev)
    shape = (p["Nz"] + 1, 1, p["Nx"])
    b = torch.from_numpy(si.rng(5).standard_normal(shape)).to(dev)
    out = {"workload": "one mixed-stage Poisson problem on the 1024 x 24 bar geometry (seeded N(0,1) "
                       "right-hand side, zero initial guess)",
           "timing": "CUDA events on the tank's stream, median of 3 solves"}
    for mname, mode in (("mixed", w.WT_MIXED), ("fp64", w.WT_FP64)):
        for cname, cyc in (("vcycle", 0), ("fmg", 1)):
            T = w.Tank(p["Nx"], 1, p["Nz"], p["L"], h, mode=mode, cycle=cyc, max_it=400)
            T.set_stream(stream.cuda_stream)
            row = {}
            for tol in (1e-4, 1e-8, 1e-12):
                x = torch.zeros(shape, dtype=torch.float64, device=dev)
                _, info = T.poisson_solve(eta, eta, b, x, tol=tol, raise_noconv=False)   # warm-up
                ms = []
                for _ in range(3):
                    x.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, info = T.poisson_solve(eta, eta, b, x, tol=tol, raise_noconv=False)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                row["%.0e" % tol] = {"iterations": info.iterations, "ms": float(np.median(ms)),
                                     "rel_residual": info.rel_residual}
            T.close()
            out["%s_%s" % (mname, cname)] = row
    return out


def bench_e2(w):
    """The paper's Sec. 5.2 accuracy study: error in u after one Runge-Kutta
    step (dt = T / 1000) from an exact stream-function wave, for kh in {0.5,
    2, 2 pi} and H/L at 0.1, 0.4, 0.7 of the Battjes limit, refining Nx at
    Nz = 24 and Nz at Nx = 64 (FP64 solver at 1e-12)."""
    out = {"workload": "stream-function waves, one wavelength per tank, flat bed h = 1, FP64 solver at 1e-12",
           "error": "max |u - u_exact(dt)| / max |u_exact|", "cases": []}
    for kh in (0.5, 2.0, 2 * math.pi):
        for frac in (0.1, 0.4, 0.7):
            k = kh
            L = 2 * math.pi / k
            H = frac * 0.1401 * math.tanh(0.8863 * kh) * 2 * math.pi / k
            row = {"kh": kh, "H_over_L_battjes_fraction": frac, "Nx_at_Nz24": {}, "Nz_at_Nx64": {}}
            for key, sizes in (("Nx_at_Nz24", [(8, 24), (16, 24), (32, 24), (64, 24)]),
                               ("Nz_at_Nx64", [(64, 4), (64, 8), (64, 12), (64, 16), (64, 24)])):
                for Nx, Nz in sizes:
                    T = w.Tank(Nx, 1, Nz, L, np.ones((1, Nx)), mode=w.WT_FP64, tol=1e-12, max_it=400)
                    eta, u, ww, c = T.stream_function_wave(1, H, 32, time=0.0)
                    dt = L / c / 1000.0
                    T.set_state(eta, u, np.zeros_like(u), ww)
                    T.step(dt, 1)
                    u1 = T.get_state()[1]
                    _, ux, _, _ = T.stream_function_wave(1, H, 32, time=dt)
                    T.close()
                    row[key][str(Nx if key.startswith("Nx") else Nz)] = float(np.abs(u1 - ux).max() /
                                                                             np.abs(ux).max())
            out["cases"].append(row)
    return out


def bench_adjoint(w, torch, args):
    """Gradient workload: bathymetry and initial-surface gradient of a gauge loss."""
    from paper_2406_00991_gb300.adjoint import gauge_series
    Nx, Nz, L = 512, 20, 16.0
    dt = 0.5 * (L / Nx) / math.sqrt(9.81)
    x = np.arange(Nx) * L / Nx
    b0, phi = si.adjoint_bathymetry(5, L=L, K=64)
    kk = np.arange(1, 65)
    C = np.cos(2.0 * math.pi * kk[:, None] * x[None, :] / L + phi[:, None])
    dev = torch.device("cuda", torch.cuda.current_device())
    T = w.Tank(Nx, 1, Nz, L, (1.0 + b0 @ C)[None], mode=w.WT_MIXED, tol=1e-10, filter=1)
    nsteps = 40
    z = torch.zeros((Nz + 1, Nx), dtype=torch.float64, device=dev)
    Ct = torch.tensor(C, device=dev)
    out = {}
    for rep in range(2):                               # the first repetition warms up
        bt = torch.tensor(b0, device=dev, requires_grad=True)
        et = torch.tensor(0.02 * np.cos(2.0 * math.pi * x / 4.0), device=dev, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        series = gauge_series(T, 1.0 + bt @ Ct, et, z, z, dt, nsteps, np.arange(0, Nx, 32), every=20)
        J = 0.5 * torch.sum(series ** 2) * dt
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out = {"workload": "2D tank L=16, Nx=512, Nz=20, 64-mode seeded bathymetry, eta0 = 0.02 cos(2 pi x/4), "
                           "%d steps, 16 gauges, checkpoints every 20 steps, mixed solver at 1e-10" % nsteps,
               "forward_ms_per_step": (t1 - t0) * 1e3 / nsteps,
               "backward_ms_per_step": (t2 - t1) * 1e3 / nsteps,
               "gradient_ms_per_step": (t2 - t0) * 1e3 / nsteps,
               "note": "backward = segment recomputation + wt_adjoint_step (stage recomputation, "
                       "five reversed stages with transposed p-multigrid solves); host clock"}
    T.close()
    return out


# ------------------------------------------------------------ oracle (CPU)
def oracle_tank(p, h):
    from oracle import rk
    return rk.Tank(p["Nx"], 1, p["Nz"], p["L"], h, tol=1e-10, coarsest_max=64, filter=True)


def oracle_state(p, x, h):
    from oracle import rk
    from oracle import spectral as sp
    sigma = sp.cgl_sigma(p["Nz"])
    st = initial_state(p, x, h, sigma)
    g = oracle_tank(p, h).grid
    return rk.State(g, st[0], st[1], st[2], st[3])


def cpu_baseline(p, x, h, budget_s=15.0):
    """Oracle Runge-Kutta stages of the same workload until ~budget_s of CPU work."""
    from oracle import rk
    tank = oracle_tank(p, h)
    st = oracle_state(p, x, h)
    n = 0
    t0 = time.perf_counter()
    while n < STAGES:
        rk.stage(tank, st, n + 1, p["dt"])
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    dof = p["Nx"] * (p["Nz"] + 1)
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    return {"value": n * dof / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d Runge-Kutta stage(s) of the first step (%.1f s, numpy float64, %d BLAS thread(s))"
                      % (n, el, threads)}


def cpu_baseline_all_cores(budget_s):
    """The same oracle sample with numpy's BLAS on every host core (a fresh
    interpreter started with the thread counts set, since they are fixed at
    import)."""
    nproc = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(nproc), OPENBLAS_NUM_THREADS=str(nproc),
               MKL_NUM_THREADS=str(nproc))
    code = ("import json, bench; p, x, h = bench.workload(); "
            "print(json.dumps(bench.cpu_baseline(p, x, h, budget_s=%r)))" % budget_s)
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        out = json.loads(r.stdout.strip().splitlines()[-1])
        out["cores"] = nproc
        out["nproc"] = nproc
        return out
    except Exception as e:          # report, do not fail the benchmark line
        return {"error": "all-cores oracle run failed: %s" % e, "nproc": nproc}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import rk
    p, x, h = workload()
    tank = oracle_tank(p, h)
    st = oracle_state(p, x, h)
    dof = p["Nx"] * (p["Nz"] + 1)
    k = 0
    for _ in range(args.warmup):
        rk.stage(tank, st, k % STAGES + 1, p["dt"])
        k += 1
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rk.stage(tank, st, k % STAGES + 1, p["dt"])
        times.append(time.perf_counter() - t0)
        k += 1
    ms = float(np.mean(times)) * 1e3
    value = dof / (ms / 1e3)
    sample = "one Runge-Kutta stage per step (a fifth of a full step), numpy float64, one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config(p, {"step": "one RK stage"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-tune", action="store_true", help="keep the default solver settings")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-tank and gradient measurements")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
