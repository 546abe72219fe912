"""Benchmark: batched RBF-FD operator build (stencils/s at kappa_T) on one GB300.

Workload (the batched-build configuration): spherical Fibonacci lattice,
N = 1,000,000 nodes, exact normals, cut into four latitude bands of 250,000
nodes with stencil sizes n = 31 / 50 / 70 / 101, IMQ kernel, per-stencil eps
searched to kappa_T = 1e12 (absolute eps tolerance 1e-4) in float64, with
the learned first guess (one network per n, trained before timing on
plain-search eps of a sphere and a torus).  One bench step = the whole hot
path once: stencils (kNN), learned guesses, the eps search, the weights (one
C-ABI build_operator call), then one CUDA-graph-replayed SBDF2 + BiCGSTAB
time step (Schnakenberg, float32) with the new operator.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launch stream, L2 flushed (256 MB write) before every step, barrier +
synchronize around the timed region, max over ranks.  Under torchrun each
rank builds its own copy (replicas: the build needs no exchange), so value
= ranks x N / time ("scaling": "weak").

The roofline of the dominant kernel (the eps search) counts algorithmic
float64 flops: per stencil E_k * m^3 / 3 (m = n + 1, one symmetric
factorisation per condition-number evaluation, E_k = the evaluations that
launch actually performed for stencil k) over the search kernel's CUDA-event
time, against the measured FP64 FMA peak.  Beside it: the same rate with every
stencil charged the oracle's median evaluation count E_n plus one final
factorisation (measured live on the CPU sample), which credits the learned
start's saved evaluations.

--profile runs the same pipeline once on a smaller version of the workload
(--profile-n nodes, default 40,000, same four stencil sizes; --profile-plain
without the learned start) inside an NVTX range "profiled", for ncu.

--impl reference times the CPU FP64 oracle on the host's cores (one
single-threaded process per core, each on its own bounded sample of the same
workload) and prints the same JSON line; the benchmark line reports that
figure and the one-core figure as its CPU baseline.
"""
from __future__ import annotations

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

SIZES = (31, 50, 70, 101)
N_NODES = 1_000_000
KAPPA_T = 1e12
METRIC = "stencils/s built at target kappa (batched mixed-n build + one IMEX step)"
UNIT = "stencils/s"
# DRAM bytes per launch of the search kernel from one ncu capture, keyed by
# the hash of build.cu at the time of the capture (None when not captured).
# The capture ran the learned 16,000-node version of this workload (same four
# stencil sizes, networks trained the same way; 16,000 lanes x ~188 KB of
# per-lane scratch, still far beyond L2): 11.0047 GB read + 2.0789 GB written;
# scaled to the 1,000,000 stencils of one bench launch by the stencil count.
SEARCH_TRAFFIC = {"6a28fbb64ea166c5": (11.004673536e9 + 2.078867712e9) * 1_000_000 / 16_000}


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations' report")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--sample", type=int, default=20, help="oracle stencils per size per step")
    ap.add_argument("--profile", action="store_true", help="one small run for ncu (NVTX 'profiled')")
    ap.add_argument("--profile-n", type=int, default=40_000, help="nodes of the --profile case")
    ap.add_argument("--profile-plain", action="store_true", help="--profile without the learned start")
    ap.add_argument("--profile-lu", action="store_true",
                    help="the banded-LU direct solve for ncu: the RCM-ordered 40k torus (n = 50), the SBDF2 "
                         "matrix factorised, 2 LU steps, then 1 step inside the NVTX range 'profiled'")
    ap.add_argument("--profile-step", action="store_true",
                    help="--profile of the IMEX step instead: after 4 graph-replayed steps, 3 steps with "
                         "the same kernels launched from the host inside the NVTX range 'profiled' "
                         "(ncu cannot replay kernels of a graph with a conditional node)")
    ap.add_argument("--horizons", action="store_true",
                    help="the long-horizon stepping studies only (C2 5000 steps, the 2M-node unit-sphere "
                         "Gray-Scott stand-in 10k steps in float32 and float64); one JSON line")
    return ap.parse_args()


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the
    slowest replica's time); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU oracle worker (single-threaded subprocess)
# ---------------------------------------------------------------------------

def cpu_worker(per_size: int, seed: int):
    import numpy as np
    from oracle import operator as oop
    from oracle import weights as ow
    from paper_1404_0812_gb300 import workloads as W
    ns = W.fibonacci_sphere(N_NODES)
    nper = W.stencil_size_groups(N_NODES, SIZES)
    rng = np.random.default_rng(seed)
    rows = np.concatenate([rng.choice(np.where(nper == n)[0], per_size, replace=False) for n in SIZES])
    t = time.perf_counter()
    op = oop.build_operator(ns.X, ns.normals, nper, ow.IMQ, kappa_T=KAPPA_T, rows=rows)
    dt = time.perf_counter() - t
    evals = {int(n): [int(e) for e, k in zip(op.evals, rows) if nper[k] == n] for n in SIZES}
    print(json.dumps(dict(count=len(rows), seconds=dt, evals=evals)))


def run_cpu_sample(per_size: int, seed: int, procs: int = 1) -> dict:
    """The oracle on ``procs`` single-threaded processes at once (separate
    interpreters, no GPU), each on its own seeded sample of ``per_size``
    stencils per n.  Throughput = all stencils / the longest worker's compute
    time (interpreter start-up and imports excluded)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    ps = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(per_size),
                            "--sample", str(seed + 7919 * i)], env=env, stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True) for i in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"oracle worker failed: {err[-500:]}")
        res.append(json.loads(out.strip().splitlines()[-1]))
    evals = {}
    for r in res:
        for n, v in r["evals"].items():
            evals.setdefault(n, []).extend(v)
    return dict(count=sum(r["count"] for r in res), seconds=max(r["seconds"] for r in res), evals=evals,
                procs=procs)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _file_hash(path):
    import hashlib
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


TRAIN_STATS = {}


def train_networks(R, W, T, torch, pairs=200_000):
    """One eps network per stencil size, trained on plain-search eps of
    Fibonacci spheres (100k and 400k nodes) and staggered tori (m = 60 and
    150): `pairs` (stencil, eps) pairs drawn at random (seed 3) per size."""
    import numpy as np
    nets = []
    sets = [W.fibonacci_sphere(100_000), W.fibonacci_sphere(400_000), W.torus_staggered(60),
            W.torus_staggered(150)]
    dev = [(T(s.X), T(s.normals)) for s in sets]
    gen = torch.Generator(device="cuda").manual_seed(3)
    for n in SIZES:
        F, Y = [], []
        for X, Nr in dev:
            op = R.build_operator(X, Nr, n, kernel="imq", kappa_target=KAPPA_T)
            f, y = R.features(op, X, Nr, n)
            F.append(f)
            Y.append(y)
            del op
        F = torch.cat(F)
        Y = torch.cat(Y)
        sel = torch.randperm(F.shape[0], generator=gen, device="cuda")[:pairs]
        net = R.EpsNet(n, W.mlp_pack(W.mlp_init(3 * n, seed=n)).astype(np.float32))
        Fs, Ys = F[sel].contiguous(), Y[sel].contiguous()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        losses = net.train(Fs, Ys, epochs=30, batch=1024, lr=1e-3, seed=0)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        # forward + backward of 3n -> 64 -> 64 -> 1 per sample: 3 x 2 x weights
        flops = 30 * Fs.shape[0] * 3 * 2 * (3 * n * 64 + 64 * 64 + 64)
        TRAIN_STATS[int(n)] = {"pairs": int(Fs.shape[0]), "epochs": 30, "ms": round(ms, 1),
                               "samples_per_s": round(30 * Fs.shape[0] / (ms * 1e-3), 1),
                               "tflops": round(flops / (ms * 1e-3) / 1e12, 3),
                               "loss_first_last": [round(losses[0], 5), round(losses[-1], 5)]}
        nets.append(net)
        del F, Y, Fs, Ys
    return nets


def configs_report(R, W, T, torch, nets):
    """The other benchmark configurations, measured after the timed steps
    (not part of the headline value).  A configuration that fails reports
    its error instead of its numbers."""
    out = {}
    for name, fn in (("sphere2562_heat", _c1), ("torus40k_schnakenberg", _c2),
                     ("torus40k_direct_lu_vs_bicgstab", _c2_lu), ("bumpy500k_learned", _c4),
                     ("bumpy2m_pointcloud", _c5), ("bumpy2m_analytic_gray_scott", _c5_bumpy),
                     ("sphere2m_gray_scott", _c5_standin),
                     ("reorder_1m_shuffled", _reorder),
                     ("sphere_heat_convergence_bdf4", _e3),
                     ("forced_sphere_convergence_bdf4", _e4), ("forced_torus_convergence_bdf4", _e5),
                     ("forced_fixed_kappa_1e14", _e6), ("forced_fixed_kappa_1e20_dd", _e6_dd)):
        try:
            out[name] = fn(R, W, T, torch, nets)
        except Exception as e:   # reported, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"[:400]}
        torch.cuda.synchronize()
    return out


def convergence_study(R, W, T, torch, problem="heat_sphere", stencil_sizes=(11, 17, 31), sizes=None,
                      kappa="grow", dt=None, t_end=None, f64_cap=1e15, dd_cap=1e24):
    """Section 6's convergence studies, IMQ, float64, BDF4 (order 4) started
    from the exact solution at t = 0, dt, 2 dt:
      heat_sphere    u_t = Delta u from the 30-term series of sectoral
                     harmonics, to t = 0.5 (dt 1e-3), icosahedral N = 642..40962;
      forced_sphere  u = exp(-5 t) sum_k exp(-10 theta_k^2), 23 centres, with
                     its source taken implicitly, to t = 0.2 (dt 1e-4);
      forced_torus   Eq. torus_forced (a = 9, b = 3), staggered N = 6 m^2,
                     m = 10..80, to t = 0.2 (dt 1e-4).
    kappa = "grow": kappa_T = 1e5 on the coarsest node set, and on every
    finer one the kappa_T that keeps the coarsest set's mean shape parameter
    (regula falsi in log kappa_T); a number: that fixed kappa_T.  Builds with
    kappa_T above f64_cap run in double-double (Section 6 computes those
    weights in quad precision).  Returns per n the relative l2 / l_inf errors
    against the exact solution and the observed orders in sqrt(N)."""
    import numpy as np
    torus = problem == "forced_torus"
    if sizes is None:
        sizes = (10, 20, 40, 80) if torus else (3, 4, 5, 6)
    if dt is None:
        dt = 1e-3 if problem == "heat_sphere" else 1e-4
    if t_end is None:
        t_end = 0.5 if problem == "heat_sphere" else 0.2
    centers = W.torus_forced_centers() if torus else W.sphere_forced_centers()
    res = {}
    for n in stencil_sizes:
        rows, eps_ref, kT_prev = [], None, 1e5
        for size in sizes:
            ns = W.torus_staggered(size) if torus else W.icosahedral_sphere(size)
            X, Nr = T(ns.X), T(ns.normals)

            def build(kT):
                prec = "dd" if kT > f64_cap * 1.0001 else "f64"
                op = R.build_operator(X, Nr, n, kernel="imq", kappa_target=kT, allow_failures=True,
                                      precision=prec)
                info = R.get_stencil_info(op)
                return op, float(info["eps"].mean().item()), bool((info["status"] == 0).all().item()), prec

            if kappa == "grow" and eps_ref is not None:
                # g(y) = ln(mean eps(kappa_T = e^y) / eps_ref) decreases in y:
                # bracket it (float64 up to f64_cap, double-double beyond),
                # then Illinois regula falsi to |g| < 1e-4
                def g(y):
                    r = build(math.exp(y))
                    return math.log(r[1] / eps_ref), r

                a = math.log(kT_prev)
                ga, ra = g(a)
                b = math.log(f64_cap)
                gb, rb = g(b)
                if gb > 0:
                    a, ga, ra = b, gb, rb
                    b = math.log(dd_cap)
                    gb, rb = g(b)
                y, gy, ry = (a, ga, ra) if abs(ga) < abs(gb) else (b, gb, rb)
                side = 0
                for _ in range(20):
                    if abs(gy) < 1e-4 or ga * gb > 0:
                        break
                    y = b - gb * (b - a) / (gb - ga)
                    gy, ry = g(y)
                    if gy * gb < 0:
                        a, ga, ra = b, gb, rb
                        side = 0
                    else:
                        ga = 0.5 * ga if side == 1 else ga
                        side = 1
                    b, gb, rb = y, gy, ry
                kT = math.exp(y)
                op, em, ok, prec = ry
            else:
                kT = 1e5 if kappa == "grow" else float(kappa)
                op, em, ok, prec = build(kT)
                if eps_ref is None:
                    eps_ref = em
            kT_prev = kT
            if problem == "heat_sphere":
                exact = lambda t: W.sphere_heat_series(ns.X, t)
                src = None
            else:
                g, h = W.torus_forced(ns.X, centers) if torus else W.sphere_forced(ns.X, centers)
                exact = lambda t: math.exp(-5.0 * t) * g
                src = T(h)
            t0 = 3 * dt
            st = R.StepState.create(T(exact(t0)), order=4)
            st.u_prev.copy_(T(exact(2 * dt)))
            st.u_prev2.copy_(T(exact(dt)))
            st.u_prev3.copy_(T(exact(0.0)))
            st.has_history = 3
            st.t = t0
            nsteps = int(round((t_end - t0) / dt))
            p = R.StepParams(model="none", nspecies=1, dtype=torch.float64, dt=dt, delta_u=1.0, tol=1e-12,
                             order=4, use_graph=True, source_u=src, source_rate=-5.0)
            rep = R.step_imex(op, st, p, nsteps, allow_failure=True)
            u = st.u.cpu().numpy()
            ex = exact(st.t)
            rows.append({"N": ns.N, "kappa_T": float(f"{kT:.3g}"), "precision": prec,
                         "eps_mean": round(em, 5), "stencils_ok": ok, "solver_status": rep["status"],
                         "l2": float(f"{np.linalg.norm(u - ex) / np.linalg.norm(ex):.3e}"),
                         "linf": float(f"{np.abs(u - ex).max() / np.abs(ex).max():.3e}")})
            del op
        for a, b in zip(rows, rows[1:]):
            hN = math.log(math.sqrt(b["N"] / a["N"]))
            b["order_l2"] = round(math.log(a["l2"] / b["l2"]) / hN, 2)
            b["order_linf"] = round(math.log(a["linf"] / b["linf"]) / hN, 2)
        res[f"n{n}"] = rows
    return res


def sphere_heat_study(R, W, T, torch, stencil_sizes=(11, 17, 31), levels=(3, 4, 5, 6), kappa="grow", **kw):
    """The heat-equation study of Section 6 (see convergence_study)."""
    return convergence_study(R, W, T, torch, "heat_sphere", stencil_sizes, levels, kappa, **kw)


def _reorder(R, W, T, torch, nets):
    """Section 4.1's reordering on a node set without any order: the 1M-node
    Fibonacci sphere shuffled (seed 9), n = 50, learned build; apply (float32)
    and SBDF2 steps (Schnakenberg float32, CUDA graph) as given, after a Morton
    renumbering and after reverse Cuthill-McKee."""
    import numpy as np
    ns = W.fibonacci_sphere(N_NODES)
    p = np.random.default_rng(9).permutation(ns.N)
    X0, N0 = ns.X[p].copy(), ns.normals[p].copy()
    net = [nets[SIZES.index(50)]] if nets is not None else None
    s = W.SCHNAKENBERG
    name, coef = R.model_coefs(s)
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    out = {}

    def measure(X, Nr, u, v):
        op = R.build_operator(T(X), T(Nr), 50, kernel="imq", kappa_target=KAPPA_T, mlps=net)
        uu = T(u, torch.float32)
        yy = torch.empty_like(uu)
        for _ in range(3):
            R.apply(op, uu, yy)
        a, b = _ev(torch)
        a.record()
        for _ in range(20):
            R.apply(op, uu, yy)
        b.record()
        torch.cuda.synchronize()
        ams = a.elapsed_time(b) / 20
        sp = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                          delta_v=s["delta_v"], coef=coef, tol=1e-6, use_graph=True)
        st = R.StepState.create(T(u, torch.float32), T(v, torch.float32))
        R.step_imex(op, st, sp, 2)
        a.record()
        R.step_imex(op, st, sp, 20)
        b.record()
        torch.cuda.synchronize()
        return op, {"apply_f32_GB_s": round(op.apply_bytes(R.F32) / (ams * 1e-3) / 1e9, 1),
                    "step_ms": round(a.elapsed_time(b) / 20, 3)}

    op, out["shuffled"] = measure(X0, N0, u0, v0)
    t0 = time.time()
    pm = R.morton_order(T(X0)).cpu().numpy()
    tm = time.time() - t0
    t0 = time.time()
    pr = R.rcm_order(op).cpu().numpy()
    tr = time.time() - t0
    del op
    for label, perm, secs in (("morton", pm, tm), ("rcm", pr, tr)):
        _, out[label] = measure(X0[perm], N0[perm], u0[perm], v0[perm])
        out[label]["ordering_s"] = round(secs, 2)
    return out


def _e3(R, W, T, torch, nets):
    return sphere_heat_study(R, W, T, torch)


def _e4(R, W, T, torch, nets):
    return convergence_study(R, W, T, torch, "forced_sphere")


def _e5(R, W, T, torch, nets):
    return convergence_study(R, W, T, torch, "forced_torus")


def _e6(R, W, T, torch, nets):
    return {"forced_sphere": convergence_study(R, W, T, torch, "forced_sphere", kappa=1e14),
            "forced_torus": convergence_study(R, W, T, torch, "forced_torus", kappa=1e14)}


def _e6_dd(R, W, T, torch, nets):
    # kappa_T = 1e20: double-double builds (Section 6 uses quad precision)
    return {"forced_sphere": convergence_study(R, W, T, torch, "forced_sphere", kappa=1e20),
            "forced_torus": convergence_study(R, W, T, torch, "forced_torus", kappa=1e20)}


def _ev(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _c1(R, W, T, torch, nets):
    import numpy as np
    ev = lambda: _ev(torch)
    stream = torch.cuda.current_stream()
    # C1: unit sphere N = 2562 (icosahedral), n = 31, Gaussian; heat equation
    # from Y_3^2 to t = 0.1 (1000 steps of 1e-4) vs exp(-12 t) decay
    ns = W.icosahedral_sphere(4)
    op = R.build_operator(T(ns.X), T(ns.normals), 31, kernel="gaussian", kappa_target=KAPPA_T)
    u0 = W.sph_harm_y32(ns.X)
    exact = math.exp(-1.2) * u0
    c1 = {}
    for dt_, tol in ((torch.float64, 1e-12), (torch.float32, 1e-6)):
        st = R.StepState.create(T(u0, dt_))
        p = R.StepParams(model="none", nspecies=1, dtype=dt_, dt=1e-4, delta_u=1.0, tol=tol, use_graph=True)
        a, b = ev()
        a.record(stream)
        rep = R.step_imex(op, st, p, 1000)
        b.record(stream)
        torch.cuda.synchronize()
        err = float(np.abs(st.u.double().cpu().numpy() - exact).max() / np.abs(exact).max())
        c1["f64" if dt_ == torch.float64 else "f32"] = {"ms_per_step": round(a.elapsed_time(b) / 1000, 4),
                                                        "rel_err_vs_exact": err,
                                                        "max_iters": rep["max_iters_u"]}
    return c1


def _c2(R, W, T, torch, nets, horizon=5000):
    ev = lambda: _ev(torch)
    stream = torch.cuda.current_stream()
    # C2: torus m = 82 (N = 40,344), n = 50, IMQ; Schnakenberg, float32 vs
    # float64 stepping over the whole 5000-step horizon (the difference after
    # 100 steps is the parity figure; the full-horizon one is reported as is:
    # pattern formation amplifies rounding differences)
    ns = W.torus_staggered(82)
    op = R.build_operator(T(ns.X), T(ns.normals), 50, kernel="imq", kappa_target=KAPPA_T)
    s = W.SCHNAKENBERG
    name, coef = R.model_coefs(s)
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    st, ms, d = {}, {}, {}
    for dt_, tol in ((torch.float64, 1e-12), (torch.float32, 1e-8)):
        st[dt_] = R.StepState.create(T(u0, dt_), T(v0, dt_))
        ms[dt_] = 0.0
    p = {dt_: R.StepParams(model=name, nspecies=2, dtype=dt_, dt=s["dt"], delta_u=s["delta_u"],
                           delta_v=s["delta_v"], coef=coef, tol=tol, use_graph=True)
         for dt_, tol in ((torch.float64, 1e-12), (torch.float32, 1e-8))}
    done = 0
    for upto in (100, horizon):
        for dt_ in (torch.float64, torch.float32):
            a, b = ev()
            a.record(stream)
            R.step_imex(op, st[dt_], p[dt_], upto - done)
            b.record(stream)
            torch.cuda.synchronize()
            ms[dt_] += a.elapsed_time(b)
        done = upto
        d[upto] = {k: float((getattr(st[torch.float32], k).double() - getattr(st[torch.float64], k)).abs().max()
                            / getattr(st[torch.float64], k).abs().max()) for k in ("u", "v")}
    u64 = st[torch.float64].u
    return {"f32_vs_f64_rel_linf_100_steps": max(d[100].values()),
            f"f32_vs_f64_rel_linf_{horizon}_steps": max(d[horizon].values()),
            "by_species": {str(k): v for k, v in d.items()},
            "ms_per_step_f64": round(ms[torch.float64] / horizon, 4),
            "ms_per_step_f32": round(ms[torch.float32] / horizon, 4),
            f"u_range_at_{horizon}_f64": [float(u64.min()), float(u64.max())]}


def _c2_lu(R, W, T, torch, nets, steps=100):
    """Section 7's direct solves against BiCGSTAB on the C2 torus (N = 40,344,
    n = 50, Schnakenberg SBDF2): nodes renumbered by reverse Cuthill-McKee
    (rbffd_rcm_order), the SBDF matrices factorised once as banded LU
    (float64 factors), then ms per step of the LU path and of BiCGSTAB
    (float32 and float64 state, CUDA graph) and the difference of their
    solutions after `steps` steps."""
    ns = W.torus_staggered(82)
    op0 = R.build_operator(T(ns.X), T(ns.normals), 50, kernel="imq", kappa_target=KAPPA_T)
    perm = R.rcm_order(op0).cpu().numpy()
    del op0
    X, Nr = ns.X[perm].copy(), ns.normals[perm].copy()
    op = R.build_operator(T(X), T(Nr), 50, kernel="imq", kappa_target=KAPPA_T)
    kl, ku = R.op_bandwidth(op)
    s = W.SCHNAKENBERG
    name, coef = R.model_coefs(s)
    u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
    u0, v0 = u0[perm].copy(), v0[perm].copy()
    out = {"N": ns.N, "bandwidths": [kl, ku]}
    t0 = time.perf_counter()
    lu = R.lu_factor(op, 3.0, 2 * s["dt"] * s["delta_v"])
    out["factor_s_one_matrix_f64"] = round(time.perf_counter() - t0, 3)
    out["factor_bytes_one_matrix"] = lu.bytes
    del lu
    res = {}
    # float32 BiCGSTAB to the float32 floor (1e-8 on the recursive residual,
    # as in C2), so that both solvers solve each step to float32 accuracy
    for dt_, tol in ((torch.float32, 1e-8), (torch.float64, 1e-12)):
        for solver in ("lu", "bicgstab"):
            p = R.StepParams(model=name, nspecies=2, dtype=dt_, dt=s["dt"], delta_u=s["delta_u"],
                             delta_v=s["delta_v"], coef=coef, tol=tol, use_graph=True, solver=solver)
            st = R.StepState.create(T(u0, dt_), T(v0, dt_))
            t1 = time.perf_counter()
            R.step_imex(op, st, p, 2)      # SBDF1 + SBDF2 factors, graph capture
            torch.cuda.synchronize()
            setup = time.perf_counter() - t1
            a, b = _ev(torch)
            a.record()
            rep = R.step_imex(op, st, p, steps)
            b.record()
            torch.cuda.synchronize()
            key = f"{solver}_{'f32' if dt_ == torch.float32 else 'f64'}"
            out[f"ms_per_step_{key}"] = round(a.elapsed_time(b) / steps, 4)
            if solver == "bicgstab":
                out[f"iters_mean_{key}"] = round(rep["total_iters"] / steps / 2, 2)
            else:
                out[f"first_two_steps_s_{key}"] = round(setup, 3)
            res[key] = st.u.double()
    for k in ("f32", "f64"):
        out[f"lu_vs_bicgstab_rel_linf_{k}"] = float((res[f"lu_{k}"] - res[f"bicgstab_{k}"]).abs().max()
                                                    / res[f"bicgstab_{k}"].abs().max())
        out[f"lu_over_bicgstab_time_{k}"] = round(out[f"ms_per_step_lu_{k}"] / out[f"ms_per_step_bicgstab_{k}"], 2)
    return out


def _c4(R, W, T, torch, nets):
    # C4: held-out bumpy sphere N = 500k, n = 50: learned start vs plain search
    ns = W.bumpy_sphere(500_000)
    X, Nr = T(ns.X), T(ns.normals)
    net50 = nets[SIZES.index(50)]
    rows = {}
    for lab, m in (("plain", None), ("learned", [net50])):
        op = R.build_operator(X, Nr, 50, kernel="imq", kappa_target=KAPPA_T, mlps=m)
        ph = R.get_build_timings(op)
        info = R.get_stencil_info(op)
        rows[lab] = {"guess_plus_search_ms": round(ph["guess"] + ph["search"], 2),
                     "build_ms": round(sum(ph.values()), 2),
                     "evals_mean": round(float(info["evals"].double().mean()), 3),
                     "accepted_fraction": round(float((info["status"] == 4).double().mean()), 4)}
        del op
    rows["speedup_search"] = round(rows["plain"]["guess_plus_search_ms"] / rows["learned"]["guess_plus_search_ms"], 3)
    rows["stencils_per_s_learned_build"] = round(ns.N / (rows["learned"]["build_ms"] * 1e-3), 1)
    return rows


def _c5(R, W, T, torch, nets):
    ev = lambda: _ev(torch)
    stream = torch.cuda.current_stream()
    # C5: bumpy sphere N = 2M, jittered, 20-NN PCA normals, n = 70, learned
    # start; apply bandwidth and Gray-Scott float32 steps
    ns = W.bumpy_sphere(2_000_000, jitter=0.25, seed=4, normals="pca")
    X, Nr = T(ns.X), T(ns.normals)
    op = R.build_operator(X, Nr, 70, kernel="imq", kappa_target=KAPPA_T, mlps=[nets[SIZES.index(70)]],
                          allow_failures=True)
    ph = R.get_build_timings(op)
    info = R.get_stencil_info(op)
    uu = torch.rand(ns.N, dtype=torch.float32, device="cuda")
    yy = torch.empty_like(uu)
    torch.cuda.nvtx.range_push("c5_apply")   # for ncu: the point cloud's applies
    for _ in range(3):
        R.apply(op, uu, yy)
    a, b = ev()
    a.record(stream)
    for _ in range(20):
        R.apply(op, uu, yy)
    b.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ams = a.elapsed_time(b) / 20
    out = {
        "build_ms": round(sum(ph.values()), 1), "phases_ms": {k: round(v, 1) for k, v in ph.items()},
        "stencils_per_s": round(ns.N / (sum(ph.values()) * 1e-3), 1),
        "stencils_ok_fraction": round(float(((info["status"] == 0) | (info["status"] == 4)).double().mean()), 6),
        "accepted_fraction": round(float((info["status"] == 4).double().mean()), 4),
        "apply_f32_GB_s": round(op.apply_bytes(R.F32) / (ams * 1e-3) / 1e9, 1)}
    g = W.GRAY_SCOTT
    name, coef = R.model_coefs(g)
    u0, v0 = W.gray_scott_initial(ns.X, seed=5, spots=50, radius=0.05)
    st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
    p = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=g["dt"], delta_u=g["delta_u"],
                     delta_v=g["delta_v"], coef=coef, tol=1e-6, use_graph=True)
    rep = R.step_imex(op, st, p, 2, allow_failure=True)
    if rep["status"] != 0:
        out["gray_scott_error"] = {k: rep[k] for k in ("status", "failed_step", "max_iters_u", "max_iters_v",
                                                       "last_relres_u", "last_relres_v")}
        return out
    a, b = ev()
    a.record(stream)
    rep = R.step_imex(op, st, p, 20, allow_failure=True)
    b.record(stream)
    torch.cuda.synchronize()
    out["gray_scott_f32_ms_per_step"] = round(a.elapsed_time(b) / 20, 3)
    out["gray_scott_max_iters"] = [rep["max_iters_u"], rep["max_iters_v"]]
    out["gray_scott_status"] = rep["status"]
    return out


def _c5_standin(R, W, T, torch, nets, steps=10_000, f64_steps=None, surface="sphere"):
    """Stand-ins of the 2M-node point-cloud Gray-Scott run (whose jittered,
    PCA-normal operator has eigenvalues far in the right half-plane, see
    test_pointcloud_spectrum): surface "bumpy" = the same bumpy sphere with
    analytic normals and no jitter (its conical poles still leave a positive
    part: reported, with the step at which BiCGSTAB fails), "sphere" = the
    unit sphere at N = 2,000,000 (Fibonacci nodes, exact normals: spectrum
    in the closed left half-plane), both n = 70, learned build.  Gray-Scott
    in float32 for `steps` steps (ms per step), float64 beside it for the
    parity window (100 steps) and, with f64_steps, to that horizon for the
    full-horizon difference.  A run stops at its first solver failure."""
    ns = (W.bumpy_sphere(2_000_000, jitter=0.0, seed=4, normals="analytic") if surface == "bumpy"
          else W.fibonacci_sphere(2_000_000))
    op = R.build_operator(T(ns.X), T(ns.normals), 70, kernel="imq", kappa_target=KAPPA_T,
                          mlps=[nets[SIZES.index(70)]], allow_failures=True)
    info = R.get_stencil_info(op)
    g = W.GRAY_SCOTT
    name, coef = R.model_coefs(g)
    u0, v0 = W.gray_scott_initial(ns.X, seed=5, spots=50, radius=0.05)
    out = {"surface": surface, "N": ns.N, "n": 70,
           "stencils_ok_fraction": round(float(((info["status"] == 0) | (info["status"] == 4)).double().mean()), 6),
           "build_ms": round(sum(R.get_build_timings(op).values()), 1)}
    st, p = {}, {}
    # float32 BiCGSTAB to the float32 floor (1e-8 on the recursive residual,
    # as in C2): a tolerance of 1e-6 leaves 1e-6 |b| of error per step, and
    # over the 100-step parity window that grew to ~5e-4
    for dt_, tol in ((torch.float32, 1e-8), (torch.float64, 1e-12)):
        st[dt_] = R.StepState.create(T(u0, dt_), T(v0, dt_))
        p[dt_] = R.StepParams(model=name, nspecies=2, dtype=dt_, dt=g["dt"], delta_u=g["delta_u"],
                              delta_v=g["delta_v"], coef=coef, tol=tol, use_graph=True)
    diffs = {}
    done = {torch.float32: 0, torch.float64: 0}
    ms32 = 0.0
    failed = False
    for upto in [100] + ([f64_steps] if f64_steps else []):
        for dt_ in (torch.float32, torch.float64):
            a, b = _ev(torch)
            a.record()
            rep = R.step_imex(op, st[dt_], p[dt_], upto - done[dt_], allow_failure=True)
            b.record()
            torch.cuda.synchronize()
            if dt_ == torch.float32:
                ms32 += a.elapsed_time(b)
            done[dt_] = upto
            if rep["status"] != 0:
                out[f"solver_failure_{'f32' if dt_ == torch.float32 else 'f64'}"] = {
                    k: rep[k] for k in ("failed_step", "max_iters_u", "max_iters_v")}
                failed = True
        diffs[upto] = max(float((getattr(st[torch.float32], k).double() - getattr(st[torch.float64], k)).abs().max()
                                / getattr(st[torch.float64], k).abs().max()) for k in ("u", "v"))
        if failed:
            break
    if not failed and steps > done[torch.float32]:
        a, b = _ev(torch)
        a.record()
        rep = R.step_imex(op, st[torch.float32], p[torch.float32], steps - done[torch.float32], allow_failure=True)
        b.record()
        torch.cuda.synchronize()
        ms32 += a.elapsed_time(b)
        done[torch.float32] = steps
        if rep["status"] != 0:
            out["solver_failure_f32"] = {k: rep[k] for k in ("failed_step", "max_iters_u", "max_iters_v")}
    out["f32_vs_f64_rel_linf"] = {str(k): v for k, v in diffs.items()}
    out["steps_f32"] = done[torch.float32]
    out["ms_per_step_f32"] = round(ms32 / max(done[torch.float32], 1), 4)
    for k in ("u", "v"):
        x = getattr(st[torch.float32], k)
        out[f"{k}_range_f32_end"] = [float(x.min()), float(x.max())]
    return out


def _c5_bumpy(R, W, T, torch, nets):
    return _c5_standin(R, W, T, torch, nets, steps=100, surface="bumpy")


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1404_0812_gb300 as R
    from paper_1404_0812_gb300 import workloads as W
    R._lib.load()
    dev = torch.device("cuda", local)
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    cpu = None
    if rank == 0 and not (args.profile or args.horizons):   # oracle sample first, before heavy GPU work
        cpu1 = run_cpu_sample(args.sample, 1234)
        cpu = run_cpu_sample(args.sample, 1234, host_cores())
    n_nodes = args.profile_n if args.profile else N_NODES

    ns = W.fibonacci_sphere(n_nodes)
    nper = W.stencil_size_groups(n_nodes, SIZES)
    X, Nr, NP = T(ns.X), T(ns.normals), T(nper, torch.int32)
    nets = None if (args.no_learned or args.profile_plain) else train_networks(R, W, T, torch)
    # hand back what the training left in torch's cache and the library's
    # pool (their blocks fragment the device memory the timed builds allocate
    # from); the warm-up steps map the build's scratch again
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    R.release_memory()
    s = W.SCHNAKENBERG
    name, coef = R.model_coefs(s)
    u0, v0 = W.schnakenberg_initial(n_nodes, seed=2)
    sp = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                      delta_v=s["delta_v"], coef=coef, tol=1e-6, use_graph=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # launch shape of the build kernels from the project's autotuner (timed on
    # a strided 1/20 subsample of this node set)
    shape = (dict(block_threads=0, blocks_per_sm=0) if args.profile else
             R.autotune_build(X, Nr, NP, kernel="imq", kappa_target=KAPPA_T, sample=max(n_nodes // 20, 2000)))

    def one_step(Xd, Nd, NPd):
        op = R.build_operator(Xd, Nd, NPd, kernel="imq", kappa_target=KAPPA_T, mlps=nets,
                              block_threads=shape["block_threads"], blocks_per_sm=shape["blocks_per_sm"])
        st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
        R.step_imex(op, st, sp, 1)
        return op

    if args.horizons:
        t0 = time.perf_counter()
        out = {"horizons": True,
               "torus40k_schnakenberg": _c2(R, W, T, torch, nets),
               "sphere2m_gray_scott": _c5_standin(R, W, T, torch, nets, steps=10_000, f64_steps=10_000)}
        out["wall_s"] = round(time.perf_counter() - t0, 1)
        print(json.dumps(out))
        return

    if args.profile_lu:
        ns = W.torus_staggered(82)
        op0 = R.build_operator(T(ns.X), T(ns.normals), 50, kernel="imq", kappa_target=KAPPA_T)
        perm = R.rcm_order(op0).cpu().numpy()
        del op0
        opl = R.build_operator(T(ns.X[perm]), T(ns.normals[perm]), 50, kernel="imq", kappa_target=KAPPA_T)
        R.release_memory()
        s = W.SCHNAKENBERG
        name, coef = R.model_coefs(s)
        u0, v0 = W.schnakenberg_initial(ns.N, seed=2)
        pl = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                          delta_v=s["delta_v"], coef=coef, use_graph=False, solver="lu")
        stl = R.StepState.create(T(u0[perm], torch.float32), T(v0[perm], torch.float32))
        R.step_imex(opl, stl, pl, 2)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        R.step_imex(opl, stl, pl, 1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": "torus_40344_rcm_lu_step", "N": ns.N, "bandwidths": list(R.op_bandwidth(opl))}))
        return

    if args.profile and args.profile_step:
        op = R.build_operator(X, Nr, NP, kernel="imq", kappa_target=KAPPA_T, mlps=nets)
        R.release_memory()
        st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
        R.step_imex(op, st, sp, 4)
        host = R.StepParams(model=name, nspecies=2, dtype=torch.float32, dt=s["dt"], delta_u=s["delta_u"],
                            delta_v=s["delta_v"], coef=coef, tol=1e-6, use_graph=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        rep = R.step_imex(op, st, host, 3)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": f"fibonacci_sphere_{n_nodes}_mixed_n_step", "N": n_nodes,
                          "nnz": op.nnz, "steps": 3, "total_iters": rep["total_iters"],
                          "max_iters": [rep["max_iters_u"], rep["max_iters_v"]]}))
        return

    if args.profile:
        for _ in range(2):
            one_step(X, Nr, NP)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        op = one_step(X, Nr, NP)
        uu = torch.rand(n_nodes, dtype=torch.float32, device=dev)
        R.apply(op, uu)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": f"fibonacci_sphere_{n_nodes}_mixed_n", "N": n_nodes,
                          "learned": nets is not None,
                          "phases_ms": R.get_build_timings(op)}))
        return

    # plain search once (untimed) for the learned-vs-plain speedup
    torch.cuda.synchronize()
    op_plain = R.build_operator(X, Nr, NP, kernel="imq", kappa_target=KAPPA_T,
                                block_threads=shape["block_threads"], blocks_per_sm=shape["blocks_per_sm"])
    plain_ms = R.get_build_timings(op_plain)
    plain_evals = R.get_stencil_info(op_plain)["evals"].double().mean().item()
    del op_plain

    for _ in range(args.warmup):
        flush.fill_(1.0)
        op = one_step(X, Nr, NP)
    torch.cuda.synchronize()

    times, phases = [], []
    l0 = R.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            op = one_step(X, Nr, NP)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            phases.append(R.get_build_timings(op))
            evals_t = R.get_stencil_info(op)["evals"]
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = R.launch_count() - l0
    if ws > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(statistics.mean(times), dev)

    # end to end through the public API: the step's inputs go up from
    # pinned host memory, and the product of the build -- the operator as
    # sliced ELL (int32 indices and float64 weights, padding included) and
    # the per-node eps -- comes back into pinned host memory, all inside the
    # timed region
    hX = torch.from_numpy(ns.X).pin_memory()
    hN = torch.from_numpy(ns.normals).pin_memory()
    hP = torch.from_numpy(nper).pin_memory()
    elems = R.get_ell(op)["elems"]
    hI = torch.empty(elems, dtype=torch.int32).pin_memory()
    hW = torch.empty(elems, dtype=torch.float64).pin_memory()
    hE = torch.empty(N_NODES, dtype=torch.float64).pin_memory()
    e2e_times, e2e_phases, e2e_split = [], [], []
    # one untimed round first (as the device-timed loop has its warm-up): the
    # first host-to-device copies into fresh device tensors take new blocks
    # from torch's allocator
    for it in range(1 + max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        sev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        t0 = time.perf_counter()
        sev[0].record(stream)
        Xd = hX.to(dev, non_blocking=True)
        Nd = hN.to(dev, non_blocking=True)
        Pd = hP.to(dev, non_blocking=True)
        sev[1].record(stream)
        op = one_step(Xd, Nd, Pd)
        sev[2].record(stream)
        e2e_phases.append(R.get_build_timings(op))
        ell = R.get_ell(op)
        sev[3].record(stream)
        hI.copy_(ell["idx"], non_blocking=True)
        sev[4].record(stream)
        hW.copy_(ell["w64"], non_blocking=True)
        sev[5].record(stream)
        hE.copy_(R.get_eps(op)[0], non_blocking=True)
        sev[6].record(stream)
        torch.cuda.synchronize()
        if it > 0:
            e2e_times.append(time.perf_counter() - t0)
            e2e_split.append([sev[i].elapsed_time(sev[i + 1]) for i in range(6)])
    h2d = hX.numel() * 8 + hN.numel() * 8 + hP.numel() * 4
    d2h = hI.numel() * 4 + hW.numel() * 8 + hE.numel() * 8
    # the same step without the networks (the plain eps search), timed once
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    op_p = R.build_operator(X, Nr, NP, kernel="imq", kappa_target=KAPPA_T,
                            block_threads=shape["block_threads"], blocks_per_sm=shape["blocks_per_sm"])
    stp = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
    R.step_imex(op_p, stp, sp, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_step_ms = e0.elapsed_time(e1)
    del op_p, stp

    info = {k: v.cpu().numpy() for k, v in R.get_stencil_info(op).items()}
    ok = bool(np.all((info["status"] == 0) | (info["status"] == 4)))

    if rank != 0:
        return
    configs = configs_report(R, W, T, torch, nets) if (nets is not None and not args.no_extras) else None
    # ---- roofline of the search kernel (float64 ALU): evaluations it performed
    E = {int(n): float(statistics.median(v)) for n, v in cpu["evals"].items()}
    ev_np = evals_t.cpu().numpy().astype(np.float64)
    alg_flops_search = sum(float(ev_np[nper == n].sum()) * (n + 1) ** 3 / 3.0 for n in SIZES)
    # the same count with every stencil charged the oracle's median number of
    # evaluations E_n plus one final factorisation (the weights), whatever the
    # launch did: the learned start's saving then shows as a higher rate
    flops_at_E = sum(float(np.sum(nper == n)) * (E[int(n)] + 1.0) * (n + 1) ** 3 / 3.0 for n in SIZES)
    search_ms = statistics.mean(p["search"] for p in phases)
    peak = R.fp64_peak() / 1e3   # TFLOP/s, measured FMA throughput
    peak_mma = R.fp64_mma_peak() / 1e3   # the FP64 tensor path, for comparison
    achieved = alg_flops_search / (search_ms * 1e-3) / 1e12
    traffic = SEARCH_TRAFFIC.get(_file_hash(os.path.join(ROOT, "paper_1404_0812_gb300", "csrc", "build.cu")))
    # apply bandwidth of the built operator (HBM; matrix far larger than L2)
    apply = {}
    for dt, code in ((torch.float32, R.F32), (torch.float64, R.F64)):
        uu = torch.rand(N_NODES, dtype=dt, device=dev)
        yy = torch.empty_like(uu)
        for _ in range(3):
            R.apply(op, uu, yy)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(20):
            R.apply(op, uu, yy)
        a1.record(stream)
        torch.cuda.synchronize()
        ams = a0.elapsed_time(a1) / 20
        gbs = op.apply_bytes(code) / (ams * 1e-3) / 1e9
        apply["f32" if code == R.F32 else "f64"] = {"ms": round(ams, 4), "GB_s": round(gbs, 1)}
    # IMEX step on the built operator: ten graph-replayed steps, each timed
    # with events and its own report, so that the ELL passes of every step
    # are exact: phase R + 2 per BiCGSTAB iteration of the slower species
    # (both species share each pass) x (nnz x 8 B: float32 weight + int32
    # index); the Krylov vectors (~152 B per node and iteration for two
    # float32 species) come on top and are not counted
    st = R.StepState.create(T(u0, torch.float32), T(v0, torch.float32))
    R.step_imex(op, st, sp, 3)
    step_times, step_passes, step_its = [], 0, []
    for _ in range(10):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s0.record(stream)
        r1 = R.step_imex(op, st, sp, 1)
        s1.record(stream)
        torch.cuda.synchronize()
        step_times.append(s0.elapsed_time(s1))
        it = max(r1["max_iters_u"], r1["max_iters_v"])
        step_its.append(it)
        step_passes += 1 + 2 * it
    step_ms = statistics.mean(step_times)
    ell_bytes = op.nnz * 8.0
    ell_gbs = step_passes * ell_bytes / (sum(step_times) * 1e-3) / 1e9
    step_info = {"ms": round(step_ms, 3), "loop_iterations_per_step": step_its,
                 "ell_passes_per_step": round(step_passes / 10.0, 2),
                 "ell_GB_s": round(ell_gbs, 1),
                 "path": ("phase kernels under a WHILE graph node"
                          if N_NODES >= 1024 * torch.cuda.get_device_properties(dev).multi_processor_count
                          else "cooperative")}
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        hbm = 6800.0
    for v in apply.values():
        v["frac_of_measured_hbm"] = round(v["GB_s"] / hbm, 3)
    step_info["ell_frac_of_measured_hbm"] = round(step_info["ell_GB_s"] / hbm, 3)
    learned_ms = statistics.mean(p["guess"] + p["search"] for p in phases)
    value = ws * N_NODES / (ms * 1e-3)
    cpu_value = cpu["count"] / cpu["seconds"]
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fibonacci_sphere_1M_mixed_n", "N": N_NODES, "n": list(SIZES),
                   "groups": "4 contiguous index bands of 250k", "kernel": "imq", "kappa_T": KAPPA_T,
                   "eps_tol": 1e-4, "learned_start": nets is not None,
                   "imex_step": "schnakenberg f32, 1 step, CUDA graph", "l2": "flushed (256 MB write) per step",
                   "launch_shape": {k: shape[k] for k in ("block_threads", "blocks_per_sm")},
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "kernel": "search_kernel (float64)", "achieved": round(achieved, 4),
                     "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "peak_source": "measured FP64 FMA microbenchmark (rbffd_fp64_peak)",
                     "fp64_tensor_peak_measured": round(peak_mma, 4),
                     "traffic": traffic, "flops_per_launch": alg_flops_search,
                     "evals_mean_by_n": {int(n): round(float(ev_np[nper == n].mean()), 3) for n in SIZES},
                     "E_oracle_median": E, "search_ms": round(search_ms, 3),
                     "charged_at_oracle_E": {"flops_per_launch": flops_at_E,
                                             "achieved": round(flops_at_E / (search_ms * 1e-3) / 1e12, 4),
                                             "frac": round(flops_at_E / (search_ms * 1e-3) / 1e12 / peak, 4)}},
        "phases_ms": {k: round(statistics.mean(p[k] for p in phases), 3) for k in phases[0]},
        "learned_speedup": {"plain_search_ms": round(plain_ms["search"], 3),
                            "learned_guess_plus_search_ms": round(learned_ms, 3),
                            "speedup": round(plain_ms["search"] / learned_ms, 3),
                            "plain_evals_mean": round(plain_evals, 3),
                            "learned_evals_mean": round(float(info["evals"].mean()), 3),
                            "accepted_fraction": round(float((info["status"] == 4).mean()), 4)},
        "apply": apply,
        "imex_step": step_info,
        "mlp_train": TRAIN_STATS or None,
        "all_stencils_ok": ok,
        "other_configs": configs,
        "e2e": {"value": round(N_NODES / statistics.mean(e2e_times), 1), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": [round(t * 1e3, 3) for t in e2e_times], "warmup": 1,
                "phases_ms": {k: round(statistics.mean(p[k] for p in e2e_phases[1:]), 3) for k in e2e_phases[0]},
                "events_ms": {k: round(statistics.mean(x[i] for x in e2e_split), 3) for i, k in enumerate(
                    ("h2d", "build_and_step", "views", "d2h_idx", "d2h_w64", "eps"))},
                "returned": "the built operator (sliced ELL: int32 indices + float64 weights) and eps"},
        "rates": {"learned_start_in_distribution": round(value, 1),
                  "plain_search_no_networks": round(N_NODES / (plain_step_ms * 1e-3), 1),
                  "learned_start_held_out_bumpy500k":
                      (configs or {}).get("bumpy500k_learned", {}).get("stencils_per_s_learned_build"),
                  "held_out_accepted_fraction":
                      (configs or {}).get("bumpy500k_learned", {}).get("learned", {}).get("accepted_fraction"),
                  "note": "value = the learned start on the networks' own distribution (networks trained on "
                          "Fibonacci spheres and tori); the plain search and the held-out bumpy sphere beside it"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": {"value": round(cpu_value, 3), "unit": UNIT, "cores": cpu["procs"], "kind": "oracle",
                         "sample": f"{cpu['count']} stencils ({args.sample} per n per core, one single-threaded "
                                   f"process per core) of the same 1M-node workload: brute-force stencil, "
                                   f"Brent eps search, full G^d weights",
                         "one_core": round(cpu1["count"] / cpu1["seconds"], 3)},
    }
    print(json.dumps(line))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    times, counts, evals = [], [], []
    cores = host_cores()
    for i in range(args.warmup + args.steps):
        r = run_cpu_sample(args.sample, 1000 + i, cores)
        if i >= args.warmup:
            times.append(r["seconds"])
            counts.append(r["count"])
    value = sum(counts) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "fibonacci_sphere_1M_mixed_n", "N": N_NODES, "n": list(SIZES),
                   "kernel": "imq", "kappa_T": KAPPA_T, "eps_tol": 1e-4},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.sample} stencils per n per core per step of the 1M-node workload "
                                   f"(one single-threaded process per core)"},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = _parse()
    if args.cpu_worker:
        cpu_worker(args.cpu_worker, args.sample)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
