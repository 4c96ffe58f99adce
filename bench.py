"""Benchmark of the 3DPIFCM hot path on GB300: IFCM voxel x particle x
iteration updates per second for whole Algorithm 1 runs.

One step = one complete 3DPIFCM run (Algorithm 1 / Algorithm 2) on the
181x217x181 brain stand-in: min-max normalisation, the FCM start, 30 swarm
generations of 20 particles (each particle one IFCM run of <= 50 iterations
stopping at max|du| < 1e-5, all particles batched), the swarm updates and the
final IFCM run at the best particle.  Inputs are resident in HBM before the
timed region; the per-step membership buffers (4.6 GB) exceed the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own volume (seed + rank): independent
problems, weak scaling, no data-path collective; timings are reduced with a
MAX over ranks.  ``--impl reference`` times the FP64 oracle on the host cores
(bounded samples of the same workload).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IFCM voxel·particle·iter updates/s (batched vs plain), % of HBM roofline"
UNIT = "updates/s"
SHAPE = (181, 217, 181)            # (nz, ny, nx)
C, M = 4, 2.0
P, GENERATIONS, MAX_ITER, EPS = 20, 30, 50, 1e-5
INIT_MAX_ITER = 300
SEED = 2
WORKLOAD = ("brain stand-in 181x217x181 (nested ellipsoids 0/0.25/0.55/0.85, +-10% bias, "
            "Rician sigma 0.07), c=4, m=2, 26-neighbourhood, 20 particles x 30 generations, "
            "<=50 IFCM iterations per fitness, stop max|du|<1e-5")
CPU_SLAB = 48                      # z-planes of the oracle's bounded sample


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ helpers
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(dist, world, seconds, updates, device):
    """Whole-job figures over the ranks (one process per GPU, each on its own
    volume): the slowest rank's seconds and the sum of all ranks' updates.
    Used only for measurement; no membership data crosses ranks."""
    if world == 1:
        return float(seconds), float(updates)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(rank):
    """Seed of rank r's phantom and swarm: independent problems per GPU."""
    return SEED + rank


def stencil_source_sha():
    """Hash of the sources that generate the FP32 pair-word stencil kernel."""
    h = hashlib.sha256()
    for name in ("stencil3d.cuh", "stencil_kernel.cuh", "ifcm_stencil_f32p_np2.cu",
                 "ifcm_math.cuh", "common.cuh", "launch.h"):
        with open(os.path.join(ROOT, "paper_2002_01981_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stencil_traffic_per_update(plan_np, plan_tz):
    """DRAM bytes per update of the stencil kernel from the committed ncu
    summary, if it was taken on the current kernel source and plan."""
    path = os.path.join(ROOT, "profiles", "stencil_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        pl = d.get("plan", {})
        if (d.get("kernel_source_sha") == stencil_source_sha() and
                pl.get("particles_per_item") == plan_np and pl.get("tz") == plan_tz):
            return float(d["dram_bytes_per_update"])
    except Exception:
        pass
    return None


def launches_per_run(init_iters_launched, generations, max_iter):
    # normalise (2) + FCM start (state init + 2 per iteration + copy) + swarm
    # init + 1/G of the volume (once) + per generation (state init + start
    # packing into pair words + 2 per iteration + swarm step) + best + final
    # run (state init + start packing + 2 per iteration + copy) + result.
    return (2 + 1 + 2 * init_iters_launched + 1 + 1 + 1 +
            generations * (1 + 1 + 2 * max_iter + 1) + 1 +
            (1 + 1 + 2 * max_iter + 1) + 1)


def plain_form_rate(G, vol, nx, prm, opts, stream, particles=2):
    """Updates/s of the plain comparison form on the same volume and
    parameters: the FCM start, then `particles` IFCM runs one after another,
    each one particle per launch with the host checking convergence after
    every iteration (the shape of the paper's Algorithm 2)."""
    import torch
    x = G.ifcm_normalize(vol, nx=nx)
    U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=prm.c, m=prm.m, max_iter=opts.init_max_iter,
                                          eps_u=prm.eps_u), (0.0, 0.0), nx=nx, plain=True)
    lam_xi = [(0.5, 0.3), (0.8, 0.6), (0.2, 0.7), (0.6, 0.1)][:particles]
    N = int(x.shape[0]) * int(x.shape[1]) * nx
    G.ifcm_fit(x, G.Params(c=prm.c, m=prm.m, max_iter=2, eps_u=0.0), lam_xi[0], nx=nx,
               u_init=U0, c_init=C0, plain=True)                       # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters = 0
    for lx in lam_xi:
        _, _, _, it = G.ifcm_fit(x, prm, lx, nx=nx, u_init=U0, c_init=C0, plain=True)
        iters += it
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"value": iters * N / el, "unit": UNIT, "iterations": iters,
            "sample": f"{particles} particles, one IFCM run each (<= {prm.max_iter} iterations, "
                      f"host stop test per iteration), plain kernel, same volume"}


# ------------------------------------------------- many volumes at once
BATCH_VOLUMES = 48
BATCH_P = 32
BATCH_BUDGET = 48 << 30            # workspace bytes: the c = 5 and c = 6 groups take two waves
BATCH_WORKLOAD = (f"{BATCH_VOLUMES} phantoms of uneven size (each side U{{64..224}}), c U{{4,5,6}}, "
                  f"Rician sigma 0.03/0.07/0.12, {BATCH_P} particles each, <= {MAX_ITER} IFCM "
                  f"iterations per fitness, stop max|du|<{EPS:g}")


def batching_leg(G, phantoms, dev):
    """Fitness of every particle of every volume of the uneven batch: the
    captured multi-volume call (volumes of one c share each launch) against
    one pso_fitness_batch call per volume, both on the same workspace."""
    import torch
    vols, nvox = [], []
    for k, (raw, c) in enumerate(phantoms.uneven_volumes(BATCH_VOLUMES, seed=3)):
        nz, ny, nx = raw.shape
        v = torch.from_numpy(phantoms.pad_pitch(raw)).to(dev)
        x = G.ifcm_normalize(v, nx=nx)
        U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=c, m=M, max_iter=INIT_MAX_ITER, eps_u=EPS),
                                  (0.0, 0.0), nx=nx)
        lam = torch.rand((BATCH_P, 2), generator=torch.Generator().manual_seed(k),
                         dtype=torch.float64).to(dev)
        vols.append(G.BatchVolume(x, c, lam, U0, C0, nx=nx))
        nvox.append(nz * ny * nx)
    prm = G.Params(m=M, max_iter=MAX_ITER, eps_u=EPS)
    ws = G.workspace(BATCH_BUDGET, dev)
    waves = G.pso_fitness_multi_waves(vols, prm, ws.numel())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed_graph():
        graph = G.pso_fitness_multi_graph(vols, prm, ws=ws)
        graph.launch()
        graph.check()
        torch.cuda.synchronize()
        ev0.record()
        graph.launch()
        ev1.record()
        graph.check()
        ms = ev0.elapsed_time(ev1)
        upd = sum(int(its.sum()) * n for (_, its), n in zip(graph.outputs, nvox))
        graph.close()
        return ms, upd

    # the built-in plan rule, then plans timed by the autotuner on one
    # uncaptured call (a stream being captured is never timed; the capture
    # then takes the cached plans)
    G.autotune(0)
    ms_batched, updates = timed_graph()
    G.autotune(1)
    t0 = time.perf_counter()
    G.pso_fitness_multi(vols, prm, ws=ws)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    ms_tuned, upd_tuned = timed_graph()
    G.autotune(0)

    torch.cuda.synchronize()
    ev0.record()
    loop_updates = 0
    for v, n in zip(vols, nvox):
        _, its, _ = G.pso_fitness_batch(v.x, G.Params(c=v.c, m=M, max_iter=MAX_ITER, eps_u=EPS),
                                        v.lam_xi, v.u0, v.c0, nx=v.nx, ws=ws)
        loop_updates += int(its.sum()) * n
    ev1.record()
    torch.cuda.synchronize()
    ms_loop = ev0.elapsed_time(ev1)
    del ws, vols
    torch.cuda.empty_cache()
    batched = updates / (ms_batched / 1e3)
    loop = loop_updates / (ms_loop / 1e3)
    return {"workload": BATCH_WORKLOAD, "volumes": BATCH_VOLUMES,
            "particles": BATCH_VOLUMES * BATCH_P, "voxels": int(sum(nvox)),
            "workspace_bytes": BATCH_BUDGET, "waves": waves,
            "batched_graph": {"value": batched, "unit": UNIT, "ms": ms_batched,
                              "updates": updates, "plans": "built-in rule"},
            "batched_graph_autotuned": {"value": upd_tuned / (ms_tuned / 1e3), "unit": UNIT,
                                        "ms": ms_tuned, "updates": upd_tuned,
                                        "tuning_call_s": tune_s,
                                        "over_rule": (upd_tuned / ms_tuned) /
                                                     (updates / ms_batched)},
            "per_volume": {"value": loop, "unit": UNIT, "ms": ms_loop,
                           "updates": loop_updates},
            "batched_over_per_volume": batched / loop}


# ------------------------------------------- membership storage precision
PREC_SHAPE = (256, 256, 256)
PREC_C, PREC_P, PREC_GEN = 6, 64, 40
PREC_WORKLOAD = ("background + 5 tissues 256^3 (0/0.2/0.35/0.5/0.7/0.9), Rician sigma 0.1, c=6, "
                 "m=2, 26-neighbourhood, one generation of 64 particles (swarm init, seed 5), "
                 f"<= {MAX_ITER} IFCM iterations per fitness, stop max|du|<{EPS:g}; full_run: "
                 f"one whole Algorithm 1 run of {PREC_P} particles x {PREC_GEN} generations")


def precision_leg(G, phantoms, dev):
    """One generation's fitness batch of the c = 6 workload with FP32
    memberships, bf16 memberships (FP64 sums) and bf16 memberships with
    compensated FP32 sums: updates/s, the stencil kernel's achieved bytes,
    and the bf16 forms' agreement with the FP32 form at full size (fitness,
    iteration counts; labels, centres and J of one run at the FP32 form's
    best particle).  Errors against the FP64 oracle are measured by the GPU
    tests on a slab of this workload."""
    import torch
    raw = phantoms.multi_tissue(PREC_SHAPE, seed=5, sigma=0.1)
    nz, ny, nx = PREC_SHAPE
    N = nz * ny * nx
    vol = torch.from_numpy(phantoms.pad_pitch(raw)).to(dev)
    del raw
    x = G.ifcm_normalize(vol, nx=nx)
    U0, C0, _, it0 = G.ifcm_fit(x, G.Params(c=PREC_C, m=M, max_iter=INIT_MAX_ITER, eps_u=EPS),
                                (0.0, 0.0), nx=nx)
    sw = G.Swarm(PREC_P, seed=5).init()
    lam_xi = sw.x.clone()
    variants = [("fp32", "fp64"), ("bf16", "fp64"), ("bf16", "comp32")]
    need = max(G.pso_fitness_batch_workspace_bytes(
        x, G.Params(c=PREC_C, u_dtype=d, reduce=r), PREC_P, nx=nx) for d, r in variants)
    ws = G.workspace(need, dev)
    hbm, _ = peaks()
    out = {"workload": PREC_WORKLOAD, "fcm_start_iterations": int(it0), "variants": {}}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fits = {}
    for d, r in variants:
        prm = G.Params(c=PREC_C, m=M, max_iter=MAX_ITER, eps_u=EPS, u_dtype=d, reduce=r)
        G.pso_fitness_batch(x, prm, lam_xi, U0, C0, nx=nx, ws=ws)        # warm
        torch.cuda.synchronize()
        G.profile_read()
        G.profile_enable(True)
        ev0.record()
        fit, its, _ = G.pso_fitness_batch(x, prm, lam_xi, U0, C0, nx=nx, ws=ws)
        ev1.record()
        torch.cuda.synchronize()
        G.profile_enable(False)
        kms, nl = G.profile_read()
        ms = ev0.elapsed_time(ev1)
        upd = int(its.sum()) * N
        np_, _, _ = G.stencil_plan(G.shape_of(x, nx), PREC_C, PREC_P)
        s_u = 4 if d == "fp32" else 2
        bpu = 2 * PREC_C * s_u + 4.0 / np_
        ach = upd * bpu / (kms / 1e3) / 1e9
        fits[(d, r)] = (fit.cpu().numpy(), its.cpu().numpy())
        out["variants"][f"{d}/{r}"] = {
            "value": upd / (ms / 1e3), "unit": UNIT, "ms": ms, "updates": upd,
            "stencil": {"bytes_per_update": bpu, "achieved_gbs": ach, "frac": ach / hbm,
                        "kernel_ms": kms, "launches": nl}}
    f32, i32 = fits[("fp32", "fp64")]
    best = int(np.argmin(f32))
    lx = lam_xi[best].cpu().numpy()
    prm32 = G.Params(c=PREC_C, m=M, max_iter=MAX_ITER, eps_u=EPS)
    U32, C32, J32, _ = G.ifcm_fit(x, prm32, lx, nx=nx, u_init=U0, c_init=C0)
    lab32 = torch.argmax(U32[..., :nx], dim=0)
    c32 = C32.cpu().numpy()
    del U32
    for d, r in variants[1:]:
        fb, ib = fits[(d, r)]
        prm = G.Params(c=PREC_C, m=M, max_iter=MAX_ITER, eps_u=EPS, u_dtype=d, reduce=r)
        Ub, Cb, Jb, _ = G.ifcm_fit(x, prm, lx, nx=nx, u_init=U0, c_init=C0)
        agree = float((torch.argmax(Ub[..., :nx], dim=0) == lab32).double().mean())
        del Ub
        out["variants"][f"{d}/{r}"]["vs_fp32"] = {
            "fitness_max_rel": float(np.max(np.abs(fb / f32 - 1.0))),
            "iterations_equal": float(np.mean(ib == i32)),
            "best_particle_run": {"labels_agree": agree,
                                  "centres_max_rel": float(np.max(np.abs(Cb.cpu().numpy() / c32
                                                                         - 1.0))),
                                  "J_rel": abs(Jb / J32 - 1.0)}}
    v32 = out["variants"]["fp32/fp64"]["value"]
    for k, v in out["variants"].items():
        v["over_fp32"] = v["value"] / v32
    del ws, x, U0
    torch.cuda.empty_cache()
    out["full_run"] = precision_full_runs(G, vol, nx)
    del vol
    torch.cuda.empty_cache()
    return out


def precision_full_runs(G, vol, nx):
    """The c = 6 workload as stated: one whole Algorithm 1 run of 64 particles
    x 40 generations (<= 50 iterations each, FCM start <= 300 iterations),
    with FP32 and with bf16 memberships (FP64 sums): seconds, updates/s, the
    best (lambda, xi), and the bf16 run's final segmentation against the FP32
    run's (labels, centres, J)."""
    import torch
    opts = G.Options(P=PREC_P, generations=PREC_GEN, seed=5, init_max_iter=INIT_MAX_ITER)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    out, ref = {}, None
    for d in ("fp32", "bf16"):
        prm = G.Params(c=PREC_C, m=M, max_iter=MAX_ITER, eps_u=EPS, u_dtype=d)
        bufs = G.pifcm3d_buffers(vol, prm, opts, nx=nx)
        torch.cuda.synchronize()
        ev0.record()
        U, res = G.pifcm3d(vol, prm, opts, nx=nx, buffers=bufs)
        ev1.record()
        torch.cuda.synchronize()
        s = ev0.elapsed_time(ev1) / 1e3
        lab = torch.argmax(U[..., :nx], dim=0)
        r = {"seconds": s, "updates": int(res["updates"]), "value": res["updates"] / s,
             "unit": UNIT, "lambda_xi": [res["lambda"], res["xi"]], "J": res["J"],
             "best_fitness": res["best_fitness"], "iters_final": res["iters_final"]}
        if ref is None:
            ref = (lab, np.asarray(res["centres"][:PREC_C]), res["J"], r["value"])
        else:
            r["vs_fp32"] = {"labels_agree": float((lab == ref[0]).double().mean()),
                            "centres_max_rel": float(np.max(np.abs(
                                np.asarray(res["centres"][:PREC_C]) / ref[1] - 1.0))),
                            "J_rel": abs(res["J"] / ref[2] - 1.0),
                            "over_fp32": r["value"] / ref[3]}
        out[d] = r
        del U, bufs, lab
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------- differentiation
DIFF_SHAPE = (128, 128, 128)
DIFF_C, DIFF_K, DIFF_P, DIFF_GEN, DIFF_STEPS = 4, 20, 20, 10, 10
DIFF_WORKLOAD = ("nested ellipsoids 128^3 (0/0.25/0.55/0.85) + Gaussian sigma 0.09, c=4, m=2, "
                 f"dJ/d(lambda, xi) through K={DIFF_K} unrolled IFCM iterations with per-iteration "
                 f"membership checkpoints; swarm of {DIFF_P} x {DIFF_GEN} generations on the same "
                 f"objective, then {DIFF_STEPS} projected gradient steps from its best particle")


def differentiation_leg(G, phantoms, dev):
    """Gradient evaluations of the c = 4 128^3 workload: time of one
    ifcm_grad (checkpointed forward + reverse) with the adjoint kernels'
    share and achieved bytes; a central-difference check of the gradient
    on the FP32 forward (h = 1e-3); and the polish of the swarm's best
    particle (J before / after)."""
    import torch
    raw = phantoms.gaussian_phantom(DIFF_SHAPE, seed=4, sigma=0.09)
    nz, ny, nx = DIFF_SHAPE
    N = nz * ny * nx
    x = G.ifcm_normalize(torch.from_numpy(phantoms.pad_pitch(raw)).to(dev), nx=nx)
    U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=DIFF_C, m=M, max_iter=INIT_MAX_ITER, eps_u=EPS),
                              (0.0, 0.0), nx=nx)
    prm = G.Params(c=DIFF_C, m=M, max_iter=DIFF_K, eps_u=0.0)
    sw = G.Swarm(DIFF_P, seed=4).init()
    for _ in range(DIFF_GEN):
        fit, _, _ = G.pso_fitness_batch(x, prm, sw.x, U0, C0, nx=nx)
        sw.step(fit)
    best = int(torch.argmin(sw.pbest_f))
    start = sw.pbest_x[best].clone()
    J0 = float(sw.pbest_f[best])
    ws = G.workspace(G.ifcm_grad_workspace_bytes(x, prm, DIFF_K, nx=nx), dev)
    G.ifcm_grad(x, prm, start, U0, C0, DIFF_K, nx=nx, ws=ws)              # warm
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for k in (G.PROF_STENCIL, G.PROF_ADJOINT_POINT, G.PROF_ADJOINT_GATHER):
        G.profile_read(k)
    G.profile_enable(True)
    reps = 5
    ev0.record()
    for _ in range(reps):
        J, g = G.ifcm_grad(x, prm, start, U0, C0, DIFF_K, nx=nx, ws=ws)
    ev1.record()
    torch.cuda.synchronize()
    G.profile_enable(False)
    ms = ev0.elapsed_time(ev1) / reps
    fwd_ms, fwd_n = G.profile_read(G.PROF_STENCIL)
    pt_ms, pt_n = G.profile_read(G.PROF_ADJOINT_POINT)
    ga_ms, ga_n = G.profile_read(G.PROF_ADJOINT_GATHER)
    g = g.cpu().numpy()
    hbm, _ = peaks()
    c = DIFF_C
    # point kernel: x, U^t, u_bar^{t+1} (not at the last iteration) read, A, B, e
    # written; gather: x, A, B, e, U^t read, u_bar^t written (4-byte elements)
    pt_bytes = N * ((8 + 16 * c) * pt_n - 4 * c * reps) / pt_n
    ga_bytes = N * (4 + 8 * c + 4 + 4 * c + 4 * c)
    # the swarm's best sits where reading R8 drives it (large lambda + xi, the
    # clamp of reading R2 active at many voxels); the derivative is checked
    # and the polish shown at an interior point as well, where it is not
    interior = np.array([0.3, 0.2])
    h = 1e-3

    def grad_check(pt):
        J_, g_ = G.ifcm_grad(x, prm, pt, U0, C0, DIFF_K, nx=nx, ws=ws)
        g_ = g_.cpu().numpy()
        f = lambda a, b: float(G.ifcm_grad(x, prm, (a, b), U0, C0, DIFF_K, nx=nx, ws=ws)[0])  # noqa
        fd = [(f(pt[0] + h, pt[1]) - f(pt[0] - h, pt[1])) / (2 * h),
              (f(pt[0], pt[1] + h) - f(pt[0], pt[1] - h)) / (2 * h)]
        return {"lambda_xi": [float(v) for v in pt], "J": float(J_), "grad": g_.tolist(),
                "central_difference_h1e-3": fd,
                "rel_diff": [abs(g_[i] / fd[i] - 1.0) if fd[i] else None for i in range(2)]}

    def polish(pt):
        J_start = float(G.ifcm_grad(x, prm, pt, U0, C0, DIFF_K, nx=nx, ws=ws)[0])
        torch.cuda.synchronize()
        ev0.record()
        lp, Jp = G.ifcm_polish(x, prm, pt, U0, C0, DIFF_K, steps=DIFF_STEPS, step0=0.05,
                               decay=0.7, nx=nx, ws=ws)
        ev1.record()
        torch.cuda.synchronize()
        return {"steps": DIFF_STEPS, "ms": ev0.elapsed_time(ev1), "J_before": J_start,
                "J_after": Jp, "lambda_xi_before": [float(v) for v in pt],
                "lambda_xi_after": lp.cpu().numpy().tolist()}

    lx = start.cpu().numpy()
    out = {"workload": DIFF_WORKLOAD,
           "grad_eval": {"ms": ms, "per_s": 1e3 / ms,
                         "forward_stencil_ms": fwd_ms / reps,
                         "adjoint_point": {"ms": pt_ms / reps,
                                           "achieved_gbs": pt_bytes * pt_n / (pt_ms / 1e3) / 1e9,
                                           "bytes_per_voxel": pt_bytes / N},
                         "adjoint_gather": {"ms": ga_ms / reps,
                                            "achieved_gbs": ga_bytes * ga_n / (ga_ms / 1e3) / 1e9,
                                            "bytes_per_voxel": ga_bytes / N},
                         "voxel_iterations_per_s": 2 * DIFF_K * N / (ms / 1e3)},
           "swarm_best": {"lambda_xi": lx.tolist(), "pbest_J": J0,
                          "grad": [float(v) for v in g]},
           "interior_point": grad_check(interior),
           "polish_from_swarm_best": polish(lx),
           "polish_from_interior_point": polish(interior)}
    for k in ("adjoint_point", "adjoint_gather"):
        out["grad_eval"][k]["frac"] = out["grad_eval"][k]["achieved_gbs"] / hbm
    del ws, x, U0
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------- 2D size sweep (Table 7)
SWEEP_WORKLOAD = ("n x n slices of the brain stand-in (Rician sigma 0.07), n = 32, 55, 95, 165, "
                  "285, 493, 854 (the sizes of the paper's Table 7); one whole Algorithm 1 run "
                  "each: c=4, m=2, 8-neighbourhood, 20 particles x 30 generations, <= 50 "
                  "iterations per fitness, stop max|du|<1e-5, FCM start <= 300 iterations")


def sweep_leg(G, phantoms, dev, runs=2):
    """Whole Algorithm 1 runs on the 2D sweep: seconds per run (mean of
    `runs` after one warm run, CUDA events) and updates/s.  Small slices are
    bound by launch latency (~3800 launches per run), large ones by the
    stencil."""
    import torch
    out = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for n in phantoms.SWEEP_SIZES:
        raw = phantoms.brain_slice(n, seed=2, sigma=0.07)
        vol = torch.from_numpy(phantoms.pad_pitch(raw)).to(dev)
        prm = G.Params(c=C, m=M, max_iter=MAX_ITER, eps_u=EPS)
        opts = G.Options(P=P, generations=GENERATIONS, seed=SEED, init_max_iter=INIT_MAX_ITER)
        bufs = G.pifcm3d_buffers(vol, prm, opts, nx=n)
        G.pifcm3d(vol, prm, opts, nx=n, buffers=bufs)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(runs):
            G.pifcm3d(vol, prm, opts, nx=n, buffers=bufs, sync=False)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / runs
        _, res = G.pifcm3d(vol, prm, opts, nx=n, buffers=bufs)
        # the same run captured once into a CUDA graph (pifcm3d_graph: the
        # ~3800 launches of a run in one graph) and replayed
        graph = G.pifcm3d_graph(vol, prm, opts, nx=n, buffers=bufs)
        graph.launch()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(runs):
            graph.launch()
        ev1.record()
        torch.cuda.synchronize()
        ms_g = ev0.elapsed_time(ev1) / runs
        res_g = graph.result()
        graph.close()
        out.append({"n": n, "seconds_per_run": ms / 1e3, "updates": res["updates"],
                    "value": res["updates"] / (ms / 1e3), "unit": UNIT,
                    "graph": {"seconds_per_run": ms_g / 1e3,
                              "value": res["updates"] / (ms_g / 1e3)},
                    "lambda_xi": [res["lambda"], res["xi"]],
                    "graph_result_equal": res_g == res})
    return {"workload": SWEEP_WORKLOAD, "sizes": out}


# ------------------------------------------------------------ CPU oracle
def _oracle_particle_iteration(args):
    """One FP64 oracle IFCM iteration of one particle on a slab (a worker of
    the all-cores baseline): returns (seconds, voxels, J)."""
    x, lam, xi = args
    from oracle import ifcm as O
    U = np.full((C,) + x.shape, 1.0 / C)
    Cc = (np.arange(C) + 0.5) / C
    t0 = time.perf_counter()
    _, _, J, _ = O.ifcm_iteration(x, U, Cc, lam, xi)
    return time.perf_counter() - t0, x.size, J


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_all_cores_rate(raw):
    """Updates/s of the FP64 oracle over all host cores: one particle per
    worker process (spawned: this process already holds a CUDA context),
    one IFCM iteration each on the 48-plane slab, 2 rounds of one task per
    core.  Timed from the first task's submission to the last result, after a
    warm-up round that starts the workers."""
    import multiprocessing as mp
    from oracle import ifcm as O
    cores = os.cpu_count() or 1
    x = O.normalize(raw)[:CPU_SLAB]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_particle_iteration, [(x[:2], 0.5, 0.5)] * cores)      # start workers
        tasks = [(x, 0.1 + 0.8 * (i % 7) / 7.0, 0.5) for i in range(2 * cores)]
        t0 = time.perf_counter()
        res = pool.map(_oracle_particle_iteration, tasks, chunksize=1)
        el = time.perf_counter() - t0
    assert all(np.isfinite(r[2]) for r in res)
    return sum(r[1] for r in res) / el, cores, len(tasks), el, x.shape


def oracle_sample_rate(raw, seconds_cap=30.0):
    """Updates/s of the FP64 oracle: IFCM iterations of one particle
    (lambda = xi = 0.5) on a 48-plane z-slab of the workload volume."""
    from oracle import ifcm as O
    x = O.normalize(raw)[:CPU_SLAB]
    U = np.full((C,) + x.shape, 1.0 / C)
    Cc = (np.arange(C) + 0.5) / C
    U, Cc, _, _ = O.ifcm_iteration(x, U, Cc, 0.0, 0.0)
    n = 0
    t0 = time.perf_counter()
    while True:
        U, Cc, _, _ = O.ifcm_iteration(x, U, Cc, 0.5, 0.5)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds_cap / 3 or n >= 3:
            break
    return n * x.size / el, n, el, x.shape


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2002_01981_gb300 import phantoms
    from oracle import ifcm as O
    raw = phantoms.brain_phantom(SHAPE, seed=SEED, sigma=0.07)
    x = O.normalize(raw)[:CPU_SLAB]
    U = np.full((C,) + x.shape, 1.0 / C)
    Cc = (np.arange(C) + 0.5) / C
    U, Cc, _, _ = O.ifcm_iteration(x, U, Cc, 0.0, 0.0)
    for _ in range(args.warmup):
        U, Cc, _, _ = O.ifcm_iteration(x, U, Cc, 0.5, 0.5)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, Cc, _, _ = O.ifcm_iteration(x, U, Cc, 0.5, 0.5)
    el = time.perf_counter() - t0
    value = args.steps * x.size / el
    sample = (f"one FP64 oracle IFCM iteration (one particle, lambda=xi=0.5) per step on a "
              f"{CPU_SLAB}-plane z-slab (181x217x{CPU_SLAB}) of the workload volume")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU arm
def run_small_kind(args):
    """Small cases for profiler captures of the F2 / F3 kernels and of the 2D
    stencil (a few GB on the device at most): 'bf16' runs 3 iterations of 8
    particles of the c = 6 256^3 workload with bf16 memberships; 'grad' runs
    ifcm_grad (K = 3) on the 128^3 differentiation workload; 'image' runs
    3 iterations of 64 particles on the 854 x 854 slice of the 2D sweep, from
    its FCM start (memberships from Eq 2, so the lean 2D kernel runs)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01981_gb300 import ifcm as G
    from paper_2002_01981_gb300 import phantoms
    dev = torch.device("cuda", 0)
    if args.small_kind == "bf16":
        raw = phantoms.multi_tissue(PREC_SHAPE, seed=5, sigma=0.1)
        nx = PREC_SHAPE[2]
        x = G.ifcm_normalize(torch.from_numpy(phantoms.pad_pitch(raw)).to(dev), nx=nx)
        U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=PREC_C, max_iter=20, eps_u=EPS), (0.0, 0.0),
                                  nx=nx)
        lam = G.Swarm(8, seed=5).init().x
        prm = G.Params(c=PREC_C, m=M, max_iter=3, eps_u=0.0, u_dtype="bf16")
        for _ in range(args.steps):
            fit, _, _ = G.pso_fitness_batch(x, prm, lam, U0, C0, nx=nx)
        torch.cuda.synchronize()
        print(json.dumps({"small_kind": "bf16", "fitness": fit.cpu().numpy().tolist()}))
    elif args.small_kind == "image":
        n = phantoms.SWEEP_SIZES[-1]
        raw = phantoms.brain_slice(n, seed=2, sigma=0.07)
        vol = torch.from_numpy(phantoms.pad_pitch(raw)).to(dev)
        # 64 particles: 298 MB of membership buffers, beyond the 129 MB L2
        opts = G.Options(P=64, generations=1, seed=SEED, init_max_iter=20)
        prm = G.Params(c=C, m=M, max_iter=3, eps_u=0.0)
        for _ in range(args.steps):
            _, res = G.pifcm3d(vol, prm, opts, nx=n)
        torch.cuda.synchronize()
        print(json.dumps({"small_kind": "image", "J": res["J"], "updates": res["updates"]}))
    else:
        raw = phantoms.gaussian_phantom(DIFF_SHAPE, seed=4, sigma=0.09)
        nx = DIFF_SHAPE[2]
        x = G.ifcm_normalize(torch.from_numpy(phantoms.pad_pitch(raw)).to(dev), nx=nx)
        U0, C0, _, _ = G.ifcm_fit(x, G.Params(c=DIFF_C, max_iter=20, eps_u=EPS), (0.0, 0.0),
                                  nx=nx)
        prm = G.Params(c=DIFF_C, m=M)
        for _ in range(args.steps):
            J, g = G.ifcm_grad(x, prm, (0.3, 0.2), U0, C0, 3, nx=nx)
        torch.cuda.synchronize()
        print(json.dumps({"small_kind": "grad", "J": float(J), "grad": g.cpu().numpy().tolist()}))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01981_gb300 import ifcm as G
    from paper_2002_01981_gb300 import phantoms

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    raw = phantoms.brain_phantom(SHAPE, seed=rank_seed(rank), sigma=0.07)
    nz, ny, nx = SHAPE
    vol_host = torch.from_numpy(phantoms.pad_pitch(raw)).pin_memory()
    vol = vol_host.to(dev)
    n_p, n_gen, n_it, n_init = P, GENERATIONS, MAX_ITER, INIT_MAX_ITER
    if args.small:       # short case for profiler captures: same volume and kernels
        n_p, n_gen, n_it, n_init = args.small_particles or P, 1, 3, 3
        if args.small_particles:
            G.force_plan(2, 1)        # the full run's plan: 2 particles per item, whole columns
    prm = G.Params(c=C, m=M, max_iter=n_it, eps_u=EPS)
    opts = G.Options(P=n_p, generations=n_gen, seed=rank_seed(rank), init_max_iter=n_init)
    bufs = G.pifcm3d_buffers(vol, prm, opts, nx=nx)
    N = nx * ny * nz

    # ---- warm-up
    for _ in range(args.warmup):
        G.pifcm3d(vol, prm, opts, nx=nx, buffers=bufs, sync=False)
    barrier()
    _, first = G.pifcm3d(vol, prm, opts, nx=nx, buffers=bufs)
    if first["status"]:
        raise RuntimeError(f"device status {first['status']}")

    # ---- timed region (device-resident inputs)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    G.profile_read()                    # drop anything recorded so far
    G.profile_enable(True)
    barrier()
    clocks.start()
    ev0.record(stream)
    for _ in range(args.steps):
        G.pifcm3d(vol, prm, opts, nx=nx, buffers=bufs, sync=False)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    G.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    k3_ms, k3_launches = G.profile_read(G.PROF_STENCIL3D)
    kernel_ms, kernel_launches = G.profile_read()
    _, res = G.pifcm3d(vol, prm, opts, nx=nx, buffers=bufs)   # same work every step
    updates_step = res["updates"]
    init_updates = res["iters_init"] * N
    # stencil3d_kernel runs every iteration of the batches (two particles per
    # item) and of the final run (one particle, clusters paired)
    final_updates = res["iters_final"] * N
    k3_updates_step = updates_step - init_updates

    s_max, total_updates = reduce_over_ranks(dist, world, ms / 1e3, updates_step * args.steps,
                                             dev)
    ms_max = s_max * 1e3
    value = total_updates / s_max

    if args.small:
        if rank == 0:
            print(json.dumps({"small_case": True, "ms_per_step": ms_max / args.steps,
                              "updates_per_step": updates_step, "kernel_ms": kernel_ms,
                              "kernel_launches": kernel_launches}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- the plain form (paper's Algorithm 2 shape): one particle per launch,
    # one thread per voxel reading neighbours from global memory, host loop
    plain = plain_form_rate(G, vol, nx, prm, opts, stream) if rank == 0 else None

    # ---- end to end through the host entry point (copies inside the region)
    u_host = torch.empty((C, nz, ny, vol.shape[2]), dtype=torch.float32).pin_memory()
    ws_host = G.pifcm3d_host_workspace(G.shape_of(vol, nx), prm, opts)
    del bufs
    G.pifcm3d_host(vol_host, prm, opts, nx=nx, u_out=u_host, ws=ws_host)   # warm
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        _, rh = G.pifcm3d_host(vol_host, prm, opts, nx=nx, u_out=u_host, ws=ws_host)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_max, e2e_updates = reduce_over_ranks(dist, world, e2e_s, e2e_steps * rh["updates"], dev)
    e2e_value = e2e_updates / e2e_max

    # ---- roofline of the dominant kernel, stencil3d_kernel<4>: its own
    # launches (CUDA events on the launching stream) and the updates they ran
    hbm, peak_kind = peaks()
    # U^t read + U^{t+1} write + x read once per item, shared by the item's particles
    plan_np, plan_tz, _ = G.stencil_plan(G.shape_of(vol, nx), C, P)
    bytes_per_update = 2 * C * 4 + 4.0 / plan_np
    step_bytes = ((k3_updates_step - final_updates) * bytes_per_update +
                  final_updates * (2 * C * 4 + 4.0))
    per_launch_updates = k3_updates_step * args.steps / max(k3_launches, 1)
    achieved = step_bytes * args.steps / (k3_ms / 1e3) / 1e9
    traffic_pu = stencil_traffic_per_update(plan_np, plan_tz)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_kind": peak_kind,
                "traffic": traffic_pu * per_launch_updates if traffic_pu else None,
                "algorithmic_bytes_per_launch": step_bytes * args.steps / max(k3_launches, 1),
                "bytes_per_update": bytes_per_update,
                "kernel": "stencil3d_kernel<4, 2> (its one-particle form <4, 1> runs the final "
                          f"run: {final_updates / k3_updates_step:.2%} of the updates, at "
                          f"{2 * C * 4 + 4} B per update)",
                "plan": {"particles_per_item": plan_np, "tz": plan_tz,
                         "tile": "32x11 columns", "memberships": "float2 pair words"},
                "kernel_ms": k3_ms, "kernel_launches": k3_launches,
                "kernel_updates_per_step": k3_updates_step,
                "kernel_share_of_step": k3_ms / ms,
                "all_stencil_ms": kernel_ms, "all_stencil_launches": kernel_launches}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "one whole Algorithm 1 run",
                       "updates_per_step": updates_step,
                       "fcm_start_updates_per_step": init_updates,
                       "l2": "inputs larger than L2 (4.6 GB of membership buffers per step)",
                       "parallelism": f"independent volume per GPU x{world}"},
            "roofline": roofline, "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(vol_host.numel() * 4),
                    "d2h_bytes_per_step": int(u_host.numel() * 4 + 120)},
            "gpu_launches": args.steps * launches_per_run(INIT_MAX_ITER, GENERATIONS, MAX_ITER)}
    if rank == 0 and not args.skip_batching:
        line["batching"] = batching_leg(G, phantoms, dev)
    if rank == 0 and not args.skip_precision:
        line["precision"] = precision_leg(G, phantoms, dev)
    if rank == 0 and not args.skip_differentiation:
        line["differentiation"] = differentiation_leg(G, phantoms, dev)
    if rank == 0 and not args.skip_sweep:
        line["sweep2d"] = sweep_leg(G, phantoms, dev)
    if plain is not None:
        line["plain"] = plain
        line["plain"]["batched_over_plain"] = value / world / plain["value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, el, shp = oracle_sample_rate(raw)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} FP64 oracle IFCM iterations of one particle "
                                          f"on a {shp[0]}x{shp[1]}x{shp[2]} z-slab, {el:.1f} s",
                                "cpu_model": cpu_model()}
        if not args.skip_all_cores:
            ra, cores, ntask, ela, shp = oracle_all_cores_rate(raw)
            line["cpu_baseline"]["all_cores"] = {
                "value": ra, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{ntask} particles x one FP64 oracle IFCM iteration on the "
                          f"{shp[0]}x{shp[1]}x{shp[2]} z-slab, one spawned worker per core, "
                          f"{ela:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def relaunch(n):
    """--gpus N under a plain interpreter: start the N ranks (one process per
    GPU) through torch.distributed.run with the same arguments, or stop with
    an error when fewer than N GPUs are visible."""
    import socket

    import torch
    have = torch.cuda.device_count() if torch.cuda.is_available() else 0
    if have < n:
        print(f"bench.py: --gpus {n} asks for {n} GPUs but {have} are visible", file=sys.stderr)
        return 2
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={n}", "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batching", action="store_true",
                    help="leave out the uneven multi-volume batch")
    ap.add_argument("--skip-precision", action="store_true",
                    help="leave out the FP32 / bf16 membership storage comparison")
    ap.add_argument("--skip-all-cores", action="store_true",
                    help="leave out the all-cores timing of the CPU oracle")
    ap.add_argument("--skip-sweep", action="store_true",
                    help="leave out the 2D size sweep (32^2 ... 854^2 slices)")
    ap.add_argument("--skip-differentiation", action="store_true",
                    help="leave out the gradient / polish leg")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: the same volume and particles, 1 generation x "
                         "3 iterations")
    ap.add_argument("--small-particles", type=int, default=0,
                    help="with --small: this many particles (a smaller capture), under the "
                         "full run's plan (2 particles per item, whole-column items)")
    ap.add_argument("--small-kind", choices=("bf16", "grad", "image"), default=None,
                    help="profiling case of the bf16 stencil, the adjoint kernels or the 2D "
                         "stencil")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch(args.gpus)
    if args.impl == "reference":
        return run_reference(args)
    if args.small_kind:
        return run_small_kind(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
