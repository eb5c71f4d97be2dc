#!/usr/bin/env python
"""Throughput of the batched differentiable rod stepper (one JSON line on stdout).

Workload: trajectory optimisation at scale -- 4096 rods x 128 vertices per GPU (one third
each inextensible cable, elastic rope, plastic wire; App. B Table "sim_params" rows
Wiring-post, Unknotting, Letter Art), two capsule grippers per rod with smooth random 6-DoF
actions, ground plane, self-contact on, dt = 1e-3 s with 5 substeps (App. B.1), a 2000-frame
rollout per step.  One step = the forward rollout (with HBM checkpoints) plus the backward
pass for dL/d(actions, material, initial state) of L = mean |x_T - target|^2.

value        rod-vertex-steps/s of forward + backward (rods x vertices x frames / time)
fwd_value    the same for the forward rollout alone
e2e          the same through the public API from pinned host buffers (copies included)
roofline     the dominant kernel (the backward) against the FP32 CUDA-core peak measured on
             the device by a register-only FMA kernel (dlo_measure_fp32_peak), with
             algorithmic operation counts per vertex-substep from tests/flop_count.cu
cpu_baseline the FP64 oracle on the host cores, on a bounded sample of the same workload
plain        the plain per-phase GPU step (dlo_step_plain) on the same rods

`--workload` selects the other configurations (batching, selfcontact, diff, separation: two
tangled ropes per environment coupled by contact) or ``cmaes``: one CMA-ES generation of the
Unknotting task per step (400 candidate rollouts of one knotted rope, forward only, each
scored on the device by its crossing sum and self-repulsion penalty).

`--impl reference` times the oracle instead (the reference arm of this benchmark).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rod-vertex-steps/s fwd and fwd+bwd at B=4096, vs plain GPU step at stated accuracy"
UNIT = "rod-vertex-steps/s"
# algorithmic FP32 operations per vertex-substep (tests/flop_count.cu counts them from the
# kernels' own element templates; tests/test_flop_count.py keeps these in step)
FLOPS_FWD_PER_VS = 912.3
FLOPS_BWD_PER_VS = 3650.0
# DRAM bytes (read + write) of the backward per rod-frame of the 128-vertex trajopt workload,
# from ncu captures (cold cache) of a 304-rod x 50-frame case of it, one 50-frame chunk:
# rev_kernel 1621.64 + 27.34 MB, rec_kernel 25.05 + 1544.64 MB
# (profiles/rec_rev_kernels_trajopt_304x128x50.md)
BWD_DRAM_BYTES_PER_ROD_FRAME = (1621.64096e6 + 27.341568e6 + 25.052928e6 + 1544.644e6) / (304 * 50)
FP32_LANES_PER_SM = 128     # for the nominal figure printed beside the measured peak


def metric_for(workload):
    if workload == "trajopt-opt":
        return "rod-vertex-steps/s fwd+bwd over Adam iterations of trajectory optimisation, fused vs plain, final losses"
    if workload == "cmaes":
        return "rod-vertex-steps/s of one CMA-ES generation (forward rollouts + device scores)"
    if workload == "trajopt":
        return METRIC
    return f"rod-vertex-steps/s fwd+bwd ({workload} configuration), vs plain GPU step"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="trajopt",
                    choices=["trajopt", "batching", "selfcontact", "diff", "cmaes", "sysid", "trajopt-opt",
                             "separation"],
                    help="trajopt is the headline line; the others measure the other configurations")
    ap.add_argument("--iters", type=int, default=50, help="trajopt-opt: Adam iterations")
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--rods", type=int, default=None)
    ap.add_argument("--verts", type=int, default=None)
    ap.add_argument("--no-self-contact", action="store_true")
    ap.add_argument("--broad-phase", default="all-pairs", choices=["all-pairs", "hash"],
                    help="self-contact candidates: every edge pair (default) or the per-rod spatial hash")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--plain-frames", type=int, default=20)
    ap.add_argument("--no-side", action="store_true",
                    help="trajopt: skip the one-shot measurements of the self-contact, batching and separation "
                         "workloads")
    return ap.parse_args()


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl == "native" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.mkdtemp(), "clocks.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        load = [float(r[1]) for r in rows if float(r[3]) > 200.0] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- reference arm
def oracle_population_rate(prob, frames, rods):
    """FP64 oracle forward rollout of `rods` candidates plus their Unknotting scores;
    returns (rod-vertex-steps/s, seconds)."""
    import numpy as np
    import torch
    from oracle import OracleSim, losses
    sub = prob.subset(rods, frames=frames)
    t0 = time.perf_counter()
    sim = OracleSim(sub)
    sim.set_state(sub.x0, sub.v0, sub.theta0, sub.omega0)
    sim.step(sub.actions[:frames], frames)
    x = torch.as_tensor(sim.get_state()["x"])
    for b, (v0, v1) in enumerate(zip(sub.vert_off[:-1], sub.vert_off[1:])):
        xb = x[v0:v1]
        losses.crossing(xb)
        losses.repulsion(xb, 2.0 * rest_edge(sub.x_rest[v0:v1]), 2)
    dt = time.perf_counter() - t0
    units = float(np.sum(sub.n_verts)) * frames
    return units / dt, dt


def sysid_cameras():
    """Two pinhole cameras over the table (rods within about 0.75 m of the origin): one looking
    straight down from 1.6 m, one from the side at 50 degrees; 256 x 256 px."""
    import math
    import numpy as np
    c = SIL_HW / 2
    down = np.concatenate([[160.0, 160.0, c, c], np.diag([1.0, -1.0, -1.0]).reshape(9), [0.0, 0.0, 1.6]])
    a = math.radians(50.0)
    R = np.array([[1.0, 0.0, 0.0], [0.0, -math.sin(a), -math.cos(a)], [0.0, math.cos(a), -math.sin(a)]])
    eye = np.array([0.0, -math.cos(a), math.sin(a)]) * 1.8
    side = np.concatenate([[150.0, 150.0, c, c], R.reshape(9), -R @ eye])
    return np.stack([down, side])


def rest_edge(x):
    """Mean rest edge length of one open rod (its initial shape)."""
    import numpy as np
    return float(np.linalg.norm(np.diff(np.asarray(x, np.float64), axis=0), axis=1).mean())


def oracle_rollout_rate(prob, frames, rods, sil=False):
    """FP64 oracle forward + reverse-mode backward on `rods` rods of the workload; returns
    (rod-vertex-steps/s, seconds).  sil: the loss is the silhouette loss against the oracle's
    own masks of the target curves (rendered before the clock starts)."""
    import numpy as np
    import torch
    from oracle import OracleSim
    from oracle import silhouette as S
    sub = prob.subset(rods, frames=frames)
    if sil:
        cams = sysid_cameras()
        masks = []
        for a, b in zip(sub.vert_off[:-1], sub.vert_off[1:]):
            xt = torch.tensor(np.asarray(sub.target[a:b], np.float64))
            masks.append(np.stack([(S.render(xt, c, SIL_HW, SIL_HW, SIL_TAU, float(sub.radius[0])) > 0.5).numpy()
                                   for c in cams]).astype(np.float64))
    t0 = time.perf_counter()
    act = torch.tensor(sub.actions[:frames], requires_grad=True)
    x0 = torch.tensor(sub.x0, requires_grad=True)
    sim = OracleSim(sub)
    sim.set_state(x0, torch.tensor(sub.v0), torch.tensor(sub.theta0), torch.tensor(sub.omega0))
    sim.step(act, frames, diff=True)
    x = sim.get_state(as_numpy=False)["x"]
    if sil:
        L = sum(S.silhouette_loss(x[a:b], cams, masks[k], SIL_TAU, float(sub.radius[k]))
                for k, (a, b) in enumerate(zip(sub.vert_off[:-1], sub.vert_off[1:])))
    else:
        L = ((x - torch.tensor(sub.target)) ** 2).sum(1).mean() if sub.target is not None else x[:, 2].mean()
    torch.autograd.grad(L, [act, x0])
    dt = time.perf_counter() - t0
    units = float(np.sum(sub.n_verts)) * frames
    return units / dt, dt


def run_reference(args, rank, ws):
    if rank != 0:
        return
    import copy
    import torch
    short = copy.copy(args)
    short.frames = 4                       # the oracle samples two frames per step
    prob, desc, R, _ = make_workload(short, 0)
    rates = []
    rate_fn = oracle_population_rate if args.workload == "cmaes" else oracle_rollout_rate
    kw = {"sil": True} if args.workload == "sysid" else {}
    for i in range(args.warmup + args.steps):
        r, dt = rate_fn(prob, 2, [0, 1], **kw)
        if i >= args.warmup:
            rates.append((r, dt))
    value = sum(r for r, _ in rates) / len(rates)
    ms = 1e3 * sum(dt for _, dt in rates) / len(rates)
    cores = torch.get_num_threads()
    sample = (f"rods 0 and 1 ({int(prob.n_verts[0])} and {int(prob.n_verts[1])} vertices) x 2 frames per step, "
              + ("FP64 forward + crossing sum and repulsion scores" if args.workload == "cmaes"
                 else "FP64 forward + silhouette loss + autograd backward" if args.workload == "sysid"
                 else "FP64 forward + autograd backward"))
    line = {"impl": "reference", "metric": metric_for(args.workload), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc + " (oracle sample)", "frames_per_step": 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- native arm
# rods, vertices per rod, frames of each workload (the configurations' own sizes)
WORKLOADS = {"trajopt": (4096, 128, 2000), "batching": (1024, None, 1000), "selfcontact": (4096, 200, 300),
             "diff": (256, 64, 500), "cmaes": (400, 128, 2000), "sysid": (256, 64, 500),
             "trajopt-opt": (512, 128, 200), "separation": (4096, 30, 2000)}
SIL_HW, SIL_TAU = 256, 0.5  # system identification: two 256 x 256 cameras, edge softness in pixels
ACTION_UNIT = 1e-3         # trajopt-opt: the optimised action corrections are in mm and mrad per frame
REPULSION_WEIGHT = 1e3     # the Unknotting penalty's weight against the crossing sum


def make_workload(args, rank):
    from paper_2606_04206_gb300 import inputs
    R0, N0, F0 = WORKLOADS[args.workload]
    R = args.rods or R0
    N = args.verts or N0
    F = args.frames or F0
    w = args.workload
    if w == "trajopt-opt":
        prob = inputs.trajopt(n_rods=R, frames=F, seed=4000 + rank, n=N, self_contact=not args.no_self_contact)
        desc = (f"trajopt-opt: {args.iters} Adam iterations (lr 1e-3 cosine to 1e-6) on the gripper actions of "
                f"{R} rods x {N} vertices per GPU, {F} frames (dt 1e-3 s, 5 substeps), cable/rope/wire thirds, "
                f"2 grippers, ground, self-contact={'on' if not args.no_self_contact else 'off'}; loss = mean squared "
                f"distance of the final vertices to seeded target curves")
    elif w == "trajopt":
        prob = inputs.trajopt(n_rods=R, frames=F, seed=4000 + rank, n=N, self_contact=not args.no_self_contact)
        desc = (f"trajopt: {R} rods x {N} vertices per GPU, {F} frames (dt 1e-3 s, 5 substeps), cable/rope/wire "
                f"thirds, 2 grippers, ground, self-contact={'on' if not args.no_self_contact else 'off'}")
    elif w == "batching":
        prob = inputs.batching(n_rods=R, frames=F, seed=1000 + rank)
        desc = (f"batching: {R} rods x 16..256 vertices, 0.3..2 m, E 1e4..1e8 Pa, plastic, 2 grippers, ground, "
                f"{F} frames, per-rod substeps")
    elif w == "sysid":
        prob = inputs.diff(n_rods=R, frames=F, seed=2000 + rank, n=N)
        desc = (f"sysid: {R} rods x {N} vertices, rope/plastic wire halves, 2 grippers, ground, {F} frames; "
                f"silhouette loss of the final state from 2 cameras of {SIL_HW} x {SIL_HW} px against binary "
                f"masks of the target curves, gradient to the material")
    elif w == "cmaes":
        prob = inputs.cmaes(pop=R, frames=F, seed=5000 + rank, n=N)
        desc = (f"cmaes: one CMA-ES generation of Unknotting, population {R} x {N} vertices (one knotted rope, "
                f"sigma 5e-2), {F} frames forward, ground, self-contact, crossing-sum + repulsion scores")
    elif w == "separation":
        prob = inputs.separation(n_envs=R, frames=F, seed=6000 + rank, n=N)
        desc = (f"separation: {R} environments x 2 tangled ropes of {N} vertices (one record of two strands, "
                f"inextensible, E 5e3 Pa, G 1e3 Pa), one gripper on each rope pulling them apart, ground, "
                f"self-contact between and within the ropes, {F} frames")
    elif w == "selfcontact":
        prob = inputs.selfcontact(n_rods=R, frames=F, seed=3000 + rank, n=N)
        desc = f"selfcontact: {R} knotted closed bands x {N} vertices, ground + box, self-contact, {F} frames"
    else:
        prob = inputs.diff(n_rods=R, frames=F, seed=2000 + rank, n=N)
        desc = f"diff: {R} rods x {N} vertices, rope/plastic wire halves, 2 grippers, ground, {F} frames"
    return prob, desc, R, F


def side_workloads(args, rank):
    """One timed forward + backward of the self-contact configuration (4096 knotted bands x 200
    vertices, 300 frames, with each broad phase), of the batching configuration (1024 rods of
    16..256 vertices, per-rod substeps; 100 of its 1000 frames) and of the Separation
    environments (4096 x two tangled 30-vertex ropes, 300 of its 2000 frames, with each broad
    phase), after one warm-up each, with the plain per-phase forward on the same rods.
    Reported beside the headline, not in it."""
    import copy
    import numpy as np
    import torch
    from paper_2606_04206_gb300 import dlo
    out = {}
    for kind, frames in (("selfcontact", 300), ("batching", 100), ("separation", 300)):
        a2 = copy.copy(args)
        a2.workload, a2.frames, a2.rods, a2.verts = kind, frames, None, None
        prob, desc, R, F = make_workload(a2, rank)
        units = float(np.sum(prob.n_verts)) * F
        res = {"workload": desc, "frames": F}
        for bp in ((0, 1) if kind in ("selfcontact", "separation") else (0,)):
            sim = dlo.DloSim(prob, broad_phase=bp)
            dev = sim.device
            stream = torch.cuda.current_stream()
            acts = torch.as_tensor(np.ascontiguousarray(prob.actions, np.float32), device=dev)
            x0, v0, th0 = sim.tensors_from_problem()
            gz = torch.zeros(sim.V, 4, device=dev)
            gz[:, 2] = 1.0 / sim.V          # L = mean height of the vertices

            def fb():
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                sim.set_state(x0, v0, th0)
                ev[0].record(stream)
                sim.begin_rollout(F)
                sim.step(acts, F)
                ev[1].record(stream)
                sim.backward(dL_dx=gz, want=("actions", "material", "x0"))
                ev[2].record(stream)
                torch.cuda.synchronize()
                return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

            fb()
            ms_f, ms_b = fb()
            key = "hash" if bp else "all_pairs"
            if bp:
                res["fwd_value_spatial_hash"] = units / (ms_f / 1e3)
                res["ms_fwd_spatial_hash"] = ms_f
            else:
                res.update({"value": units / ((ms_f + ms_b) / 1e3), "fwd_value": units / (ms_f / 1e3),
                            "ms_fwd": ms_f, "ms_bwd": ms_b, "substeps_max": int(np.max(sim.query(dlo.Q_SUBSTEPS))),
                            "pairs_max_per_rod": int(np.max(sim.query(dlo.Q_PAIRS)))})
                pf = 5
                sim.set_state(x0, v0, th0)
                sim.step_plain(acts[:2].contiguous(), 2)
                sim.set_state(x0, v0, th0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step_plain(acts[:pf].contiguous(), pf)
                e1.record(stream)
                torch.cuda.synchronize()
                pv = float(np.sum(prob.n_verts)) * pf / (e0.elapsed_time(e1) / 1e3)
                res["plain_fwd_value"] = pv
                res["speedup_fwd_vs_plain"] = res["fwd_value"] / pv
            sim.close()
            del sim
            torch.cuda.empty_cache()
        out[kind] = res
    return out


def run_native(args, rank, ws):
    import numpy as np
    import torch
    from paper_2606_04206_gb300 import build, dlo, inputs

    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    prob, desc, R, F = make_workload(args, rank)
    sim = dlo.DloSim(prob, broad_phase=int(args.broad_phase == "hash"))
    V = sim.V
    N = int(np.max(prob.n_verts))
    units = float(np.sum(prob.n_verts)) * F
    acts = torch.as_tensor(np.ascontiguousarray(prob.actions, np.float32), device=dev)
    target = torch.zeros(V, 4, device=dev)
    if prob.target is not None:
        target[:, :3] = torch.as_tensor(prob.target, dtype=torch.float32, device=dev)
    x0, v0, th0 = sim.tensors_from_problem()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()
    mean_z = torch.zeros(V, 4, device=dev)
    mean_z[:, 2] = 1.0 / V

    sil = args.workload == "sysid"
    if sil:
        cams = torch.tensor(sysid_cameras(), dtype=torch.float32, device=dev)
        blank = torch.zeros(R, 2, SIL_HW, SIL_HW, dtype=torch.uint8, device=dev)
        _, _, img = sim.silhouette(target, cams, blank, SIL_TAU, grad=False, render=True)
        masks = (img > 0.5).to(torch.uint8)
        del img, blank

    def loss_grad(x):
        """dL/dx_T: the silhouette loss for system identification, else the mean squared
        distance to the target curve, or the mean height without one."""
        if sil:
            return sim.silhouette(x, cams, masks, SIL_TAU)[1]
        if prob.target is not None:
            return (2.0 / V) * (x - target)
        return mean_z

    def dL_dx():
        x, _, _ = sim.get_state()
        return loss_grad(x)

    pop = args.workload == "cmaes"          # forward-only rollouts scored on the device
    if pop:
        prm = torch.zeros(R, 4, device=dev)
        prm[:, 0] = torch.as_tensor([2.0 * rest_edge(prob.x_rest[a:b]) for a, b in
                                     zip(prob.vert_off[:-1], prob.vert_off[1:])], device=dev)
        prm[:, 1] = 2.0

    def scores():
        x, _, _ = sim.get_state()
        qc, _ = sim.loss(dlo.LOSS_CROSSING, x, grad=False)
        qr, _ = sim.loss(dlo.LOSS_REPULSION, x, prm, grad=False)
        return qc, qr

    def one_step(record):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        l0 = sim.query(dlo.Q_LAUNCHES)
        ev[0].record(stream)
        sim.set_state(x0, v0, th0)
        gb = torch.cuda.Event(enable_timing=True)
        if pop:
            sim.step(acts, F)
            ev[1].record(stream)
            gb.record(stream)
            scores()
        else:
            sim.begin_rollout(F)
            sim.step(acts, F)
            ev[1].record(stream)
            g = dL_dx()
            gb.record(stream)
            sim.backward(dL_dx=g, want=("actions", "material", "x0"))
        ev[2].record(stream)
        torch.cuda.synchronize()
        l1 = sim.query(dlo.Q_LAUNCHES)
        return ev[0].elapsed_time(ev[1]), gb.elapsed_time(ev[2]), ev[0].elapsed_time(ev[2]), l1 - l0

    for _ in range(args.warmup):
        one_step(False)
    clocks = Clocks(torch.cuda.current_device())
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    t_fwd, t_bwd, t_all, launches = [], [], [], []
    for _ in range(args.steps):
        a, b, c, n = one_step(True)
        t_fwd.append(a)
        t_bwd.append(b)
        t_all.append(c)
        launches.append(n)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms_step = max_over_ranks(sum(t_all) / len(t_all), ws)
    ms_fwd = max_over_ranks(sum(t_fwd) / len(t_fwd), ws)
    ms_bwd = max_over_ranks(sum(t_bwd) / len(t_bwd), ws)
    value = units * ws / (ms_step / 1e3)
    fwd_value = units * ws / (ms_fwd / 1e3)

    # end-to-end through the public API from pinned host memory
    h_acts = torch.empty_like(acts, device="cpu").pin_memory()
    h_acts.copy_(acts)
    h_state = [t.cpu().pin_memory() for t in (x0, v0, th0)]
    h_target = target.cpu().pin_memory()
    h_gact = torch.empty(F, R, 2, 6).pin_memory()
    h_loss = torch.empty(1).pin_memory()
    h_scores = torch.empty(2, R).pin_memory()
    h_masks = masks.cpu().pin_memory() if sil else None
    def e2e_step():
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_acts = h_acts.to(dev, non_blocking=True)
        xs, vs, ts = (t.to(dev, non_blocking=True) for t in h_state)
        tg = h_target.to(dev, non_blocking=True)
        sim.set_state(xs, vs, ts)
        if pop:
            sim.step(d_acts, F)
            qc, qr = scores()
            h_scores[0].copy_(qc, non_blocking=True)
            h_scores[1].copy_(qr, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        sim.begin_rollout(F)
        sim.step(d_acts, F)
        x, _, _ = sim.get_state()
        if sil:
            d_masks = h_masks.to(dev, non_blocking=True)
            qs, gs, _ = sim.silhouette(x, cams, d_masks, SIL_TAU)
            loss = qs.sum()
            g = sim.backward(dL_dx=gs, want=("actions", "material", "x0"))
        else:
            loss = ((x - tg)[:, :3] ** 2).sum(1).mean() if prob.target is not None else x[:, 2].mean()
            g = sim.backward(dL_dx=(2.0 / V) * (x - tg) if prob.target is not None else mean_z,
                             want=("actions", "material", "x0"))
        h_gact.copy_(g["actions"], non_blocking=True)
        h_loss.copy_(loss.reshape(1), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    e2e_step()   # warm-up: first use of the host buffers and of the device copies' allocations
    e2e = [e2e_step() for _ in range(args.e2e_steps)]
    ms_e2e = max_over_ranks(sum(e2e) / len(e2e), ws)
    if pop:
        h2d = h_acts.numel() * 4 + sum(t.numel() * 4 for t in h_state)
        d2h = h_scores.numel() * 4
    else:
        h2d = h_acts.numel() * 4 + sum(t.numel() * 4 for t in h_state) + h_target.numel() * 4
        if sil:
            h2d += h_masks.numel()
        d2h = h_gact.numel() * 4 + 4

    # roofline of the dominant kernel (the backward): algorithmic FP32 operations per launch
    nsub_rod = np.asarray(sim.query(dlo.Q_SUBSTEPS), np.float64)
    nsub = int(np.max(nsub_rod))
    vs_units = float(F) * float(np.sum(np.asarray(prob.n_verts, np.float64) * nsub_rod))
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    peak_tflops = dlo.measure_fp32_peak(2.0)
    bwd_tflops = FLOPS_BWD_PER_VS * vs_units / (ms_bwd / 1e3) / 1e12
    fwd_tflops = FLOPS_FWD_PER_VS * vs_units / (ms_fwd / 1e3) / 1e12
    traffic = (BWD_DRAM_BYTES_PER_ROD_FRAME * R * F
               if (args.workload == "trajopt" and N == 128 and not args.no_self_contact) else None)
    basis = (f"measured: register-only FMA kernel over {sms} SMs for 2 s (dlo_measure_fp32_peak), "
             f"{peak_tflops:.1f} TFLOP/s; nominal {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {max_mhz:.0f} MHz = "
             f"{nominal:.1f}")
    if pop:
        roofline = {"bound": "alu", "kernel": "fwd_kernel (dlo_step)", "achieved": fwd_tflops,
                    "peak": peak_tflops, "unit": "TFLOP/s", "frac": fwd_tflops / peak_tflops, "traffic": None,
                    "peak_basis": basis}
    else:
        roofline = {"bound": "alu", "kernel": "backward: rec_kernel + rev_kernel (dlo_backward)", "achieved": bwd_tflops,
                    "peak": peak_tflops, "unit": "TFLOP/s", "frac": bwd_tflops / peak_tflops, "traffic": traffic,
                    "peak_basis": basis, "forward": {"achieved": fwd_tflops, "frac": fwd_tflops / peak_tflops}}

    # plain per-phase GPU step on the same rods (short rollout, forward only)
    plain = None
    try:
        pf = args.plain_frames
        sim.set_state(x0, v0, th0)
        sim.step_plain(acts[:2].contiguous(), 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sim.set_state(x0, v0, th0)
        e0.record(stream)
        sim.step_plain(acts[:pf].contiguous(), pf)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        pv = float(np.sum(prob.n_verts)) * pf / (ms_p / 1e3)
        plain = {"fwd_value": pv, "unit": UNIT, "frames": pf, "speedup_fwd": fwd_value / ws / pv}
    except Exception as exc:   # the comparator is optional for the line; say why it is missing
        plain = {"unavailable": str(exc)[:200]}

    # CPU baseline: the FP64 oracle on a bounded sample of the same workload (rank 0 only)
    cpu = None
    if rank == 0:
        rate_fn = oracle_population_rate if pop else oracle_rollout_rate
        kw = {"sil": True} if sil else {}
        rate, dt = rate_fn(prob, 1, [0, 1], **kw)
        frames = max(1, min(20, int(args.cpu_seconds / max(dt, 1e-3))))
        rate, dt = rate_fn(prob, frames, [0, 1], **kw)
        what = ("crossing sum and repulsion scores" if pop else
                "silhouette loss + autograd backward" if sil else "autograd backward")
        cpu = {"value": rate, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"2 rods x {N} vertices x {frames} frames of the same workload, FP64 forward + "
                         f"{what}, {dt:.1f} s"}

    ck_used = int(sim.query(dlo.Q_CONFIG)[1])
    side = None
    if args.workload == "trajopt" and not args.no_side and rank == 0:
        sim.close()
        del sim
        torch.cuda.empty_cache()
        try:
            side = side_workloads(args, rank)
        except Exception as exc:   # supplementary: say why it is missing rather than lose the line
            side = {"unavailable": str(exc)[:200]}

    if rank == 0:
        line = {"metric": metric_for(args.workload), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": desc,
                           "rods_per_gpu": R, "verts_per_rod": N, "frames": F, "substeps": nsub,
                           "n_iter_pbd": 10, "checkpoint_every": ck_used,
                           "broad_phase": args.broad_phase,
                           "l2": "256 MiB buffer written before every timed step"},
                "fwd_value": fwd_value, "ms_fwd": ms_fwd, ("ms_score" if pop else "ms_bwd"): ms_bwd,
                "e2e": {"value": units * ws / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(max(launches)), "roofline": roofline, "cpu_baseline": cpu, "plain": plain,
                "clocks": clk}
        if side is not None:
            line["workloads"] = side
        print(json.dumps(line), flush=True)


def run_trajopt_opt(args, rank, ws):
    """Trajectory optimisation (App. B's gradient-descent setting): Adam on the per-frame gripper
    actions through DloRollout, once with the fused kernels and once with the plain per-phase
    comparator, from identical inputs.  One step = one iteration (rollout, loss, backward, Adam
    update).  value = fused fwd+bwd rod-vertex-steps/s over the iterations."""
    import numpy as np
    import torch
    from paper_2606_04206_gb300 import build, dlo

    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    prob, desc, R, F = make_workload(args, rank)
    units = float(np.sum(prob.n_verts)) * F
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    h_acts = torch.as_tensor(np.ascontiguousarray(prob.actions, np.float32)).pin_memory()
    h_target = torch.zeros(int(prob.vert_off[-1]), 4)
    h_target[:, :3] = torch.as_tensor(prob.target, dtype=torch.float32)
    h_target = h_target.pin_memory()
    h_loss = torch.empty(1).pin_memory()

    def optimise(plain, iters, clocks=None):
        sim = dlo.DloSim(prob)
        stream = torch.cuda.current_stream()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        acts0 = h_acts.to(dev, non_blocking=True)
        target = h_target.to(dev, non_blocking=True)
        x0, v0, th0 = sim.tensors_from_problem()
        # decision variables: corrections to the per-frame actions in mm and mrad per frame
        u = torch.zeros_like(acts0, requires_grad=True)
        opt = torch.optim.Adam([u], lr=1e-3)
        sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=max(1, iters - 1), eta_min=1e-6)
        losses = []
        n_bad = torch.zeros((), dtype=torch.int64, device=dev)
        for _ in range(iters):
            opt.zero_grad(set_to_none=True)
            x, _, _ = dlo.rollout(sim, x0, v0, th0, acts0 + ACTION_UNIT * u, plain=plain)
            loss = ((x - target)[:, :3] ** 2).sum(1).mean()
            loss.backward()
            # where a rod's sensitivity overflows float32 (self-contact can make it grow without
            # bound: ~1e48 in FP64 for some rods over 200 frames), those entries are zeroed
            bad = ~torch.isfinite(u.grad)
            n_bad += bad.sum()
            u.grad.masked_fill_(bad, 0.0)
            opt.step()
            sched.step()
            losses.append(loss.detach())
        x, _, _ = dlo.rollout(sim, x0, v0, th0, (acts0 + ACTION_UNIT * u).detach(), plain=plain)
        final = ((x - target)[:, :3] ** 2).sum(1).mean()
        h_loss.copy_(final.reshape(1), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = sim.query(dlo.Q_LAUNCHES)
        sim.close()
        return ms, float(h_loss[0]), [float(l) for l in losses], launches, int(n_bad)

    for _ in range(args.warmup):        # warm-up: one short run of each path
        optimise(False, 1)
        optimise(True, 1)
    clocks = Clocks(torch.cuda.current_device())
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ms_f, loss_f, hist_f, launches, bad_f = optimise(False, args.iters)
    clk = clocks.stop()
    ms_p, loss_p, hist_p, _, bad_p = optimise(True, args.iters)
    ms_f = max_over_ranks(ms_f, ws)
    ms_p = max_over_ranks(ms_p, ws)
    total_units = units * (args.iters + 1)   # iterations plus the final evaluation rollout
    value = total_units * ws / (ms_f / 1e3)
    plain_value = total_units * ws / (ms_p / 1e3)
    if rank == 0:
        line = {"metric": metric_for(args.workload), "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.iters, "warmup": args.warmup, "ms_per_step": ms_f / args.iters,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": desc, "rods_per_gpu": R, "verts_per_rod": int(np.max(prob.n_verts)),
                           "frames": F, "iterations": args.iters,
                           "optimizer": "Adam, lr 1e-3 cosine to 1e-6, on action corrections in mm / mrad per frame",
                           "l2": "256 MiB buffer written before each timed optimisation"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h_acts.numel() * 4 + h_target.numel() * 4),
                        "d2h_bytes_per_step": 4},
                "gpu_launches": int(launches),
                "loss": {"initial": hist_f[0], "final_fused": loss_f, "final_plain": loss_p,
                         "rel_diff": abs(loss_f - loss_p) / max(abs(loss_p), 1e-30),
                         "history_fused": hist_f[:: max(1, args.iters // 10)],
                         "history_plain": hist_p[:: max(1, args.iters // 10)],
                         "nonfinite_gradient_entries_zeroed": {"fused": bad_f, "plain": bad_p}},
                "plain": {"value": plain_value, "unit": UNIT, "ms_total": ms_p, "speedup": value / plain_value},
                "clocks": clk}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, ws = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, ws)
    elif args.workload == "trajopt-opt":
        run_trajopt_opt(args, rank, ws)
    else:
        run_native(args, rank, ws)


if __name__ == "__main__":
    main()
