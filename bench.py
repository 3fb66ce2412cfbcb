#!/usr/bin/env python
"""DG-RK3 throughput (dof-updates/s) of the nodal DG hot path on GB300: the
mixed-precision path with the learned con2prim guess (headline `value`), the
same path warm-started from the previous pass's pressures (`mixed_warm_start`),
and the plain FP64 path (`plain_fp64`).  The guess network is trained first
(untimed) on pairs the method generates.

Workload: 3D special-relativistic blast on a periodic unit cube, 16^3 affine
elements, 5 LGL nodes per axis (512,000 nodes x 5 conserved variables),
gamma = 4/3, rho = 10, p = 13.33 for r < 0.3 else rho = 1, p = 1e-6, v = 0,
1 % seeded density noise; HLL flux, MinModN limiter and SR fix after every
stage, con2prim at every node, CFL 0.2 (dt computed on the device each step).
A step is one full SSP-RK3 step (three RHS evaluations, limiter, fix).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (launched by torch.distributed.run) runs
N independent replicas, one per GPU; the path has no data exchange to shard.
The state (20.5 MB) is smaller than L2, so a 256 MiB buffer is written between
timed steps (outside the per-step event pairs).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dg_inputs  # noqa: E402  (seeded input generator, no method arithmetic)

WORKLOAD = dict(system=1, K=(16, 16, 16), n=5, flux=1, limiter=1, gamma=4.0 / 3.0, cfl=0.2, seed=1)
METRIC = "DG-RK3 dof-updates/s on 1 GB300: plain FP64 vs mixed+learned at equal L2 error"
UNIT = "dof-updates/s"


def _config(extra=None):
    w = WORKLOAD
    cfg = {"workload": "SR blast, 16^3 elements, 5 LGL nodes/axis, HLL, MinModN, con2prim per node, CFL 0.2",
           "system": "special-relativistic hydro", "elements": list(w["K"]), "lgl_nodes_per_axis": w["n"],
           "nodes": int(np.prod(w["K"]) * w["n"] ** 3), "vars": 5, "flux": "HLL", "limiter": "MinModN",
           "cfl": w["cfl"], "seed": w["seed"], "l2_between_steps": "flushed (256 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(total_ms: float, dist=None) -> float:
    """The slowest rank's time: the whole job is done when the last replica is.
    NCCL reduces on the GPU, gloo (CPU tests) on the host."""
    if not dist:
        return float(total_ms)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank: int, world_size: int, steps: int, total_ms: float) -> float:
    """dof-updates/s of all replicas together: every rank advances its own copy
    of the workload (weak scaling), and the job takes the slowest rank's time."""
    return world_size * nodes_per_rank * 5 * steps / (total_ms / 1e3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"dg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _init_state(pkg, mesh, torch):
    import dg_inputs as di
    xyz = mesh.coords().cpu().numpy()
    prim = di.blast_sr(xyz, seed=WORKLOAD["seed"])
    return mesh.from_prim(torch.from_numpy(prim).cuda())


# DRAM bytes per k_stage_mixed launch of the learned-guess steps on this workload
# (mean over the three stages of a step: stage 1 runs the variant that takes the
# CFL pass's primitives, stages 2-3 the in-kernel network), from the ncu launch
# list summarised in profiles/launches_sr_blast_16x16x16_n5.md.  Reported only
# while the kernel's sources and the step's dispatch still hash to the value they
# had when it was taken.
TRAFFIC_BYTES_PER_LAUNCH = 38690727.0
TRAFFIC_SOURCES = ("paper_1609_00098_gb300/csrc/dg_mixed.cuh", "paper_1609_00098_gb300/csrc/dg_physics.cuh",
                   "paper_1609_00098_gb300/csrc/dg_internal.h", "paper_1609_00098_gb300/csrc/dg_c2p_net.cuh",
                   "paper_1609_00098_gb300/csrc/dg_api.cu")
TRAFFIC_SOURCES_SHA256 = "b2f0d951b38752a732040ff7c665d4a125ae41b1c6a8c7c5cf13899394c49ee4"
TRAFFIC_VARIANT = "learned"


def _traffic(variant):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    ok = h.hexdigest() == TRAFFIC_SOURCES_SHA256 and variant == TRAFFIC_VARIANT
    return TRAFFIC_BYTES_PER_LAUNCH if ok else None


def _algorithmic(nodes, precision, learned=False):
    """Compulsory HBM bytes of one fused stage launch, averaged over the 3 stages.
    Both paths keep FP64 stage states: stage 1 reads U^n and writes U^1 (80 B/node);
    stages 2, 3 read U_s and U^n and write U_{s+1} (120 B/node).  The warm-started
    mixed SR path also reads the previous pass's FP32 pressure (4 B) and writes its
    own (4 B).  Stage 1 of an SR CFL step reads the CFL pass's FP32 primitives of
    U^n (20 B) instead of solving con2prim; with the learned guess computed in the
    kernel, stages 2, 3 carry no pressure."""
    if precision == 0:
        return nodes * (80 + 120 + 120) / 3.0
    if learned:
        return nodes * (100 + 120 + 120) / 3.0
    return nodes * (104 + 128 + 128) / 3.0


def _train_guess_net(pkg, torch):
    """Train the learned con2prim guess (untimed) on pairs the method generates for
    this problem class: the conserved states and FP64 pressures of the first six
    FP64 steps of the same blast with another noise seed (2), 2^18 pairs sampled
    from them, plus 2^16 states of the generic con2prim distribution (rho
    log-uniform [1e-8, 10], W uniform [1, 10], eps log-uniform [1e-6, 1e2]).
    Twenty epochs of Adam, batch 2048."""
    w = WORKLOAD
    g = w["gamma"]
    mesh = pkg.Mesh(system=w["system"], K=w["K"], n=w["n"], flux=w["flux"], limiter=w["limiter"], gamma=g)
    xyz = mesh.coords().cpu().numpy()
    U = mesh.from_prim(torch.from_numpy(dg_inputs.blast_sr(xyz, seed=2)).cuda())
    cons, pres = [], []
    P = torch.empty((mesh.E, 4, mesh.nn), dtype=torch.float64, device="cuda")
    for _ in range(6):
        pkg.abi.dg_primitives(mesh.h, U, P)
        cons.append(U.permute(1, 0, 2).reshape(5, -1).clone())
        pres.append(P[:, 3, :].reshape(-1).clone())
        mesh.rk3_step(U, cfl=w["cfl"])
    mesh.close()
    cons, pres = torch.cat(cons, 1), torch.cat(pres)
    gen = torch.Generator().manual_seed(2)
    pick = torch.randperm(cons.shape[1], generator=gen)[: 1 << 18].cuda()
    n_gen = 1 << 16
    prim = torch.from_numpy(np.ascontiguousarray(dg_inputs.c2p_samples(7, n_gen, gamma=g))).cuda()
    helper = pkg.Mesh(system=1, K=(16, 8, 8), n=4, gamma=g)   # 1024 x 64 = 2^16 nodes
    Ug = helper.state()
    pkg.abi.dg_prim2con(helper.h, prim, Ug)
    helper.close()
    cons = torch.cat([cons[:, pick], Ug.permute(1, 0, 2).reshape(5, n_gen)], 1).contiguous()
    pres = torch.cat([pres[pick], prim[4]]).contiguous()
    n_samp = cons.shape[1]
    init = dg_inputs.uniform(5, 9, np.arange(pkg.abi.N_NET_PARAMS))
    params = np.zeros(pkg.abi.N_NET_PARAMS)
    for o, fan, cnt in ((0, 3, 192), (256, 64, 4096), (4416, 64, 64)):  # W1, W2, W3: U(+-sqrt(3/fan_in))
        params[o:o + cnt] = np.sqrt(3.0 / fan) * (2.0 * init[o:o + cnt] - 1.0)
    net = pkg.abi.dg_c2p_net_create(params.astype(np.float32), (-5.0, 4.0, -9.0, 3.0, -4.5, 4.5))
    epochs = 20
    losses = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    t0 = time.time()
    pkg.abi.dg_c2p_net_train(net, n_samp, cons, pres, epochs, 2048, 2e-3, losses)
    torch.cuda.synchronize()
    info = {"pairs": n_samp, "source": "blast seed 2, FP64 steps 0-5 (2^18) + generic con2prim states (2^16)",
            "epochs": epochs, "batch": 2048, "train_s": round(time.time() - t0, 3),
            "loss_first_last": [float(losses[0]), float(losses[-1])]}
    return net, info


def _ensemble(pkg, torch, net, args):
    """Ragged ensemble (untimed setup): 256 meshes from the seeded recipe -- system
    NE or SR with probability 1/2, K uniform in [2, 16] per axis, n uniform in
    [3, 8].  NE meshes carry the smooth density wave (LLF, no limiter), SR meshes
    the blast (HLL, MinModN, learned con2prim guess); mixed precision, CFL 0.2.
    Times `ens_steps` steps of (a) the batched per-group launches replayed as one
    CUDA graph per step, after the launch-shape autotuner, and (b) the same meshes
    stepped one by one with dg_rk3_step.  The states (2.7 GB each) exceed L2."""
    recipe = dg_inputs.ensemble_recipe(5)
    meshes, states = [], []
    for system, K, n in recipe:
        g = 4.0 / 3.0 if system else 1.4
        m = pkg.Mesh(system=system, K=(K, K, K), n=n, flux=1 if system else 0, limiter=1 if system else 0,
                     gamma=g, precision=1)
        if system:
            m.set_c2p_net(net)
        xyz = m.coords().cpu().numpy()
        prim = dg_inputs.blast_sr(xyz, seed=1) if system else dg_inputs.smooth_wave_ne(
            xyz, k=dg_inputs.wave_numbers(1))
        states.append(m.from_prim(torch.from_numpy(prim).cuda()))
        meshes.append(m)
    nodes = sum(m.E * m.nn for m in meshes)
    ens = pkg.abi.dg_ensemble_create([m.h for m in meshes], states)
    t0 = time.time()
    pkg.abi.dg_ensemble_tune(ens)
    tune_s = time.time() - t0
    stream = torch.cuda.current_stream()

    def timed(step_all):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.ens_steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            step_all()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    for _ in range(3):
        pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=True)
    batched_ms = timed(lambda: pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=True))

    def one_by_one():
        for m, U in zip(meshes, states):
            m.rk3_step(U, cfl=0.2)
    one_by_one()
    permesh_ms = timed(one_by_one)
    status = max(m.sync_status() for m in meshes)
    groups = pkg.abi.dg_ensemble_groups(ens)
    for g in groups:
        g.pop("members", None)
    pkg.abi.dg_ensemble_destroy(ens)
    for m in meshes:
        m.close()
    dof = nodes * 5 * args.ens_steps
    return {"workload": "256 meshes: NE smooth wave (LLF) or SR blast (HLL, MinModN, learned guess), "
                        "K in [2,16], n in [3,8], seed 5, mixed precision, CFL 0.2",
            "meshes": len(recipe), "nodes": nodes, "steps": args.ens_steps,
            "batched_graph": {"value": dof / (batched_ms / 1e3), "unit": UNIT,
                              "ms_per_step": batched_ms / args.ens_steps},
            "per_mesh_launches": {"value": dof / (permesh_ms / 1e3), "unit": UNIT,
                                  "ms_per_step": permesh_ms / args.ens_steps},
            "speedup": permesh_ms / batched_ms, "tune_s": round(tune_s, 3), "groups": groups,
            "device_status": status}


def _measure(pkg, torch, precision, args, dist, U0, net=None):
    """Warm-up, then K graph-replayed steps timed with per-step CUDA events (L2
    flushed between steps, outside the event pairs), then K profiled steps for
    per-kernel durations."""
    w = WORKLOAD
    mesh = pkg.Mesh(system=w["system"], K=w["K"], n=w["n"], flux=w["flux"], limiter=w["limiter"],
                    gamma=w["gamma"], precision=precision)
    if net is not None:
        mesh.set_c2p_net(net)
    shape = None
    U = U0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        mesh.rk3_step(U, cfl=w["cfl"])
    torch.cuda.synchronize()
    if mesh.sync_status() != 0:
        raise RuntimeError("warm-up steps reported a device error")
    if precision == 1:
        # tuned on the warmed-up state, the one the timed steps start from
        shape = _tune_launch_shape(pkg, mesh, U)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        mesh.rk3_step(U, cfl=w["cfl"])  # one more warm step on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        mesh.rk3_step(U, cfl=w["cfl"])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        graph.replay()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    status = mesh.sync_status()
    # per-kernel durations: the same steps launched directly with event pairs
    pkg.abi.dg_profile_enable(mesh.h, True)
    for k in range(args.steps):
        flush.fill_(float(k))
        mesh.rk3_step(U, cfl=w["cfl"])
    torch.cuda.synchronize()
    prof = pkg.abi.dg_profile_read(mesh.h)
    pkg.abi.dg_profile_enable(mesh.h, False)
    return mesh, graph, step_ms, prof, status, U, shape


def _tune_launch_shape(pkg, mesh, U0):
    """Pick the stage kernel's elements per CTA and volume contraction for this
    mesh with the library's autotuner (a one-mesh ensemble times the candidates
    on a copy of the given state), and set them on the mesh (untimed)."""
    U = U0.clone()
    ens = pkg.abi.dg_ensemble_create([mesh.h], [U])
    try:
        pkg.abi.dg_ensemble_tune(ens)
        g = pkg.abi.dg_ensemble_groups(ens)[0]
    finally:
        pkg.abi.dg_ensemble_destroy(ens)
    mesh.set_option(pkg.abi.OPT_ELEMENTS_PER_CTA, g["epb"])
    mesh.set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, g["tc"])
    return {"elements_per_cta": g["epb"], "volume_contraction": "tensor cores (split-BF16x3)" if g["tc"]
            else "FP32 FMA"}


def run_ours(args):
    import torch
    import paper_1609_00098_gb300 as pkg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOAD
    setup = pkg.Mesh(system=w["system"], K=w["K"], n=w["n"], flux=w["flux"], limiter=w["limiter"],
                     gamma=w["gamma"])
    nodes = setup.E * setup.nn
    U0 = _init_state(pkg, setup, torch)
    net, net_info = _train_guess_net(pkg, torch)

    # accuracy at equal time steps (untimed): mixed (learned guess, and warm
    # start) vs plain FP64 after a few steps
    mixed_acc = None
    if not args.no_accuracy:
        mixed_acc = {}
        for name, use_net in (("learned", net), ("warm_start", None)):
            mix = pkg.Mesh(system=w["system"], K=w["K"], n=w["n"], flux=w["flux"], limiter=w["limiter"],
                           gamma=w["gamma"], precision=1)
            if use_net is not None:
                mix.set_c2p_net(use_net)
            Uf, Um = U0.clone(), U0.clone()
            dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
            for _ in range(args.acc_steps):
                setup.rk3_step(Uf, cfl=w["cfl"], dt_used=dtv)
                mix.rk3_step(Um, dt=float(dtv.item()))
            torch.cuda.synchronize()
            num = torch.sqrt(((Um - Uf) ** 2).sum(dim=(0, 2)))
            den = torch.sqrt((Uf ** 2).sum(dim=(0, 2)))
            rel = (num / torch.clamp(den, min=1e-3 * float(den.max()))).cpu().tolist()
            mixed_acc[name] = {"steps": args.acc_steps, "rel_l2_vs_fp64_per_var": rel, "max": max(rel)}
            mix.close()
    setup.close()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    results = {}
    for key, precision, use_net in (("learned", 1, net), ("warm_start", 1, None), ("fp64", 0, None)):
        results[key] = _measure(pkg, torch, precision, args, dist, U0, use_net)
    clk = clocks.stop()

    def agg(ms):
        return max_over_ranks(float(sum(ms)), dist)

    mesh, graph, step_ms, prof, status, mesh_state, shape = results["learned"]
    total_ms = agg(step_ms)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(nodes, ws, args.steps, total_ms)
    f_mesh, f_graph, f_ms, f_prof, f_status, _, _ = results["fp64"]
    f_total = agg(f_ms)
    w_mesh, w_graph, w_ms, w_prof, w_status, _, w_shape = results["warm_start"]
    w_total = agg(w_ms)

    # end to end through the C ABI with host buffers (mixed path): every step copies
    # the state from pinned host memory to the device, advances it with
    # dg_rk3_step, and copies it back, so the host copy evolves as the device state
    # did above.  The three are captured once into a CUDA graph (as the device-timed
    # steps are) and replayed; per-step event pairs, the L2 flush between steps
    # outside them.
    host_state = mesh_state.cpu().pin_memory()
    Ud = torch.empty_like(U0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # one eager end-to-end step before the capture
        Ud.copy_(host_state, non_blocking=True)
        mesh.rk3_step(Ud, cfl=w["cfl"])
        host_state.copy_(Ud, non_blocking=True)
    torch.cuda.current_stream().wait_stream(side)
    e2e_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(e2e_graph):
        Ud.copy_(host_state, non_blocking=True)
        mesh.rk3_step(Ud, cfl=w["cfl"])
        host_state.copy_(Ud, non_blocking=True)
    stream = torch.cuda.current_stream()
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        e_s[k].record(stream)
        e2e_graph.replay()
        e_e[k].record(stream)
    torch.cuda.synchronize()
    e2e_ms = agg([a.elapsed_time(b) for a, b in zip(e_s, e_e)])
    e2e = ws * nodes * 5 * args.steps / (e2e_ms / 1e3)
    state_bytes = nodes * 5 * 8

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))

    def kern(pr):
        tot = max(1e-12, sum(x[0] for x in pr.values()))
        return {c: {"ms_total": round(v[0], 4), "launches": int(v[1]), "share": round(v[0] / tot, 4)}
                for c, v in pr.items() if v[1]}

    st_ms, st_n = prof["stage"]
    stage_avg_s = (st_ms / st_n) / 1e3 if st_n else float("nan")
    achieved = _algorithmic(nodes, 1, learned=True) / stage_avg_s / 1e9
    launches = int(sum(c for _, c in prof.values()))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 arithmetic, f64 state and RK accumulation",
        "data": "synthetic (seeded blast initial data)",
        "config": _config({"precision": "mixed", "c2p_guess": "learned (in-kernel MLP; stage 1 reuses the CFL pass's solve of U^n)",
                           "launch_shape": dict(shape, picked_by="dg_ensemble_tune"),
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "step_launch": "CUDA graph replay"}),
        "variant": "mixed+learned (FP32 con2prim from the in-kernel MLP guess, FP32 fluxes/contraction/face "
                   "fluxes, FP64 stage states and RK accumulation)",
        "plain_fp64": {"value": ws * nodes * 5 * args.steps / (f_total / 1e3), "unit": UNIT,
                       "ms_per_step": f_total / args.steps, "kernels": kern(f_prof), "device_status": f_status},
        "speedup_vs_plain_fp64": f_total / total_ms,
        "mixed_warm_start": {"value": ws * nodes * 5 * args.steps / (w_total / 1e3), "unit": UNIT,
                             "ms_per_step": w_total / args.steps, "kernels": kern(w_prof),
                             "device_status": w_status, "launch_shape": w_shape,
                             "note": "con2prim starts from the previous pass's pressure (8 B/node/stage carried)"},
        "c2p_net": net_info,
        "mixed_accuracy": mixed_acc,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
        "gpu_launches": launches,
        "kernels": kern(prof),
        "roofline": {"kernel": "k_stage_mixed (fused con2prim + RHS + SSP-RK3 stage update + limiter summaries)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": _traffic("learned"), "bytes_per_launch": _algorithmic(nodes, 1, learned=True),
                     "avg_launch_ms": stage_avg_s * 1e3,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"},
        "clocks": clk,
        "device_status": status,
    }
    if not args.no_ensemble:
        out["ensemble"] = _ensemble(pkg, torch, net, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    for r in results.values():
        r[0].close()
    pkg.abi.dg_c2p_net_destroy(net)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _oracle_mesh():
    import oracle
    w = WORKLOAD
    spec = oracle.MeshSpec(system=w["system"], K=w["K"], n=w["n"], flux=w["flux"], limiter=w["limiter"],
                           gamma=w["gamma"])
    return oracle.Mesh(spec)


def cpu_baseline(seconds: float = 15.0):
    """The FP64 oracle, as it stands, on the host cores: as many steps of the same
    workload as fit in about `seconds` (at least one)."""
    import dg_inputs as di
    om = _oracle_mesh()
    U = om.from_prim(di.blast_sr(om.coords(), seed=WORKLOAD["seed"]))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    steps = 0
    while True:
        h = om.cfl_dt(U, WORKLOAD["cfl"])
        U = om.rk3_step(U, h)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    nodes = om.E * om.nn
    return {"value": nodes * 5 * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} CFL steps of the full workload from its initial state ({el:.1f} s)"}


def run_reference(args):
    """The oracle timed as the reference arm: each step is one full step of the
    workload on the host cores."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    import dg_inputs as di
    om = _oracle_mesh()
    U = om.from_prim(di.blast_sr(om.coords(), seed=WORKLOAD["seed"]))
    for _ in range(args.warmup):
        U = om.rk3_step(U, om.cfl_dt(U, WORKLOAD["cfl"]))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = om.rk3_step(U, om.cfl_dt(U, WORKLOAD["cfl"]))
    el = time.perf_counter() - t0
    nodes = om.E * om.nn
    value = nodes * 5 * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded blast initial data)",
           "config": _config({"precision": "fp64", "implementation": "FP64 CPU oracle (C, OpenMP)"}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} full steps after {args.warmup} warm-up steps"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--acc-steps", type=int, default=10)
    ap.add_argument("--ens-steps", type=int, default=20)
    ap.add_argument("--no-ensemble", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
