#!/usr/bin/env python
"""DG-RK3 throughput (dof-updates/s) of the nodal DG hot path on GB300.

Headline workload: the 3D Newtonian Kelvin-Helmholtz shear layer, gamma = 5/3,
periodic [-0.5, 0.5]^3, 64^3 affine elements, 6 LGL nodes per axis (56,623,104
nodes x 5 conserved variables), rho = 2 and vx = +0.5 for |y| < 0.25, else rho = 1
and vx = -0.5, p = 2.5, vy = 0.01 (2u - 1) seeded per node; HLL flux, MinModN
limiter after every stage, CFL 0.2 (dt computed on the device every step).  A
step is one full SSP-RK3 step (three right-hand sides, the limiter after each
stage).  `value` is the mixed-precision path (FP32 arithmetic, FP64 state and RK
accumulation); the Newtonian system has no con2prim, so the learned guess does
not apply to it.  `plain_fp64` is the FP64 path on the same workload, and
`mixed_accuracy` compares the two after ten steps at equal dt.

Secondary objects: `sr_blast` (the relativistic blast, 16^3 x 5^3 nodes: mixed
with the learned con2prim guess, mixed warm-started, FP64), `con2prim` (2^24
standalone FP64 con2prim solves from the standard and the learned guess, the
network trained on 2^22 generated pairs), `ensemble` (256 ragged meshes).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (launched by torch.distributed.run) runs
N independent replicas, one per GPU; the path has no data exchange to shard.
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

KH = dict(system=0, K=(64, 64, 64), n=6, flux=1, limiter=1, gamma=5.0 / 3.0, lo=(-0.5,) * 3, hi=(0.5,) * 3,
          cfl=0.2, seed=1)
BLAST = dict(system=1, K=(16, 16, 16), n=5, flux=1, limiter=1, gamma=4.0 / 3.0, lo=(0.0,) * 3, hi=(1.0,) * 3,
             cfl=0.2, seed=1)
KH_SAMPLE_K = (16, 16, 16)   # the CPU oracle's bounded sample of the KH workload
METRIC = "DG-RK3 dof-updates/s on 1 GB300: plain FP64 vs mixed+learned at equal L2 error"
UNIT = "dof-updates/s"
# Compulsory HBM bytes per node of one stage launch in the roofline model with FP64
# stage states: stage 1 reads U^n and writes U^1 (80 B), stages 2 and 3 read U_s and
# U^n and write U_{s+1} (120 B each): 320 B per node-step, 64 B per dof-update.
FP64_STATE_BYTES_PER_NODE_STAGE = (80.0 + 120.0 + 120.0) / 3.0


def _nodes(w):
    return int(np.prod(w["K"])) * w["n"] ** 3


def _mesh_kw(w, **extra):
    kw = {k: w[k] for k in ("system", "K", "n", "flux", "limiter", "gamma", "lo", "hi")}
    kw.update(extra)
    return kw


def _config(extra=None):
    w = KH
    k, nodes = w["K"][0], _nodes(w)
    cfg = {"workload": "Newtonian Kelvin-Helmholtz shear layer, %d^3 elements, %d LGL nodes/axis (%.1fM nodes), "
                       "gamma 5/3, HLL, MinModN, CFL 0.2" % (k, w["n"], nodes / 1e6),
           "system": "Newtonian Euler", "elements": list(w["K"]), "lgl_nodes_per_axis": w["n"], "nodes": nodes,
           "vars": 5, "flux": "HLL", "limiter": "MinModN", "cfl": w["cfl"], "seed": w["seed"],
           "l2_between_steps": "inputs larger than L2 (state %.2f GB per copy; no flush)" % (nodes * 40 / 1e9)}
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



def _state(pkg, torch, w, mesh, seed=None):
    """Initial conserved state on the device: the library's node coordinates, the
    seeded primitive fields of dg_inputs, the library's prim -> cons."""
    xyz = mesh.coords().cpu().numpy()
    seed = w["seed"] if seed is None else seed
    prim = dg_inputs.kh_ne(xyz, seed=seed) if w["system"] == 0 else dg_inputs.blast_sr(xyz, seed=seed)
    del xyz
    return mesh.from_prim(torch.from_numpy(prim).cuda())


def _lgl_weights3(pkg, n):
    _, w, _, _ = pkg.abi.dg_lgl_tables(n)
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


def _rel_l2(torch, w3, a, b):
    """Per-variable relative L2 distance of a to b (LGL quadrature on the uniform
    affine mesh, each norm floored at 1 % of the largest variable's norm)."""
    wt = torch.from_numpy(w3).to(a.device)
    d = torch.sqrt(((a - b) ** 2 * wt).sum(dim=(0, 2)))
    r = torch.sqrt((b ** 2 * wt).sum(dim=(0, 2)))
    return (d / torch.clamp(r, min=1e-2 * float(r.max()))).cpu().tolist()


def _replay(torch, graph, steps, dist, flush, after=None):
    """`steps` replays of `graph`, each bracketed by CUDA events on the replay stream
    (L2 flushed before each when `flush` is given, outside the events)."""
    stream = torch.cuda.current_stream()
    s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        if flush is not None:
            flush.fill_(float(k))
        s_ev[k].record(stream)
        graph.replay()
        e_ev[k].record(stream)
        if after is not None:
            torch.cuda.synchronize()
            after()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return [s.elapsed_time(e) for s, e in zip(s_ev, e_ev)]


def _capture(pkg, torch, mesh, U, w):
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        mesh.rk3_step(U, cfl=w["cfl"])  # one more warm step on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    pkg.abi.dg_profile_read(mesh.h)  # drop the eager warm step's events, if any
    with torch.cuda.graph(graph):
        mesh.rk3_step(U, cfl=w["cfl"])
    torch.cuda.synchronize()
    return graph


def _timed_steps(pkg, torch, mesh, U, w, steps, dist, flush=None):
    """Graph-replayed steps, timed twice: (1) the step alone, each replay bracketed
    by CUDA events on the replay stream: the step time; (2) the same steps with
    the library's per-kernel events captured into the graph (external event
    nodes), so that kernel durations come from replays of the step that is timed.
    Returns (step times of 1, per-kernel totals of 2, step times of 2): the
    difference of the step times is what the event nodes cost."""
    graph = _capture(pkg, torch, mesh, U, w)
    step_ms = _replay(torch, graph, steps, dist, flush)
    del graph
    pkg.abi.dg_profile_enable(mesh.h, True)
    graph = _capture(pkg, torch, mesh, U, w)
    prof = {}

    def collect():
        for c, (ms, n) in pkg.abi.dg_profile_read(mesh.h).items():
            acc = prof.setdefault(c, [0.0, 0])
            acc[0] += ms
            acc[1] += n
    prof_ms = _replay(torch, graph, steps, dist, flush, after=collect)
    pkg.abi.dg_profile_enable(mesh.h, False)
    del graph  # before the mesh that owns the graph's events goes
    torch.cuda.synchronize()
    return step_ms, prof, prof_ms


def _kern(prof):
    tot = max(1e-12, sum(v[0] for v in prof.values()))
    return {c: {"ms_total": round(v[0], 4), "launches": int(v[1]), "share": round(v[0] / tot, 4)}
            for c, v in prof.items() if v[1]}


def _kh_accuracy(pkg, torch, U0, steps):
    """Mixed vs FP64 after `steps` KH steps at equal dt (the FP64 path's CFL dt;
    the FP64 path is bitwise equal to the FP64 oracle in the tests), with the
    number of elements whose last-stage limiter flags differ."""
    w = KH
    f = pkg.Mesh(precision=0, **_mesh_kw(w))
    m = pkg.Mesh(precision=1, **_mesh_kw(w))
    Uf, Um = U0.clone(), U0.clone()
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    tf = torch.zeros(f.E, dtype=torch.uint8, device="cuda")
    tm = torch.zeros(f.E, dtype=torch.uint8, device="cuda")
    for _ in range(steps):
        f.rk3_step(Uf, cfl=w["cfl"], dt_used=dtv, troubled=tf)
        m.rk3_step(Um, dt=float(dtv.item()), troubled=tm)
    torch.cuda.synchronize()
    rel = _rel_l2(torch, _lgl_weights3(pkg, w["n"]), Um, Uf)
    flips = int((tf != tm).sum().item())
    out = {"steps": steps, "rel_l2_vs_fp64_per_var": rel, "max": max(rel), "bar": 1e-6,
           "norm": "LGL-quadrature L2 per conserved variable, floored at 1 % of the largest",
           "reference": "the FP64 GPU path at the same dt (bitwise equal to the FP64 oracle in the tests)",
           "limiter_flag_differences_last_stage": flips, "elements": f.E,
           "device_status": [f.sync_status(), m.sync_status()]}
    f.close()
    m.close()
    del Uf, Um
    return out


def _new_net(pkg):
    """A network with seeded uniform initial weights U(+-sqrt(3 / fan_in))."""
    init = dg_inputs.uniform(5, 9, np.arange(pkg.abi.N_NET_PARAMS))
    params = np.zeros(pkg.abi.N_NET_PARAMS)
    for o, fan, cnt in ((0, 3, 192), (256, 64, 4096), (4416, 64, 64)):
        params[o:o + cnt] = np.sqrt(3.0 / fan) * (2.0 * init[o:o + cnt] - 1.0)
    return pkg.abi.dg_c2p_net_create(params.astype(np.float32), (-5.0, 4.0, -9.0, 3.0, -4.5, 4.5))


def _c2p_states(pkg, torch, seed, count, gamma):
    """`count` (a multiple of 64) seeded primitive states of the con2prim
    distribution (rho log-uniform [1e-8, 10], W uniform [1, 10] on uniform
    directions, eps log-uniform [1e-6, 1e2]) and their conserved states from the
    library's prim -> cons (a helper mesh of 4^3-node elements holds them)."""
    prim = torch.from_numpy(np.ascontiguousarray(dg_inputs.c2p_samples(seed, count, gamma=gamma))).cuda()
    E = count // 64
    kx = min(E, 64)
    ky = min(E // kx, 64)
    kz = E // (kx * ky)
    helper = pkg.Mesh(system=1, K=(kx, ky, kz), n=4, gamma=gamma)
    assert helper.E * 64 == count
    Ug = helper.state()
    pkg.abi.dg_prim2con(helper.h, prim, Ug)
    helper.close()
    return Ug.permute(1, 0, 2).reshape(5, count).contiguous(), prim


def _train_guess_net(pkg, torch, w):
    """Train the learned con2prim guess (untimed) on pairs the method generates for
    the blast: the conserved states and FP64 pressures of the first six FP64 steps
    of the same blast with another noise seed (2), 2^18 pairs sampled from them,
    plus 2^16 states of the generic con2prim distribution.  Twenty epochs of
    Adam, batch 2048."""
    g = w["gamma"]
    mesh = pkg.Mesh(precision=0, **_mesh_kw(w))
    U = _state(pkg, torch, w, mesh, seed=2)
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
    Ug, prim = _c2p_states(pkg, torch, 7, 1 << 16, g)
    cons = torch.cat([cons[:, pick], Ug], 1).contiguous()
    pres = torch.cat([pres[pick], prim[4]]).contiguous()
    net = _new_net(pkg)
    epochs = 20
    losses = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    t0 = time.time()
    pkg.abi.dg_c2p_net_train(net, cons.shape[1], cons, pres, epochs, 2048, 2e-3, losses)
    torch.cuda.synchronize()
    info = {"pairs": int(cons.shape[1]),
            "source": "blast seed 2, FP64 steps 0-5 (2^18) + generic con2prim states (2^16)",
            "epochs": epochs, "batch": 2048, "train_s": round(time.time() - t0, 3),
            "loss_first_last": [float(losses[0]), float(losses[-1])]}
    return net, info


def _con2prim_bench(pkg, torch, reps=3):
    """Config 3: 2^24 FP64 con2prim solves (Sec. 2.1.2) from the standard guess and
    from the learned guess (network trained on 2^22 generated pairs, disjoint
    seed), timed with CUDA events; the results agree to the solver's resolution."""
    g = 4.0 / 3.0
    tr_cons, tr_prim = _c2p_states(pkg, torch, 11, 1 << 22, g)
    net = _new_net(pkg)
    epochs = 8
    losses = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    pkg.abi.dg_c2p_net_train(net, 1 << 22, tr_cons, tr_prim[4].contiguous(), epochs, 4096, 2e-3, losses)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    del tr_cons, tr_prim
    N = 1 << 24
    cons, prim_true = _c2p_states(pkg, torch, 3, N, g)
    del prim_true
    guess = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.empty((5, N), dtype=torch.float64, device="cuda")
    it = torch.empty(N, dtype=torch.int32, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    res, prims = {}, {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for name in ("standard", "learned"):
        times, gtimes = [], []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            ev[0].record()
            if name == "learned":
                pkg.abi.dg_c2p_net_guess(net, N, g, cons, guess)
            ev[1].record()
            pkg.abi.dg_con2prim(N, g, cons, out, guess if name == "learned" else None, it, st)
            ev[2].record()
            torch.cuda.synchronize()
            if r:  # the first repetition is a warm-up
                gtimes.append(ev[0].elapsed_time(ev[1]))
                times.append(ev[1].elapsed_time(ev[2]))
        itn = it.to(torch.float64)
        ms = float(np.median(times))
        gms = float(np.median(gtimes)) if name == "learned" else 0.0
        res[name] = {"con2prim_ms": ms, "guess_ms": gms, "total_ms": ms + gms,
                     "solves_per_s": N / ((ms + gms) / 1e3), "mean_iters": float(itn.mean()),
                     "max_iters": int(it.max()), "failed": int((st != 0).sum())}
        prims[name] = out[4].clone()
    p0, p1 = prims["standard"], prims["learned"]
    rel = ((p1 - p0).abs() / p0.abs()).max().item()
    pkg.abi.dg_c2p_net_destroy(net)
    return {"workload": "2^24 con2prim solves, gamma 4/3, rho log-uniform [1e-8, 10], W uniform [1, 10], "
                        "eps log-uniform [1e-6, 1e2], seed 3; FP64 bracketed Newton",
            "states": N, "net": {"pairs": 1 << 22, "seed": 11, "epochs": epochs, "batch": 4096,
                                  "train_s": round(train_s, 3),
                                  "loss_first_last": [float(losses[0]), float(losses[-1])]},
            "standard_guess": res["standard"], "learned_guess": res["learned"],
            "speedup_con2prim_only": res["standard"]["con2prim_ms"] / res["learned"]["con2prim_ms"],
            "speedup_with_guess": res["standard"]["total_ms"] / res["learned"]["total_ms"],
            "max_rel_diff_pressure": rel}


# Arithmetic of one k_stage_mixed launch on the relativistic blast with the learned
# guess, mean over the three stages of a step, from one ncu capture of three
# launches: FP64 flops = 2 DFMA + DADD + DMUL, FP32 flops = 2 FFMA + FADD + FMUL
# (+ twice that for the paired FFMA2 / FADD2 / FMUL2), SASS thread instructions
# with all predicates true.  Reported only while the kernel's sources hash to
# their state at capture.
# The same capture's pipe utilisation (ncu, % of peak sustained while active, mean
# of the three launches) is reported beside the flop fractions.
SR_STAGE_FLOPS = {"fp64": 18911529, "fp32": 348447061}
SR_STAGE_PIPES = {"fp64_pipe_pct": 35.2, "fma_pipe_pct": 13.9, "alu_pipe_pct": 22.1, "tensor_pipe_pct": 4.6,
                  "issue_active_pct": 40.8}
SR_STAGE_SOURCES = ("paper_1609_00098_gb300/csrc/dg_mixed.cuh", "paper_1609_00098_gb300/csrc/dg_physics.cuh",
                    "paper_1609_00098_gb300/csrc/dg_c2p_net.cuh", "paper_1609_00098_gb300/csrc/dg_internal.h")
SR_STAGE_SOURCES_SHA256 = "8d675640bc064200bd0ad8de38aa766def3ba352f8d371be08a4ad4bbbc41120"
# FMA throughput of this GPU (independent dependent-FMA chains, every SM busy;
# flops count an FMA as two): FP64 1.20 TFLOP/s, FP32 75.0 TFLOP/s.
FP64_PEAK_TFLOPS = 1.20
FP32_PEAK_TFLOPS = 75.0


def _sources_match(files, digest):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == digest


def _alu_roofline(avg_launch_ms):
    """FP64- and FP32-pipe roofline of the SR stage kernel: the captured flops of
    one launch over the live CUDA-event launch time, against the FMA peaks."""
    out = {"kernel": "k_stage_mixed<5, SR, HLL, learned guess>", "bound": "alu", "unit": "TFLOP/s",
           "avg_launch_ms": avg_launch_ms, "peak_fp64": FP64_PEAK_TFLOPS, "peak_fp32": FP32_PEAK_TFLOPS,
           "peak_source": "FMA-chain micro-benchmark on this GPU (measured)",
           "timing": "CUDA events captured as graph nodes into replays of the timed step (second pass of the same steps)"}
    if SR_STAGE_FLOPS is None or not _sources_match(SR_STAGE_SOURCES, SR_STAGE_SOURCES_SHA256):
        out.update({"achieved": None, "peak": FP64_PEAK_TFLOPS, "frac": None,
                    "note": "no flop count captured for the current kernel sources"})
        return out
    s = avg_launch_ms / 1e3
    f64 = SR_STAGE_FLOPS["fp64"] / s / 1e12
    f32 = SR_STAGE_FLOPS["fp32"] / s / 1e12
    out.update({"achieved": f64, "peak": FP64_PEAK_TFLOPS, "frac": f64 / FP64_PEAK_TFLOPS,
                "ncu_pipes": SR_STAGE_PIPES,
                "fp64": {"flops_per_launch": SR_STAGE_FLOPS["fp64"], "achieved": f64,
                         "frac": f64 / FP64_PEAK_TFLOPS},
                "fp32": {"flops_per_launch": SR_STAGE_FLOPS["fp32"], "achieved": f32,
                         "frac": f32 / FP32_PEAK_TFLOPS}})
    return out


def _tc_ab(pkg, torch, args):
    """Volume contraction of the SR stage kernel on the tensor cores (split-BF16x3
    mma.sync) vs FP32 FMA, per n: the blast at about 512k nodes, mixed, warm
    start; mean stage-launch time over 5 graph-replayed steps each."""
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    table = {}
    for n in range(3, 9):
        k = max(4, int(round((512000.0 / n ** 3) ** (1.0 / 3.0))))
        w = dict(BLAST, K=(k, k, k), n=n)
        setup = pkg.Mesh(precision=0, **_mesh_kw(w))
        U0 = _state(pkg, torch, w, setup)
        setup.close()
        row = {"elements": k ** 3, "nodes": k ** 3 * n ** 3}
        for key, tc in (("tensor_core_ms", 1), ("fma_ms", 0)):
            m = pkg.Mesh(precision=1, **_mesh_kw(w))
            m.set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, tc)
            U = U0.clone()
            for _ in range(3):
                m.rk3_step(U, cfl=w["cfl"])
            _, prof, _ = _timed_steps(pkg, torch, m, U, w, 5, None, flush=flush)
            row[key] = prof["stage"][0] / prof["stage"][1]
            m.close()
        row["faster"] = "tensor_core" if row["tensor_core_ms"] < row["fma_ms"] else "fma"
        table[str(n)] = row
    return {"workload": "SR blast, K^3 elements with K^3 n^3 about 512k nodes, mixed, warm start, HLL, MinModN",
            "stat": "mean k_stage_mixed launch, CUDA events in graph replays, L2 flushed per step", "per_n": table}


def _sr_blast(pkg, torch, args):
    """The relativistic blast (secondary): mixed with the learned guess, mixed
    warm-started, FP64; L2 flushed between steps (its state fits in L2)."""
    w = BLAST
    setup = pkg.Mesh(precision=0, **_mesh_kw(w))
    U0 = _state(pkg, torch, w, setup)
    setup.close()
    net, net_info = _train_guess_net(pkg, torch, w)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"workload": "SR blast, 16^3 elements, 5 LGL nodes/axis (512,000 nodes), HLL, MinModN, con2prim per node, "
                       "CFL 0.2", "l2_between_steps": "flushed (256 MiB write)", "c2p_net": net_info}
    nodes = _nodes(w)
    steps = args.sr_steps
    for key, precision, use_net in (("mixed_learned", 1, net), ("mixed_warm_start", 1, None), ("plain_fp64", 0, None)):
        m = pkg.Mesh(precision=precision, **_mesh_kw(w))
        if use_net is not None:
            m.set_c2p_net(use_net)
        if precision:
            m.set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, 0)  # FP32 FMA (faster at every n: tc_contraction)
        U = U0.clone()
        for _ in range(max(3, args.warmup)):
            m.rk3_step(U, cfl=w["cfl"])
        ms, prof, pms = _timed_steps(pkg, torch, m, U, w, steps, None, flush=flush)
        out[key] = {"value": nodes * 5 * steps / (sum(ms) / 1e3), "unit": UNIT, "ms_per_step": sum(ms) / steps,
                    "ms_per_step_with_kernel_events": sum(pms) / steps,
                    "kernels": _kern(prof), "device_status": m.sync_status()}
        if key == "mixed_learned":
            roof = _alu_roofline(prof["stage"][0] / prof["stage"][1])
            # the event nodes stretch these short launches: the same launch time scaled
            # to the step time measured without them
            scaled = prof["stage"][0] / prof["stage"][1] * (sum(ms) / sum(pms))
            roof["avg_launch_ms_scaled_to_plain_step"] = scaled
            if roof.get("fp64"):
                roof["fp64"]["frac_scaled"] = roof["fp64"]["frac"] * roof["avg_launch_ms"] / scaled
                roof["fp32"]["frac_scaled"] = roof["fp32"]["frac"] * roof["avg_launch_ms"] / scaled
            out["alu_roofline"] = roof
        m.close()
    acc = {}
    for name, use_net in (("learned", net), ("warm_start", None)):
        f = pkg.Mesh(precision=0, **_mesh_kw(w))
        m = pkg.Mesh(precision=1, **_mesh_kw(w))
        if use_net is not None:
            m.set_c2p_net(use_net)
        Uf, Um = U0.clone(), U0.clone()
        dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(10):
            f.rk3_step(Uf, cfl=w["cfl"], dt_used=dtv)
            m.rk3_step(Um, dt=float(dtv.item()))
        rel = _rel_l2(torch, _lgl_weights3(pkg, w["n"]), Um, Uf)
        acc[name] = {"steps": 10, "rel_l2_vs_fp64_per_var": rel, "max": max(rel)}
        f.close()
        m.close()
    out["mixed_accuracy"] = acc
    out["speedup_learned_vs_fp64"] = out["plain_fp64"]["ms_per_step"] / out["mixed_learned"]["ms_per_step"]
    pkg.abi.dg_c2p_net_destroy(net)
    return out


def _hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except Exception:
        return 6800.0, "fallback"


def _ensemble_roofline(nodes, ms_per_step):
    """Whole-step HBM roofline of the batched ensemble: the FP64-state model's 64 B per
    dof-update (320 B per node-step) over the graph-timed step."""
    peak, src = _hbm_peak()
    achieved = 320.0 * nodes / (ms_per_step / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "bytes_per_step": 320.0 * nodes, "rule": "64 B per dof-update over the graph-timed step",
            "peak_source": src}


def _ensemble(pkg, torch, args):
    """Ragged ensemble (untimed setup): 256 meshes from the seeded recipe -- system
    NE or SR with probability 1/2, K uniform in [2, 16] per axis, n uniform in
    [3, 8].  NE meshes carry the smooth density wave (LLF, no limiter), SR meshes
    the blast (HLL, MinModN, learned con2prim guess); mixed precision, CFL 0.2.
    Times `ens_steps` steps of (a) the batched per-group launches replayed as one
    CUDA graph per step, after the launch-shape autotuner, with the groups one
    after the other and, for comparison, on parallel graph branches, and (b) the same
    meshes stepped one by one with dg_rk3_step.  The states (2.7 GB each) exceed L2."""
    net, _ = _train_guess_net(pkg, torch, BLAST)
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
        pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=1)
    # every variant starts from the same states (the blast evolves, and with it the
    # limiter's and con2prim's work), after one untimed step of its own
    snapshot = [U.clone() for U in states]

    def restore():
        for U, S in zip(states, snapshot):
            U.copy_(S)

    def one_by_one():
        for m, U in zip(meshes, states):
            m.rk3_step(U, cfl=0.2)

    restore()
    pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=1)
    batched_ms = timed(lambda: pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=1))
    restore()
    pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=2)
    branches_ms = timed(lambda: pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=2))
    restore()
    one_by_one()
    permesh_ms = timed(one_by_one)
    del snapshot
    status = max(m.sync_status() for m in meshes)
    groups = pkg.abi.dg_ensemble_groups(ens)
    for g in groups:
        g.pop("members", None)
    pkg.abi.dg_ensemble_destroy(ens)
    for m in meshes:
        m.close()
    pkg.abi.dg_c2p_net_destroy(net)
    dof = nodes * 5 * args.ens_steps
    return {"workload": "256 meshes: NE smooth wave (LLF) or SR blast (HLL, MinModN, learned guess), "
                        "K in [2,16], n in [3,8], seed 5, mixed precision, CFL 0.2",
            "meshes": len(recipe), "nodes": nodes, "steps": args.ens_steps,
            "batched_graph": {"value": dof / (batched_ms / 1e3), "unit": UNIT,
                              "ms_per_step": batched_ms / args.ens_steps,
                              "launch": "one CUDA graph per step, the groups one after the other"},
            "batched_graph_parallel_branches": {"value": dof / (branches_ms / 1e3), "unit": UNIT,
                                                "ms_per_step": branches_ms / args.ens_steps,
                                                "launch": "one CUDA graph per step, each group on its own branch"},
            "per_mesh_launches": {"value": dof / (permesh_ms / 1e3), "unit": UNIT,
                                  "ms_per_step": permesh_ms / args.ens_steps},
            "speedup": permesh_ms / batched_ms, "tune_s": round(tune_s, 3), "groups": groups,
            "roofline": _ensemble_roofline(nodes, batched_ms / args.ens_steps),
            "device_status": status}


# DRAM bytes per k_ne_stage launch on the headline workload (mean over the three
# stages of a step), from a one-kernel ncu capture of the same kernel on the
# 32^3-element case of the same problem scaled by the node count (64^3 / 32^3 = 8).
# Reported only while the kernel's sources still hash to their state at capture.
# (409.7 MB per launch at 32^3, 57.9 B per node.)
TRAFFIC_BYTES_PER_LAUNCH = 3277945515
TRAFFIC_SOURCES = ("paper_1609_00098_gb300/csrc/dg_ne_mixed.cuh", "paper_1609_00098_gb300/csrc/dg_internal.h")
TRAFFIC_SOURCES_SHA256 = "55ff2325c3b9ad59fcdbeb0a4866b7772eff667623c900db9cdc2798eb3aa4ac"


def _traffic():
    if TRAFFIC_BYTES_PER_LAUNCH is None or not _sources_match(TRAFFIC_SOURCES, TRAFFIC_SOURCES_SHA256):
        return None
    return TRAFFIC_BYTES_PER_LAUNCH


def _design_bytes_per_node_stage(masked_all):
    """Compulsory bytes per node of one k_ne_stage launch of this design (FP64 U^n,
    FP32 stage differences), mean over the three stages: stage 1 reads U^n (40 B)
    and writes R(U^n) (20 B); stages 2 and 3 read U^n and, where a variable is not
    limited, its difference (20 B), and write the next difference (20 B).  With
    every variable limited (the shear layer after its first stage) the differences
    of stages 2 and 3 are not read."""
    return (60.0 + 2 * (60.0 if masked_all else 80.0)) / 3.0


def _headline(pkg, torch, args, ws, local, dist):
    """The KH workload: mixed (timed), FP64, accuracy, end to end, roofline."""
    w = KH
    nodes = _nodes(w)
    setup = pkg.Mesh(precision=0, **_mesh_kw(w))
    U0 = _state(pkg, torch, w, setup)
    setup.close()

    mixed_acc = None if args.no_accuracy else _kh_accuracy(pkg, torch, U0, args.acc_steps)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    runs = {}
    for key, precision in (("mixed", 1), ("fp64", 0)):
        m = pkg.Mesh(precision=precision, **_mesh_kw(w))
        U = U0.clone()
        for _ in range(args.warmup):
            m.rk3_step(U, cfl=w["cfl"])
        torch.cuda.synchronize()
        if m.sync_status() != 0:
            raise RuntimeError("warm-up steps reported a device error")
        ms, prof, pms = _timed_steps(pkg, torch, m, U, w, args.steps if key == "mixed" else args.fp64_steps, dist)
        runs[key] = (m, ms, prof, m.sync_status(), U, pms)
    clk = clocks.stop()
    mesh, step_ms, prof, status, mesh_state, prof_step_ms = runs["mixed"]
    total_ms = max_over_ranks(float(sum(step_ms)), dist)
    value = whole_job_rate(nodes, ws, args.steps, total_ms)
    f_mesh, f_ms, f_prof, f_status, _, _ = runs["fp64"]
    f_total = max_over_ranks(float(sum(f_ms)), dist)
    f_value = whole_job_rate(nodes, ws, args.fp64_steps, f_total)
    f_mesh.close()
    del runs["fp64"]

    # end to end through the C ABI with host buffers (mixed path): every step copies
    # the state from pinned host memory to the device, advances it with
    # dg_rk3_step, and copies it back, so the host copy evolves as the device state
    # did above.  The three are captured into a CUDA graph (as the device-timed
    # steps are) and replayed; per-step event pairs.
    host_state = mesh_state.cpu().pin_memory()
    Ud = torch.empty_like(U0)
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
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps)]
    torch.cuda.synchronize()
    for k in range(args.e2e_steps):
        e_s[k].record(stream)
        e2e_graph.replay()
        e_e[k].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in zip(e_s, e_e))), dist)
    e2e = ws * nodes * 5 * args.e2e_steps / (e2e_ms / 1e3)
    state_bytes = nodes * 5 * 8
    del e2e_graph, Ud, host_state

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    st_ms, st_n = prof["stage"]
    stage_avg_s = (st_ms / st_n) / 1e3
    bytes_8d = FP64_STATE_BYTES_PER_NODE_STAGE * nodes
    bytes_design = _design_bytes_per_node_stage(True) * nodes
    achieved = bytes_8d / stage_avg_s / 1e9
    launches = int(sum(v[1] for v in prof.values()))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 arithmetic, f64 state and RK accumulation",
        "data": "synthetic (seeded Kelvin-Helmholtz initial data)",
        "config": _config({"precision": "mixed", "parallelism": "replicas" if ws > 1 else "single GPU",
                           "step_launch": "CUDA graph replay (7 kernels per step)"}),
        "variant": "mixed (Newtonian: no con2prim, so the learned guess does not apply; the learned form is "
                   "measured on the relativistic blast in sr_blast and standalone in con2prim)",
        "plain_fp64": {"value": f_value, "unit": UNIT, "ms_per_step": f_total / args.fp64_steps,
                       "steps": args.fp64_steps, "kernels": _kern(f_prof), "device_status": f_status},
        "speedup_vs_plain_fp64": value / f_value,
        "mixed_accuracy": mixed_acc,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "steps": args.e2e_steps},
        "gpu_launches": launches,
        "kernels": _kern(prof),
        "ms_per_step_with_kernel_events": max_over_ranks(float(sum(prof_step_ms)), dist) / args.steps,
        "roofline": {"kernel": "k_ne_stage (fused RHS of eq:411 + SSP-RK3 stage difference + limiter summaries)",
                     "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": _traffic(),
                     "bytes_per_launch": bytes_8d, "bytes_per_node": FP64_STATE_BYTES_PER_NODE_STAGE,
                     "bytes_rule": "FP64-state roofline model: FP64 stage states, 320 B per node-step, mean 106.7 B per "
                                   "node and stage launch",
                     "design_bytes_per_launch": bytes_design,
                     "design_frac": bytes_design / stage_avg_s / 1e9 / hbm_peak,
                     "avg_launch_ms": stage_avg_s * 1e3, "launches_timed": int(st_n),
                     "timing": "CUDA events captured as graph nodes into replays of the timed step (second pass of the same steps)",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"},
        "step_roofline": {"ceiling_dof_updates_per_s": hbm_peak * 1e9 / 64.0,
                          "frac": value / (hbm_peak * 1e9 / 64.0),
                          "rule": "64 B per dof-update (320 B per node-step) over the measured HBM bandwidth"},
        "clocks": clk,
        "device_status": status,
    }
    mesh.close()
    del mesh_state, runs
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import paper_1609_00098_gb300 as pkg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.skip_kh:
        out = {"metric": METRIC, "unit": UNIT, "n_gpus": ws, "note": "--skip-kh: secondary objects only"}
    else:
        out = _headline(pkg, torch, args, ws, local, dist)
    if not args.no_sr:
        out["sr_blast"] = _sr_blast(pkg, torch, args)
    if not args.no_con2prim:
        out["con2prim"] = _con2prim_bench(pkg, torch)
    if not args.no_ensemble:
        out["ensemble"] = _ensemble(pkg, torch, args)
    if not args.no_tc_ab:
        out["tc_contraction"] = _tc_ab(pkg, torch, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _oracle_sample_mesh():
    """The oracle's bounded sample of the headline workload: the same problem on
    a 16^3-element periodic box (1/64 of the elements)."""
    import oracle
    w = KH
    spec = oracle.MeshSpec(system=w["system"], K=KH_SAMPLE_K, n=w["n"], flux=w["flux"], limiter=w["limiter"],
                           gamma=w["gamma"], lo=w["lo"], hi=w["hi"])
    return oracle.Mesh(spec)


def cpu_baseline(seconds: float = 15.0):
    """The FP64 oracle, as it stands, on the host cores: as many CFL steps of the
    bounded sample as fit in about `seconds` (at least one)."""
    om = _oracle_sample_mesh()
    U = om.from_prim(dg_inputs.kh_ne(om.coords(), seed=KH["seed"]))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    steps = 0
    while True:
        U = om.rk3_step(U, om.cfl_dt(U, KH["cfl"]))
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    nodes = om.E * om.nn
    return {"value": nodes * 5 * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} CFL steps of the Kelvin-Helmholtz problem on a 16^3-element box, n = 6 "
                      f"({nodes} nodes, 1/64 of the workload) from its initial state ({el:.1f} s)"}


def run_reference(args):
    """The oracle timed as the reference arm: each step is one CFL step of the
    bounded sample of the workload on the host cores."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    om = _oracle_sample_mesh()
    U = om.from_prim(dg_inputs.kh_ne(om.coords(), seed=KH["seed"]))
    for _ in range(args.warmup):
        U = om.rk3_step(U, om.cfl_dt(U, KH["cfl"]))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = om.rk3_step(U, om.cfl_dt(U, KH["cfl"]))
    el = time.perf_counter() - t0
    nodes = om.E * om.nn
    value = nodes * 5 * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Kelvin-Helmholtz initial data)",
           "config": _config({"precision": "fp64", "implementation": "FP64 CPU oracle (C, OpenMP)",
                              "sample": "each step: one CFL step of the same problem on a 16^3-element box "
                                        f"({nodes} nodes, 1/64 of the workload)"}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} CFL steps of the 16^3-element box after {args.warmup} warm-up "
                                      "steps"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--sr-steps", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--acc-steps", type=int, default=10)
    ap.add_argument("--ens-steps", type=int, default=20)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-sr", action="store_true")
    ap.add_argument("--no-con2prim", action="store_true")
    ap.add_argument("--no-tc-ab", action="store_true")
    ap.add_argument("--kh-k", type=int, default=KH["K"][0],
                    help="elements per axis of the KH problem (smaller for profiling captures)")
    ap.add_argument("--skip-kh", action="store_true",
                    help="time only the secondary objects (profiling captures of their kernels)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.kh_k < 1:
        ap.error("--kh-k must be >= 1")
    KH["K"] = (args.kh_k,) * 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
