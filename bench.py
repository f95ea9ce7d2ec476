#!/usr/bin/env python3
"""Benchmark of the PLBM stream-and-collide step on GB300.

Default workload: D2Q25 ({0,+-1,+-3}^2) Kelvin-Helmholtz double shear layer on
a periodic 2048 x 2048 grid, FP32 populations, theta0 = 1, omega = 1.3.  The two
population arrays (2 x 839 MB) are far larger than the 129 MB L2, so every
timed step streams its inputs from HBM.

Prints ONE JSON line (rank 0).  ``value`` is whole-job MLUPS (node updates per
microsecond summed over ranks) measured with CUDA events on the solver's stream,
the median of five timed runs of --steps steps each (all five are reported);
``e2e`` is the same metric through the public API with host (pinned) buffers:
plbm_init from host fields, K steps, plbm_moments back to host.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload and prints the same metric with "impl": "reference".
Under torchrun every rank runs an independent replica (the build is
single-GPU: replicas only); rank 0 prints.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1402_5487_gb300 import inputs as I  # noqa: E402

V5 = I.SET_013
OMEGA = 1.3
REPEATS = 5            # timed runs of --steps steps in the bench line; the median is reported
SURROGATE_NOISE = 0.2  # input perturbation of the surrogate's training (normalised units)
THETA0 = 1.0
ELEM = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}


KERNEL_NAME = {"f32": "k_stream_collide_pair<float>", "f16dev": "k_stream_collide_pair2<__half>",
               "bf16dev": "k_stream_collide_pair<__nv_bfloat16>", "f64": "k_stream_collide<double,5,2>"}


def kernel_fingerprint(sources):
    """SHA-256 over the source text a kernel is compiled from.  An entry is a path,
    or [path, first line, last line] for the part of a shared header the kernel
    uses (the text from the first occurrence of one to the next of the other)."""
    import hashlib
    h = hashlib.sha256()
    for src in sources:
        path, part = (src, None) if isinstance(src, str) else (src[0], src[1:])
        with open(os.path.join(ROOT, path), "rb") as fh:
            text = fh.read()
        if part:
            a = text.index(part[0].encode())
            b = text.index(part[1].encode(), a) + len(part[1])
            text = text[a:b]
        h.update(text)
    return h.hexdigest()


def read_traffic(prec):
    """DRAM bytes per launch from the committed ncu capture, or None when absent or
    when the kernel's sources changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)[KERNEL_NAME[prec]]
        if kernel_fingerprint(d["kernel_sources"]) != d["kernel_sources_sha256"]:
            return None
        return float(d["bytes_per_launch"])
    except Exception:
        return None


def json_safe(obj):
    """The object with every non-finite float replaced by None (strict JSON)."""
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: json_safe(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [json_safe(v) for v in obj]
    return obj


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
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
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(torch, t_local, node_updates, dist=None, device="cuda"):
    """Whole-job time and throughput of N independent replicas (one per rank, the
    same node_updates each): the job time is the maximum of the ranks' times and
    the throughput N x node_updates / that time, in MLUPS."""
    t_max, ws = float(t_local), 1
    if dist is not None:
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, ws = float(tt.item()), dist.get_world_size()
    return t_max, ws * node_updates / t_max / 1e6


def time_device(solver, steps: int, warmup: int, torch, barrier):
    """CUDA-event time of `steps` plbm_step launches on the solver's stream."""
    solver.step(warmup)
    st = solver.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(st)
    solver.step(steps)
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) * 1e-3


def run_variant(torch, L, prec, steps, warmup, barrier, dim=2, v=V5, bc="periodic", fields=None,
                theta0=THETA0, omega=OMEGA, left=None, right=None, nx=None):
    from paper_1402_5487_gb300 import plbm
    nx = L if nx is None else nx
    ny = L if dim == 2 else 1
    s = plbm.Solver(dim, v, omega, nx, ny, theta0=theta0, prec=prec, bc=bc, left_state=left,
                    right_state=right)
    fields = I.kh_fields(L) if fields is None else fields
    s.init(*fields)
    t = time_device(s, steps, warmup, torch, barrier)
    st = s.check()
    s.close()
    q = len(v) ** dim
    return {"mlups": nx * ny * steps / t / 1e6, "ms_per_step": t / steps * 1e3,
            "gbs_algorithmic": 2 * q * ELEM[prec] * nx * ny * steps / t / 1e9,
            "status": "ok" if st == 0 else "diverged"}


def run_slabs(torch, L, nslabs, steps, warmup, prec="f32"):
    """KH L x L decomposed into nslabs y-slabs on this GPU (halo exchange + slab steps),
    against the undivided lattice: the cost of the exchange."""
    from paper_1402_5487_gb300 import plbm
    st = torch.cuda.Stream()
    sl = plbm.Slabs(V5, OMEGA, L, L, nslabs, theta0=THETA0, prec=prec, stream=st)
    sl.init(*I.kh_fields(L))
    sl.step(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    sl.step(steps)
    e1.record(st)
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    rows = [sl.slab(k)[2] for k in range(nslabs)]
    sl.close()
    return {"mlups": L * L * steps / t / 1e6, "ms_per_step": t / steps * 1e3, "slab_rows": rows,
            "gbs_algorithmic": 2 * 25 * ELEM[prec] * L * L * steps / t / 1e9,
            "launches_per_step": 1 + nslabs}


def run_diag_overhead(torch, L, steps, every):
    """Cost of FP64 diagnostics every `every` steps: `steps` steps as
    plbm_step_diagnostics(every) calls (each a host synchronisation) against plain
    steps, both wall-timed with a synchronisation at the end."""
    from paper_1402_5487_gb300 import plbm
    s = plbm.Solver(2, V5, OMEGA, L, L, theta0=THETA0, prec="f32")
    s.init(*I.kh_fields(L))
    s.step(20)
    times = {}
    for mode in ("plain", "fused", "plain", "fused"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if mode == "plain":
            s.step(steps)
        else:
            for _ in range(steps // every):
                d = s.step_diagnostics(every)
        torch.cuda.synchronize()
        times[mode] = time.perf_counter() - t0
    s.close()
    return {"steps": steps, "every": every, "plain_ms_per_step": times["plain"] / steps * 1e3,
            "fused_ms_per_step": times["fused"] / steps * 1e3,
            "overhead": times["fused"] / times["plain"] - 1.0, "last_mass": d["mass"]}


def run_variant3(torch, n, prec, steps, warmup):
    """D3Q125 {0,+-1,+-3}^3 double shear layer on an n^3 periodic grid."""
    from paper_1402_5487_gb300 import plbm
    s = plbm.Solver(3, V5, OMEGA, n, n, nz=n, theta0=THETA0, prec=prec)
    rho, ux, uy, uz, th = I.kh3_fields(n, n, n)
    s.init(rho, ux, uy, th, uz=uz)
    t = time_device(s, steps, warmup, torch, lambda: None)
    st = s.check()
    s.close()
    nodes = n ** 3
    gbs = 2 * 125 * ELEM[prec] * nodes * steps / t / 1e9
    peak, _ = read_peaks()
    return {"grid": [n, n, n], "mlups": nodes * steps / t / 1e6, "ms_per_step": t / steps * 1e3,
            "gbs_algorithmic": gbs, "frac_of_measured_hbm": gbs / peak,
            "status": "ok" if st == 0 else "diverged"}


def run_batched(torch, steps=400, warmup=4, n=256, config=None):
    """Batched sweep of n admissible instances (FP32): persistent graph vs per-instance launches.
    config = (block_x, ctas_per_sm, order) fixes the persistent launch instead of autotuning."""
    from paper_1402_5487_gb300 import batch as B
    t0 = time.perf_counter()
    inst, stats = B.draw_instances(n)
    t_draw = time.perf_counter() - t0
    b = B.Batch(inst, prec="f32")
    b.init()
    if config:
        b.set_config(int(config[0]), int(config[1]))
        b.set_order(config[2])
        tuned = {"block_x": int(config[0]), "ctas_per_sm": int(config[1]), "order": config[2], "fixed": True}
    else:
        cache = os.path.join(ROOT, "paper_1402_5487_gb300", "_build", "autotune.json")
        tuned = b.autotune(steps_per_trial=6, cache_path=cache)
        b.init()
    nodes = b.nodes
    out = {"instances": n, "nodes": nodes, "draw_seconds": t_draw, "acceptance": stats["acceptance"],
           "autotune": tuned, "launch": b.info()}
    st = b.stream
    for mode in ("persistent_graph", "persistent", "per_instance", "per_instance_graph"):
        b.step(warmup, mode)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        b.step(steps, mode)
        e1.record(st)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        out[mode] = {"mlups": nodes * steps / t / 1e6, "ms_per_step": t / steps * 1e3,
                     "gbs_algorithmic": 200.0 * nodes * steps / t / 1e9}
    out["speedup_persistent_graph_vs_per_instance"] = (out["persistent_graph"]["mlups"] /
                                                      out["per_instance"]["mlups"])
    out["speedup_persistent_graph_vs_per_instance_graph"] = (out["persistent_graph"]["mlups"] /
                                                            out["per_instance_graph"]["mlups"])
    out["status"] = "ok" if b.check()[0] == 0 else "diverged"
    b.close()
    return out


def _field_err(mg, mr):
    rho = float(np.max(np.abs(mg[0] - mr[0])) / np.max(np.abs(mr[0])))
    u = float(np.max(np.hypot(mg[1] - mr[1], mg[2] - mr[2])) / np.max(np.hypot(mr[1], mr[2])))
    th = float(np.max(np.abs(mg[3] - mr[3])) / np.max(np.abs(mr[3])))
    return {"rho": rho, "u": u, "theta": th}


def run_surrogate(torch, n_train=2000, n_test=100, train_steps=2000, batch=16, K=32, L=256, mean_penalty=0.0,
                  noise=SURROGATE_NOISE):
    """Learned surrogate: data from the batched solver, training (loss: MSE plus
    mean_penalty x the squared lattice-mean error; inputs perturbed by `noise` x
    N(0, 1) in normalised units), held-out errors, speed."""
    import oracle as O
    from paper_1402_5487_gb300 import plbm, surrogate as SG
    from paper_1402_5487_gb300.batch import Batch
    out = {"grid": [L, L], "K": K, "train_trajectories": n_train, "test_trajectories": n_test}
    t0 = time.perf_counter()
    stack = SG.generate(range(n_train), L=L, K=K, snaps=17)
    out["generate_seconds"] = time.perf_counter() - t0
    pairs = SG.pairs_of(n_train, 17)
    norm = SG.fit_norm(stack, pairs)
    net = SG.Surrogate(64, L, L, seed=0)
    net.set_norm(*norm)
    net.set_mean_penalty(mean_penalty)
    out["mean_penalty"] = mean_penalty
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(stack, pairs, train_steps, batch=batch, lr=1e-3, lr_end=1e-4, log_every=train_steps // 4,
                       noise=noise)
    out["input_noise"] = noise
    t_train = time.perf_counter() - t0
    flops_sample = 3 * 2.0 * L * L * (9 * 4 * 64 + 4 * 9 * 64 * 64 + 9 * 64 * 4)
    out["training"] = {"steps": train_steps, "batch": batch, "seconds": t_train,
                       "samples_per_s": train_steps * batch / t_train,
                       "tflops": train_steps * batch * flops_sample / t_train / 1e12,
                       "loss": losses}
    del stack
    torch.cuda.empty_cache()
    snaps = 17
    test_seeds = list(range(10000, 10000 + n_test))
    tstack = SG.generate(test_seeds, L=L, K=K, snaps=snaps)
    mse_net, mse_p = net.evaluate(tstack, SG.pairs_of(n_test, snaps))
    out["test_mse_normalised"] = {"network": mse_net, "persistence": mse_p}
    # rollouts: the LBM trajectory (FP32, parity-checked against the FP64 oracle) is the reference
    nroll = min(n_test, 64)

    def rollout(tol, checkpoints=(1, 4, 16)):
        solvers = [plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32") for _ in range(nroll)]
        for s, seed in zip(solvers, test_seeds):
            s.init(*SG.trajectory_fields(seed, L))
            s.step(64)
        errs, drifts = {}, []
        fell = calls = 0
        t_roll = 0.0
        for k in range(1, 17):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            flags = net.advance(solvers, K=K, tol=tol)
            torch.cuda.synchronize()
            t_roll += time.perf_counter() - t0
            drifts.append(net.last_drift())
            fell += sum(flags)
            calls += len(flags)
            if k in checkpoints:
                e_net, e_pers = [], []
                for j, s in enumerate(solvers):
                    ref = tstack[j * snaps + k].cpu().numpy().astype(np.float64)
                    ref = [ref[:, c].reshape(L, L) for c in range(4)]
                    ini = tstack[j * snaps].cpu().numpy().astype(np.float64)
                    ini = [ini[:, c].reshape(L, L) for c in range(4)]
                    e_net.append(_field_err(s.moments(), ref))
                    e_pers.append(_field_err(ini, ref))
                fin = [e for e in e_net if all(np.isfinite(e[f]) for f in ("rho", "u", "theta"))]
                errs[str(k)] = {"surrogate_vs_lbm": {f: (float(np.mean([e[f] for e in fin])) if fin else None)
                                                     for f in ("rho", "u", "theta")},
                                "persistence_vs_lbm": {f: float(np.mean([e[f] for e in e_pers])) for f in ("rho", "u", "theta")},
                                "non_finite_lattices": len(e_net) - len(fin)}
        for s in solvers:
            s.close()
        return t_roll, fell / calls, np.concatenate(drifts), errs

    t_roll, rate, d, errs = rollout(1e-4)
    out["rollout_errors_mean_over_%d_seeds" % nroll] = errs
    out["fallback_rate"] = rate
    out["drift"] = {"tol": 1e-4, "median": float(np.median(d)), "p10": float(np.percentile(d, 10)),
                    "p90": float(np.percentile(d, 90)), "fraction_within_tol": float(np.mean(d <= 1e-4))}
    sweep = {"1e-4": (t_roll, rate, errs["16"]["surrogate_vs_lbm"]["u"], errs["16"]["non_finite_lattices"],
                      errs["4"]["surrogate_vs_lbm"]["u"])}
    for tol in (3e-4, 1e-3, float("inf")):
        t_r, r_r, _, e_r = rollout(tol, checkpoints=(4, 16))
        sweep["%g" % tol if tol < 1 else "no gate"] = (t_r, r_r, e_r["16"]["surrogate_vs_lbm"]["u"],
                                                       e_r["16"]["non_finite_lattices"],
                                                       e_r["4"]["surrogate_vs_lbm"]["u"])
    # the same gate after projecting each prediction onto the old global sums
    net.set_conserve(True)
    t_r, r_r, _, e_r = rollout(1e-4, checkpoints=(4, 16))
    net.set_conserve(False)
    sweep["1e-4, conservative projection"] = (t_r, r_r, e_r["16"]["surrogate_vs_lbm"]["u"],
                                              e_r["16"]["non_finite_lattices"], e_r["4"]["surrogate_vs_lbm"]["u"])
    # gain test: the same lattices and horizon (16 x K steps) with plain batched LBM
    insts = [SG.trajectory_instance(sd, L)[0] for sd in test_seeds[:nroll]]
    bt = Batch(insts, prec="f32")
    for sol, sd in zip(bt.solvers, test_seeds[:nroll]):
        sol.init(*SG.trajectory_fields(sd, L))
    bt.step(64, "persistent_graph")
    bt.stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(bt.stream)
    bt.step(16 * K, "persistent_graph")
    e1.record(bt.stream)
    e1.synchronize()
    t_lbm_roll = e0.elapsed_time(e1) * 1e-3
    bt.close()
    out["gain_test"] = {"lattices": nroll, "horizon_steps": 16 * K, "lbm_s": t_lbm_roll,
                        "by_tol": {k: {"surrogate_with_fallback_s": v[0], "speedup": t_lbm_roll / v[0],
                                       "fallback_rate": v[1], "u_error_at_horizon_vs_lbm": v[2],
                                       "non_finite_lattices_at_horizon": v[3],
                                       "u_error_after_4_advances_vs_lbm": v[4]}
                                   for k, v in sweep.items()}}
    # FP64 oracle check on two held-out seeds after one advance
    orc = []
    for seed in test_seeds[:2]:
        lat = O.Lattice(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0)
        mo = lat.moments(lat.run(lat.init(*SG.trajectory_fields(seed, L)), 64 + K))
        s = plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32")
        s.init(*SG.trajectory_fields(seed, L))
        s.step(64)
        net.advance([s], K=K, tol=1.0)
        e_sur = _field_err(s.moments(), mo)
        s.init(*SG.trajectory_fields(seed, L))
        s.step(64 + K)
        e_lbm = _field_err(s.moments(), mo)
        s.close()
        orc.append({"seed": seed, "surrogate_vs_fp64_oracle": e_sur, "lbm_f32_vs_fp64_oracle": e_lbm})
    out["one_advance_vs_fp64_oracle"] = orc
    # speed: one surrogate advance of B lattices vs K LBM steps of the same lattices
    speed = {}
    for B in (1, 16, 64):
        sols = [plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32") for _ in range(B)]
        for s, seed in zip(sols, test_seeds):
            s.init(*SG.trajectory_fields(seed, L))
        net.advance(sols, K=K, tol=1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.advance(sols, K=K, tol=1.0)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t0
        for s in sols:
            s.close()
        insts = [SG.trajectory_instance(sd, L)[0] for sd in test_seeds[:B]]
        bt = Batch(insts, prec="f32")
        bt.init()
        bt.step(2, "persistent_graph")
        bt.stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(bt.stream)
        bt.step(K, "persistent_graph")
        e1.record(bt.stream)
        e1.synchronize()
        t_lbm = e0.elapsed_time(e1) * 1e-3
        bt.close()
        speed[str(B)] = {"surrogate_advance_ms": t_sur * 1e3, "lbm_K_steps_ms": t_lbm * 1e3,
                         "speedup_vs_lbm": t_lbm / t_sur}
    out["speed_one_advance"] = speed
    net.close()
    del tstack
    torch.cuda.empty_cache()
    return out


def _long_errors(mg, mr):
    """Per-field errors of a run against stored FP64 oracle fields: relative
    maximum (velocity as a vector), relative L2 and absolute maximum."""
    out = _field_err(mg, mr)
    du = np.hypot(mg[1] - mr[1], mg[2] - mr[2])
    out["rho_l2"] = float(np.sqrt(np.mean((mg[0] - mr[0]) ** 2) / np.mean(mr[0] ** 2)))
    out["u_l2"] = float(np.sqrt(np.mean(du ** 2) / np.mean(mr[1] ** 2 + mr[2] ** 2)))
    out["theta_l2"] = float(np.sqrt(np.mean((mg[3] - mr[3]) ** 2) / np.mean(mr[3] ** 2)))
    out["rho_abs"] = float(np.max(np.abs(mg[0] - mr[0])))
    out["u_abs"] = float(np.max(du))
    out["theta_abs"] = float(np.max(np.abs(mg[3] - mr[3])))
    return out


def run_longrun(torch, paths, precs=("f64", "f32", "f16dev", "bf16dev")):
    """Errors of each storage precision against FP64 oracle snapshots of the double
    shear layer (files written by the oracle's long-run script), with the
    plausibility bounds of the flow (rho, theta within 1 +- 0.01, |u| <= 0.12)."""
    from paper_1402_5487_gb300 import plbm
    res = []
    for path in paths:
        d = np.load(path)
        L, stride = int(d["size"]), int(d["stride"])
        omega, theta0, seed = float(d["omega"]), float(d["theta0"]), int(d["seed"])
        steps = [int(n) for n in d["steps"]]
        fields = I.kh_fields(L, theta0=theta0, seed=seed)
        entry = {"grid": [L, L], "omega": omega, "theta0": theta0, "seed": seed,
                 "sampled": "every %d-th node in x and y" % stride if stride > 1 else "all nodes",
                 "precisions": {}}
        for prec in precs:
            s = plbm.Solver(2, V5, omega, L, L, theta0=theta0, prec=prec)
            s.init(*fields)
            done, per = 0, {}
            t0 = time.perf_counter()
            for n in steps:
                s.step(n - done)
                done = n
                st = s.check()
                if st != 0:
                    per[str(n)] = {"status": "diverged"}
                    break
                mg = [a[::stride, ::stride] for a in s.moments()]
                mr = [d["%s_%d" % (k, n)] for k in ("rho", "ux", "uy", "theta")]
                e = _long_errors(mg, mr)
                e["plausible"] = bool(np.all(np.abs(mg[0] - 1) <= 0.01) and np.all(np.abs(mg[3] - 1) <= 0.01)
                                      and np.max(np.hypot(mg[1], mg[2])) <= 0.12)
                e["status"] = "ok"
                per[str(n)] = e
            per["seconds"] = time.perf_counter() - t0
            s.close()
            entry["precisions"][prec] = per
        res.append(entry)
    return res


def run_case(torch, args):
    """One secondary workload alone: the surrogate network on a batch of 256 x 256
    lattices (forward passes and Adam steps on seeded random tensors), the
    batched 256-instance sweep, or the D3Q125 shear layer on a size^3 grid."""
    if args.case == "batched":
        cfg = args.batch_config.split(",") if args.batch_config else None
        return {"case": "batched", **run_batched(torch, steps=args.steps, warmup=args.warmup, config=cfg,
                                                 n=args.batch_instances)}
    if args.case == "longrun":
        return {"case": "longrun", "runs": run_longrun(torch, args.snapshots)}
    if args.case == "surrogate_gain":
        return {"case": "surrogate_gain", **run_surrogate(torch, n_train=args.surrogate_train,
                                                          train_steps=args.surrogate_steps,
                                                          noise=args.surrogate_noise)}
    if args.case == "d3q125":
        return {"case": "d3q125", "prec": args.prec,
                **run_variant3(torch, args.size, args.prec, args.steps, args.warmup)}
    import ctypes
    from paper_1402_5487_gb300 import plbm, surrogate as SG
    B, L = args.batch, 256
    net = SG.Surrogate(B, L, L, seed=0)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((B, L, L, 4), generator=g, device="cuda").to(torch.bfloat16)
    y = torch.randn((B, L, L, 4), generator=g, device="cuda")
    out = {"case": "surrogate", "batch": B, "grid": [L, L]}
    fwd_flops = 2.0 * L * L * (9 * 4 * 64 + 4 * 9 * 64 * 64 + 9 * 64 * 4)
    for name, call, flops in (
            ("forward", lambda: plbm.lib().plbm_sur_forward(net.h, B, x.data_ptr(), None), fwd_flops),
            ("train_step", lambda: plbm.lib().plbm_sur_train_step(net.h, B, x.data_ptr(), y.data_ptr(),
                                                                  ctypes.c_float(1e-4), None), 3 * fwd_flops)):
        for _ in range(args.warmup):
            call()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(net.stream)
        for _ in range(args.steps):
            call()
        e1.record(net.stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3 / args.steps
        out[name] = {"ms": t * 1e3, "tflops": B * flops / t / 1e12}
    out["status"] = "ok" if net.check() == 0 else "timeout"
    net.close()
    return out


def variant_summary(variants, peak):
    """The variants' headline figures in a few hundred characters, last on the line (a reader
    that keeps only the end of a long line still sees them): MLUPS, fraction of the measured
    copy bandwidth for the HBM-bound ones, the surrogate's speedups and errors."""
    out = {}

    def put(key, name, field="mlups", nd=0):
        v = variants.get(name) or {}
        if field in v and v[field] is not None:
            out[key] = round(v[field], nd) if nd else int(round(v[field]))

    put("f16dev_mlups", "kh2048_f16dev")
    put("bf16dev_mlups", "kh2048_bf16dev")
    put("f16dev_vs_f32", "kh2048_f16dev", "speedup_vs_f32", 2)
    put("f64_mlups", "kh2048_f64")
    put("odd2047_f32_mlups", "kh2047_f32_plain_layout")
    put("slabs4_f32_mlups", "kh2048_f32_4slabs")
    put("diag_every10_overhead", "kh2048_f32_diagnostics_every_10", "overhead", 3)
    for prec in ("f32", "f16dev", "bf16dev"):
        put("d3q125_256_%s_frac" % prec, "kh3d256_d3q125_%s" % prec, "frac_of_measured_hbm", 3)
    b = next((v for k, v in variants.items() if k.startswith("batched_")), None) or {}
    if "persistent_graph" in b:
        out["batched_mlups"] = int(round(b["persistent_graph"]["mlups"]))
        out["batched_frac"] = round(b["persistent_graph"]["gbs_algorithmic"] / peak, 3)
        out["batched_vs_per_instance"] = round(b.get("speedup_persistent_graph_vs_per_instance", 0.0), 2)
    s = variants.get("surrogate_kh256") or {}
    if "gain_test" in s:
        g = {}
        for tol, r in s["gain_test"]["by_tol"].items():
            g[tol] = [round(r["speedup"], 2), round(r["fallback_rate"], 2),
                      round(r["u_error_after_4_advances_vs_lbm"], 3)]
        out["surrogate_gain_speedup_fallback_uerr4"] = g
        out["surrogate_advance_speedup_b64"] = round(s["speed_one_advance"]["64"]["speedup_vs_lbm"], 2)
        out["surrogate_train_tflops"] = round(s["training"]["tflops"], 1)
        out["surrogate_heldout_mse"] = round(s["test_mse_normalised"]["network"], 3)
    return out


def cpu_oracle_sample(L, seconds=12.0, max_steps=50):
    """Time the FP64 oracle as it stands on this host's cores on an L x L KH grid."""
    import oracle as O
    lat = O.Lattice(2, V5, OMEGA, L, L, theta0=THETA0)
    f = lat.init(*I.kh_fields(L))
    cores = O.max_threads()
    f = lat.step(f)  # one untimed step (page-in)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps and time.perf_counter() - t0 < seconds:
        f = lat.step(f)
        n += 1
    dt = time.perf_counter() - t0
    out = {"value": L * L * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": "%dx%d D2Q25 KH, %d FP64 steps of the C oracle (OpenMP over rows)" % (L, L, n)}
    out["per_config"] = oracle_configs(O, cores)
    return out


def oracle_configs(O, cores, seconds=2.0):
    """The oracle on one host thread and on all of them, for the 1000-node D1Q5 shock
    tube, the 512 x 512 and the 2048 x 2048 D2Q25 shear layers (short samples)."""
    left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
    cases = {
        "shock1000_d1q5": (lambda: O.Lattice(1, V5, 1.5, 1000, 1, bc="fixed", theta0=0.5, left_state=left,
                                             right_state=right), lambda: I.shock_tube_fields(1000, left, right),
                           1000),
        "kh512_d2q25": (lambda: O.Lattice(2, V5, OMEGA, 512, 512, theta0=THETA0), lambda: I.kh_fields(512),
                        512 * 512),
        "kh2048_d2q25": (lambda: O.Lattice(2, V5, OMEGA, 2048, 2048, theta0=THETA0), lambda: I.kh_fields(2048),
                         2048 * 2048),
    }
    res = {}
    try:
        for name, (mk, fields, nodes) in cases.items():
            lat = mk()
            rho, ux, uy, th = fields()
            f = lat.init(rho, ux, uy if lat.dim == 2 else None, th)
            row = {}
            for threads in (1, cores):
                O.set_threads(threads)
                f = lat.step(f)
                n, t0 = 0, time.perf_counter()
                while n < 1000 and (n < 1 or time.perf_counter() - t0 < seconds):
                    f = lat.step(f)
                    n += 1
                row["threads_%d" % threads] = nodes * n / (time.perf_counter() - t0) / 1e6
            res[name] = row
    finally:
        O.set_threads(cores)
    return res


def end_to_end(torch, plbm, fields, L, args, local, barrier, dist, ws):
    """Public-API job with pinned host buffers: init from host, K steps, moments to host."""
    pinned = [torch.from_numpy(a).pin_memory() for a in fields]
    host_fields = [p.numpy() for p in pinned]
    outs = [torch.empty((L, L), dtype=torch.float64).pin_memory() for _ in range(4)]
    host_outs = [o.numpy() for o in outs]
    e2e_steps = args.steps
    solver2 = plbm.Solver(2, V5, OMEGA, L, L, theta0=THETA0, prec=args.prec, device=local)
    solver2.init(*host_fields)
    solver2.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    solver2.init(*host_fields)
    solver2.step(e2e_steps)
    from paper_1402_5487_gb300.plbm import lib as _lib
    ptrs = [o.ctypes.data for o in host_outs]
    stt = _lib().plbm_moments(solver2.h, *ptrs, 0)
    assert stt == 0
    t_e2e = time.perf_counter() - t0
    barrier()
    solver2.close()
    t_e2e, e2e_value = replica_throughput(torch, t_e2e, L * L * e2e_steps, dist)
    h2d = 4 * L * L * 8
    d2h = 4 * L * L * 8
    e2e = {"value": e2e_value, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
           "job": "plbm_init from pinned host fields + %d steps + plbm_moments to pinned host" % e2e_steps}

    return e2e


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--prec", default="f32", choices=list(ELEM))
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-config", default=None,
                    help="block_x,ctas_per_sm,order (contiguous|interleaved): fixed persistent launch "
                         "instead of the autotuner (--case batched)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-train", type=int, default=2000, help="training trajectories")
    ap.add_argument("--surrogate-steps", type=int, default=6000, help="Adam steps")
    ap.add_argument("--surrogate-noise", type=float, default=SURROGATE_NOISE,
                    help="input noise of the surrogate's training (normalised units)")
    ap.add_argument("--case", default="main", choices=["main", "surrogate", "surrogate_gain", "batched", "d3q125",
                                                       "longrun"],
                    help="main: the bench line; any other: one secondary workload alone (a JSON "
                         "line of its own); longrun: errors against FP64 oracle snapshots")
    ap.add_argument("--batch", type=int, default=16, help="lattices per surrogate call (--case surrogate)")
    ap.add_argument("--snapshots", nargs="+", default=[],
                    help="FP64 oracle snapshot files (.npz) for --case longrun")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    L = args.size
    q = 25
    metric = "D2Q25 MLUPS"
    config = {"workload": "kh%d_d2q25_%s" % (L, args.prec),
              "description": "Kelvin-Helmholtz double shear layer, D2Q25 {0,+-1,+-3}^2, %dx%d periodic, "
                             "theta0=1, omega=1.3, %s populations" % (L, L, args.prec),
              "grid": [L, L], "velocities": list(V5), "omega": OMEGA, "theta0": THETA0,
              "l2": "inputs larger than L2 (2 population arrays of %.0f MB each)" % (
                  q * ELEM[args.prec] * L * L / 1e6),
              "parallelism": "replicas" if ws > 1 else "single-gpu"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle as O
        lat = O.Lattice(2, V5, OMEGA, L, L, theta0=THETA0)
        f = lat.init(*I.kh_fields(L))
        f = lat.run(f, args.warmup)
        t0 = time.perf_counter()
        f = lat.run(f, args.steps)
        dt = time.perf_counter() - t0
        val = L * L * args.steps / dt / 1e6
        cores = O.max_threads()
        line = {"impl": "reference", "metric": metric, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                 "sample": "%dx%d D2Q25 KH, %d timed FP64 steps of the C oracle" % (
                                     L, L, args.steps)},
                "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(json_safe(line)))
        return 0

    import torch
    from paper_1402_5487_gb300 import build, plbm
    dist = None
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = td
    torch.cuda.set_device(local)
    build.build()
    if args.case != "main":
        if rank == 0:
            print(json.dumps(json_safe(run_case(torch, args))))
        return 0

    def barrier():
        if dist is not None:
            dist.barrier()

    fields = I.kh_fields(L)
    solver = plbm.Solver(2, V5, OMEGA, L, L, theta0=THETA0, prec=args.prec, device=local)
    solver.init(*fields)
    solver.step(args.warmup)
    st = solver.stream
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    time.sleep(0.3)
    # REPEATS timed runs of exactly --steps steps each, every one bracketed by
    # CUDA events on the solver's stream with a synchronisation and a barrier on
    # both sides; the run of median duration is the reported one.
    runs = []
    for _ in range(REPEATS):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(st)
        solver.step(args.steps)
        e1.record(st)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        runs.append(e0.elapsed_time(e1) * 1e-3)
    clock_info = clocks.stop()
    t = statistics.median(runs)
    healthy = solver.check() == 0
    solver.close()
    t_max, value = replica_throughput(torch, t, L * L * args.steps, dist)
    per_launch = t / args.steps
    alg_bytes = 2 * q * ELEM[args.prec] * L * L
    peak, peak_kind = read_peaks()
    achieved = alg_bytes / per_launch / 1e9

    # End to end through the public API with pinned host buffers.
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(torch, plbm, fields, L, args, local, barrier, dist, ws)

    variants = {}
    if not args.no_variants and rank == 0:
        for prec in ("f16dev", "bf16dev", "f64"):
            if prec == args.prec:
                continue
            variants["kh%d_%s" % (L, prec)] = run_variant(torch, L, prec, 200, 10, lambda: None)
        variants["kh2048_f32_diagnostics_every_10"] = run_diag_overhead(torch, 2048, 400, 10)
        # odd side: the plain layout, one node per thread (no row pairs)
        variants["kh%d_f32_plain_layout" % (L - 1)] = run_variant(torch, L - 1, "f32", 200, 10, lambda: None)
        variants["kh%d_f32_4slabs" % L] = run_slabs(torch, L, 4, 200, 10)
        variants["kh512_f32"] = run_variant(torch, 512, "f32", 1000, 50, lambda: None)
        variants["kh512_f64"] = run_variant(torch, 512, "f64", 200, 20, lambda: None)
        pf, pth = I.paper_kh_fields()
        # the paper's own shear layer to its last printed step: FP64, as FP32 storage rounding
        # seeds a mode that grows at omega = 1.9 and diverges near step 3000
        variants["paper_kh128_d2q25_f64"] = run_variant(torch, 128, "f64", 3695, 10, lambda: None, v=I.SET_012,
                                                        fields=pf, theta0=pth, omega=1.9)
        for prec in ("f32", "f16dev", "bf16dev"):
            variants["kh3d256_d3q125_%s" % prec] = run_variant3(torch, 256, prec, 40, 4)
        variants["kh3d64_d3q125_f64"] = run_variant3(torch, 64, "f64", 20, 3)
        left, right = (1.1, 0.0, 0.5), (1.0, 0.0, 0.5)
        variants["shock1000_d1q5_f64"] = run_variant(
            torch, 1000, "f64", 500, 20, lambda: None, dim=1, bc="fixed",
            fields=I.shock_tube_fields(1000, left, right), theta0=0.5, omega=1.5, left=left, right=right)
        if not args.no_batch:
            variants["batched_%d_f32" % args.batch_instances] = run_batched(torch, n=args.batch_instances)
        if not args.no_surrogate:
            variants["surrogate_kh256"] = run_surrogate(torch, n_train=args.surrogate_train,
                                                        train_steps=args.surrogate_steps, noise=args.surrogate_noise)
        base = value / ws
        for k, vv in variants.items():
            if k.startswith("kh%d_" % L) and "mlups" in vv:
                vv["speedup_vs_f32"] = vv["mlups"] / base

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        cpu = cpu_oracle_sample(L)

    if rank == 0:
        line = {"metric": metric, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
                "config": config, "healthy": healthy,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": read_traffic(args.prec),
                             "peak_source": peak_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
                             "algorithmic_bytes_per_launch": alg_bytes,
                             "kernel": KERNEL_NAME[args.prec]},
                "repeats": {"n": REPEATS, "reported": "median",
                            "ms_per_step_each": [r / args.steps * 1e3 for r in runs],
                            "spread": (max(runs) - min(runs)) / t},
                "e2e": e2e, "gpu_launches": args.steps, "clocks": clock_info,
                "cpu_baseline": cpu, "variants": variants, "variant_summary": variant_summary(variants, peak)}
        print(json.dumps(json_safe(line)))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
