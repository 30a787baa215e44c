#!/usr/bin/env python
"""FEWHA benchmark: MAORY-size frames/s and p99 frame latency on GB300.

One step = one frame of Algorithm 1 (right-hand side, explicit initial residual, 4 PCG
iterations, DM fit and gain) of the MAORY-size instance (39 m, 6 LGS 80x80 + 3 NGS
2x2, 9 layers, 3 DMs), warm-started from the previous frame, slopes resident on the
device.  Timed per frame with CUDA events; a 512 MiB memset flushes L2 between frames
(outside the events).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (single thread) on the same workload.
With N > 1 (torchrun) every rank runs an independent replica (the path does not
shard); rank 0 prints the aggregate.
"""

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")     # the CPU baseline runs single-threaded

import argparse
import hashlib
import json
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "FEWHA frames/s and p99 frame latency, MAORY-size, FP32 form vs FP64 plain, 1 GB300"
UNIT = "frames/s"
N_FRAMES_INPUT = 8          # distinct seeded frames, cycled through the timed loop
FLUSH_BYTES = 512 << 20     # > 129 MB L2
_CSRC = os.path.join(ROOT, "paper_2202_11945_gb300", "csrc")
# source file of each stage's kernel (the traffic record is tied to its hash)
STAGE_SRC = {"idwt": "fewha_cluster.cuh", "sensor": "fewha_cluster.cuh", "layer": "fewha_cluster.cuh",
             "rhs": "fewha_cluster.cuh", "proj": "fewha_pair.cuh", "projT": "fewha_pair.cuh",
             "vector": "fewha_kernels.cuh", "fit": "fewha_kernels.cuh"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_maory_fp32.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-frames", type=int, default=20, help="oracle frames of the CPU baseline")
    ap.add_argument("--batch-count", type=int, default=64, help="instances of the batched workload")
    ap.add_argument("--batch-steps", type=int, default=50, help="timed batched frames")
    ap.add_argument("--backward-frames", type=int, default=8,
                    help="frames of the differentiable-reconstruction leg (0: leave it out)")
    ap.add_argument("--aug-steps", type=int, default=500,
                    help="timed frames per configuration of the augmented-PCG, closed-loop and "
                         "paper-geometry runs")
    ap.add_argument("--loop-frames", type=int, default=2000,
                    help="frames of the 1 kHz real-time loop (8 m single-conjugate geometry)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(wl):
    atm = synth.TruthAtmosphere(wl["truth"])
    return [synth.simulate_slopes(wl, t, atm=atm) for t in range(N_FRAMES_INPUT)]


def max_over_ranks(values, world, device):
    """Element-wise maximum over the ranks of per-rank timed totals: the slowest replica
    sets the job's time (every rank gets the result)."""
    if world == 1:
        return [float(v) for v in values]
    import torch.distributed as dist
    v = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return [float(x) for x in v.tolist()]


def replica_throughput(world, steps, total_ms):
    """Frames per second of the whole job: every rank runs `steps` frames of its own
    replica in at most `total_ms` (the path does not shard; no data-path collective)."""
    return world * steps / (total_ms * 1e-3)


def time_frames(R, S, steps, warmup, flush, dm):
    """Per-frame device times (ms) of `steps` warm-started frames, L2 flushed between."""
    n = S.shape[0]
    for k in range(warmup):
        R.reconstruct(S[k % n], dm_out=dm)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    # a lead of device work (L2 flushes, ~0.6 ms) so that the host's submissions run ahead
    # of the timed frames: a host stall between a frame's start event and its launch would
    # otherwise be timed as part of that frame
    for _ in range(8):
        flush.zero_()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        R.reconstruct(S[k % n], dm_out=dm)
        ev[k][1].record()
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def stage_bytes(R, b):
    """Algorithmic (compulsory) bytes per launch of each hot-path stage."""
    nc, nn, ns, na = R.n_coeffs, R.n_nodes, R.n_slopes, R.n_act
    return {
        "idwt": 4 * nc * b,               # read z, p; write p, phi
        "proj": (nc + nn) * b,            # read phi; write P phi on the aperture nodes
        "sensor": 2 * nn * b,             # read P phi; write the aperture-node adjoint u
        "projT": (nn + nc) * b,           # read u; write P^T u on the layers
        "layer": 3 * nc * b,              # read P^T u and p; write q (D: one value per level)
        "vector": 11 * nc * b,            # read c, p, r, q, J^-1, phi_c, phi_p; write c, r, z, phi_c
        "rhs": (ns + nn) * b,             # read slopes; write u
        "fit": (nc + 3 * na) * b,         # read phi, a_prev; write a_prev, dm
    }


def stage_launches(iters):
    """Launches of each stage's kernel in one explicit-residual frame: the initial residual's
    chain (inverse transform, P, the sensor kernel on the slopes' residual, P^T, the forward
    kernel with the vector step) and one apply plus one CG update per iteration; the fit
    reads the carried layers (no inverse transform) and no right-hand side is formed."""
    return {"idwt": iters + 1, "proj": iters + 1, "sensor": iters + 1, "projT": iters + 1,
            "layer": iters + 1, "vector": iters, "rhs": 0, "fit": 1}


def time_stages(R, flush, reps=100):
    """Per-launch device time of each stage's kernel: `reps` back-to-back launches
    captured in a CUDA graph (so the host launch rate does not pace them), after a flush."""
    out = {}
    cap = torch.cuda.Stream()
    for st in ("idwt", "proj", "sensor", "projT", "layer", "vector", "rhs", "fit"):
        R.bench_stage(st, 3)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            R.bench_stage(st, reps)
        g.replay()
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        out[st] = a.elapsed_time(b) / reps
    return out


def recorded_traffic():
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary.

    The summary records the SHA-256 of the kernel source it was taken with; a changed
    kernel makes the figure stale and it is dropped (null).
    """
    if not os.path.exists(TRAFFIC_FILE):
        return None, None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    stage = kv.get("stage")
    if stage not in STAGE_SRC:
        return None, stage
    sha = hashlib.sha256(open(os.path.join(_CSRC, STAGE_SRC[stage]), "rb").read()).hexdigest()
    if kv.get("kernel_source_sha256") != sha:
        return None, kv.get("stage")
    return float(kv["dram_bytes_per_launch"]), kv.get("stage")


def cpu_baseline(wl, frames, S_np, R_gpu_factory):
    """The FP64 oracle, single thread, on the first `frames` frames; plus parity."""
    import oracle as O
    t0 = time.perf_counter()
    ref = O.Reconstructor(wl)
    t_setup = time.perf_counter() - t0
    refs = []
    t0 = time.perf_counter()
    for k in range(frames):
        refs.append(ref.frame(S_np[k % len(S_np)]))
    t = time.perf_counter() - t0
    parity = {}
    for prec in (32, 64):
        R = R_gpu_factory(prec)
        dt = torch.float32 if prec == 32 else torch.float64
        worst = 0.0
        for k in range(frames):
            a = R.reconstruct(torch.as_tensor(S_np[k % len(S_np)], dtype=dt, device="cuda"))
            a = a.double().cpu().numpy()
            worst = max(worst, float(np.linalg.norm(a - refs[k]) / np.linalg.norm(refs[k])))
        parity["fp%d_max_rel_l2_dm" % prec] = worst
        R.close()
    return {"value": frames / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d warm-started MAORY frames (frame 0 cold), numpy FP64, 1 thread; "
                      "set-up (D, exact J) %.2f s not timed" % (frames, t_setup)}, parity


def time_loop(frames, warmup=100, period_us=1000.0):
    """The real-time loop: the 8 m single-conjugate geometry, frozen flow, frames released
    every `period_us` from pinned host slopes, commands back on the host per frame."""
    from paper_2202_11945_gb300 import Reconstructor
    wl = synth.realtime_loop()
    S = synth.slope_sequence(wl, frames)
    R = Reconstructor(wl, precision=32, graph=True)
    R.run_loop(S[:min(warmup, frames)], period_us=0.0)
    R.reset()
    dm, wall, dev, late = R.run_loop(S, period_us=period_us)
    Rw = Reconstructor(wl, precision=32, graph=True, warm_residual=True)
    dmw, _, _, _ = Rw.run_loop(S, period_us=0.0)
    Rr = Reconstructor(wl, precision=32, graph=True, warm_residual=True, warm_refresh=20)
    dmr, _, _, _ = Rr.run_loop(S, period_us=0.0)
    R.close()
    Rw.close()
    Rr.close()
    wall, dev = wall.numpy().astype(float), dev.numpy().astype(float)
    out = {"workload": wl["name"], "frames": frames, "period_us": period_us,
           "form": "FP32 operators, FP64 dots, CUDA graph; host slopes in, host commands out",
           "latency_us": {"p50": float(np.percentile(wall, 50)), "p99": float(np.percentile(wall, 99)),
                          "max": float(wall.max())},
           "device_us": {"p50": float(np.percentile(dev, 50)), "p99": float(np.percentile(dev, 99))},
           "late_frames": late}
    return out, wl, S, dm.double().numpy(), (dmw.double().numpy(), dmr.double().numpy())


def frame_bytes(R, b=4):
    """Algorithmic bytes of one frame of an instance (stage bytes x launches per frame)."""
    nb = stage_bytes(R, b)
    la = stage_launches(R.iters)
    return sum(nb[k] * la[k] for k in nb)


def time_batched(count, steps, warmup, flush):
    """Uneven instances: one-by-one frames (each instance's own graph, one after another)
    against the batched frame (one launch per step over all instances), autotuned."""
    from paper_2202_11945_gb300 import Batch, Reconstructor
    wls = synth.batched_instances(count)
    S = []
    for wl in wls:
        atm = synth.TruthAtmosphere(wl["truth"])
        S.append([torch.as_tensor(synth.simulate_slopes(wl, t, atm=atm), dtype=torch.float32,
                                  device="cuda") for t in range(2)])
    solo = [Reconstructor(wl, precision=32, graph=True) for wl in wls]
    mem = [Reconstructor(wl, precision=32, graph=True) for wl in wls]
    B = Batch(mem)
    cfg, tuned_us = B.autotune([s[0] for s in S], reps=5)
    for R in mem:
        R.reset()
    torch.cuda.synchronize()

    def run(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record()
            fn(k)
            ev[k][1].record()
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ev])

    dm_solo = [torch.empty(R.n_act, dtype=torch.float32, device="cuda") for R in solo]
    dm_b = [torch.empty(R.n_act, dtype=torch.float32, device="cuda") for R in mem]

    def one_by_one(k):
        for i, R in enumerate(solo):
            R.reconstruct(S[i][k % 2], dm_out=dm_solo[i])

    def batched(k):
        B.reconstruct([s[k % 2] for s in S], dm_out=dm_b)

    run(one_by_one, warmup)
    run(batched, warmup)
    t1 = run(one_by_one, steps)
    tb = run(batched, steps)
    # same frame count on both sides and the same inputs: compare the last commands
    diff = max(float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))
               for a, b in zip(dm_b, dm_solo))
    nbytes = sum(frame_bytes(R) for R in mem)
    # every instance against the FP64 oracle: two fresh frames (cold, then warm-started)
    import oracle as O
    for R in mem:
        R.reset()
    torch.cuda.synchronize()
    vs_oracle = 0.0
    got = []
    for t in range(2):
        B.reconstruct([s[t] for s in S], dm_out=dm_b)
        got.append([d.double().cpu().numpy() for d in dm_b])
    for i, wl in enumerate(wls):
        ref = O.Reconstructor(wl)
        for t in range(2):
            a_ref = ref.frame(S[i][t].double().cpu().numpy())
            vs_oracle = max(vs_oracle, float(np.linalg.norm(got[t][i] - a_ref) / np.linalg.norm(a_ref)))
    out = {"workload": "batched_%d_uneven_instances" % count, "instances": count,
           "frames_per_s": count / (tb.mean() * 1e-3),
           "one_by_one_frames_per_s": count / (t1.mean() * 1e-3),
           "speedup": float(t1.mean() / tb.mean()),
           "ms_per_batch": float(tb.mean()), "p99_ms_per_batch": float(np.percentile(tb, 99)),
           "ms_one_by_one": float(t1.mean()),
           "config": cfg, "autotune_us": tuned_us,
           "max_rel_l2_vs_one_by_one": diff,
           "max_rel_l2_vs_oracle": vs_oracle,
           "oracle_check": "every instance, 2 frames from a reset (cold, then warm-started)",
           "algorithmic_gb_s": nbytes / (tb.mean() * 1e-3) / 1e9,
           "l2": "512 MiB memset between timed batches", "steps": steps}
    B.close()
    for R in solo + mem:
        R.close()
    return out


def time_batched_maory(count, steps, flush):
    """Throughput of independent MAORY-size frames: `count` instances of the MAORY workload
    (each its own frame stream of seeded slopes) reconstructed in one batched frame, autotuned;
    the aggregate frames/s and the algorithmic GB/s of the frame's kernels."""
    from paper_2202_11945_gb300 import Batch, Reconstructor
    wl = synth.maory()
    atm = synth.TruthAtmosphere(wl["truth"])
    S = [torch.as_tensor(synth.simulate_slopes(wl, t, atm=atm), dtype=torch.float32, device="cuda")
         for t in range(4)]
    mem = [Reconstructor(wl, precision=32, graph=True) for _ in range(count)]
    B = Batch(mem)
    cfg, tuned_us = B.autotune([S[i % 4] for i in range(count)], reps=3)
    dm = [torch.empty(R.n_act, dtype=torch.float32, device="cuda") for R in mem]
    for k in range(3):
        B.reconstruct([S[(i + k) % 4] for i in range(count)], dm_out=dm)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        B.reconstruct([S[(i + k) % 4] for i in range(count)], dm_out=dm)
        ev[k][1].record()
    torch.cuda.synchronize()
    t = np.array([a.elapsed_time(b) for a, b in ev])
    nbytes = count * frame_bytes(mem[0])
    # one cold frame per instance from a reset, against the FP64 oracle on its four inputs
    import oracle as O
    for R in mem:
        R.reset()
    B.reconstruct([S[i % 4] for i in range(count)], dm_out=dm)
    ref = [O.Reconstructor(wl).frame(S[k].double().cpu().numpy()) for k in range(4)]
    vs_oracle = max(float(np.linalg.norm(dm[i].double().cpu().numpy() - ref[i % 4]) / np.linalg.norm(ref[i % 4]))
                    for i in range(count))
    out = {"workload": "%d x %s" % (count, wl["name"]), "instances": count,
           "frames_per_s": count / (t.mean() * 1e-3), "ms_per_batch": float(t.mean()),
           "p99_ms_per_batch": float(np.percentile(t, 99)), "config": cfg, "autotune_us": tuned_us,
           "algorithmic_gb_s": nbytes / (t.mean() * 1e-3) / 1e9, "steps": steps,
           "max_rel_l2_vs_oracle": vs_oracle, "oracle_check": "every instance, 1 cold frame",
           "l2": "512 MiB memset between timed batches"}
    B.close()
    for R in mem:
        R.close()
    return out


def time_backward(frames=8):
    """The differentiable 8 m workload: converged reconstruction and backward (adjoint PCG
    and adjoint operator kernels) of J = ||Pi (a~ - true on-axis phase)||^2 (Pi removes the
    piston) per frame, FP32 and FP64, solves warm-started from the previous frame; wall
    time of each synchronous call, and the FP32 gradients against the FP64 ones."""
    from paper_2202_11945_gb300 import Reconstructor
    wl = synth.differentiable()
    atm = synth.TruthAtmosphere(wl["truth"])
    na = sum(m["n_act"] ** 2 for m in wl["dms"])
    xs, ys = [], []
    for m in wl["dms"]:
        k = (np.arange(m["n_act"]) - (m["n_act"] - 1) / 2.0) * m["spacing"]
        X, Y = np.meshgrid(k, k)
        xs.append(X.ravel())
        ys.append(Y.ravel())
    xa, ya = np.concatenate(xs), np.concatenate(ys)
    assert len(xa) == na
    out = {"workload": wl["name"], "frames": frames,
           "objective": "||a~ - true on-axis phase||^2 over the actuators, piston removed"}
    grads = {}
    for prec, dt in ((32, torch.float32), (64, torch.float64)):
        R = Reconstructor(wl, precision=prec, graph=False)
        tf, tb, its, gl = [], [], [], []
        for t in range(frames + 1):
            s = torch.as_tensor(synth.simulate_slopes(wl, t, atm=atm), dtype=dt, device="cuda")
            target = synth.true_phase_at(wl, xa, ya, t, atm=atm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dm, it, rel = R.reconstruct_converged(s)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            d = dm.double().cpu().numpy() - target
            g = torch.as_tensor(2.0 * (d - d.mean()), dtype=dt, device="cuda")
            t2 = time.perf_counter()
            gs, ga, gw = R.backward(g)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            gl.append((gs.double().cpu().numpy(), ga, np.array(gw)))
            if t > 0:                       # frame 0 starts cold
                tf.append(t1 - t0)
                tb.append(t3 - t2)
                its.append(it)
        grads[prec] = gl
        out["fp%d" % prec] = {"forward_ms": 1e3 * float(np.mean(tf)), "backward_ms": 1e3 * float(np.mean(tb)),
                              "forward_iters": float(np.mean(its)), "tol": R.default_tol()}
        R.close()
    e = [(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0]), abs(a[1] - b[1]) / abs(b[1]),
          np.linalg.norm(a[2] - b[2]) / np.linalg.norm(b[2])) for a, b in zip(grads[32], grads[64])]
    out["fp32_vs_fp64_max_rel"] = {"slopes": float(max(x[0] for x in e)), "alpha": float(max(x[1] for x in e)),
                                   "cn2": float(max(x[2] for x in e))}
    return out


def time_augmented(wl, S32, S_np, flush, steps, parity=True):
    """Augmented PCG (Sec. 3.4) on the MAORY workload against the plain warm start, at 4,
    3 and 2 iterations: frames/s of the graph-replayed frame, and the mean relative
    residual ||r|| / ||b|| that the fixed iteration count leaves (frames 2..7 of the
    frozen-flow sequence, each configuration from a cold start)."""
    from paper_2202_11945_gb300 import Reconstructor
    out = {"workload": wl["name"], "form": "FP32 operators, FP64 dots, CUDA graph"}
    for it in (4, 3, 2):
        for aug in (False, True):
            R = Reconstructor(wl, precision=32, graph=True, augmented=aug)
            if it != wl["params"]["iters"]:
                R.update_params(iters=it)
            rel = []
            for k in range(S32.shape[0]):
                R.reconstruct(S32[k])
                r, _ = R.residual(with_b=False)
                b = R.rhs(S32[k])            # the plain frame does not form b
                rel.append(float(torch.linalg.norm(r.double()) / torch.linalg.norm(b.double())))
            dm = torch.empty(R.n_act, dtype=torch.float32, device="cuda")
            t = time_frames(R, S32, steps, 20, flush, dm)
            out["%s_iters%d" % ("augmented" if aug else "plain", it)] = {
                "frames_per_s": 1e3 / float(t.mean()), "p99_ms": float(np.percentile(t, 99)),
                "mean_rel_residual": float(np.mean(rel[2:])), "launches_per_frame": R.frame_launches()}
            R.close()
    out["steps"] = steps
    if parity:
        # the first frames against the oracle's augmented frames
        import oracle as O
        R = Reconstructor(wl, precision=32, graph=True, augmented=True)
        ref = O.Reconstructor(wl)
        err = []
        for k in range(3):
            a = R.reconstruct(S32[k]).double().cpu().numpy()
            a_ref = ref.frame(S_np[k], augmented=True)
            err.append(float(np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)))
        R.close()
        out["parity_max_rel_l2_dm"] = max(err)
    return out


def time_iteration_sweep(wl, S32, flush, steps, iters=(1, 2, 3, 4, 6, 8)):
    """Frame time against the PCG iteration count (the paper finds its run-time linear in
    the iterations, Sec. 4.3): the FP32 graph form of the MAORY frame at each count, and the
    least-squares line through the mean frame times (its slope is one iteration, its
    intercept the initial residual and the fit)."""
    from paper_2202_11945_gb300 import Reconstructor
    out = {"workload": wl["name"], "form": "FP32 operators, FP64 dots, CUDA graph", "steps": steps}
    try:
        ms = []
        for it in iters:
            R = Reconstructor(wl, precision=32, graph=True)
            if it != wl["params"]["iters"]:
                R.update_params(iters=it)
            dm = torch.empty(R.n_act, dtype=torch.float32, device="cuda")
            t = time_frames(R, S32, steps, 20, flush, dm)
            ms.append(float(t.mean()))
            out["iters%d" % it] = {"frames_per_s": 1e3 / ms[-1], "mean_ms": ms[-1],
                                   "p99_ms": float(np.percentile(t, 99)), "launches_per_frame": R.frame_launches()}
            R.close()
        slope, icpt = np.polyfit(np.array(iters, float), np.array(ms), 1)
        line = icpt + slope * np.array(iters, float)
        out["us_per_iteration"] = 1e3 * float(slope)
        out["us_fixed"] = 1e3 * float(icpt)
        out["max_rel_deviation_from_line"] = float(np.max(np.abs(line - np.array(ms)) / np.array(ms)))
    except Exception as e:  # a failing leg is reported, not fatal to the line
        out["error"] = "%s: %s" % (type(e).__name__, e)
    return out


def time_persistent(wl, S32, S_np, flush, steps, parity=True):
    """The persistent frame (one cooperative launch per frame, grid-wide waits between the
    stages) on the MAORY workload, FP32 and graph-captured, against the graph of separate
    launches; parity of its first frames against the oracle."""
    from paper_2202_11945_gb300 import Reconstructor
    out = {"workload": wl["name"], "steps": steps}
    for name, kw in (("launches", {}), ("persistent", {"persistent": True})):
        R = Reconstructor(wl, precision=32, graph=True, **kw)
        dm = torch.empty(R.n_act, dtype=torch.float32, device="cuda")
        t = time_frames(R, S32, steps, 20, flush, dm)
        out[name] = {"frames_per_s": 1e3 / float(t.mean()), "p50_ms": float(np.percentile(t, 50)),
                     "p99_ms": float(np.percentile(t, 99)), "launches_per_frame": R.frame_launches()}
        R.close()
    if parity:
        import oracle as O
        ref = O.Reconstructor(wl)
        R = Reconstructor(wl, precision=32, graph=True, persistent=True)
        err = []
        for k in range(3):
            a = R.reconstruct(S32[k]).double().cpu().numpy()
            a_ref = ref.frame(S_np[k])
            err.append(float(np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)))
        R.close()
        out["parity_max_rel_l2_dm"] = max(err)
    return out


def footprint(wl, S32, S_np):
    """Device memory of the MAORY instance (Sec. 4.3 compares 16 MB for FEWHA with 53 GB for
    a matrix-vector method): the instance's own accounting (fewha_device_bytes) and the drop
    of the device's free memory, at creation and after the options' first use."""
    from paper_2202_11945_gb300 import Reconstructor

    def free():
        torch.cuda.synchronize()
        return torch.cuda.mem_get_info()[0]
    out = {"workload": wl["name"], "unit": "MB"}
    for prec in (32, 64):
        dt = torch.float32 if prec == 32 else torch.float64
        f0 = free()
        R = Reconstructor(wl, precision=prec, graph=True)
        rec = {"created": R.device_bytes() / 1e6, "created_free_drop": (f0 - free()) / 1e6}
        R.close()
        R = Reconstructor(wl, precision=prec, graph=True, augmented=True)
        R.reconstruct(S32[0].to(dt))
        rec["augmented"] = R.device_bytes() / 1e6
        R.close()
        R = Reconstructor(wl, precision=prec, graph=False)
        s = S32[1].to(dt)
        c0 = torch.zeros(R.n_coeffs, dtype=dt, device="cuda")
        R.frame_vjp(s, c0, torch.ones(R.n_act, dtype=dt, device="cuda"))
        rec["with_reverse_record"] = R.device_bytes() / 1e6
        R.reconstruct_converged(s, tol=1e-3, max_iters=200)
        rec["with_reverse_record_and_converged"] = R.device_bytes() / 1e6
        R.close()
        out["fp%d" % prec] = rec
    return out


def time_closed_loop(wl, S32, S_np, flush, steps, parity=True):
    """Closed-loop frames (Algorithm 1: pseudo-open-loop slopes from the commands of two
    frames back, delayed control law) on the MAORY workload, FP32 graph form; the timed
    inputs are the benchmark's slope frames taken as residual slopes."""
    from paper_2202_11945_gb300 import Reconstructor
    R = Reconstructor(wl, precision=32, graph=True, closed_loop=True)
    dm = torch.empty(R.n_act, dtype=torch.float32, device="cuda")
    t = time_frames(R, S32, steps, 20, flush, dm)
    out = {"workload": wl["name"], "form": "FP32 operators, FP64 dots, CUDA graph",
           "frames_per_s": 1e3 / float(t.mean()), "p50_ms": float(np.percentile(t, 50)),
           "p99_ms": float(np.percentile(t, 99)), "launches_per_frame": R.frame_launches(),
           "steps": steps}
    R.close()
    if parity:
        # residual slopes synthesised from the oracle's own commands (the sensors saw the
        # DM shape of two frames back), the same slopes to both sides
        import oracle as O
        ref = O.Reconstructor(wl)
        R = Reconstructor(wl, precision=32, graph=True, closed_loop=True)
        A = [np.zeros(ref.geo.n_a), np.zeros(ref.geo.n_a)]
        err = []
        for k in range(3):
            s_cl = S_np[k] - O.dm_slopes(ref.geo, A[-2])
            A.append(ref.frame(s_cl, closed_loop=True))
            a = R.reconstruct(torch.as_tensor(s_cl, dtype=torch.float32, device="cuda")).double().cpu().numpy()
            err.append(float(np.linalg.norm(a - A[-1]) / np.linalg.norm(A[-1])))
        R.close()
        out["parity_max_rel_l2_dm"] = max(err)
    return out


def time_paper_geometry(flush, steps, parity=True):
    """The paper's own MAORY simulation geometry (37 m, 6 LGS 74x74 with spot elongation,
    3 NGS 2x2, 3 layers at the DM altitudes, F the identity) at 2 and 4 iterations, FP32
    graph form: context for the paper's 1.48 ms per frame (2 iterations, 9 threads)."""
    from paper_2202_11945_gb300 import Reconstructor
    wl = synth.paper_mcao()
    S_np = make_inputs(wl)
    S = torch.as_tensor(np.stack(S_np), dtype=torch.float32, device="cuda").contiguous()
    out = {"workload": wl["name"], "form": "FP32 operators, FP64 dots, CUDA graph",
           "alpha_eta": wl["params"]["alpha_eta"], "steps": steps}
    for it in (2, 4):
        R = Reconstructor(wl, precision=32, graph=True)
        if it != wl["params"]["iters"]:
            R.update_params(iters=it)
        dm = torch.empty(R.n_act, dtype=torch.float32, device="cuda")
        t = time_frames(R, S, steps, 20, flush, dm)
        out["iters%d" % it] = {"frames_per_s": 1e3 / float(t.mean()), "p50_ms": float(np.percentile(t, 50)),
                               "p99_ms": float(np.percentile(t, 99))}
        R.close()
    if parity:
        import oracle as O
        ref = O.Reconstructor(wl)
        R = Reconstructor(wl, precision=32, graph=True)
        err = []
        for k in range(3):
            a = R.reconstruct(S[k]).double().cpu().numpy()
            a_ref = ref.frame(S_np[k])
            err.append(float(np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)))
        R.close()
        out["parity_max_rel_l2_dm"] = max(err)
    return out


def time_ls_fit(wl, reps=3):
    """Least-squares DM fitting over fitting directions (fewha_fit_ls, Sec. 4.1) on the
    MAORY geometry: a 3 x 3 grid of directions 20 arcsec apart, 81 x 81 pupil nodes,
    eps = 1e-2, seeded random coefficients.  Wall time per call (the CG is host-paced: a
    convergence check every 64 steps), CG steps to 1e-7 (FP32) / 1e-12 (FP64), and the
    FP32 commands against the FP64 ones (oracle parity is in the GPU tests)."""
    from paper_2202_11945_gb300 import Reconstructor
    dirs = [(synth.arcsec(x), synth.arcsec(y)) for y in (-20, 0, 20) for x in (-20, 0, 20)]
    w, n_fit, eps = [1.0] * 9, 80, 1e-2
    out = {"directions": "3 x 3 grid, 20 arcsec apart", "n_fit": n_fit, "eps": eps,
           "input": "seeded random wavelet coefficients"}
    try:
        res = {}
        for prec in (32, 64):
            R = Reconstructor(wl, precision=prec, graph=False)
            dt = torch.float32 if prec == 32 else torch.float64
            c_np = np.random.default_rng(11).standard_normal(R.n_coeffs)
            c = torch.as_tensor(c_np, dtype=dt, device="cuda")
            R.fit_ls(c, dirs, w, n_fit, eps)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                a, it, rel = R.fit_ls(c, dirs, w, n_fit, eps)
                ts.append(time.perf_counter() - t0)
            res[prec] = a.double().cpu().numpy()
            out["fp%d" % prec] = {"ms_per_call": 1e3 * float(np.median(ts)), "cg_steps": it,
                                  "us_per_step": 1e6 * float(np.median(ts)) / max(it, 1),
                                  "rel_residual": rel}
            R.close()
        out["fp32_vs_fp64_rel_l2"] = float(np.linalg.norm(res[32] - res[64]) / np.linalg.norm(res[64]))
    except Exception as e:  # a failing leg is reported, not fatal to the line
        out["error"] = "%s: %s" % (type(e).__name__, e)
    return out


def time_unrolled(wl, S_np, reps=10, parity=True):
    """Reverse mode through the fixed-iteration MAORY frame (fewha_frame_vjp): wall time of
    forward + reverse per call (synchronous), FP32 and FP64, and the FP32 gradient against
    the oracle's reverse pass on one frame."""
    from paper_2202_11945_gb300 import Reconstructor
    rng = np.random.default_rng(21)
    out = {"workload": wl["name"], "iters": wl["params"]["iters"]}
    for prec, dt in ((32, torch.float32), (64, torch.float64)):
        R = Reconstructor(wl, precision=prec, graph=False)
        s = torch.as_tensor(S_np[1], dtype=dt, device="cuda")
        c0 = torch.zeros(R.n_coeffs, dtype=dt, device="cuda")
        g = torch.as_tensor(rng.standard_normal(R.n_act), dtype=dt, device="cuda")
        R.frame_vjp(s, c0, g)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            R.frame_vjp(s, c0, g)
        torch.cuda.synchronize()
        out["fp%d_ms" % prec] = 1e3 * (time.perf_counter() - t0) / reps
        if parity and prec == 32:
            from oracle import fewha_grad as G
            import oracle as O
            geo = O.Geometry(wl)
            a_ref, _, tape = G.unrolled_frame(geo, S_np[1], np.zeros(geo.n_c), wl["params"]["iters"])
            gs_ref = G.unrolled_frame_vjp(geo, tape, g.double().cpu().numpy())
            _, gs = R.frame_vjp(s, c0, g)
            gs = gs.double().cpu().numpy()
            out["fp32_grad_rel_l2_vs_oracle"] = float(np.linalg.norm(gs - gs_ref) / np.linalg.norm(gs_ref))
        R.close()
    return out


def loop_parity(wl, S, dm, dmw):
    """Per-frame relative L2 error of the loop's commands against the FP64 oracle run on
    the same sequence (explicit initial residual), of the warm-residual recurrence's
    commands without and with an explicit refresh every 20th frame, and the oracle's own
    frame rate."""
    dmw, dmr = dmw
    import oracle as O
    ref = O.Reconstructor(wl)
    t0 = time.perf_counter()
    a = np.stack([ref.frame(s) for s in S])
    t = time.perf_counter() - t0
    e = np.array([np.linalg.norm(x - y) / np.linalg.norm(y) for x, y in zip(dm, a)])
    ew = np.array([np.linalg.norm(x - y) / np.linalg.norm(y) for x, y in zip(dmw, a)])
    return {"max_rel_l2_dm": float(e.max()), "p99_rel_l2_dm": float(np.percentile(e, 99)),
            "warm_residual_max_rel_l2_dm": float(ew.max()),
            "warm_residual_last_rel_l2_dm": float(ew[-1]),
            "warm_residual_refresh20_max_rel_l2_dm": float(max(np.linalg.norm(x - y) / np.linalg.norm(y)
                                                               for x, y in zip(dmr, a))),
            "oracle_frames_per_s": len(S) / t}


def bench_config(wl, n_coeffs, n_slopes, n_act, world):
    """The workload of the JSON line, the same for the native and the reference arm."""
    return {"workload": wl["name"], "n_coeffs": n_coeffs, "n_slopes": n_slopes, "n_act": n_act,
            "iters": wl["params"]["iters"], "warm_start": True, "initial_residual": "explicit b - M c0",
            "l2": "512 MiB memset between timed frames (native arm)",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    wl = synth.maory()
    S_np = make_inputs(wl)
    ref = O.Reconstructor(wl)
    # a bounded sample: at most 10 warm-up and 60 timed frames (~0.3-0.5 s each)
    warm = min(args.warmup, 10)
    steps = min(args.steps, 60)
    for k in range(warm):
        ref.frame(S_np[k % len(S_np)])
    ts = []
    for k in range(steps):
        t0 = time.perf_counter()
        ref.frame(S_np[(warm + k) % len(S_np)])
        ts.append(time.perf_counter() - t0)
    ts = np.array(ts) * 1e3
    value = 1e3 / ts.mean()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": float(ts.mean()),
        "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(wl, ref.geo.n_c, ref.geo.n_s, ref.geo.n_a, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d warm-started MAORY frames after %d warm-up (requested "
                                   "%d/%d), numpy FP64, 1 thread" % (steps, warm, args.steps,
                                                                      args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    assert args.warmup >= 3, "at least 3 warm-up frames"
    torch.cuda.set_device(local)
    from paper_2202_11945_gb300 import Reconstructor

    wl = synth.maory()
    S_np = make_inputs(wl)
    S32 = torch.as_tensor(np.stack(S_np), dtype=torch.float32, device="cuda").contiguous()
    S64 = torch.as_tensor(np.stack(S_np), dtype=torch.float64, device="cuda").contiguous()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    R32 = Reconstructor(wl, precision=32, graph=True)
    R64 = Reconstructor(wl, precision=64, graph=False)
    dm32 = torch.empty(R32.n_act, dtype=torch.float32, device="cuda")
    dm64 = torch.empty(R64.n_act, dtype=torch.float64, device="cuda")

    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t32 = time_frames(R32, S32, args.steps, args.warmup, flush, dm32)
    torch.cuda.synchronize()
    t64 = time_frames(R64, S64, args.steps, args.warmup, flush, dm64)
    torch.cuda.synchronize()
    # end to end through the host-buffer entry point (pinned buffers, copies inside)
    Re = Reconstructor(wl, precision=32, graph=True)
    hs = [torch.as_tensor(s, dtype=torch.float32).pin_memory() for s in S_np]
    hd = torch.empty(Re.n_act, dtype=torch.float32).pin_memory()
    for k in range(args.warmup):
        Re.reconstruct_host(hs[k % len(hs)], hd)
    e2e_steps = min(args.steps, 1000)
    te = []
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Re.reconstruct_host(hs[k % len(hs)], hd)
        te.append(time.perf_counter() - t0)
    te = np.array(te) * 1e3
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()

    # per-stage kernel times (dedicated handle; back-to-back launches after a flush)
    Rb = Reconstructor(wl, precision=32, graph=False)
    Rb.reconstruct(S32[0])
    st_ms = time_stages(Rb, flush)
    nbytes = stage_bytes(Rb, 4)
    launches = stage_launches(wl["params"]["iters"])
    share = {k: st_ms[k] * launches[k] for k in st_ms}
    dom = max(share, key=share.get)
    peak, peak_kind = measured_peaks()
    achieved = nbytes[dom] / (st_ms[dom] * 1e-3) / 1e9
    traffic, traffic_stage = recorded_traffic()
    if traffic_stage is not None and traffic_stage != dom:
        traffic = None
    Rb.close()

    loop, wl3, S3, dm3, dm3w = time_loop(args.loop_frames)
    batched = time_batched(args.batch_count, args.batch_steps, 3, flush) if args.batch_count > 0 else None
    batched_maory = time_batched_maory(32, args.batch_steps, flush) if args.batch_count > 0 else None
    backward = time_backward(args.backward_frames) if args.backward_frames > 0 else None
    augmented = (time_augmented(wl, S32, S_np, flush, args.aug_steps, parity=(rank == 0 and world == 1))
                 if args.aug_steps > 0 else None)
    closed = (time_closed_loop(wl, S32, S_np, flush, args.aug_steps, parity=(rank == 0 and world == 1))
              if args.aug_steps > 0 else None)
    pers = (time_persistent(wl, S32, S_np, flush, args.aug_steps, parity=(rank == 0 and world == 1))
            if args.aug_steps > 0 else None)
    foot = footprint(wl, S32, S_np)
    paper = (time_paper_geometry(flush, args.aug_steps, parity=(rank == 0 and world == 1))
             if args.aug_steps > 0 else None)
    unrolled = time_unrolled(wl, S_np, parity=(rank == 0 and world == 1)) if args.backward_frames > 0 else None
    lsfit = time_ls_fit(wl) if args.aug_steps > 0 else None
    sweep = time_iteration_sweep(wl, S32, flush, args.aug_steps) if args.aug_steps > 0 else None

    total32, total64, tot_e2e = max_over_ranks([float(t32.sum()), float(t64.sum()), float(te.sum())],
                                               world, "cuda")
    value = replica_throughput(world, args.steps, total32)

    base, parity = (None, None)
    if rank == 0 and world == 1:
        base, parity = cpu_baseline(wl, args.cpu_frames, S_np,
                                    lambda p: Reconstructor(wl, precision=p, graph=(p == 32)))
        loop["parity"] = loop_parity(wl3, S3, dm3, dm3w)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total32 / args.steps,
            "p50_ms": float(np.percentile(t32, 50)), "p99_ms": float(np.percentile(t32, 99)),
            "max_ms": float(t32.max()),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "form": "FP32 operators, FP64 dots, CUDA graph",
            "data": "synthetic: seeded 35-layer von Karman atmosphere with frozen flow, "
                    "simulated SH slopes + noise; %d distinct frames cycled" % N_FRAMES_INPUT,
            "config": bench_config(wl, R32.n_coeffs, R32.n_slopes, R32.n_act, world),
            "fp64_plain": {"value": replica_throughput(world, args.steps, total64), "unit": UNIT,
                           "ms_per_step": total64 / args.steps,
                           "p50_ms": float(np.percentile(t64, 50)),
                           "p99_ms": float(np.percentile(t64, 99)), "form": "FP64, stream launches"},
            "clocks": clk,
            "e2e": {"value": replica_throughput(world, e2e_steps, tot_e2e), "unit": UNIT,
                    "p99_ms": float(np.percentile(te, 99)),
                    "h2d_bytes_per_step": R32.n_slopes * 4, "d2h_bytes_per_step": R32.n_act * 4 + 4,
                    "api": "fewha_reconstruct_host (pinned host buffers, wall clock)"},
            "gpu_launches": R32.frame_launches() * args.steps,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes_per_launch": nbytes[dom],
                         "launch_us": st_ms[dom] * 1e3,
                         "note": "single MAORY frame: L2-resident, latency-bound"},
            "stages_us": {k: round(v * 1e3, 3) for k, v in st_ms.items()},
            "stage_share": {k: round(v / sum(share.values()), 4) for k, v in share.items()},
            "cpu_baseline": base,
            "parity": parity,
            "realtime_loop": loop,
            "batched": batched,
            "batched_maory": batched_maory,
            "backward": backward,
            "augmented": augmented,
            "closed_loop": closed,
            "persistent": pers,
            "footprint": foot,
            "paper_geometry": paper,
            "unrolled_backward": unrolled,
            "ls_fit": lsfit,
            "iteration_sweep": sweep,
        }
        print(json.dumps(line), flush=True)
    for R in (R32, R64, Re):
        R.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
