#!/usr/bin/env python
"""Throughput benchmark of the staggered space-time DG solver (arXiv:1802.04516).

Workload: the 2D layered medium on [0,2]x[0,1] with 448x224x2 = 200,704 jittered
triangles, 1% slivers, free surface, p = p_gamma = 3, one Ricker point source, 16
receivers, dt at 10x the explicit CFL.  One "step" is one space-time slab of the whole
path: right-hand side, the preconditioned Krylov solve of the Schur velocity system to
1e-8 relative residual (stencil preconditioner Pre2 by default, --pre), stress
back-substitution, traces and receivers.

Metric: space-time DOF-steps/s = (velocity + stress space-time DOFs per slab) x steps x
shots / time.  `value` is the mixed-precision path (FP32 operator and Krylov, FP64
refinement); the FP64 path is reported under "fp64".  With --gpus N (torchrun) every rank
runs its own independent shot on its own GPU (weak scaling, no collective on the data
path); the timed region is bracketed by barriers and the max over ranks is used.

--impl reference times the CPU oracle (explicit sparse assembly + SuperLU) on a bounded
sample of the same construction.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25       # nominal dense FP64 of one GB300: only if the probe below fails


METRIC = "space-time DOF-steps/s (velocity+stress) at 1e-8 rel residual, mixed FP32/FP64"


def dofs_per_slab(w, n_face):
    from math import comb
    nphi = comb(w.p + w.dim, w.dim)
    ng = w.p_gamma + 1
    s = 3 if w.dim == 2 else 6
    return w.n_elem * w.dim * nphi * ng + n_face * s * nphi * ng


def velocity_dofs_per_slab(w):
    """Velocity space-time DOFs alone (d N_phi N_gamma per element): the count that compares
    with the paper's, whose 2D dual basis carries more stress DOFs than ours."""
    from math import comb
    return w.n_elem * w.dim * comb(w.p + w.dim, w.dim) * (w.p_gamma + 1)


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def max_over_ranks(torch, dist, x):
    """This rank's x -> the maximum over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_shot_offset(rank):
    """x-shift of this rank's Ricker shot: with N ranks every rank runs its own independent
    shot (weak scaling, no collective on the data path)."""
    return 0.01 * rank


def build_solver(w, precision, stream, shot_offset=0.0, restart=20, inner_tol=1e-4, use_graph=True, pre=2):
    from paper_1802_04516_gb300.binding import Solver
    s = Solver(w.dim, w.p, w.p_gamma, w.scheme, precision, rel_tol=1e-8, max_iters=20000, gmres_restart=restart,
               inner_tol=inner_tol, use_graph=use_graph, stream=stream, preconditioner=pre)
    s.set_mesh(w.xyz, w.elem_vert, w.period)
    s.set_material(w.lam, w.mu, w.rho)
    if w.shots_xs is not None:
        xs = np.array(w.shots_xs) + np.array([shot_offset, 0.0])
        s.set_sources(xs, w.shots_dir, w.f0, w.t_delay, w.a1)
    else:                                   # ragged union: one point source per mesh part, one shot
        xs = w.extra["part_sources"]
        s.set_point_sources(xs, np.tile([0.0, 1.0], (xs.shape[0], 1)), w.f0, w.t_delay, w.a1)
    s.set_receivers(w.receivers)
    return s


def time_steps(torch, s, w, steps, warmup, stream, dist, start=0):
    if start > 0:          # untimed spin-up into the run before the warm-up and the timed window
        s.step(w.dt, start)
    for _ in range(warmup):
        s.step(w.dt, 1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters, launches = [], 0
    e0.record(stream)
    for _ in range(steps):
        st = s.step(w.dt, 1)
        iters.append(st["iters_max"])
        launches += s.query(11)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(torch, dist, e0.elapsed_time(e1))
    if dist is not None:
        dist.barrier()
    return ms, iters, launches, st


def e2e_steps(torch, s, w, steps, stream):
    """Same metric through the C ABI with host buffers: per step, upload the carried state
    from pinned host memory, step, read the state and the receivers back to the host."""
    v0, s0 = s.get_state()
    v = torch.empty(v0.shape, dtype=torch.float64, pin_memory=True).numpy()
    sig = torch.empty(s0.shape, dtype=torch.float64, pin_memory=True).numpy()
    v[...] = v0
    sig[...] = s0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rec_bytes = 0
    for _ in range(steps):
        s.set_state(v, sig)
        s.step(w.dt, 1)
        s.get_state(out=(v, sig))
    rec = s.read_receivers()
    rec_bytes = rec.nbytes // max(1, rec.shape[1])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dt * 1e3, v.nbytes + sig.nbytes, v.nbytes + sig.nbytes + rec_bytes


# DRAM bytes per unit measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum), scaled
# by the units one launch processes; valid for the 2D p = p_gamma = 3 shape only: the tiled
# face kernel per face on the 102,400-triangle copy of the construction
# (profiles/face_tile_c2_102k.md), the Pre2 local step per element on the 16,384-triangle copy
# (FP32 blocks, profiles/traffic_face_pre2_c2_16k.md) and on the 102,400-triangle copy (FP16
# blocks, profiles/pre1_pre2_single_shot_c2_102k.md).
TRAFFIC_PER_UNIT = {"face_fp32": (344876032 + 27466752) / 154080, "pre2_local_fp32": (429949184 + 2444032) / 16384,
                    "pre2_local_fp16": (1450097000 + 32895744) / 102400}


def _traffic(w, key, units):
    if key in TRAFFIC_PER_UNIT and w.dim == 2 and w.p == 3 and w.p_gamma == 3:
        return int(TRAFFIC_PER_UNIT[key] * units)
    return None


def fp64_peak():
    """The FP64 FMA rate this GPU sustains, from the library's own probe kernel
    (stdg_measure_fma_peak: 8 independent FMA chains per thread on every SM)."""
    from paper_1802_04516_gb300.binding import measure_fma_peak
    try:
        return measure_fma_peak(fp64=True), "measured FP64 FMA rate (stdg_measure_fma_peak)"
    except Exception:
        return FP64_NOMINAL_TFLOPS, "nominal FP64 1.25 TFLOP/s"


def face_kernel_roofline(s, w, fp32, n_face, pk, fp64_pk=None):
    """Algorithmic bytes / FLOPs of one launch of the operator's face kernel, its measured
    average duration (CUDA events on the library stream) and the fraction of peak."""
    from math import comb
    nphi = comb(w.p + w.dim, w.dim)
    ng = w.p_gamma + 1
    d = w.dim
    ns = 3 if d == 2 else 6
    wsz = 4 if fp32 else 8
    nvel = w.n_elem * d * ng * nphi
    bytes_alg = n_face * (2 * d * nphi * nphi * wsz + 2 * wsz + 8) + nvel * wsz * 3
    per_face = (2 * (d * d * ng * nphi) * nphi * 2          # D~^T v, both sides
                + ns * ng * nphi * (d + 3)                 # E : g
                + ns * ng * nphi * ng * 2                  # time factor S
                + 2 * (d * ng * nphi) * (d * nphi) * 2)    # D~ h, both sides
    flops = n_face * per_face
    ms = s.time_operator(w.dt, fp32=fp32, n=20)
    if fp32:
        peak = float(pk.get("hbm_gbs", 6800.0))
        achieved = bytes_alg / (ms * 1e-3) / 1e9
        # the tiled kernels serve 2D p = 3 and 3D p = 2; other shapes, the one-face-per-warp kernel
        tiled = (d == 2 and w.p == 3 and w.p_gamma == 3) or (d == 3 and w.p == 2 and w.p_gamma == 2)
        name = ("face_apply_tile_kernel" if d == 2 else "face_apply_tile3_kernel") if tiled else "face_apply_tma_kernel<float>"
        return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": _traffic(w, "face_fp32", n_face),
                "alg_bytes_per_launch": int(bytes_alg), "alg_flops_per_launch": int(flops), "ms_per_launch": round(ms, 4),
                "peak_source": "measured hbm_gbs" if "hbm_gbs" in pk else "fallback"}
    achieved = flops / (ms * 1e-3) / 1e12
    peak, src = fp64_pk if fp64_pk else (FP64_NOMINAL_TFLOPS, "nominal FP64 1.25 TFLOP/s")
    return {"kernel": "face_apply_kernel<double>", "bound": "alu", "achieved": round(achieved, 4),
            "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "alg_bytes_per_launch": int(bytes_alg), "alg_flops_per_launch": int(flops), "ms_per_launch": round(ms, 4),
            "peak_source": src}


def multishot_section(torch, args, stream, dist, world):
    """The 64-shot batch on the layered sliver mesh at p = 2: all shots of a slab as one
    stacked mixed-precision solve, against the plain FP64 path run one shot at a time on
    the same mesh.  Both at 1e-8 relative residual; shot-steps/s and DOF-steps/s."""
    import synth
    w = synth.c4_multishot(ny=args.ny, n_shots=args.shots, steps=args.ms_steps)
    s = build_solver(w, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol,
                     use_graph=not args.host_loop, pre=args.pre)
    tuning = s.autotune(w.dt)
    n_face = s.n_face
    ms, iters, launches, st = time_steps(torch, s, w, args.ms_steps, 1, stream, dist)
    local = pre2_local_batch_roofline(s, w, peaks()) if args.pre == 2 else None
    s.close()
    dofs_shot = dofs_per_slab(w, n_face)
    w1 = synth.c4_multishot(ny=args.ny, n_shots=1, steps=args.ms_steps)
    w1.shots_xs, w1.shots_dir = w.shots_xs[:1], w.shots_dir[:1]
    s1 = build_solver(w1, "fp64", stream.cuda_stream, restart=args.restart, use_graph=not args.host_loop, pre=args.pre)
    ms1, it1, _, _ = time_steps(torch, s1, w1, args.ms_steps, 1, stream, dist)
    s1.close()
    multi = world * w.n_shots * args.ms_steps / (ms * 1e-3)
    single = world * args.ms_steps / (ms1 * 1e-3)
    return {"workload": "c4_multishot: %d triangles (layered, 1%% slivers), p=p_gamma=2, %d Ricker shots on a line, "
                        "dt=%.4g (10x CFL)" % (w.n_elem, w.n_shots, w.dt),
            "mixed_multishot": {"shot_steps_per_s": multi, "dof_steps_per_s": multi * dofs_shot,
                                "ms_per_step": ms / args.ms_steps, "krylov_iters_per_step": iters,
                                "final_rel_res": st["final_rel_res"], "gpu_launches": launches},
            "fp64_single_shot": {"shot_steps_per_s": single, "dof_steps_per_s": single * dofs_shot,
                                 "ms_per_step": ms1 / args.ms_steps, "krylov_iters_per_step": it1},
            "speedup_shot_steps": multi / single, "dofs_per_slab_per_shot": dofs_shot, "steps": args.ms_steps,
            "pre2_local_batch_roofline": local, "tuning": tuning}


def c3_solver(w, precision, stream, args, pre):
    from paper_1802_04516_gb300.binding import Solver
    s = Solver(w.dim, w.p, w.p_gamma, w.scheme, precision, rel_tol=1e-8, max_iters=20000, gmres_restart=args.restart,
               inner_tol=args.inner_tol, use_graph=not args.host_loop, stream=stream, preconditioner=pre)
    s.set_mesh(w.xyz, w.elem_vert, w.period)
    s.set_material(w.lam, w.mu, w.rho)
    s.set_shots(1)
    pw = w.plane_wave
    s.set_plane_wave(pw["kind"], pw["n"], pw["pol"], pw["amp"])
    s.tuning = s.autotune(w.dt)   # also builds the preconditioner for dt, before any timed slab
    return s


def c3_section(torch, args, stream, dist, world, pk, fp64_pk):
    """The 3D configuration: [0,1]^3 periodic, 6 x 64^3 = 1,572,864 jittered Kuhn tetrahedra,
    p = p_gamma = 2, homogeneous (vp = sqrt 3, vs = 1, rho = 1), plane S wave along x polarised
    in y, dt = 0.02 (33x the explicit CFL), mixed precision and FP64 at 1e-8 with the stencil
    preconditioner Pre2 (its blocks hold (3 N_phi N_gamma)^2 = 8,100 values per element: 51 GB
    in FP32 for the mixed path, 102 GB in FP64 for the FP64 path).  Reports DOF-steps/s of
    both paths and the rooflines of the operator's face kernel (3, 10, 3): FP32 against the
    measured HBM bandwidth, FP64 against the measured FP64 FMA rate."""
    import synth
    w = synth.c3_cube_swave(n=args.c3_n, steps=args.c3_steps)
    out = {"workload": "c3_cube_swave: %d tetrahedra (6 x %d^3, Kuhn, jitter 0.2h), p=p_gamma=2, plane S wave, dt=%.3g, "
                       "stencil Pre2" % (w.n_elem, args.c3_n, w.dt)}
    t0 = time.perf_counter()
    s = c3_solver(w, "mixed", stream.cuda_stream, args, 2)
    out["setup_s_mixed"] = time.perf_counter() - t0
    n_face = s.n_face
    dofs = dofs_per_slab(w, n_face)
    ms, iters, launches, st = time_steps(torch, s, w, args.c3_steps, 1, stream, dist)
    out["mixed"] = {"dof_steps_per_s": world * dofs * args.c3_steps / (ms * 1e-3), "ms_per_step": ms / args.c3_steps,
                    "krylov_iters_per_step": iters, "final_rel_res": st["final_rel_res"], "gpu_launches": launches,
                    "tuning": s.tuning}
    out["face_fp32"] = face_kernel_roofline(s, w, True, n_face, pk)
    out["face_fp64"] = face_kernel_roofline(s, w, False, n_face, pk, fp64_pk)
    out["face_fp64"]["kernel"] = "face_apply_kernel<3,10,double>"
    s.close()
    if args.c3_fp64_steps > 0:
        s = c3_solver(w, "fp64", stream.cuda_stream, args, 2)
        ms, iters, _, st = time_steps(torch, s, w, args.c3_fp64_steps, 0, stream, dist)
        out["fp64"] = {"dof_steps_per_s": world * dofs * args.c3_fp64_steps / (ms * 1e-3),
                       "ms_per_step": ms / args.c3_fp64_steps, "krylov_iters_per_step": iters,
                       "final_rel_res": st["final_rel_res"],
                       "note": "no warm-up slab (graph capture included; the preconditioner is built before)"}
        s.close()
    out["dofs_per_slab"] = dofs
    return out


def order_section(torch, args, stream, dist, world):
    """Element order: the benchmark mesh as generated (raster order) and the same mesh with its
    elements and vertices renumbered by a random permutation, mixed precision, same slabs;
    ms per slab of both (the face kernels gather and scatter whole element rows, and the
    129 MB L2 holds the FP32 velocity vectors of this mesh)."""
    import synth
    out = {}
    for name, w in (("raster", synth.c2_layered_slivers(ny=args.ny, steps=args.steps)),
                    ("permuted", synth.permuted(synth.c2_layered_slivers(ny=args.ny, steps=args.steps), seed=5))):
        s = build_solver(w, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol,
                         use_graph=not args.host_loop, pre=args.pre)
        ms, iters, _, st = time_steps(torch, s, w, args.steps, args.warmup, stream, dist)
        face_ms = s.time_operator(w.dt, fp32=True, n=20)
        s.close()
        out[name] = {"ms_per_step": ms / args.steps, "krylov_iters_per_step": iters, "face_fp32_ms": face_ms}
    out["slowdown"] = out["permuted"]["ms_per_step"] / out["raster"]["ms_per_step"]
    return out


def ragged_section(torch, args, stream, dist, world):
    """The ragged batch: 16 meshes of ~5k to ~80k triangles side by side as one disconnected
    mesh, one source per part, every part at its own 10x-CFL time step (a per-element time
    scale, stdg_set_time_scale), advanced by one mixed-precision solve per slab."""
    import synth
    w, spans = synth.ragged_union(steps=args.ms_steps)
    s = build_solver(w, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol,
                     use_graph=not args.host_loop, pre=args.pre)
    s.set_time_scale(w.extra["alpha"])
    pdt = w.extra["part_dt"]
    n_face = s.n_face
    ms, iters, launches, st = time_steps(torch, s, w, args.ms_steps, 1, stream, dist)
    s.close()
    dofs = dofs_per_slab(w, n_face)
    return {"workload": "c4_ragged: %d meshes of %d..%d triangles (%d total), p=p_gamma=2, each at its own 10x-CFL "
                        "dt (%.4g..%.4g)" % (len(spans), min(n for _, n in spans), max(n for _, n in spans), w.n_elem,
                                             min(pdt), max(pdt)),
            "dof_steps_per_s": world * dofs * args.ms_steps / (ms * 1e-3),
            "mesh_steps_per_s": world * len(spans) * args.ms_steps / (ms * 1e-3),
            "ms_per_step": ms / args.ms_steps, "krylov_iters_per_step": iters, "final_rel_res": st["final_rel_res"],
            "gpu_launches": launches, "steps": args.ms_steps}


def adjoint_section(torch, args, stream, dist, world):
    """Full-waveform-inversion gradient on the 60,024-triangle random medium (p = p_gamma = 2,
    8 Ricker shots, 100 receivers, 10x CFL, checkpoints every 20 slabs): one complete
    stdg_misfit_grad per gradient -- forward run with checkpoints, misfit, segment
    recompute and adjoint solves for all 8 shots -- in mixed precision.  The data are a
    forward run of the perturbed ("true") model, made before the timed region."""
    import synth
    w = synth.c5_adjoint(steps=args.adj_steps)
    wt = synth.c5_adjoint(steps=args.adj_steps, true_model=True)
    gen = build_solver(wt, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol, pre=args.pre)
    gen.step(wt.dt, wt.n_steps)
    data = gen.read_receivers()
    gen.close()
    s = build_solver(w, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol, pre=args.pre)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    loss, gl, gm, gr, gs, st = s.misfit_grad(w.dt, w.n_steps, data, checkpoint_every=20, source_grad=True)
    torch.cuda.synchronize()
    sec = max_over_ranks(torch, dist, time.perf_counter() - t0)
    s.close()
    return {"workload": "c5_adjoint: %d triangles, p=p_gamma=2, %d shots, %d receivers, %d slabs%s, dt=%.4g, "
                        "checkpoint every 20" % (w.n_elem, w.n_shots, len(w.receivers), w.n_steps,
                                                 "" if w.n_steps == 300 else " (of the workload's 300)", w.dt),
            "grads_per_s": world / sec, "seconds_per_gradient": sec, "loss": loss,
            "grad_norms": {"lambda": float(np.linalg.norm(gl)), "mu": float(np.linalg.norm(gm)),
                           "rho": float(np.linalg.norm(gr)), "sources": float(np.linalg.norm(gs))},
            "krylov_iters_total": st["iters_total"], "precision": "mixed FP32/FP64 (1e-8 rel residual)",
            "timing": "wall clock of one call, no warm-up (includes graph capture of the step and solve graphs)"}


def pre2_local_roofline(s, w, pk):
    """Element-local step of the stencil preconditioner, z = S^{-1} (2 r - w) in FP32 arithmetic:
    one dense (d N_phi N_gamma)^2 block per element streamed from HBM -- FP16 balanced (H plus
    2N FP32 scales) by default, or FP32 padded to 16 bytes -- plus r, w read and z written."""
    from math import comb
    nphi = comb(w.p + w.dim, w.dim)
    N = w.dim * nphi * (w.p_gamma + 1)
    nvel = w.n_elem * N
    bits = s.pre2_bits
    if bits == 16:
        block, name, tkey = N * N * 2 + 2 * N * 4, "pre2_local_half_kernel", "pre2_local_fp16"
    else:
        block, name, tkey = ((N * N + 3) // 4 * 4) * 4, "pre2_local_kernel<float,float,1>", "pre2_local_fp32"
    bytes_alg = w.n_elem * block + 3 * nvel * 4
    ms = s.time_kernel(w.dt, 2, fp32=True, n=20)
    peak = float(pk.get("hbm_gbs", 6800.0))
    achieved = bytes_alg / (ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": _traffic(w, tkey, w.n_elem),
            "alg_bytes_per_launch": int(bytes_alg), "alg_flops_per_launch": int(2 * w.n_elem * N * N),
            "ms_per_launch": round(ms, 4), "peak_source": "measured hbm_gbs" if "hbm_gbs" in pk else "fallback"}


def pre2_local_batch_roofline(s, w, pk):
    """Element-local step of the stencil preconditioner for all shots of a stacked solve (FP32;
    with d N_phi N_gamma = 36 the tensor-core kernel, kind::tf32): one (d N_phi N_gamma)^2 block
    per element read once for all shots, r and w read and z written for every shot."""
    from math import comb
    nphi = comb(w.p + w.dim, w.dim)
    N = w.dim * nphi * (w.p_gamma + 1)
    ns = w.n_shots
    nvel = w.n_elem * N
    bytes_alg = w.n_elem * N * N * 4 + 3 * ns * nvel * 4
    flops = 2 * w.n_elem * N * N * ns
    ms = s.time_kernel(w.dt, 4, fp32=True, n=10)
    peak = float(pk.get("hbm_gbs", 6800.0))
    achieved = bytes_alg / (ms * 1e-3) / 1e9
    return {"kernel": "pre2_local_mma_kernel<36> (tcgen05.mma kind::tf32, TMEM accumulator)" if N == 36
            else "pre2_local_kernel<float,float,4>", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None, "shots": ns,
            "alg_bytes_per_launch": int(bytes_alg), "alg_flops_per_launch": int(flops),
            "tensor_tflops_useful": round(flops / (ms * 1e-3) / 1e12, 2), "ms_per_launch": round(ms, 4),
            "peak_source": "measured hbm_gbs" if "hbm_gbs" in pk else "fallback"}


def full_run(torch, w, args, stream):
    """The whole 200-slab configuration once, untimed per slab, from rest: Krylov iterations of
    every slab (the timed window covers a few slabs early in the run, before the Ricker pulse
    has spread) and the whole run's DOF-steps/s from CUDA events around it."""
    s = build_solver(w, "mixed", stream.cuda_stream, restart=args.restart, inner_tol=args.inner_tol,
                     use_graph=not args.host_loop, pre=args.pre)
    dofs = dofs_per_slab(w, s.n_face)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    its = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.full_slabs):
        its.append(s.step(w.dt, 1)["iters_max"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    a = np.array(its, dtype=float)
    return {"slabs": args.full_slabs, "ms": ms, "dof_steps_per_s": dofs * args.full_slabs / (ms * 1e-3),
            "krylov_iters_per_slab": {"min": int(a.min()), "median": float(np.median(a)), "max": int(a.max()),
                                      "mean": float(a.mean())},
            "krylov_iters_by_decile": [float(x.mean()) for x in np.array_split(a, 10)],
            "note": "first-slab graph capture included; per-slab host call (stdg_step with one slab)"}


def dominant_roofline(cands, per_iter):
    """The candidate with the largest device time per Krylov iteration (ms per launch x
    launches per iteration); all candidates are reported under "kernels"."""
    best = max(cands, key=lambda k: cands[k]["ms_per_launch"] * per_iter[k])
    out = dict(cands[best])
    out["launches_per_krylov_iteration"] = per_iter[best]
    return out


def cpu_baseline(max_seconds=25.0, ny=12, steps=20):
    """The oracle as it stands (assembly + SuperLU, one core) on a bounded sample of the
    same construction: ny x 2ny cells, steps slabs; DOF-steps/s over the solve phase."""
    import synth
    from oracle.stepper import Simulation
    w = synth.scaled("c2", ny=ny, steps=steps)
    t0 = time.perf_counter()
    sim = Simulation.from_workload(w)
    sim.set_source(w.shots_xs[0], w.shots_dir[0], w.f0, w.t_delay, w.a1)
    sim.step(1)                                    # factorisation happens here
    import resource
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    t1 = time.perf_counter()
    k = 0
    while k < steps and time.perf_counter() - t1 < max_seconds:
        sim.step(1)
        k += 1
    t2 = time.perf_counter()
    r2 = resource.getrusage(resource.RUSAGE_SELF)
    busy = (r2.ru_utime - r1.ru_utime + r2.ru_stime - r1.ru_stime) / (t2 - t1)   # cores kept busy
    rate = dofs_per_slab(w, sim.mesh.n_face) * k / (t2 - t1)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": rate, "unit": "DOF-steps/s", "cores": max(1, int(round(busy))), "cpu_seconds_per_second":
            round(busy, 2), "cores_available": cores, "kind": "oracle",
            "sample": "%d-triangle copy of the construction (%dx%d cells), %d slabs after assembly+LU (%.1fs)"
                      % (w.n_elem, 2 * ny, ny, k, t1 - t0), "seconds": round(t2 - t0, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = max(1, args.steps)
    cb = cpu_baseline(max_seconds=max(5.0, 4.0 * steps), steps=max(steps + args.warmup, 3))
    line = {"impl": "reference", "metric": METRIC,
            "value": cb["value"], "unit": "DOF-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "c2_layered_slivers_p3 (scaled copy, CPU oracle)",
                                            "sample": cb["sample"]},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "DOF-steps/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--start-slab", type=int, default=100,
                    help="untimed slabs before the warm-up and the timed window (the benchmark run has 200: the "
                         "window then lies mid-run, where the Krylov counts are typical of the whole run)")
    ap.add_argument("--ny", type=int, default=224, help="cells in y (224 = the 200,704-triangle mesh)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--restart", type=int, default=20, help="GMRES restart length")
    ap.add_argument("--inner-tol", type=float, default=1e-4, help="relative tolerance of the FP32 inner solve")
    ap.add_argument("--pre", type=int, default=2, choices=[0, 1, 2],
                    help="preconditioner: 0 none, 1 block Jacobi (Pre1), 2 stencil (Pre2)")
    ap.add_argument("--shots", type=int, default=64, help="shots of the multi-shot batch")
    ap.add_argument("--ms-steps", type=int, default=2, help="timed slabs of the multi-shot and ragged batches")
    ap.add_argument("--no-multishot", action="store_true")
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--c3-n", type=int, default=64, help="cubes per direction of the 3D configuration (64: 1.57M tets)")
    ap.add_argument("--c3-steps", type=int, default=2, help="timed mixed-precision slabs of the 3D configuration")
    ap.add_argument("--c3-fp64-steps", type=int, default=1, help="timed FP64 slabs of the 3D configuration (0: skip)")
    ap.add_argument("--adj-steps", type=int, default=300, help="slabs of the misfit-gradient run (the workload's 300)")
    ap.add_argument("--full-slabs", type=int, default=200,
                    help="slabs of the untimed-per-slab full run of the benchmark configuration (0: skip)")
    ap.add_argument("--only", choices=["multishot", "ragged", "adjoint", "c3", "order"],
                    help="run this one section alone and print its object (profiling runs)")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the solver loops from the host instead of CUDA-graph while nodes (for kernel profilers)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        dist = tdist
    torch.cuda.set_device(local)
    from paper_1802_04516_gb300 import build as _b
    if rank == 0:
        _b.build()
    if dist is not None:
        dist.barrier()
    import synth
    stream = torch.cuda.Stream()
    pk = peaks()
    if args.only:
        with torch.cuda.stream(stream):
            sec = {"multishot": lambda: multishot_section(torch, args, stream, dist, world),
                   "ragged": lambda: ragged_section(torch, args, stream, dist, world),
                   "adjoint": lambda: adjoint_section(torch, args, stream, dist, world),
                   "c3": lambda: c3_section(torch, args, stream, dist, world, pk, fp64_peak()),
                   "order": lambda: order_section(torch, args, stream, dist, world)}[args.only]()
        if rank == 0:
            print(json.dumps({"section": args.only, "result": sec}))
        return
    w = synth.c2_layered_slivers(ny=args.ny, steps=args.steps)
    with torch.cuda.stream(stream):
        s = build_solver(w, "mixed", stream.cuda_stream, shot_offset=rank_shot_offset(rank), restart=args.restart,
                         inner_tol=args.inner_tol, use_graph=not args.host_loop, pre=args.pre)
        tuning = s.autotune(w.dt)   # launch shapes picked on this mesh before the step graph is captured
        n_face = s.n_face
        dofs = dofs_per_slab(w, n_face)
        sampler = ClockSampler(local)
        sampler.start()
        ms, iters, launches, st = time_steps(torch, s, w, args.steps, args.warmup, stream, dist, start=args.start_slab)
        clocks = sampler.stop()
        value = world * dofs * args.steps / (ms * 1e-3)
        cands = {"face": face_kernel_roofline(s, w, True, n_face, pk)}
        per_iter = {"face": 2 if args.pre == 2 else 1}   # the Krylov operator, plus one inside Pre2
        if args.pre == 2:
            cands["pre2_local"] = pre2_local_roofline(s, w, pk)
            per_iter["pre2_local"] = 1
        roof = dominant_roofline(cands, per_iter)
        e2e_ms, h2d, d2h = e2e_steps(torch, s, w, max(1, args.steps // 2), stream)
        e2e_ms = max_over_ranks(torch, dist, e2e_ms)
        e2e_value = dofs * max(1, args.steps // 2) / (e2e_ms * 1e-3) * world
        full = full_run(torch, synth.c2_layered_slivers(ny=args.ny, steps=args.full_slabs), args, stream) \
            if args.full_slabs > 0 else None
        fp64 = None
        fp64_pk = fp64_peak()
        if not args.no_fp64 and args.fp64_steps > 0:
            s64 = build_solver(w, "fp64", stream.cuda_stream, shot_offset=rank_shot_offset(rank), restart=args.restart,
                               use_graph=not args.host_loop, pre=args.pre)
            ms64, it64, _, _ = time_steps(torch, s64, w, args.fp64_steps, 1, stream, dist)
            fp64 = {"value": world * dofs * args.fp64_steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.fp64_steps,
                    "krylov_iters_per_step": it64, "roofline": face_kernel_roofline(s64, w, False, n_face, pk, fp64_pk)}
            s64.close()
        s.close()
        multishot = None if args.no_multishot else multishot_section(torch, args, stream, dist, world)
        ragged = None if args.no_ragged else ragged_section(torch, args, stream, dist, world)
        adjoint = None if args.no_adjoint else adjoint_section(torch, args, stream, dist, world)
        c3 = None if args.no_c3 else c3_section(torch, args, stream, dist, world, pk, fp64_pk)
    if rank != 0:
        return
    cb = None if args.no_cpu_baseline else cpu_baseline()
    line = {
        "metric": METRIC,
        "value": value, "unit": "DOF-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "velocity_dof_steps_per_s": value * velocity_dofs_per_slab(w) / dofs,
        "dtype": "f32 operator/Krylov + f64 refinement", "data": "synthetic",
        "config": {"workload": "c2_layered_slivers_p3: %d triangles (448x224x2, 1%% slivers), p=p_gamma=3, "
                               "1 Ricker shot/GPU, 16 receivers, dt=%.4g (10x CFL)" % (w.n_elem, w.dt),
                   "dofs_per_slab": dofs, "n_face": n_face,
                   "preconditioner": {0: "none", 1: "block Jacobi (Pre1)", 2: "stencil (Pre2)"}[args.pre],
                   "gmres_restart": args.restart, "inner_tol": args.inner_tol,
                   "control": "host loop" if args.host_loop else "CUDA graph per step (device while loops)", "l2": "working set (blocks, Krylov basis) > 129 MB L2; no flush",
                   "parallelism": "independent shot per GPU", "tuning": tuning,
                   "window": "slabs %d..%d of the %d-slab run (after %d untimed and %d warm-up slabs)"
                             % (args.start_slab + args.warmup + 1, args.start_slab + args.warmup + args.steps,
                                200, args.start_slab, args.warmup)},
        "krylov_iters_per_step": iters, "final_rel_res": st["final_rel_res"], "refinements_last": st["refinements"],
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roof,
        "kernels": cands,
        "e2e": {"value": e2e_value, "unit": "DOF-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "full_run": full,
        "fp64": fp64,
        "multishot": multishot,
        "ragged": ragged,
        "adjoint": adjoint,
        "c3": c3,
        "cpu_baseline": cb,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
