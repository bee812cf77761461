"""Benchmark of the lattice Boltzmann hot path on one GB300 (or N replicas).

Headline: MLUPS of the D3Q19 BGK lid-driven cavity on a 256^3 lattice, FP32
storage, halfway bounce-back on five walls and a moving lid u = (0.05, 0, 0),
Re = 1000 (nu = u L / Re with L = 254).  One benchmark step is one lattice
update of all 256^3 cells (the paper's MLUPS counts every cell, collision +
streaming + boundary conditions).  The populations (2 x 1.27 GB) are far larger
than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extra]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (the paper ships no runnable reference here).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CAV = 256
LID_U = 0.05
RE = 1000.0
BYTES_PER_CELL_F32 = 2 * 19 * 4   # one read + one write of 19 FP32 populations
REPEATS = 5                       # timed regions per run; the median is reported
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def cavity_omega(n=N_CAV):
    nu = LID_U * (n - 2) / RE
    return 1.0 / (3.0 * nu + 0.5)


def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, dist=None, device="cpu"):
    """Slowest rank's time (the whole job ends when the slowest replica ends)."""
    if not dist:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells_per_rank, steps, world, ms_max):
    """Whole-job throughput of N independent replicas: all ranks' updates over
    the slowest rank's time (weak scaling)."""
    return world * cells_per_rank * steps / (ms_max * 1e3)


# ---------------------------------------------------------------------------
# our arm

def _cavity_sim(torch, X, I, n, storage, stream):
    mask = I.lid_driven_cavity_mask(n)
    sim = X.Simulation(19, (n, n, n), cavity_omega(n), "bgk", storage, stream=stream)
    sim.set_mask(mask)
    sim.set_bc(X.XLB_CELL_LID, 1.0, (LID_U, 0.0, 0.0))
    sim.init()
    return sim, mask


def run_ours(args, rank, world, dist):
    import torch
    from paper_2311_16080_gb300 import inputs as I
    from paper_2311_16080_gb300 import xlb as X

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    # a dedicated (non-default) stream: the library queues every kernel on it
    # and the CUDA events below are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    n = args.size
    cells = n ** 3
    sim, mask = _cavity_sim(torch, X, I, n, args.storage, stream.cuda_stream)
    if args.kernel != "auto":
        sim.set_kernel(args.kernel)
    st_name = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16"}[args.storage]
    kname = (f"k_sc_vec<19,{st_name},BGK,4> (4 cells per thread)" if sim.kernel() == X.XLB_KERNEL_VEC
             else f"k_stream_collide<19,{st_name},BGK> (one cell per thread)")
    fluid = int((mask == 0).sum())
    n_links, n_fix = X.xlb_boundary_links(sim.ctx)
    split = n_links + n_fix > 0
    if split:
        kname += " + k_boundary (%d ghost links, %d inlet/outlet cells)" % (n_links, n_fix)

    # warm-up (also takes the one local collision after initialisation)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    # the timed region (exactly K steps, barrier + synchronize on both sides)
    # is taken REPEATS times; the median run gives the value
    runs = []
    with ClockSampler(dev) as clk:
        for _ in range(REPEATS):
            if dist:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            runs.append(max_over_ranks(e0.elapsed_time(e1), dist, "cuda"))
    ms_max = float(np.median(runs))
    mass, _ = sim.reduce()  # FP64 conservation check on every benchmark run
    ms_step = ms_max / args.steps
    mlups = job_mlups(cells, args.steps, world, ms_max)

    # end to end through the public API with host buffers: upload mask and
    # initial fields from pinned memory, K steps, read rho and u back.
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_mask = pin(mask)
    h_rho = pin(np.ones(mask.shape, np.float32))
    h_u = pin(np.zeros((3,) + mask.shape, np.float32))
    o_rho = torch.empty(mask.shape, dtype=torch.float32).pin_memory()
    o_u = torch.empty((3,) + mask.shape, dtype=torch.float32).pin_memory()
    sim2 = X.Simulation(19, (n, n, n), cavity_omega(n), "bgk", "f32", stream=stream.cuda_stream)  # noqa
    sim2.set_bc(X.XLB_CELL_LID, 1.0, (LID_U, 0.0, 0.0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim2.set_mask(h_mask)
    t1 = time.perf_counter()
    sim2.init(h_rho, h_u)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sim2.step(args.steps)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    X.xlb_macroscopic(sim2.ctx, o_rho, o_u)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    e2e_s = t4 - t0
    sim2.close()
    e2e = {"value": world * cells * args.steps / (e2e_s * 1e6), "unit": "MLUPS",
           "h2d_bytes_per_step": (h_mask.numel() + 4 * (h_rho.numel() + h_u.numel())) / args.steps,
           "d2h_bytes_per_step": 4 * (o_rho.numel() + o_u.numel()) / args.steps,
           "phases_ms": {"set_mask": round(1e3 * (t1 - t0), 3), "init_upload": round(1e3 * (t2 - t1), 3),
                         "steps": round(1e3 * (t3 - t2), 3), "readback": round(1e3 * (t4 - t3), 3)}}

    peak, peak_kind = hbm_peak()
    esz = 4 if args.storage == "f32" else 2
    # one read and one write of every population of every cell per update
    # (the paper's MLUPS counts all cells; the bulk pass updates all of them)
    algo_bytes = 2 * 19 * esz * cells
    achieved = algo_bytes / (ms_step * 1e-3) / 1e9
    if achieved > 1.15 * peak:
        raise RuntimeError(f"timed kernel exceeds the measured copy bandwidth ({achieved:.0f} GB/s): "
                           "the events do not bracket the work")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
            "kernel": kname,
            "algorithmic_bytes_per_launch": algo_bytes,
            "bytes_per_cell": 2 * 19 * esz,
            "frac_of_8TBs_nominal": round(achieved / 8000.0, 4)}
    prof_traffic = _profile_traffic() if args.storage == "f32" else None
    if prof_traffic:
        roof["traffic"] = prof_traffic
        roof["traffic_over_algorithmic"] = round(prof_traffic / algo_bytes, 4)

    out = {"metric": "MLUPS", "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
           "timed_runs_ms": [round(r, 4) for r in runs], "timed_runs": REPEATS,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "D3Q19 BGK lid-driven cavity 256^3, FP32 storage, halfway bounce-back "
                                  "walls + moving lid u=(0.05,0,0), Re=1000",
                      "lattice": "D3Q19", "cells": cells, "fluid_cells": fluid, "omega": cavity_omega(n),
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2 (2.55 GB of populations per step), no flush"},
           "e2e": e2e, "roofline": roof, "gpu_launches": args.steps * (2 if split else 1),
           "clocks": clk.summary(), "mass_fp64": mass}
    sim.close()
    torch.cuda.synchronize()
    if rank == 0 and not args.no_extra:
        out["extra"] = extras(args, torch, X, I, stream)
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    return out


def _profile_traffic():
    """DRAM bytes per launch of the stream-collide kernel from a committed ncu
    summary (profiles/stream_collide_d3q19_cavity.txt), if present."""
    p = os.path.join(ROOT, "profiles", "stream_collide_d3q19_cavity.txt")
    try:
        for line in open(p):
            if line.strip().startswith("traffic_bytes_per_launch_256cube:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


def extras(args, torch, X, I, stream):
    """Secondary figures of the metric: low-precision storage MLUPS and error,
    KBC D3Q27 MLUPS, adjoint MLUPS (kernel and end-to-end)."""
    res = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(sim, k):
        a, b = ev(), ev()
        a.record(stream)
        sim.step(k)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    n = N_CAV
    for st in ("f16", "bf16"):
        sim, _ = _cavity_sim(torch, X, I, n, st, stream.cuda_stream)
        sim.step(10)
        ms = timed(sim, 300)
        res[f"cavity256_{st}_mlups"] = round(n ** 3 / (ms * 1e3), 1)
        res[f"cavity256_{st}_algo_GBs"] = round(2 * 19 * 2 * n ** 3 / (ms * 1e-3) / 1e9, 1)
        sim.close()

    # the paper's own performance cavity (Section 5): full-way bounce-back
    # walls and an equilibrium-BC lid, same lattice, size and viscosity
    pmask = I.paper_cavity_mask(n)
    for st in ("f32", "f16"):
        sim = X.Simulation(19, (n, n, n), cavity_omega(n), "bgk", st, stream=stream.cuda_stream)
        sim.set_mask(pmask)
        sim.set_bc(X.XLB_CELL_EQ, 1.0, (LID_U, 0.0, 0.0))
        sim.init()
        sim.step(10)
        ms = timed(sim, 300)
        esz = 4 if st == "f32" else 2
        res[f"paper_cavity256_fullway_eq_lid_{st}_mlups"] = round(n ** 3 / (ms * 1e3), 1)
        res[f"paper_cavity256_fullway_eq_lid_{st}_algo_GBs"] = round(2 * 19 * esz * n ** 3 / (ms * 1e-3) / 1e9, 1)
        sim.close()
    del pmask

    # KBC D3Q27 flow past a sphere, 512 x 256 x 256, Zou-He inlet + outflow
    mask = I.sphere_channel_mask(512, 256, 256, radius=32, center=(128, 128, 128))
    for st in ("f32", "f16", "bf16"):
        sim = X.Simulation(27, (512, 256, 256), 1.857, "kbc", st, stream=stream.cuda_stream)
        sim.set_mask(mask)
        sim.set_bc(X.XLB_CELL_INLET, 1.0, (0.04, 0.0, 0.0))
        sim.init()
        sim.step(5)
        ms = timed(sim, 50)
        cells = 512 * 256 * 256
        res[f"kbc_d3q27_sphere_{st}_mlups"] = round(cells / (ms * 1e3), 1)
        res[f"kbc_d3q27_sphere_{st}_algo_GBs"] = round(2 * 27 * (4 if st == "f32" else 2) * cells / (ms * 1e-3) / 1e9, 1)
        sim.close()
    del mask

    # Section 4.2's high-Reynolds cavity: D3Q27 KBC with a regularized moving
    # lid (INLET cells on the top plane, inward normal -z, u = (0.06, 0, 0)),
    # N = 256 as in the paper, Re = 10,000; a stability demonstration (no
    # reference data): 20,000 steps must stay finite
    try:
        n3, U3, re3 = 256, 0.06, 10000.0
        om3 = 1.0 / (3.0 * U3 * (n3 - 2) / re3 + 0.5)
        m3 = I.lid_driven_cavity_mask(n3)
        m3[n3 - 1, 1:n3 - 1, 1:n3 - 1] = I.INLET
        sim = X.Simulation(27, (n3, n3, n3), om3, "kbc", "f32", stream=stream.cuda_stream)
        sim.set_mask(m3)
        sim.set_bc(X.XLB_CELL_INLET, 1.0, (U3, 0.0, 0.0))
        sim.set_inlet_scheme("regularized")
        sim.set_inlet_normal(2, -1)
        sim.init()
        sim.step(1)
        ms = timed(sim, 20000 - 1)
        r3, u3 = sim.macroscopic()
        sim.close()
        fl3 = np.isin(m3, (0, 3, 4))
        res["kbc_cavity256_re10000_regularized_lid"] = {
            "steps": 20000, "omega": om3, "finite": bool(np.isfinite(u3).all() and np.isfinite(r3).all()),
            "max_u_over_lid": float(np.abs(u3[:, fl3]).max() / U3), "mean_rho": float(r3[fl3].mean()),
            "mlups": round(n3 ** 3 / (ms * 1e3), 1)}
        del m3, r3, u3
    except Exception as e:  # secondary figures; keep the line
        res["kbc_cavity256_re10000_error"] = repr(e)

    # the same flow on the 128 x 64 x 64 crop (radius 8), 1000 steps, in the
    # three storage forms, against the FP64 oracle's velocity stored at
    # 16,384 sampled fluid cells by tests/golden/make_kbc_sphere_crop.py
    try:
        import importlib.util
        path = os.path.join(ROOT, "tests", "golden", "make_kbc_sphere_crop.py")
        spec = importlib.util.spec_from_file_location("make_kbc_sphere_crop", path)
        crop = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(crop)
        ref = np.load(crop.OUT)
        _, cmask, crho, cu, _ = crop.setup()
        for st in ("f32", "f16", "bf16"):
            sim = X.Simulation(27, (crop.NX, crop.NY, crop.NZ), crop.OMEGA, "kbc", st, stream=stream.cuda_stream)
            sim.set_mask(cmask)
            sim.set_bc(X.XLB_CELL_INLET, 1.0, (crop.U_IN, 0.0, 0.0))
            sim.init(crho.astype(np.float32), cu.astype(np.float32))
            sim.step(int(ref["steps"]))
            _, ug = sim.macroscopic()
            sim.close()
            got = ug.reshape(3, -1)[:, ref["index"]].astype(np.float64)
            res[f"kbc_crop128_{st}_rel_l2_u_sampled"] = float(np.sqrt(((got - ref["u"]) ** 2).sum()
                                                                        / (ref["u"] ** 2).sum()))
    except Exception as e:  # secondary figures; keep the line
        res["kbc_crop128_error"] = repr(e)

    # adjoint: D3Q19 128^3 periodic, 500 steps, checkpoints every 50; the
    # gradient is computed twice on one context and the second (warm: the
    # tape memory is reused) is timed end to end
    m = 128
    rho0 = (1.0 + I.density_perturbation((m, m, m), 1e-3, seed=1234)).astype(np.float32)
    sim = X.Simulation(19, (m, m, m), 1.25, "bgk", "f32", stream=stream.cuda_stream)
    rho0_d = torch.from_numpy(rho0).cuda()
    box = (slice(48, 80),) * 3

    def gradient(profile):
        # the differentiable rollout: tape, 500 steps, FP64 kinetic-energy
        # loss on the device; backward seeds the adjoint with the loss
        # cotangent (formed on the GPU) and returns dL/drho0
        X.xlb_profile_enable(sim.ctx, profile)
        r0 = rho0_d.clone().requires_grad_(True)
        loss = X.rollout(sim, r0, 500, 50, box)
        (grad,) = torch.autograd.grad(loss, [r0])
        return loss, grad

    gradient(False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, g = gradient(False)
    torch.cuda.synchronize()
    grad_s = time.perf_counter() - t0
    gradient(True)
    adj_ms, adj_n = X.xlb_profile_read(sim.ctx, 1)
    res["adjoint_loss_fp64"] = float(loss)
    res["adjoint_grad_norm"] = float(np.sqrt(X.xlb_sum_squares(sim.ctx, g)))  # FP64 on the GPU
    sim.close()
    cells = m ** 3
    if adj_n:
        per = adj_ms / adj_n
        res["adjoint_d3q19_128_kernel_mlups"] = round(cells / (per * 1e3), 1)
        res["adjoint_d3q19_128_kernel_algo_GBs"] = round(228 * cells / (per * 1e-3) / 1e9, 1)
    res["adjoint_d3q19_128_gradient_e2e_s"] = round(grad_s, 4)
    # forward + recompute + adjoint: about 3 updates per step of the rollout
    res["adjoint_d3q19_128_gradient_rollout_mlups"] = round(500 * cells / (grad_s * 1e6), 1)

    # batched channels: 4096 D2Q9 domains (32..256 x 32..128, 1-5 discs, body
    # force), autotuned launch shape, 5000 steps in one persistent CUDA-graph
    # launch; the launch-per-domain baseline runs 50 steps (extrapolated)
    doms = I.batched_channels(4096, seed=1234, nu=(1.0 / 1.25 - 0.5) / 3.0, u_max=0.05)
    bt = X.Batch(doms, 1.25, "f32", stream=stream.cuda_stream)
    bt.set_masks()
    bt.init()
    bt.step(2)
    th, ct = bt.tune(20)
    cells = sum(bt.cells)
    a, b2 = ev(), ev()
    bt.step(10)
    torch.cuda.synchronize()
    a.record(stream)
    bt.step(5000)
    b2.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b2)
    res["batch4096_cells"] = cells
    res["batch4096_launch"] = {"threads": th, "ctas_per_sm": ct}
    res["batch4096_persistent_mlups"] = round(cells * 5000 / (ms * 1e3), 1)
    res["batch4096_persistent_algo_GBs"] = round(72 * cells * 5000 / (ms * 1e-3) / 1e9, 1)
    a, b2 = ev(), ev()
    a.record(stream)
    bt.step_per_domain(50)
    b2.record(stream)
    torch.cuda.synchronize()
    ms_pd = a.elapsed_time(b2)
    res["batch4096_per_domain_mlups_50_steps"] = round(cells * 50 / (ms_pd * 1e3), 1)
    res["batch4096_per_domain_5000_steps_s_extrapolated"] = round(ms_pd / 50 * 5000 / 1e3, 2)
    res["batch4096_persistent_5000_steps_s"] = round(ms / 1e3, 3)
    bt.close()

    # Taylor-Green 128^2 D2Q9 FP32 (16,384 cells: launch-bound), 1000 steps:
    # one launch per update against graph replay of 100 updates per graph
    nt = 128
    r0, u0 = I.taylor_green_2d(nt, nt, 0.04)
    for mode, g in (("launch", 0), ("graph", 100)):
        s = X.Simulation(9, (nt, nt), 1.25, "bgk", "f32", stream=stream.cuda_stream)
        s.set_step_graph(g)
        s.init(r0.astype(np.float32), u0.astype(np.float32))
        s.step(201)  # local collision, then a capture and a replay
        ms = timed(s, 1000)
        res[f"tg128_f32_{mode}_mlups"] = round(nt * nt / (ms * 1e3), 1)
        s.close()

    # Section 4.3's cylinder: Schafer-Turek 2D at Re = 100, 80 cells per
    # diameter, u = 0.003, to t = 100 D/U (2.67 M steps), C_d, C_l, St
    try:
        res.update(schafer_turek(torch, X, I, stream))
    except Exception as e:  # secondary figures; keep the line
        res["schafer_turek_error"] = repr(e)

    # storage error: Taylor-Green 128^2, 1000 steps, against the FP64 oracle
    try:
        from oracle import lbm as O
        nt = 128
        r0, u0 = I.taylor_green_2d(nt, nt, 0.04)
        lat = O.Lattice(9)
        msk = np.zeros((nt, nt), np.uint8)
        p = O.Params(lat, 1.25)
        f = O.run(lat, O.init_state(lat, r0, u0, msk, p), msk, p, 1000)
        _, uo = O.macroscopic(lat, f, msk, p)
        for st in ("f32", "f16", "bf16"):
            s = X.Simulation(9, (nt, nt), 1.25, "bgk", st, stream=stream.cuda_stream)
            s.init(r0.astype(np.float32), u0.astype(np.float32))
            s.step(1000)
            _, ug = s.macroscopic()
            s.close()
            err = float(np.sqrt(((ug - uo) ** 2).sum() / (uo ** 2).sum()))
            res[f"tg128_{st}_store_rel_l2_u"] = err
    except Exception as e:  # the error figures are secondary; keep the line
        res["tg128_error"] = repr(e)
    return res


def schafer_turek(torch, X, I, stream, n_d=80, u=0.003, re=100.0, t_end=100.0, every=100):
    """The flow around a cylinder of Section 4.3 (Schafer-Turek 2D benchmark):
    BGK, Bouzidi walls on the cylinder, regularized Poiseuille inflow,
    outflow, halfway channel walls, FP32; the momentum-exchange force is
    recorded on the device every `every` steps (graph replay in between).
    Maxima of C_d, C_l and the Strouhal number over 50 <= t <= 100."""
    c, _ = X.xlb_lattice_table(9)
    m, ctr, radius, uin = I.schafer_turek_2d(n_d, u)
    cells, dirs, q = I.ball_links(m, ctr, radius, c[:, :2])
    omega = 1.0 / (3.0 * u * n_d / re + 0.5)
    ny, nx = m.shape
    sim = X.Simulation(9, (nx, ny), omega, "bgk", "f32", stream=stream.cuda_stream)
    sim.set_mask(m)
    sim.set_inlet_profile(uin.astype(np.float32))
    sim.set_inlet_scheme("regularized")
    sim.set_wall_distances(cells, dirs, q.astype(np.float32))
    u0 = (uin * np.isin(m, (0, 3, 4))).astype(np.float32)
    sim.init(np.ones(m.shape, np.float32), u0)
    sim.set_step_graph(every)
    steps = int(round(t_end * n_d / u))
    n = steps // every
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    base = F.data_ptr()
    sim.step(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(n):
        sim.step(every)
        sim.wall_force(base + 24 * k)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    sim.close()
    Fh = F.cpu().numpy()
    t = (1 + every * (np.arange(n) + 1)) * u / n_d
    cd = 2.0 * Fh[:, 0] / (u * u * n_d)
    cl = 2.0 * Fh[:, 1] / (u * u * n_d)
    win = t >= 50.0
    if not win.any():  # a short run (profiling): timing only
        return {"schafer_turek_steps": steps, "schafer_turek_s": round(ms / 1e3, 3)}
    x = cl[win] - cl[win].mean()
    tw = t[win]
    k = np.flatnonzero((x[:-1] < 0) & (x[1:] >= 0))
    tc = tw[k] - x[k] * (tw[k + 1] - tw[k]) / (x[k + 1] - x[k])
    st = (len(tc) - 1) / (tc[-1] - tc[0]) if len(tc) > 1 else float("nan")
    return {"schafer_turek_re100_cd_max": round(float(cd[win].max()), 4),
            "schafer_turek_re100_cl_max": round(float(cl[win].max()), 4),
            "schafer_turek_re100_strouhal": round(float(st), 4),
            "schafer_turek_re100_paper": {"cd_max": 3.25, "cl_max": 0.985, "strouhal": 0.300},
            "schafer_turek_re100_steps": steps, "schafer_turek_re100_cells": int(m.size),
            "schafer_turek_re100_s": round(ms / 1e3, 2),
            "schafer_turek_re100_mlups": round(m.size * steps * 1.0 / (ms * 1e3), 1)}


# ---------------------------------------------------------------------------
# CPU oracle legs

def _oracle_cavity_steps(n, steps_or_seconds, by_time):
    from oracle import lbm as O
    from paper_2311_16080_gb300 import inputs as I
    lat = O.Lattice(19)
    mask = I.lid_driven_cavity_mask(n)
    p = O.Params(lat, cavity_omega(N_CAV), bc=O.BC(3, lid_u=(LID_U, 0.0, 0.0)))
    f = O.init_state(lat, np.ones(mask.shape), np.zeros((3,) + mask.shape), mask, p)
    f = O.step(lat, f, mask, p)
    done = 0
    t0 = time.perf_counter()
    while True:
        f = O.step(lat, f, mask, p)
        done += 1
        el = time.perf_counter() - t0
        if (by_time and el >= steps_or_seconds) or (not by_time and done >= steps_or_seconds):
            break
    return done, el


def _oracle_procs(k, seconds, n):
    """k concurrent single-threaded child processes, each timing the oracle
    on its own n^3 cavity for `seconds`; returns [(steps, elapsed), ...]."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench, json; "
            f"d, el = bench._oracle_cavity_steps({n}, {seconds}, True); print(json.dumps([d, el]))")
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True) for _ in range(k)]
    out = []
    for pr in procs:
        so, _ = pr.communicate(timeout=seconds * 6 + 180)
        out.append(tuple(json.loads(so.strip().splitlines()[-1])))
    return out


def cpu_baseline(seconds=15.0, n=48):
    """Oracle timed on the host cores on a bounded sample of the workload:
    one single-threaded child process, then one per core at once (independent
    n^3 cavities; the oracle itself is not parallelised), whose summed
    throughput is the all-core figure reported as the value."""
    cores = os.cpu_count() or 1
    try:
        (d1, e1), = _oracle_procs(1, seconds, n)
        allc = _oracle_procs(cores, seconds, n)
    except Exception as e:
        return {"value": None, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": f"failed: {e!r}"}
    single = n ** 3 * d1 / (e1 * 1e6)
    total = sum(n ** 3 * d / (el * 1e6) for d, el in allc)
    return {"value": round(total, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_thread_value": round(single, 4),
            "sample": f"{n}^3 lid-driven cavity (same mask recipe, omega and lid), FP64 numpy oracle, ~{seconds:.0f} s: "
                      f"{cores} concurrent one-thread processes (sum of their MLUPS; {sum(d for d, _ in allc)} steps "
                      f"in total) and, alone, one thread ({d1} steps in {e1:.1f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    n = 32
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench, json; "
            f"bench._oracle_cavity_steps({n}, {args.warmup}, False); "
            f"d, el = bench._oracle_cavity_steps({n}, {args.steps}, False); print(json.dumps([d, el]))")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    done, el = json.loads(r.stdout.strip().splitlines()[-1])
    v = n ** 3 * done / (el * 1e6)
    return {"impl": "reference", "metric": "MLUPS", "value": round(v, 4), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / done, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "D3Q19 BGK lid-driven cavity 256^3, FP32 storage, halfway bounce-back "
                                   "walls + moving lid u=(0.05,0,0), Re=1000",
                       "sample": f"{n}^3 crop of the same recipe per step"},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"{n}^3 lid-driven cavity per step, FP64 numpy oracle, one thread"},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """One secondary workload's loop only, for a profiler: the adjoint on a
    128^3 periodic D3Q19 lattice (60 steps, checkpoints every 20), the KBC
    D3Q27 sphere channel at 256 x 128 x 128 (args.steps steps), or the
    Section 4.3 cylinder at full resolution (100 * args.steps steps, graph
    replay, the wall force every 100 steps)."""
    import torch
    from paper_2311_16080_gb300 import inputs as I
    from paper_2311_16080_gb300 import xlb as X
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    if args.profile_case == "cylinder":
        r = schafer_turek(torch, X, I, stream, t_end=100 * args.steps * 0.003 / 80)
        print(json.dumps({"profile_case": "cylinder", **r, "seconds": round(time.perf_counter() - t0, 3)}))
        return
    if args.profile_case == "adjoint":
        m, T = 128, 60
        rho0 = torch.from_numpy((1.0 + I.density_perturbation((m, m, m), 1e-3, seed=1234)).astype(np.float32)).cuda()
        sim = X.Simulation(19, (m, m, m), 1.25, "bgk", "f32", stream=stream.cuda_stream)
        sim.init(rho0, None)
        X.xlb_tape_begin(sim.ctx, T, 20)
        sim.step(T)
        rb = torch.ones((m, m, m), dtype=torch.float32, device="cuda") * 1e-3
        X.xlb_adjoint_seed_macro(sim.ctx, rb, None)
        X.xlb_adjoint_step(sim.ctx, T)
        X.xlb_tape_end(sim.ctx)
    else:
        mask = I.sphere_channel_mask(256, 128, 128, radius=16, center=(64, 64, 64))
        sim = X.Simulation(27, (256, 128, 128), 1.857, "kbc", args.storage, stream=stream.cuda_stream)
        sim.set_mask(mask)
        sim.set_bc(X.XLB_CELL_INLET, 1.0, (0.04, 0.0, 0.0))
        sim.init()
        sim.step(args.steps)
    torch.cuda.synchronize()
    sim.close()
    print(json.dumps({"profile_case": args.profile_case, "seconds": round(time.perf_counter() - t0, 3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--kernel", choices=["auto", "direct", "vec"], default="auto")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32",
                    help="population storage (default f32, the benchmark workload; others for profiling)")
    ap.add_argument("--profile-case", choices=["adjoint", "kbc", "cylinder"], default=None,
                    help="run only one secondary workload's loop (for profilers); prints no bench line")
    ap.add_argument("--size", type=int, default=N_CAV,
                    help="cavity edge (default 256, the benchmark workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_case:
        run_profile_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
