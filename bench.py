"""Benchmark: slices/s to a fixed photoelectric-image error for UDM1-PCG1 ADMM
(Sec. 3.3) on the 512x512, 720-view, 1024-bin fan-beam baggage slice.

One step = reconstruct the batch to the workload's iteration count: the
initial estimate plus 100 ADMM iterations, everything in libdect kernels, with
the measurements already resident in HBM. The fixed PE error is the FP64
oracle's xi_p (Eq. 14) after those 100 iterations on the same seeded slice
(tests/golden/baggage_fan_512_xi.json); the line reports whether the GPU's
xi_p lands within 0.5 dB of it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl dect|reference]

Prints one JSON line on rank 0. Multi-GPU: one process per GPU (torchrun),
each rank reconstructs its own slices (weak scaling, no collective on the
data path); timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slices/s to fixed PE error (UDM1-PCG1, 100 ADMM iterations), 512^2 x 720 views fan beam"
UNIT = "slices/s"
ITERS = 100
GOLDEN = os.path.join(ROOT, "tests", "golden", "baggage_fan_512_xi.json")
GOLDEN_CDM_FBP = os.path.join(ROOT, "tests", "golden", "baggage_fan_512_cdm_fbp.json")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _golden(path=None):
    try:
        with open(path or GOLDEN) as f:
            return json.load(f)
    except Exception:
        return None


def joseph_weight_count(g) -> int:
    """Non-zero weights of the projection matrix R (one channel) for geometry g: every sample of the
    Joseph interpolation (Eq. 2-3's R, one sample per column or row along each ray) has up to two
    in-image neighbours. Counted in float64 from the same ray parameters the projector tabulates;
    samples landing exactly on a pixel centre (a zero upper weight) are counted too."""
    px, py, dx, dy = g.rays()
    total = 0
    for v0 in range(0, g.n_views, 16):
        X, Y, DX, DY = (a[v0:v0 + 16].ravel() for a in (px, py, dx, dy))
        ax0 = np.abs(DX) >= np.abs(DY)
        for m, (pa, pb, da, db, n_along, n_across) in ((ax0, (X, Y, DX, DY, g.nx, g.ny)),
                                                        (~ax0, (Y, X, DY, DX, g.ny, g.nx))):
            if not m.any():
                continue
            slope = db[m] / da[m]
            q0 = (pb[m] - pa[m] * slope) / g.pixel_cm + 0.5 * (n_across - 1) - 0.5 * (n_along - 1) * slope
            h = np.floor(q0[:, None] + np.arange(n_along)[None, :] * slope[:, None])
            total += int(((h >= 0) & (h < n_across)).sum() + ((h >= -1) & (h < n_across - 1)).sum())
    return total


# the workload both arms of the bench line name (the reference arm times a bounded sample of it)
WORKLOAD = "fan 512x512, 720 views x 1024 bins, 40 objects, I0 2e5, UDM1-PCG1 x 100 + init"

# Shared-memory wavefronts per slice of the backprojector sweep on the same workload (ncu
# l1tex__data_pipe_lsu_wavefronts_mem_shared.sum), keyed by (tile side, slices per CTA); the count
# follows the samples and staged rays, not the view-group count. The SM serves one wavefront per clock.
SWEEP_SMEM_WAVEFRONTS = {(32, 2): 8.01e7}

# DRAM bytes (read + write) per launch of the backprojector sweep at the bench workload (8 slices),
# keyed by the launch shape they were captured with (slices, view groups, tile side, cluster form,
# slices per CTA, reduced form); from the counter captures in profiles/k_bp_sweep_512x720x1024.txt.
# Reported only when the run uses one of these shapes.
SWEEP_TRAFFIC = {(8, 6, 32, 0, 2, 1): 56.4e6, (8, 8, 32, 0, 2, 1): 57.8e6, (8, 10, 32, 0, 2, 1): 58.3e6}


# ------------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle as it stands, on a bounded sample of the workload

def _oracle_sample(n_iters: int, case=None):
    """Times the oracle's initial image and n_iters ADMM iterations on one slice."""
    from oracle import _clib, admm
    from synth.workloads import BAGGAGE_KAPPA, baggage_fan_case

    c = case if case is not None else baggage_fan_case()
    P = admm.Params(kappa=BAGGAGE_KAPPA)
    t0 = time.perf_counter()
    prob = admm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], P)
    x0 = admm.initial_image(prob)
    st = admm.state_from_image(prob, *x0)
    t_init = time.perf_counter() - t0
    times = []
    for _ in range(n_iters):
        t1 = time.perf_counter()
        st = admm.admm_iteration(prob, st)
        times.append(time.perf_counter() - t1)
    return t_init, times, _clib.num_threads(), (prob, st)


def _oracle_phases(prob, st):
    """Seconds of one application of each phase of an iteration in the oracle, on its current state:
    R and R^T of both bases, the preconditioner on both bases, one LM iteration of every ray (Eq. 13)."""
    from oracle import spectral

    out = {}
    t = time.perf_counter()
    prob.R(st.x)
    out["R_both_bases"] = time.perf_counter() - t
    t = time.perf_counter()
    prob.RT(st.a)
    out["RT_both_bases"] = time.perf_counter() - t
    t = time.perf_counter()
    prob.M(st.x, prob.H)
    out["preconditioner_both_bases"] = time.perf_counter() - t
    v = st.Rx - st.ua
    t = time.perf_counter()
    spectral.udm(prob.spec, prob.m_h, prob.m_l, prob.w_h, prob.w_l, v[0], v[1], st.rho[0], st.rho[1], 1,
                 st.a[0], st.a[1], st.mu.copy())
    out["udm_one_lm_iteration"] = time.perf_counter() - t
    return {k: round(v, 4) for k, v in out.items()}


def cpu_baseline():
    t_init, times, cores, (prob, st) = _oracle_sample(2)
    per_slice = t_init + ITERS * float(np.mean(times))
    return {"value": 1.0 / per_slice, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle on one 512^2 slice: set-up + initial image ({t_init:.1f} s) and 2 of the "
                      f"{ITERS} ADMM iterations ({np.mean(times):.2f} s each), iterations scaled x{ITERS // 2}",
            "phases_s": _oracle_phases(prob, st)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from synth.workloads import baggage_fan_case

    case = baggage_fan_case()
    t_init, _, cores, (prob, st) = _oracle_sample(0, case)
    from oracle import admm

    for _ in range(args.warmup):
        st = admm.admm_iteration(prob, st)
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        st = admm.admm_iteration(prob, st)
        times.append(time.perf_counter() - t1)
    per_slice = t_init + ITERS * float(np.mean(times))
    value = 1.0 / per_slice
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "batch": 1, "step": "one ADMM iteration of the FP64 oracle (a bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"initial image ({t_init:.1f} s) + {args.steps} timed ADMM iterations, "
                                   f"scaled to {ITERS} iterations"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------

CDM_ITERS = 20  # LM iterations of the CDM decomposition (the same LM as UDM, rho = 0)


def _timed_reconstruct(sol, steps, warmup, stream, flush, barrier=None):
    """Device ms per step of reconstruct(ITERS) (L2 flushed between steps, outside the events)."""
    import torch

    for _ in range(warmup):
        sol.reconstruct(ITERS)
    (barrier or torch.cuda.synchronize)()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sol.reconstruct(ITERS)
        ev[k][1].record(stream)
    (barrier or torch.cuda.synchronize)()
    return [a.elapsed_time(b) for a, b in ev]


def _plain_ms(make_single, n, stream, flush, iters=ITERS):
    """Device ms for the slices reconstructed one after another by single-slice solvers."""
    import torch

    singles = [make_single(b) for b in range(n)]
    for s1 in singles:
        s1.reconstruct(iters)  # warm-up (graph capture)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(0.0)
    p0.record(stream)
    for s1 in singles:
        s1.reconstruct(iters)
    p1.record(stream)
    torch.cuda.synchronize()
    del singles
    return p0.elapsed_time(p1)


# a plain single-slice solver: eager launches, backprojector view groups from the occupancy rule
PLAIN = dict(use_graph=0, bp_view_groups=-1, bp_tile=32, bp_cluster=-1, proj_views=2)


def _phase_ms(sol, iters=5):
    prof = sol.profile(iters)
    return {p: prof[p][0] / iters for p in prof}


def run_dect(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__

    # one build per node: local rank 0 compiles while the other ranks wait, then every rank loads it
    if ws == 1 or local == 0:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
        if local != 0:
            __graft_entry__.build()  # up to date: only checks and loads
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect, shard
    from synth.workloads import BAGGAGE_KAPPA, baggage_fan_case

    B = args.batch
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=min(B, 16)) as ex:  # numpy releases the GIL in the heavy loops
        # weak scaling: ws * B equal slices, each rank its contiguous share (no data-path collective)
        mine = list(shard.rank_slices([1.0] * (ws * B), rank, ws))
        cases = list(ex.map(lambda s: baggage_fan_case(slice_index=s), mine))
    geo = [Geometry(c["geom"]) for c in cases]
    spec = Spectra.from_tables(cases[0]["spectra"])
    storage = {"f32": 0, "f16": 1, "bf16": 2}[args.storage]
    # the backprojector's launch shape: autotuned at creation unless fixed on the command line
    shape = dict(bp_view_groups=args.bp_view_groups, bp_tile=args.bp_tile, bp_cluster=args.bp_cluster,
                 bp_slices=args.bp_slices, bp_reduce=args.bp_reduce, proj_views=args.proj_views)
    sol = Solver(geo, spec, kappa=BAGGAGE_KAPPA, storage=storage, **shape)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    dev_data = [[f32(c[k]) for k in ("m_h", "m_l", "w_h", "w_l")] for c in cases]
    truths = [f32(np.stack([c["truth_c"], c["truth_p"]])) for c in cases]
    for b in range(B):
        sol.set_data(b, *dev_data[b])
        sol.set_truth(b, truths[b])
    stream = torch.cuda.current_stream()
    if args.profile_run:
        # one untimed reconstruction of the workload, for profiler captures
        sol.reconstruct(args.profile_run)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": args.profile_run, "batch": B, "stats": sol.stats(0)}), flush=True)
        return 0
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > 129 MB L2

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- the headline: B slices batched per launch, reconstruct to the workload's iteration count ----
    launches0 = sol.stats(0)["count_launches"]
    with ClockSampler(torch.cuda.current_device()) as clk:
        step_ms = _timed_reconstruct(sol, args.steps, args.warmup, stream, flush, barrier)
    clocks = clk.summary()
    # every step launches the same kernels: the timed steps' share of the warm-up and timed launches
    launches = (sol.stats(0)["count_launches"] - launches0) * args.steps // (args.steps + args.warmup)
    total_ms = shard.max_over_ranks(float(sum(step_ms)), dev)
    value = ws * B * args.steps / (total_ms / 1e3)
    st0 = sol.stats(0)

    # end to end through the C ABI: pinned host measurements in, image out, every step
    host_in = [[t.cpu().pin_memory() for t in d] for d in dev_data]
    host_out = [torch.empty((2, c["geom"].ny, c["geom"].nx), dtype=torch.float32).pin_memory() for c in cases]
    h2d = sum(t.numel() * 4 for d in host_in for t in d)
    d2h = sum(t.numel() * 4 for t in host_out)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        for b in range(B):
            sol.set_data(b, *host_in[b])
        sol.reconstruct(ITERS)
        for b in range(B):
            dect.admm_get(sol.handle, b, dect.X, host_out[b])
    e1.record(stream)
    barrier()
    e2e_ms = shard.max_over_ranks(e0.elapsed_time(e1), dev)
    e2e_value = ws * B * e2e_steps / (e2e_ms / 1e3)
    for b in range(B):  # back to the device-resident data
        sol.set_data(b, *dev_data[b])
    if ws > 1:
        torch.distributed.destroy_process_group()  # the rank-0 legs below use no collective
    if rank != 0:
        return 0

    cfg = {"workload": WORKLOAD,
           "iterations_fixed": ITERS, "batch_per_gpu": B, "l2": "flushed between steps (512 MB write)",
           "storage": args.storage, "bp_view_groups": st0["bp_view_groups"], "bp_tile": st0["bp_tile"],
           "bp_cluster": st0["bp_cluster"], "bp_slices": st0["bp_slices"], "bp_reduce": st0["bp_reduce"],
           "proj_views": st0["proj_views"]}
    phases = _phase_ms(sol, 10)
    for p_, ms in phases.items():
        cfg[f"{args.storage}_ms_{p_}"] = round(ms, 4)
    cfg[f"{args.storage}_ms_iteration"] = round(sum(phases.values()), 4)

    # ---- the plain form of the metric and the batched mixed-precision arms ----
    extras = not args.no_extras
    if B > 1 and extras:
        def single(params):
            def make(b):
                s1 = Solver([geo[b]], spec, kappa=BAGGAGE_KAPPA, **params)
                s1.set_data(0, *dev_data[b])
                return s1
            return make

        plain_ms = _plain_ms(single(PLAIN), B, stream, flush)
        best_ms = _plain_ms(single({}), B, stream, flush)
        plain = B / (plain_ms / 1e3)
        cfg.update({"plain": "single-slice solvers in turn: eager, occupancy view groups, FP32",
                    "plain_slices_per_s": plain, "batched_over_plain": value / plain,
                    "plain_graph_autotuned_slices_per_s": B / (best_ms / 1e3),
                    "batched_over_plain_graph_autotuned": value / (B / (best_ms / 1e3))})
        for name, code in (("f16", 1), ("bf16", 2)):
            if name == args.storage:
                continue
            try:
                s16 = Solver(geo, spec, kappa=BAGGAGE_KAPPA, storage=code, **shape)
                for b in range(B):
                    s16.set_data(b, *dev_data[b])
                    s16.set_truth(b, truths[b])
                ms16 = _timed_reconstruct(s16, 2, 1, stream, flush)
                v16 = B * 2 / (sum(ms16) / 1e3)
                cfg[f"batched_{name}_slices_per_s"] = v16
                cfg[f"batched_{name}_over_plain"] = v16 / plain
                cfg[f"batched_{name}_xi_p_db"] = s16.stats(0)["xi_db"][1]
                ph = _phase_ms(s16, 5)
                for p_, ms in ph.items():
                    cfg[f"{name}_ms_{p_}"] = round(ms, 4)
                cfg[f"{name}_ms_iteration"] = round(sum(ph.values()), 4)
                del s16
            except Exception as exc:
                cfg[f"batched_{name}_error"] = f"{type(exc).__name__}: {exc}"[:90]
        # the float64 decomposition option: its cost per slice-iteration next to the default's
        try:
            s64 = Solver(geo, spec, kappa=BAGGAGE_KAPPA, udm_f64=1, **shape)
            for b in range(B):
                s64.set_data(b, *dev_data[b])
            s64.reconstruct(1)
            cfg["udm_us_per_slice"] = round(1e3 * phases["udm"] / B, 2)
            cfg["udm_f64_us_per_slice"] = round(1e3 * _phase_ms(s64, 3)["udm"] / B, 2)
            del s64
        except Exception as exc:
            cfg["udm_f64_error"] = f"{type(exc).__name__}: {exc}"[:90]

    # ---- quality gate: xi_p of slice 0 after the workload's iterations vs the FP64 oracle's ----
    gold = _golden()
    cfg["pe_gate_xi_p_db"] = st0["xi_db"][1]
    cfg["pe_gate_xi_c_db"] = st0["xi_db"][0]
    if gold is not None:
        target = gold["xi_p"][ITERS]
        cfg["pe_gate_oracle_xi_p_db"] = target
        cfg["pe_gate_ok"] = bool(abs(st0["xi_db"][1] - target) <= 0.5)

    # ---- roofline of the dominant kernel group (live events of one captured iteration) ----
    prof = sol.profile(10)
    top = max(prof, key=lambda p_: prof[p_][0])
    g = cases[0]["geom"]
    M, Np = g.n_views * g.n_bins, g.nx * g.ny
    peak, peak_kind = _peaks()
    nnz = joseph_weight_count(g)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12

    def kernel_roof(name, launches_per_iter):
        ms_total, n_launch = prof[name]
        avg_ms = ms_total / max(n_launch, 1)
        tf = B * 2 * 2 * nnz / (avg_ms / 1e3) / 1e12
        # algorithmic bytes: R reads the image once and writes the sinogram (both bases, FP32); R^T reads
        # the sinogram and writes the image
        nbytes = B * 8 * (M + Np)
        gbs = nbytes / (avg_ms / 1e3) / 1e9
        return avg_ms, tf, gbs, nbytes

    bp_ms, bp_tf, bp_gbs, bp_bytes = kernel_roof("backproject", 2)
    pr_ms, pr_tf, pr_gbs, pr_bytes = kernel_roof("project", 1)
    cfg.update({"project_tflops": pr_tf, "project_tflops_frac": pr_tf / fp32_peak, "project_hbm_gbs": pr_gbs,
                "project_hbm_frac": pr_gbs / peak, "backproject_hbm_frac": bp_gbs / peak})
    traffic = SWEEP_TRAFFIC.get((B, st0["bp_view_groups"], st0["bp_tile"], st0["bp_cluster"], st0["bp_slices"],
                                 st0["bp_reduce"]))
    roof = {"kernel": "backproject" if top == "backproject" else top, "bound": "alu", "achieved": bp_tf,
            "peak": fp32_peak, "unit": "TFLOP/s", "frac": bp_tf / fp32_peak,
            "traffic": traffic, "traffic_source": "stored ncu capture of this kernel and launch shape "
                                                  "(profiles/k_bp_sweep_512x720x1024.txt)" if traffic else None,
            "peak_kind": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x max SM clock",
            "avg_launch_ms": bp_ms, "algorithmic_flops_per_launch": B * 4 * nnz,
            "algorithmic_bytes_per_launch": bp_bytes, "hbm_achieved_gbs": bp_gbs, "hbm_peak_gbs": peak,
            "hbm_frac": bp_gbs / peak, "hbm_peak_kind": peak_kind}
    wf = SWEEP_SMEM_WAVEFRONTS.get((st0["bp_tile"], st0["bp_slices"]))
    if wf and top == "backproject":
        # the sweep's actual limit: shared-memory wavefronts (accumulator read-modify-writes and staging)
        clk = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
        achieved_wf = B * wf / (bp_ms / 1e3)
        roof["onchip"] = {"resource": "shared-memory wavefronts", "per_launch": B * wf,
                          "achieved_per_s": achieved_wf, "peak_per_s": n_sm * clk, "frac": achieved_wf / (n_sm * clk),
                          "source": "per-slice count from a stored ncu capture "
                                    "(profiles/k_bp_sweep_512x720x1024.txt); peak one per SM per clock"}
    # the HBM-bound phases (data read and written once per iteration; 8 slices exceed L2): the four
    # element-wise kernels of an iteration (b = a + u^a - R x: 32 B/ray; x, R x += alpha p, q: 24 B/pixel
    # + 24 B/ray; y, z, u^y, u^z of Eq. 9-11 with x: 104 B/pixel; the dual rescale moves nothing when
    # rho stays) and the two backprojector finalize passes (partial images of 8 B, plus 64 B/pixel of
    # epilogue images for r0 and 16 B/pixel for A p)
    parts = 1 if st0["bp_cluster"] or st0["bp_reduce"] else st0["bp_view_groups"]
    for p_, nbytes in (("update", B * (56 * M + 128 * Np)), ("bp_finalize", B * ((16 * parts + 80) * Np))):
        ms = prof[p_][0] / 10
        cfg[f"{p_}_hbm_frac"] = nbytes / (ms / 1e3) / 1e9 / peak

    # ---- batching on other workloads: slice-size scan, and the 64 uneven slices ----
    if extras:
        try:
            cfg.update(size_scan(args, stream, flush))
        except Exception as exc:
            cfg["size_scan_error"] = f"{type(exc).__name__}: {exc}"[:90]
        if args.uneven_slices:
            try:
                cfg.update(uneven_leg(args.uneven_slices, stream))
            except Exception as exc:
                cfg["uneven_error"] = f"{type(exc).__name__}: {exc}"[:90]
        if args.stack_slices:
            try:
                cfg.update(stack_leg(args.stack_slices, stream))
            except Exception as exc:
                cfg["stack_error"] = f"{type(exc).__name__}: {exc}"[:90]

    # ---- the paper's comparison (Sec. 4): time to the same PE error, new splitting vs LM x CG ----
    if gold is not None and not args.no_comparison:
        try:
            cfg.update(scheme_comparison(geo, spec, cases, dev_data, truths, gold, B, stream))
        except Exception as exc:  # an optional measurement must not cost the bench line
            cfg["comparison_error"] = f"{type(exc).__name__}: {exc}"[:90]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else args.storage,
        "data": "synthetic", "config": cfg, "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": int(launches),
        "roofline": roof,
    }
    if ws == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as exc:  # the oracle leg is a reported baseline, not the measurement
            line["cpu_baseline"] = {"error": f"{type(exc).__name__}: {exc}"}
    print(json.dumps(line), flush=True)
    return 0


def size_scan(args, stream, flush):
    """Batched vs the plain single-slice loop for 8 fan slices at smaller sizes (per ADMM iteration after
    the initial image, device time): where batching pays beyond launch overheads."""
    import torch

    from paper_1905_00934_gb300 import Geometry, Solver, Spectra
    from synth.workloads import BAGGAGE_KAPPA, quick_fan_case

    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for n, v, nb in ((128, 180, 256), (256, 360, 512)):
        cases = [quick_fan_case(s, n, v, nb) for s in range(8)]
        spec = Spectra.from_tables(cases[0]["spectra"])
        geo = [Geometry(c["geom"]) for c in cases]
        data = [[torch.tensor(np.ascontiguousarray(c[k]), dtype=torch.float32, device=dev)
                 for k in ("m_h", "m_l", "w_h", "w_l")] for c in cases]

        def per_iter(solvers, iters=10):
            for s1 in solvers:
                s1.reconstruct(0)
                s1.step(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s1 in solvers:
                s1.step(iters)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / iters

        bt = Solver(geo, spec, kappa=BAGGAGE_KAPPA)
        for b in range(8):
            bt.set_data(b, *data[b])
        t_b = per_iter([bt])
        singles = []
        for b in range(8):
            s1 = Solver([geo[b]], spec, kappa=BAGGAGE_KAPPA, **PLAIN)
            s1.set_data(0, *data[b])
            singles.append(s1)
        t_p = per_iter(singles)
        out[f"scan{n}_batched_over_plain"] = t_p / t_b
        out[f"scan{n}_batched_ms_per_iter"] = t_b
    return out


def stack_leg(n_slices, stream):
    """The mixed-precision stack: n_slices fan slices of 1024^2 with 1440 views and 2048 bins in one solver
    per storage format (one seeded slice's measurements on every slice: the kernels' work does not
    depend on the values), device ms per ADMM iteration after the initial image, against the plain
    single-slice FP32 solver on one slice, times n_slices; and the 16-bit formats' xi_p after the
    initial image and 10 iterations next to FP32's on that slice."""
    import torch

    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect
    from synth.workloads import BAGGAGE_KAPPA, MIXED_SEED_BASE, baggage_fan_case

    dev = torch.device("cuda", torch.cuda.current_device())
    c = baggage_fan_case(slice_index=MIXED_SEED_BASE, n=1024, n_views=1440, n_bins=2048)
    spec = Spectra.from_tables(c["spectra"])
    geo = Geometry(c["geom"])
    data = [torch.tensor(np.ascontiguousarray(c[k]), dtype=torch.float32, device=dev)
            for k in ("m_h", "m_l", "w_h", "w_l")]
    truth = torch.tensor(np.stack([c["truth_c"], c["truth_p"]]), dtype=torch.float32, device=dev)
    del c

    def per_iter(sol, iters):
        sol.reconstruct(0)
        sol.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol.step(iters)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / iters

    out = {"stack_slices": n_slices, "stack_workload": "fan 1024x1024, 1440 views x 2048 bins"}
    one = Solver([geo], spec, kappa=BAGGAGE_KAPPA, **PLAIN)
    one.set_data(0, *data)
    t_plain = per_iter(one, 3) * n_slices
    del one
    out["stack_plain_ms_per_iter"] = t_plain
    for name, code in (("f32", dect.STORE_F32), ("f16", dect.STORE_F16), ("bf16", dect.STORE_BF16)):
        sol = Solver([geo] * n_slices, spec, kappa=BAGGAGE_KAPPA, storage=code)
        for b in range(n_slices):
            sol.set_data(b, *data)
        sol.set_truth(0, truth)
        t = per_iter(sol, 3)
        sol.step(10 - 4)
        out[f"stack_{name}_ms_per_iter"] = t
        out[f"stack_{name}_over_plain"] = t_plain / t
        out[f"stack_{name}_xi_p_db_at_10"] = sol.stats(0)["xi_db"][1]
        del sol
        torch.cuda.empty_cache()
    return out


def uneven_leg(n_slices, stream):
    """The uneven-batch workload (seeded 256..1024 px, 360..1440 views, 512..2048 bins): one batched
    solver (graph, autotuned backprojector) against single-slice solvers in turn, plain (eager,
    occupancy view groups) and with graph and autotuner; device ms per ADMM iteration after the
    initial image."""
    import torch

    from paper_1905_00934_gb300 import Geometry, Solver, Spectra
    from synth.workloads import BAGGAGE_KAPPA, quick_fan_case, uneven_batch_shapes
    from concurrent.futures import ThreadPoolExecutor

    dev = torch.device("cuda", torch.cuda.current_device())
    shapes = uneven_batch_shapes(n_slices)
    with ThreadPoolExecutor(max_workers=16) as ex:
        cases = list(ex.map(lambda b: quick_fan_case(b, *shapes[b]), range(len(shapes))))
    spec = Spectra.from_tables(cases[0]["spectra"])
    geo = [Geometry(c["geom"]) for c in cases]
    data = [[torch.tensor(np.ascontiguousarray(c[k]), dtype=torch.float32, device=dev)
             for k in ("m_h", "m_l", "w_h", "w_l")] for c in cases]
    del cases
    iters = 5

    def timed(make_solvers):
        solvers = make_solvers()
        for s1 in solvers:
            s1.reconstruct(0)
            s1.step(1)  # graph capture outside the timing
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s1 in solvers:
            s1.step(iters)
        e1.record(stream)
        e1.synchronize()
        del solvers
        return e0.elapsed_time(e1) / iters

    def batched():
        s = Solver(geo, spec, kappa=BAGGAGE_KAPPA)
        for b in range(len(geo)):
            s.set_data(b, *data[b])
        return [s]

    def singles(params):
        def make():
            out = []
            for b in range(len(geo)):
                s1 = Solver([geo[b]], spec, kappa=BAGGAGE_KAPPA, **params)
                s1.set_data(0, *data[b])
                out.append(s1)
            return out
        return make

    t_b = timed(batched)
    t_p = timed(singles(PLAIN))
    t_g = timed(singles({"bp_tile": 32, "bp_cluster": -1}))
    return {"uneven_slices": len(geo), "uneven_batched_ms_per_iter": t_b, "uneven_plain_ms_per_iter": t_p,
            "uneven_plain_graph_autotuned_ms_per_iter": t_g, "uneven_batched_over_plain": t_p / t_b,
            "uneven_batched_over_plain_graph_autotuned": t_g / t_b}


def scheme_comparison(geo, spec, cases, dev_data, truths, gold, B, stream):
    """Time to the same PE error (slice 0's xi_p, checked every 5 iterations, against the oracle's value
    after the workload's iterations + 0.5 dB, up to twice the workload's iterations) for UDM1-PCG1 and
    the old splitting LM1 x CG1 on the same slices; and the one-pass CDM-FBP baseline."""
    import torch

    from paper_1905_00934_gb300 import Solver, cdm_fbp, dect
    from synth.workloads import BAGGAGE_KAPPA

    target = gold["xi_p"][ITERS] + 0.5
    out = {"cmp_target_xi_p_db": target}
    for name, scheme in (("udm", dect.SCHEME_UDM_PCG), ("lmcg", dect.SCHEME_LM_CG)):
        s2 = Solver(geo, spec, kappa=BAGGAGE_KAPPA, scheme=scheme)
        for b in range(B):
            s2.set_data(b, *dev_data[b])
            s2.set_truth(b, truths[b])
        s2.reconstruct(0)
        s2.step(5)  # graph capture outside the timing
        s2.reconstruct(0)
        torch.cuda.synchronize()
        t_ms, it, hit, xi_p = 0.0, 0, None, None
        while it < 2 * ITERS:
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            s2.step(5)
            c1.record(stream)
            c1.synchronize()
            t_ms += c0.elapsed_time(c1)
            it += 5
            xi_p = s2.stats(0)["xi_db"][1]
            if xi_p <= target:
                hit = it
                break
        out[f"cmp_{name}_iters_to_target"] = hit
        out[f"cmp_{name}_ms_to_target"] = t_ms if hit else None
        out[f"cmp_{name}_ms_per_iter"] = t_ms / it
        out[f"cmp_{name}_xi_p_db_at_stop"] = xi_p
        del s2
    cdm_fbp(geo[0], spec, *dev_data[0][:4], iters=CDM_ITERS)  # one-time per-geometry tables
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    xs = [cdm_fbp(geo[b], spec, *dev_data[b][:4], iters=CDM_ITERS) for b in range(B)]
    c1.record(stream)
    c1.synchronize()
    x0 = xs[0].cpu().numpy().astype(np.float64)
    xi = [float(20.0 * np.log10(np.linalg.norm(x0[k] - t) / np.linalg.norm(t)))
          for k, t in enumerate((cases[0]["truth_c"], cases[0]["truth_p"]))]
    out.update({"cmp_cdm_fbp_ms_per_slice": c0.elapsed_time(c1) / B, "cmp_cdm_fbp_xi_c_db": xi[0],
                "cmp_cdm_fbp_xi_p_db": xi[1]})
    gold_cdm = _golden(GOLDEN_CDM_FBP)
    if gold_cdm is not None and gold_cdm.get("decomposition_iterations") == CDM_ITERS:
        out["cmp_cdm_fbp_oracle_xi_p_db"] = gold_cdm["xi_p"]
    return out


def run_study(args):
    """The paper's evaluation protocol on the synthetic workload (Sec. 4, Fig. 2): xi_c, xi_p (Eq. 14,
    mean over the batch) every 10 iterations and the device time per iteration, for UDM(m)-PCG(n)
    variants (circulant preconditioner), with the plain ramp-filter preconditioner, with plain CG (no
    preconditioner) and the LM(m) x CG(n) splitting; and the one-pass CDM-FBP baseline."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect
    from synth.workloads import BAGGAGE_KAPPA, baggage_fan_case
    from concurrent.futures import ThreadPoolExecutor

    dev = torch.device("cuda", 0)
    B = args.batch
    with ThreadPoolExecutor(max_workers=min(B, 16)) as ex:
        cases = list(ex.map(lambda b: baggage_fan_case(slice_index=b), range(B)))
    geo = [Geometry(c["geom"]) for c in cases]
    spec = Spectra.from_tables(cases[0]["spectra"])
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    configs = [("UDM1-PCG1", dict(m_udm=1, n_pcg=1)), ("UDM1-PCG2", dict(m_udm=1, n_pcg=2)),
               ("UDM2-PCG1", dict(m_udm=2, n_pcg=1)), ("UDM1-PCG5", dict(m_udm=1, n_pcg=5)),
               ("UDM1-PCG1 CDM-FBP start", dict(m_udm=1, n_pcg=1, init=dect.INIT_CDM_FBP)),
               ("UDM1-PCG1 ramp", dict(m_udm=1, n_pcg=1, precondition=dect.PRECOND_RAMP)),
               ("UDM1-PCG5 ramp", dict(m_udm=1, n_pcg=5, precondition=dect.PRECOND_RAMP)),
               ("UDM1-CG1", dict(m_udm=1, n_pcg=1, precondition=0)),
               ("UDM1-CG5", dict(m_udm=1, n_pcg=5, precondition=0)),
               ("LM1xCG1", dict(m_udm=1, n_pcg=1, scheme=dect.SCHEME_LM_CG)),
               ("LM1xCG5", dict(m_udm=1, n_pcg=5, scheme=dect.SCHEME_LM_CG))]
    iters = args.study_iters
    rows = {}
    for name, params in configs:
        sol = Solver(geo, spec, kappa=BAGGAGE_KAPPA, **params)
        for b, c in enumerate(cases):
            sol.set_data(b, *[f32(c[k]) for k in ("m_h", "m_l", "w_h", "w_l")])
            sol.set_truth(b, f32(np.stack([c["truth_c"], c["truth_p"]])))
        sol.reconstruct(0)
        xi0 = np.mean([sol.stats(b)["xi_db"] for b in range(B)], axis=0)
        traj, t_ms = [(0, 0.0, float(xi0[0]), float(xi0[1]))], 0.0
        for k in range(iters // 10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sol.step(10)
            e1.record()
            e1.synchronize()
            t_ms += e0.elapsed_time(e1)
            xi = np.mean([sol.stats(b)["xi_db"] for b in range(B)], axis=0)
            traj.append((10 * (k + 1), round(t_ms, 2), round(float(xi[0]), 4), round(float(xi[1]), 4)))
        rows[name] = {"ms_per_iteration": t_ms / iters, "params": params,
                      "xi": traj, "best_xi_p_db": min(r[3] for r in traj)}
        del sol
    # the paper's baseline (i), CDM-FBP: one pass, no iterations
    from paper_1905_00934_gb300 import cdm_fbp

    data = [[f32(c[k]) for k in ("m_h", "m_l", "w_h", "w_l")] for c in cases]
    cdm_fbp(geo[0], spec, *data[0], iters=CDM_ITERS)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    xs = [cdm_fbp(geo[b], spec, *data[b], iters=CDM_ITERS) for b in range(B)]
    e1.record()
    e1.synchronize()
    xi = np.mean([[20.0 * np.log10(np.linalg.norm(xs[b][k].cpu().numpy().astype(np.float64) - t) / np.linalg.norm(t))
                   for k, t in enumerate((cases[b]["truth_c"], cases[b]["truth_p"]))] for b in range(B)], axis=0)
    rows["CDM-FBP"] = {"ms_per_slice": e0.elapsed_time(e1) / B, "decomposition_iterations": CDM_ITERS,
                       "xi_c_db": float(xi[0]), "xi_p_db": float(xi[1])}
    print(json.dumps({"study": "xi vs iteration and time, mean over the batch", "batch": B,
                      "workload": "fan beam 512x512, 720 views x 1024 bins", "trajectories": rows}), flush=True)
    return 0


def run_uneven(args):
    """Batching on the uneven-slice workload: one batched solver against the plain form (single-slice
    solvers one after another, eager launches, occupancy view groups) and single-slice solvers with
    graph and autotuner, as device time per ADMM iteration (after the initial image, CUDA events)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra
    from synth.workloads import BAGGAGE_KAPPA, quick_fan_case, uneven_batch_shapes
    from concurrent.futures import ThreadPoolExecutor

    dev = torch.device("cuda", 0)
    shapes = uneven_batch_shapes(args.uneven)
    with ThreadPoolExecutor(max_workers=16) as ex:
        cases = list(ex.map(lambda b: quick_fan_case(b, *shapes[b]), range(len(shapes))))
    spec = Spectra.from_tables(cases[0]["spectra"])
    geo = [Geometry(c["geom"]) for c in cases]
    data = [[torch.tensor(np.ascontiguousarray(c[k]), dtype=torch.float32, device=dev)
             for k in ("m_h", "m_l", "w_h", "w_l")] for c in cases]
    iters = 10

    def timed(solvers):
        for s in solvers:
            s.reconstruct(0)
            s.step(2)  # graph capture outside the timing
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in solvers:
            s.step(iters)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / iters

    out = {}
    batched = Solver(geo, spec, kappa=BAGGAGE_KAPPA)
    for b in range(len(cases)):
        batched.set_data(b, *data[b])
    out["batched_ms_per_iteration"] = timed([batched])
    del batched
    for name, params in (("plain", dict(use_graph=0, bp_view_groups=-1)), ("plain_graph_autotuned", {})):
        singles = []
        for b in range(len(cases)):
            s1 = Solver([geo[b]], spec, kappa=BAGGAGE_KAPPA, **params)
            s1.set_data(0, *data[b])
            singles.append(s1)
        out[name + "_ms_per_iteration"] = timed(singles)
        del singles
    out["batched_over_plain"] = out["plain_ms_per_iteration"] / out["batched_ms_per_iteration"]
    out["batched_over_plain_graph_autotuned"] = (out["plain_graph_autotuned_ms_per_iteration"]
                                                 / out["batched_ms_per_iteration"])
    print(json.dumps({"uneven_batch": {"slices": len(cases), "shapes_n_views_bins": shapes, "iterations_timed": iters,
                                       **out}}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--impl", default="dect", choices=["dect", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage of the sinogram vectors and projector textures (arithmetic stays f32/f64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparison", action="store_true",
                    help="skip the time-to-target comparison with the LM x CG splitting")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain forms, the 16-bit arms, the slice-size scan and the uneven batch")
    ap.add_argument("--stack-slices", type=int, default=128,
                    help="slices of the 1024^2 mixed-precision stack leg of the bench line (0 skips it)")
    ap.add_argument("--uneven-slices", type=int, default=64,
                    help="slices of the uneven-batch leg of the bench line (0 skips it)")
    ap.add_argument("--bp-view-groups", type=int, default=0,
                    help="backprojector view groups per tile (0: autotuned, -1: occupancy rule)")
    ap.add_argument("--bp-tile", type=int, default=0, help="backprojector tile side, 32 or 64 (0: autotuned)")
    ap.add_argument("--bp-cluster", type=int, default=0, help="1 cluster form, -1 plain form, 0 autotuned")
    ap.add_argument("--bp-slices", type=int, default=0, help="slices per backprojector CTA, 1 or 2 (0: autotuned)")
    ap.add_argument("--proj-views", type=int, default=0, help="views per projector CTA, 2, 4 or 8 (0: autotuned)")
    ap.add_argument("--bp-reduce", type=int, default=0,
                    help="-1: the finalize pass sums the view groups' partial images; 0/1: the last CTA of a tile does")
    ap.add_argument("--profile-run", type=int, default=0, metavar="ITERS",
                    help="set up the workload, run one untimed reconstruction of ITERS iterations and exit "
                         "(for profiler captures; prints no bench line)")
    ap.add_argument("--study", action="store_true",
                    help="print xi trajectories of UDM-PCG variants, plain CG and LM x CG instead of the bench line")
    ap.add_argument("--study-iters", type=int, default=200)
    ap.add_argument("--uneven", type=int, default=0, metavar="SLICES",
                    help="batched vs plain on SLICES seeded uneven fan slices (256..1024 px, 360..1440 views, "
                         "512..2048 bins), per ADMM iteration")
    args = ap.parse_args()
    if args.study:
        return run_study(args)
    if args.uneven:
        return run_uneven(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_dect(args)


if __name__ == "__main__":
    sys.exit(main())
