"""Writes the FP64 oracle reference for the mixed-precision workload (4-slice subset) using oracle/ only.

Workload: fan-beam slices of 1024 x 1024 pixels, 1440 views, 2048 bins (seeded baggage phantoms,
I0 2e5), UDM1-PCG1 for 100 ADMM iterations from the oracle's initial image. Stored per slice:
xi_c, xi_p (Eq. 14) every 10 iterations, and the final Compton and PE values at 2048 seeded pixel
positions each, so the GPU runs (float32 / float16 / bfloat16 storage) can be compared with the
oracle pixel by pixel without storing whole images.

With --early K it instead writes mixed_1024_early.json: for each slice, the sampled pixels after the
initial image and after each of the first K iterations, from float32-rounded measurements (the
values the GPU receives), for a pixel-by-pixel comparison before float32 rounding of the per-ray
decisions has had time to accumulate.

With --from-x0 it writes mixed_1024_from_x0.json for slice 0: float32-rounded measurements and the
oracle's initial image rounded to float32 (both as the GPU receives them), then xi every 10
iterations and the sampled pixels after iterations 10, 20, 50 and 100, so a GPU run started from the
same image can be compared pixel by pixel at several depths of the trajectory.

Usage: python tests/golden/make_golden_mixed.py [--slices 4] [--iters 100] [--early K] [--from-x0]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import _clib, admm  # noqa: E402
from synth.workloads import BAGGAGE_KAPPA, MIXED_SEED_BASE, baggage_fan_case  # noqa: E402

N, VIEWS, BINS = 1024, 1440, 2048
SAMPLES = 2048


def sample_pixels(slice_index: int):
    rng = np.random.Generator(np.random.PCG64(MIXED_SEED_BASE + 500 + slice_index))
    return rng.integers(0, N * N, SAMPLES)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--slices", type=int, default=4)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--early", type=int, default=-1)
    ap.add_argument("--from-x0", action="store_true")
    args = ap.parse_args()
    if args.early >= 0:
        return early(args)
    if args.from_x0:
        return from_x0(args)
    args.out = args.out or os.path.join(HERE, "mixed_1024_oracle.json")
    out = {"what": "FP64 oracle, UDM1-PCG1, fan beam 1024x1024, 1440 views, 2048 bins, E_ref 100 keV, kappa 0.25; "
                   "xi every 10 iterations (entry 0 = initial image) and final x at seeded pixels",
           "iterations": args.iters, "slices": []}
    for s in range(args.slices):
        t0 = time.time()
        c = baggage_fan_case(slice_index=MIXED_SEED_BASE + s, n=N, n_views=VIEWS, n_bins=BINS)
        prob = admm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"],
                            admm.Params(kappa=BAGGAGE_KAPPA))
        xc0, xp0 = admm.initial_image(prob)
        st = admm.state_from_image(prob, xc0, xp0)
        xi = [[admm.xi_db(xc0, c["truth_c"]), admm.xi_db(xp0, c["truth_p"])]]
        for it in range(args.iters):
            st = admm.admm_iteration(prob, st)
            if (it + 1) % 10 == 0:
                xi.append([admm.xi_db(st.x[0], c["truth_c"]), admm.xi_db(st.x[1], c["truth_p"])])
                print(s, it + 1, xi[-1], flush=True)
        idx = sample_pixels(s)
        out["slices"].append({"slice_index": MIXED_SEED_BASE + s, "xi": xi, "pixels": idx.tolist(),
                              "x_c": st.x[0].ravel()[idx].tolist(), "x_p": st.x[1].ravel()[idx].tolist(),
                              "norm_x_c": float(np.linalg.norm(st.x[0])), "norm_x_p": float(np.linalg.norm(st.x[1])),
                              "seconds": time.time() - t0})
        with open(args.out, "w") as f:
            json.dump(out, f)
    out["oracle_threads"] = _clib.num_threads()
    with open(args.out, "w") as f:
        json.dump(out, f)


def early(args):
    out_path = args.out or os.path.join(HERE, "mixed_1024_early.json")
    out = {"what": "FP64 oracle from float32-rounded measurements, fan beam 1024x1024, 1440 views, 2048 bins, "
                   "E_ref 100 keV, kappa 0.25: sampled x after the initial image (entry 0) and after each of the "
                   "first iterations", "iterations": args.early, "slices": []}
    for s in range(args.slices):
        c = baggage_fan_case(slice_index=MIXED_SEED_BASE + s, n=N, n_views=VIEWS, n_bins=BINS)
        meas = [np.float32(c[k]).astype(np.float64) for k in ("m_h", "m_l", "w_h", "w_l")]
        prob = admm.Problem(c["geom"], c["spectra"], *meas, admm.Params(kappa=BAGGAGE_KAPPA))
        xc0, xp0 = admm.initial_image(prob)
        st = admm.state_from_image(prob, xc0, xp0)
        idx = sample_pixels(s)
        xs = [[xc0.ravel()[idx].tolist(), xp0.ravel()[idx].tolist()]]
        for _ in range(args.early):
            st = admm.admm_iteration(prob, st)
            xs.append([st.x[0].ravel()[idx].tolist(), st.x[1].ravel()[idx].tolist()])
        out["slices"].append({"slice_index": MIXED_SEED_BASE + s, "pixels": idx.tolist(), "x": xs})
        print(s, "done", flush=True)
    with open(out_path, "w") as f:
        json.dump(out, f)


FROM_X0_CHECKPOINTS = (10, 20, 50, 100)


def from_x0(args):
    out_path = args.out or os.path.join(HERE, "mixed_1024_from_x0.json")
    c = baggage_fan_case(slice_index=MIXED_SEED_BASE, n=N, n_views=VIEWS, n_bins=BINS)
    meas = [np.float32(c[k]).astype(np.float64) for k in ("m_h", "m_l", "w_h", "w_l")]
    prob = admm.Problem(c["geom"], c["spectra"], *meas, admm.Params(kappa=BAGGAGE_KAPPA))
    x0 = np.float32(np.stack(admm.initial_image(prob))).astype(np.float64)
    st = admm.state_from_image(prob, x0[0], x0[1])
    idx = sample_pixels(0)
    out = {"what": "FP64 oracle from float32-rounded measurements and its own initial image rounded to float32, "
                   "fan beam 1024x1024, 1440 views, 2048 bins, E_ref 100 keV, kappa 0.25, UDM1-PCG1: xi every 10 "
                   "iterations (entry 0 = start) and sampled x after the listed iterations",
           "slice_index": MIXED_SEED_BASE, "pixels": idx.tolist(), "checkpoints": list(FROM_X0_CHECKPOINTS),
           "xi": [[admm.xi_db(x0[0], c["truth_c"]), admm.xi_db(x0[1], c["truth_p"])]], "x": {}}
    for it in range(1, max(FROM_X0_CHECKPOINTS) + 1):
        st = admm.admm_iteration(prob, st)
        if it % 10 == 0:
            out["xi"].append([admm.xi_db(st.x[0], c["truth_c"]), admm.xi_db(st.x[1], c["truth_p"])])
            print(it, out["xi"][-1], flush=True)
        if it in FROM_X0_CHECKPOINTS:
            out["x"][str(it)] = [st.x[0].ravel()[idx].tolist(), st.x[1].ravel()[idx].tolist()]
            with open(out_path, "w") as f:
                json.dump(out, f)
    out["oracle_threads"] = _clib.num_threads()
    with open(out_path, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
