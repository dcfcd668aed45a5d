"""Writes the stored expected values of the benchmark's quality gate using the FP64 oracle only.

The benchmark's metric is slices/s to a fixed photoelectric-image error: the error
xi_p (Eq. 14) that the FP64 oracle reaches after the workload's iteration count on
the same seeded slice. This script runs the oracle (initial image + 100 ADMM
iterations of UDM1-PCG1 on the 512x512, 720-view, 1024-bin fan-beam slice) and
stores xi_c, xi_p per iteration in baggage_fan_512_xi.json.

Usage: python tests/golden/make_golden.py [--iters 100]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import _clib, admm  # noqa: E402
from synth.workloads import BAGGAGE_E_REF_KEV, BAGGAGE_KAPPA, baggage_fan_case  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--out", default=os.path.join(HERE, "baggage_fan_512_xi.json"))
    args = ap.parse_args()
    c = baggage_fan_case(e_ref_kev=BAGGAGE_E_REF_KEV)
    P = admm.Params(kappa=BAGGAGE_KAPPA)
    prob = admm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], P)
    t0 = time.time()
    xc0, xp0 = admm.initial_image(prob)
    st = admm.state_from_image(prob, xc0, xp0)
    hist = [[admm.xi_db(xc0, c["truth_c"]), admm.xi_db(xp0, c["truth_p"])]]
    rho = []
    for it in range(args.iters):
        st = admm.admm_iteration(prob, st)
        hist.append([admm.xi_db(st.x[0], c["truth_c"]), admm.xi_db(st.x[1], c["truth_p"])])
        rho.append(list(st.rho))
        print(it + 1, hist[-1], st.rho, flush=True)
    out = {
        "what": "FP64 oracle xi (Eq. 14, dB) per ADMM iteration, UDM1-PCG1, fan-beam 512x512, 720 views, "
                "1024 bins, seed 1905, I0 2e5, E_ref 100 keV, kappa 0.25; entry 0 is the initial image",
        "iterations": args.iters,
        "xi_c": [h[0] for h in hist],
        "xi_p": [h[1] for h in hist],
        "rho": rho,
        "oracle_seconds": time.time() - t0,
        "oracle_threads": _clib.num_threads(),
    }
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
