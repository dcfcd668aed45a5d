"""Writes the stored xi of the comparison method CDM-FBP (Sec. 2, Sec. 4) on the benchmark's slice,
using the FP64 oracle only (oracle/fbp.py: per-ray decomposition with rho = 0, a >= 0, FBP).

Usage: python tests/golden/make_golden_cdm_fbp.py [--iters 20]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import _clib, admm, fbp  # noqa: E402
from synth.workloads import BAGGAGE_E_REF_KEV, baggage_fan_case  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--out", default=os.path.join(HERE, "baggage_fan_512_cdm_fbp.json"))
    args = ap.parse_args()
    c = baggage_fan_case(e_ref_kev=BAGGAGE_E_REF_KEV)
    t0 = time.time()
    xc, xp = fbp.cdm_fbp(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], args.iters)
    out = {
        "what": "FP64 oracle CDM-FBP on the fan-beam 512x512, 720-view, 1024-bin slice (seed 1905, I0 2e5, "
                "E_ref 100 keV): xi (Eq. 14, dB) of the Compton and PE images",
        "decomposition_iterations": args.iters,
        "xi_c": admm.xi_db(xc, c["truth_c"]),
        "xi_p": admm.xi_db(xp, c["truth_p"]),
        "oracle_seconds": time.time() - t0,
        "oracle_threads": _clib.num_threads(),
    }
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
