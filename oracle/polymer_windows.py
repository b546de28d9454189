"""Writes paper_1312_2213_gb300/polymer_windows.json: the multicanonical energy window of the
bead-spring polymer for each chain length.  Calls only oracle/.

The paper restricts the polymer run to "an energy range around the collapse transition" without
giving numbers.  Reading used here: canonical Metropolis pilots (oracle, 8 walkers, seeded) at
T = 1.5 (coil) and T = 0.3 (globule); E_hi = <E>_{1.5} + 2 sigma, E_lo = <E>_{0.3} - 2 sigma,
both rounded outward to the 0.1 bin grid.

Usage: python oracle/polymer_windows.py [sweeps]
       python oracle/polymer_windows.py --paper-model [sweeps]   (model 1, N = 40 and 80)
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(HERE), "paper_1312_2213_gb300", "polymer_windows.json")


def pilot(N, T, sweeps, seed, model=0):
    r = oracle.PolyRun(N, 8, seed, -1e6, 1e6, beta=1.0 / T, model=model)
    r.init()
    chunks, samples = 20, []
    for c in range(chunks):
        r.iterate(max(1, sweeps // chunks), os.cpu_count() or 1)
        if c >= chunks // 2:
            samples.extend(r.energy().tolist())
    return float(np.mean(samples)), float(np.std(samples))


def window(N, sweeps, model):
    hi_m, hi_s = pilot(N, 1.5, sweeps, 100 + N, model)
    lo_m, lo_s = pilot(N, 0.3, sweeps, 200 + N, model)
    e_lo = math.floor((lo_m - 2 * lo_s) * 10) / 10
    e_hi = math.ceil((hi_m + 2 * hi_s) * 10) / 10
    return {"e_lo": e_lo, "e_hi": e_hi, "pilot": {"T1.5": [hi_m, hi_s], "T0.3": [lo_m, lo_s]}}


def main_paper_model(sweeps):
    """Model 1 (the paper's parameters of Eq. 7) at its chain lengths N = 40, 80: merged into the
    existing file under "paper_model"."""
    out = json.load(open(OUT))
    pm = {"reading": "model 1 (FENE K = 40, r0 = 0.7, r_max = 1; LJ sigma = 2^(-1/6) r0, no cutoff); same "
                     "pilot rule, %d sweeps" % sweeps, "windows": {}}
    for N in (40, 80):
        pm["windows"][str(N)] = window(N, sweeps, 1)
        print(N, pm["windows"][str(N)], flush=True)
    out["paper_model"] = pm
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


def main():
    if "--paper-model" in sys.argv:
        args = [a for a in sys.argv[1:] if a != "--paper-model"]
        return main_paper_model(int(args[0]) if args else 10000)
    sweeps = int(sys.argv[1]) if len(sys.argv) > 1 else 10000
    out = {"reading": "E_lo = <E>_{T=0.3} - 2 sigma, E_hi = <E>_{T=1.5} + 2 sigma (canonical oracle pilots, "
                      "8 walkers, %d sweeps, second half averaged), rounded outward to 0.1" % sweeps,
           "fene_K": 40.0, "fene_R": 1.5, "lj_cutoff": 2.5, "bin_width": 0.1, "windows": {}}
    for N in (13, 32, 64, 128):
        hi_m, hi_s = pilot(N, 1.5, sweeps, 100 + N)
        lo_m, lo_s = pilot(N, 0.3, sweeps, 200 + N)
        e_lo = math.floor((lo_m - 2 * lo_s) * 10) / 10
        e_hi = math.ceil((hi_m + 2 * hi_s) * 10) / 10
        out["windows"][str(N)] = {"e_lo": e_lo, "e_hi": e_hi, "pilot": {"T1.5": [hi_m, hi_s], "T0.3": [lo_m, lo_s]}}
        print(N, out["windows"][str(N)], flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
