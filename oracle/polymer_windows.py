"""Writes paper_1312_2213_gb300/polymer_windows.json: the multicanonical energy window of the
bead-spring polymer for each chain length.  Calls only oracle/.

The paper restricts the polymer run to "an energy range around the collapse transition" without
giving numbers.  Reading used here: canonical Metropolis pilots (oracle, 8 walkers, seeded) at
T = 1.5 (coil) and T = 0.3 (globule); E_hi = <E>_{1.5} + 2 sigma, E_lo = <E>_{0.3} - 2 sigma,
both rounded outward to the 0.1 bin grid.

Usage: python oracle/polymer_windows.py [sweeps]
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


def pilot(N, T, sweeps, seed):
    r = oracle.PolyRun(N, 8, seed, -1e6, 1e6, beta=1.0 / T)
    r.init()
    chunks, samples = 20, []
    for c in range(chunks):
        r.iterate(max(1, sweeps // chunks), os.cpu_count() or 1)
        if c >= chunks // 2:
            samples.extend(r.energy().tolist())
    return float(np.mean(samples)), float(np.std(samples))


def main():
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
