"""Write pm128_run.txt: the FP64 oracle's whole run of the 128^3 workload
(128^3 particles and mesh, 1000 Mpc/h, P(k) ~ k^-1.5 exp(-k^2/2k_c^2),
k_c = k_Ny/2, seed 1, 100 steps uniform in a from 0.02 to 1, shrinking with
the lightcone; the paper's step order, Table 2, and its final P(k)
comparison, Sec. 3).  Calls only oracle/ and the seeded input generator.

    python tests/golden/make_pm128_run.py      # about 10 minutes on one core

Contents (whitespace-separated text):
  n_active  <100 ints>          active particles at the start of each step
  n_lightcone <int>             catalogue size at the end
  pk <bin> <k h/Mpc> <P (Mpc/h)^3> <modes>   oracle.pk.power_spectrum of the
                                lightcone records plus the survivors, wrapped
                                into the box, n/2 linear bins
  rec <id> <a_cross> <x> <y> <z>  a seeded sample of 4096 particle ids:
                                a_cross of their lightcone record (0 for a
                                survivor) and the recorded position (cells)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cosmology as cz  # noqa: E402
from oracle import pm as opm  # noqa: E402
from oracle.pk import power_spectrum as opk  # noqa: E402
from paper_1709_04703_gb300 import ics  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pm128_run.txt")
N_SAMPLE = 4096


def main():
    cfg = ics.WORKLOADS["pm128"]
    n = cfg["n"]
    pos, mom, ids = ics.workload_ics("pm128")
    sched = cz.schedule(n, cfg["box"], ics.OMEGA_M, ics.OMEGA_L, cfg["a_init"],
                        cfg["a_final"], cfg["steps"])
    out = opm.run(pos, mom, ids, sched, n, ics.OMEGA_M, 1.0)
    allx = np.concatenate([out["pos"], out["lc_pos"]]) % n
    k, p, modes = opk(allx, n, cfg["box"], n // 2)
    sample = np.sort(np.random.default_rng(0).choice(n**3, N_SAMPLE, replace=False))
    rec_id = np.concatenate([out["ids"], out["lc_ids"]])
    rec_a = np.concatenate([np.zeros(len(out["ids"])), out["lc_a"]])
    rec_x = np.concatenate([out["pos"], out["lc_pos"]])
    where = np.empty(n**3, dtype=np.int64)
    where[rec_id] = np.arange(len(rec_id))
    lines = ["# FP64 oracle run of the 128^3 workload; written by make_pm128_run.py "
             "(calls oracle/ only)",
             "n_active " + " ".join(str(int(v)) for v in out["n_active"]),
             f"n_lightcone {len(out['lc_ids'])}"]
    for b in range(len(k)):
        lines.append(f"pk {b} {k[b]:.17g} {p[b]:.17g} {int(modes[b])}")
    for i in sample:
        j = where[i]
        x = rec_x[j]
        lines.append(f"rec {i} {rec_a[j]:.17g} {x[0]:.17g} {x[1]:.17g} {x[2]:.17g}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
