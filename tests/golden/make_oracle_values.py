"""Write the stored expected values of the large parity cases (FP64 oracle only).

Each case is a seeded workload decoded by the same-chi FP64 sweep of the oracle
(oracle/su.py, Sec. 4 of the paper).  The GPU tests regenerate the same detector bits from
the seeded stream (td_inputs) and compare element by element.  Run from the repository
root:  python tests/golden/make_oracle_values.py [--jobs N]
The oracle takes about 1 s (rotated d = 9, chi = 8), 5 s (chi = 16) and several minutes
(chi = 32) per shot; the cases are split over N spawned processes (--only NAME: one case).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))

# name -> (workload, builder arguments, seed, shots, chi, chi_mps)
CASES = {
    "rotated_d9_r9_p0.03_chi8_mps8": ("rotated", (9, 9, 0.03, 0.03), 2000, 64, 8, 8),
    "rotated_d9_r9_p0.03_chi16_mps16": ("rotated", (9, 9, 0.03, 0.03), 2000, 64, 16, 16),
    "point_d7_p0.1_chi16_mps8": ("point", (7, 0.1), 4007, 48, 16, 8),
    "rotated_d9_r9_p0.03_chi32_mps8": ("rotated", (9, 9, 0.03, 0.03), 2000, 4, 32, 8),
}


def make_dem(kind, args):
    from td_inputs import point_sector_3d, rotated_phenomenological
    return rotated_phenomenological(*args) if kind == "rotated" else point_sector_3d(*args)


def _one(job):
    name, b = job
    from oracle import su
    from td_inputs import sample_shots
    kind, args, seed, _, chi, chi_mps = CASES[name]
    dem = make_dem(kind, args)
    det, _ = sample_shots(dem, 1, seed=seed, first_shot=b)
    return name, b, su.su_logprob(dem, det, chi=chi, chi_mps=chi_mps)[0]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    names = [n for n in CASES if a.only is None or n == a.only]
    jobs = [(n, b) for n in names for b in range(CASES[n][3])]
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    out = {n: np.zeros((CASES[n][3], 2)) for n in names}
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        for name, b, lp in pool.imap_unordered(_one, jobs):
            out[name][b] = lp
    for n in names:
        kind, args, seed, shots, chi, chi_mps = CASES[n]
        np.savez(os.path.join(HERE, n + ".npz"), logp=out[n], kind=kind, args=np.array(args, dtype=float),
                 seed=seed, shots=shots, chi=chi, chi_mps=chi_mps)
        print(n, out[n][:2])


if __name__ == "__main__":
    main()
