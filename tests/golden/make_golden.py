"""Writes the fixtures of tests/golden/ from the CPU oracle alone (test
infrastructure: nothing here is used by the library).

config1_L16_series.txt -- 2D Ising ferromagnet L = 16, beta = 0.4406868,
    all-up start, Philox seed 1, instance 0, replica 0 (the 10^4-sweep series
    workload): E (Eq. (7)) and M after each of the first 500 checkerboard
    Metropolis sweeps (Sec. 3.1, Eq. (8); the per-site Philox counters of
    Sec. 4 in the mapping the oracle documents).
pa_L8_R2000.txt -- population annealing (Sec. 5.4, Eq. (13)) of the 2D Ising
    ferromagnet L = 8, R = 2000, beta_i = i/40 (i = 0..40), theta = 3 sweeps
    per temperature, Philox seed 6, instance 0: per step beta_i, the exact
    population sum of E and ln Z_i = N ln 2 + sum_k ln Q_k.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

SERIES = dict(L=16, beta=0.4406868, seed=1, sweeps=500)
PA = dict(L=8, R=2000, S=40, theta=3, seed=6)


def series():
    s = oracle.init_spins(2, SERIES["L"], SERIES["seed"], 0, 0, False)
    rows = []
    for t in range(SERIES["sweeps"]):
        oracle.sweeps(2, SERIES["L"], s, None, SERIES["beta"], SERIES["seed"], 0, 0, t, 1)
        rows.append(oracle.observables(2, SERIES["L"], s))
    return rows


def pa():
    betas = oracle.linear_betas(1.0, PA["S"])
    r = oracle.pa_run(2, PA["L"], PA["seed"], 0, PA["R"], betas, PA["theta"])
    return [(float(b), int(e), float(z)) for b, e, z in zip(r["betas"], r["sumE"], r["lnZ"])]


def main():
    with open(os.path.join(HERE, "config1_L16_series.txt"), "w") as f:
        f.write("# 2D Ising L=16, beta=0.4406868, all-up, Philox seed 1, instance 0, replica 0\n")
        f.write("# E and M after sweep t (Sec. 3.1, Eqs. (7), (8)); written by make_golden.py from the oracle\n")
        f.write("# t E M\n")
        for t, (E, M) in enumerate(series()):
            f.write("%d %d %d\n" % (t, E, M))
    with open(os.path.join(HERE, "pa_L8_R2000.txt"), "w") as f:
        f.write("# population annealing 2D Ising L=8, R=2000, beta_i=i/40, theta=3, Philox seed 6, instance 0\n")
        f.write("# per step: beta_i, sum of E over the population, ln Z_i (Sec. 5.4, Eq. (13)); "
                "written by make_golden.py from the oracle\n")
        f.write("# i beta sumE lnZ\n")
        for i, (b, e, z) in enumerate(pa()):
            f.write("%d %.17g %d %.17g\n" % (i, b, e, z))


if __name__ == "__main__":
    main()
