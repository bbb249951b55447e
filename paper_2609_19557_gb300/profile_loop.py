"""Profiling driver: one persistent trial-loop launch (k_trials) running a
fixed number of accepted trials of the first inner solve on the large
synthetic workload (n = 1e6, m = 5e5 by default).  The periodic checks are
switched off (k_chk = 1e9) and the accepted-iteration budget equals the trial
count, so the first k_trials launch of the process does exactly that work;
profile it with `-k regex:k_trials -s 0 -c 1`.

    python -m paper_2609_19557_gb300.profile_loop --trials 200 --precision 32
"""
import argparse
import json
import time

from . import instances as I
from . import pdnqp as P


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=500_000)
    ap.add_argument("--trials", type=int, default=200)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    a = ap.parse_args()
    P.load()
    inst = I.large_qp(0, n=a.n, m=a.m)
    h = P.create_from_instance(inst, precision=a.precision)
    P.pdnqp_set_param(h, "k_chk", 1e9)
    P.pdnqp_set_param(h, "iter_budget", a.trials)
    t = time.time()
    st = P.pdnqp_solve(h, 1e-4, 1e-4)
    wall = time.time() - t
    _, _, r = P.pdnqp_get(h)
    lt = max(1, r["loop_trials"])
    print(json.dumps({"status": P.STATUS_NAMES[st], "trials": r["trials"], "loop_trials": r["loop_trials"],
                      "loop_us_per_trial": 1e6 * r["loop_seconds"] / lt,
                      "phase_us_per_trial": [1e6 * v / lt for v in r["loop_phase_seconds"]],
                      "wall_s": wall, "loop_blocks": r["loop_blocks"]}))
    h.close()


if __name__ == "__main__":
    main()
