"""Writes tests/golden/plain_fp64_2000x1500_k20.json from the FP64 oracle only.

The file pins the oracle's own output on the plain FP64 workload (2000 x 1500,
rank 20 + N(0, 1e-6) noise, k = 20, 5 k-means iterations, seed 1607) so that an
unintended change to the oracle shows up as a diff. Run from the repository
root: ``python tests/golden/make_golden.py``.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cabs_ref as o  # noqa: E402
from workloads import synth  # noqa: E402


def main():
    A = synth.plain_lowrank()
    out = {}
    for mode in ("pinv", "stabilized"):
        r = o.cabs(o.DenseSource(A), k1=20, iters=5, seed=1607, mode=mode)
        out[mode] = dict(
            pilot_rows=r.pilot_rows.tolist(), pilot_cols=r.pilot_cols.tolist(),
            pilot_rows_drawn=r.pilot_rows_drawn.tolist(), pilot_cols_drawn=r.pilot_cols_drawn.tolist(),
            rows=r.rows.tolist(), cols=r.cols.tolist(),
            pilot_err=o.rel_fro_error_dense(A, r.pilot.U, r.pilot.S, r.pilot.V),
            final_err=o.rel_fro_error_dense(A, r.final.U, r.final.S, r.final.V),
            final_S=r.final.S.tolist(), energy_rows=r.km_rows.energy, energy_cols=r.km_cols.energy)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plain_fp64_2000x1500_k20.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
