"""Writes tests/golden/cfg2_oracle_run.json: the oracle's own run of the
benchmark workload (PDF-like, n = 3000, m = 2000, k = 4, 1e-3 relative noise,
data seed 0, the U[0,1] start of seed 0) to relative KKT 1e-8 -- Alg. "anls"
(Sec. 2) with the Sec. 5.1 stopping test in the relative form used
throughout.  It calls only oracle/ (and synth/ for the inputs) and takes
about half an hour on one core:

    python tests/golden/make_cfg2_reference.py

Stored: the sweep count, f, E_abs and relative KKT of the final iterate,
the passive sets of every column and row (hex), and every 250th point of the
trace, which shows how slowly f still falls at relative KKT ~ 1e-8.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

N, M_COLS, K, NOISE, SEED, TARGET, CAP = 3000, 2000, 4, 1e-3, 0, 1e-8, 40000


def main():
    M, _, _ = synth.pdf_like(N, M_COLS, K, noise=NOISE, relative=True, seed=SEED)
    X0, Y0 = synth.init_factors(N, M_COLS, K, seed=SEED)
    X, Y, xm, ym, sweeps, tr, st = oracle.anls(M, X0, Y0, max_sweeps=CAP, kkt_target=TARGET, want_trace=True)
    assert st == oracle.OK, st
    out = {"workload": "PDF-like n=%d m=%d k=%d, %g relative noise, data seed %d, U[0,1] start seed %d"
                       % (N, M_COLS, K, NOISE, SEED, SEED),
           "target_kkt_rel": TARGET, "sweeps": int(sweeps),
           "f": float(tr[-1, 0]), "E_abs": float(tr[-1, 1]), "kkt_rel": float(tr[-1, 2]),
           "ymask_hex": ["%x" % int(v) for v in ym], "xmask_hex": ["%x" % int(v) for v in xm],
           "trace_every_250": [[i] + [float(v) for v in tr[i, :3]] for i in range(0, len(tr), 250)]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_oracle_run.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print("wrote %s: %d sweeps, f %.15e, rel KKT %.3e" % (path, sweeps, out["f"], out["kkt_rel"]))


if __name__ == "__main__":
    main()
