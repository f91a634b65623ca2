"""Runs the trace cases of the precision contract on whichever engine
library the process loads (MC_STRICT=1: the IEEE-strict build) and saves the
raw traces to the .npz named on the command line. Used by
tests/test_gpu_trace_precision.py."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5
N_TRACE = 4096
# (name, phase, tau, mu_a, run keywords): every optical depth of the sweep,
# Mie table and H-G, plus absorption with roulette inside the 32 events
CASES = [("mie-tau%g" % t, "table", t, 0.0, {}) for t in (1.0, 2.0, 5.0, 10.0, 20.0)] + \
        [("hg-tau%g" % t, "hg", t, 0.0, {}) for t in (1.0, 5.0, 20.0)] + \
        [("mie-tau20-absorb", "table", 20.0, 0.08, dict(rr_threshold=0.02)),
         ("hg-tau20-absorb", "hg", 20.0, 0.08, dict(rr_threshold=0.02))]


def main(out):
    import paper_2507_23189_gb300 as E
    tab = E.PhaseTable(5.0, 1.59, 1.33, 532.0, 4096)
    res = {}
    for name, phase, tau, mu_a, kw in CASES:
        med = E.Medium(tau / LX - mu_a, mu_a, phase, tab.info["g"], tab)
        e = E.Engine(E.Camera(64, 64, 128, R_MAX), E.Geometry(LX, LY, LZ))
        res[name] = e.trace(med, N_TRACE, N_TRACE, 32, seed=11, **kw).cpu().numpy()
        e.check()
    res["library"] = np.array(os.path.basename(E.lib()._name))
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
