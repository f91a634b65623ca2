"""Runs a fixed set of small workloads on whichever engine library the
process loads (MC_CHECKED=1: the index-checked build) and saves every raw
tally and the error words to the .npz named on the command line. Used by
tests/test_gpu_checked.py."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(out):
    import torch
    import paper_2507_23189_gb300 as E
    from paper_2507_23189_gb300 import workloads as W
    res = {}
    tab = E.PhaseTable()
    paper = E.PaperTable(n_theta=3000)
    cases = [("table_band", E.Medium(5 / 45.0, 0.002, "table", 0.0, tab), E.Geometry(), E.Camera(256, 256), {}),
             ("table_global", E.Medium(5 / 45.0, 0.0, "table", 0.0, tab), E.Geometry(), E.Camera(128, 96),
              dict(image_mode=2)),
             ("hg_beam", E.Medium(2 / 45.0, 0.0, "hg", 0.8, None), E.Geometry(45.0, 10.0, 10.0, 1.25),
              E.Camera(64, 64), {}),
             ("paper", E.Medium(8 / 30.0, 0.0, "paper", 0.0, paper), E.Geometry(30.0, 10.0, 45.0, 1.25),
              E.Camera(60, 90, 64, 23.05), dict(rr_threshold=1e-3, rr_survival=0.0)),
             ("cube", E.Medium(0.2, 0.0, "hg", 0.0, None), E.Geometry(10.0, 10.0, 10.0), E.Camera(32, 32), {})]
    for name, med, geo, cam, kw in cases:
        e = E.Engine(cam, geo)
        e.run(med, 2_000_000, seed=3, **kw)
        err = int(e.error.cpu().numpy()[0])     # read before check(), which clears it
        e.check()
        r = e.result()
        res[name + "_img"], res[name + "_tot"] = r["raw_image"], r["raw_totals"]
        res[name + "_rad"], res[name + "_err"] = e.radial.cpu().numpy(), np.array(err)
    # heterogeneous medium: walk and density gradient
    dens = torch.from_numpy(np.ascontiguousarray(W.rough_grid((16, 16, 64), 4, mean=2000.0),
                                                 dtype=np.float32)).cuda()
    geo = E.Geometry()
    g = E.Grid(dens, 4e-5, 3.6e-5, 0.002, (8, 4, 4)).prepare(geo)
    e = E.Engine(E.Camera(64, 64), geo)
    med = E.Medium(1.0, 0.0, "table", 0.0, tab)
    e.run_grid(g, med, 1_000_000, seed=2)
    err = int(e.error.cpu().numpy()[0])
    e.check()
    r = e.result()
    res["grid_img"], res["grid_tot"], res["grid_err"] = r["raw_image"], r["raw_totals"], np.array(err)
    adj = torch.from_numpy(np.random.default_rng(1).uniform(0, 1, (64, 64)).astype(np.float32))
    val, grad = e.grid_adjoint(g, med, adj, 300_000, seed=4)
    err = int(e.error.cpu().numpy()[0])
    e.check()
    res["gadj_val"], res["gadj_grad"], res["gadj_err"] = val.cpu().numpy(), grad.cpu().numpy(), np.array(err)
    # homogeneous adjoint with phase weights
    e = E.Engine(E.Camera(128, 128), E.Geometry())
    gvec = e.adjoint(E.Medium(5 / 45.0, 0.01, "table", 0.0, tab), adj.repeat(2, 2), 1_000_000, n_w=64, seed=5)
    err = int(e.error.cpu().numpy()[0])
    e.check()
    res["adj"], res["adj_err"] = gvec.cpu().numpy(), np.array(err)
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
