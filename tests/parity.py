"""Comparison rules shared by the GPU parity tests.

Trace rule: the first 32 events of every photon must agree with the
double-precision oracle within 1e-5 relative (positions relative to the
cuvette length, directions absolutely, weights and camera contributions
relative; two camera contributions both below NEE_FLOOR, which no tally
can register, agree). A discrete decision (wall hit, exit face, pixel, table bin,
roulette) may differ only where the oracle's branch quantity lies within
1e-5 of its threshold; that photon's later events are then excluded.
At least 99.9 % of photons must match.

Tally rule: every image bin within 3 sigma of the oracle's estimate, and a
pooled chi-square over well-populated bins with p > 0.01.
"""
import math

import numpy as np

TOL = 1e-5
# Two camera terms that are both below this floor agree; otherwise they are
# compared relative to the larger of the oracle's value and the floor. A
# term below it can reach no fixed-point tally: the finest
# image unit is 2^-48, and one run adds at most 2^31 photons times 10^6
# events (2.1e15 terms, 2.1e-16 in all). Single precision cannot hold such a
# term at all where the camera path's optical depth passes about 87: it
# flushes to zero while the double-precision oracle keeps, say, 1e-98.
NEE_FLOOR = 1e-31


def compare_traces(g, o, mu_ext, lx=45.0, tol=TOL, nee_slope=None, hy=None):
    """g: decode_trace() dict of the GPU trace; o: oracle trace array
    [n, ev, 13]. nee_slope(mu_c): |d log p_sr / d mu_c| of a camera density
    that varies continuously with the direction (the paper's table); the
    camera term then also carries the direction difference of the previous
    event times that slope. hy (half the cuvette's height along the camera
    axis): the camera term's transmittance exp(-D) in single precision
    carries a relative error of about D 2^-23 (D, its argument and the fused
    multiply-add forming it are each rounded), so with hy given the term is
    also allowed 2^-22 D, D bounded by mu_ext (hy - r_y) with mu_ext the
    largest extinction. Returns dict(n, matched, flips, bad, worst...)."""
    n, ev = o.shape[0], o.shape[1]
    st_o = o[..., 0].astype(int)
    # nee_net: the camera term's deviation beyond what the position (and,
    # with nee_slope, the direction) deviations carry into it
    worst = dict(pos=0.0, dir=0.0, w=0.0, nee=0.0, nee_net=0.0)
    bad, causes, flips, checked_events = [], [], 0, 0
    for p in range(n):
        ok = True
        muc, ddir_prev = 0.0, 0.0     # direction before the first collision is +x
        for e in range(ev):
            so, sg = st_o[p, e], int(g["status"][p, e])
            if so < 0 and sg < 0:
                break
            rec = o[p, e]
            margin = rec[12]
            disc_o = (so, int(rec[9]), int(rec[10]), int(rec[11]))
            disc_g = (sg, int(g["pix"][p, e]), int(g["nee_bin"][p, e]), int(g["rad_bin"][p, e]))
            if disc_o != disc_g:
                if margin < tol:
                    flips += 1
                    break
                ok = False
                causes.append((p, e, "discrete (status, pixel, bin, radial) %s vs oracle %s, margin %.3g"
                               % (disc_g, disc_o, margin)))
                break
            if so == 6:
                break
            checked_events += 1
            dpos = float(np.max(np.abs(g["r"][p, e] - rec[1:4])))
            ddir = float(np.max(np.abs(g["d"][p, e] - rec[4:7])))
            dw = abs(g["w"][p, e] - rec[7]) / max(abs(rec[7]), 1e-300) if rec[7] else abs(g["w"][p, e])
            dnee_abs = abs(g["nee"][p, e] - rec[8])
            # the camera term depends on r_y through exp(-mu_ext (ly/2 - r_y))
            # two terms below what any tally can register agree
            tiny = max(abs(g["nee"][p, e]), abs(rec[8])) < NEE_FLOOR
            dnee = 0.0 if tiny else dnee_abs / max(abs(rec[8]), NEE_FLOOR)
            nee_tol = tol + mu_ext * dpos
            if nee_slope is not None:
                nee_tol += nee_slope(muc) * ddir_prev
            if hy is not None:
                nee_tol += 2.0 ** -22 * mu_ext * max(hy - rec[2], 0.0)
            worst["pos"] = max(worst["pos"], dpos / lx)
            worst["dir"] = max(worst["dir"], ddir)
            worst["w"] = max(worst["w"], dw)
            worst["nee"] = max(worst["nee"], dnee)
            worst["nee_net"] = max(worst["nee_net"], dnee - (nee_tol - tol))
            if dpos > tol * lx or ddir > tol or dw > tol or dnee > nee_tol:
                if margin < tol:
                    flips += 1
                    break
                ok = False
                causes.append((p, e, "position %.3g mm, direction %.3g, weight %.3g, camera %.3g (allowed %.3g), "
                               "margin %.3g" % (dpos, ddir, dw, dnee, nee_tol, margin)))
                break
            if so != 0:
                break
            muc, ddir_prev = float(rec[5]), ddir
        if not ok:
            bad.append(p)
    return dict(n=n, matched=n - len(bad), flips=flips, bad=bad[:20], causes=causes, worst=worst,
                events=checked_events)


def report_unmatched(cmp, label=""):
    """Print every photon that compare_traces did not match, with its cause
    (photon, event, what differed and the oracle's margin), so a tolerated
    mismatch is always on record in the test output."""
    for p, e, why in cmp["causes"]:
        print("unmatched%s: photon %d event %d: %s" % ((" " + label) if label else "", p, e, why))


def chi2_sf(x, k):
    """Survival function of the chi-square distribution (Wilson-Hilferty
    approximation for large k, exact series otherwise via scipy if present)."""
    try:
        from scipy.stats import chi2
        return float(chi2.sf(x, k))
    except Exception:  # pragma: no cover
        z = ((x / k) ** (1 / 3) - (1 - 2 / (9 * k))) / math.sqrt(2 / (9 * k))
        return 0.5 * math.erfc(z / math.sqrt(2))


def tally_agreement(a, b, var, hits=None, min_hits=20):
    """a, b: images; var: variance of (a - b); hits: oracle contributions per
    bin. Returns (max |z| over bins with var > 0, chi2, dof, p) with the
    chi-square pooled over bins holding at least min_hits contributions."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    var = np.asarray(var, dtype=np.float64).ravel()
    sig = np.sqrt(np.maximum(var, 0))
    ok = sig > 0
    z = np.zeros_like(a)
    z[ok] = (a - b)[ok] / sig[ok]
    pop = ok if hits is None else ok & (np.asarray(hits).ravel() >= min_hits)
    zmax = float(np.max(np.abs(z))) if z.size else 0.0
    chi2 = float(np.sum(z[pop] ** 2))
    dof = int(np.count_nonzero(pop))
    return zmax, chi2, dof, chi2_sf(chi2, max(dof, 1)), z


def oracle_var(res):
    """Per-bin variance of an oracle image sum from its per-photon squares."""
    n = res["n_photons"]
    img, sq = res["image"], res["image_sq"]
    return np.maximum(sq - img ** 2 / n, 0) * n / max(n - 1, 1)


def gpu_batches(gpu, med, n, batches, camera, geometry, offset=0, seed=1, **kw):
    """Run photons [offset, offset + n) as `batches` separate launches and
    return the summed result plus the batch-means variance of the image sum
    (the engine keeps integer sums only, so its spread comes from batches)."""
    # one image scale for every batch: the whole budget's (as one launch of
    # all n photons would use), so the integer sums add up exactly
    kw = dict(kw)
    if not kw.get("image_frac_bits"):
        kw["image_frac_bits"] = gpu.auto_frac_bits(n)
    imgs, tot, steps = [], None, 0
    raw_img = None
    edges = [offset + (n * k) // batches for k in range(batches + 1)]
    for k in range(batches):
        e = gpu.Engine(camera, geometry)
        e.run(med, edges[k + 1] - edges[k], seed=seed, photon_offset=edges[k], **kw)
        e.check()
        r = e.result()
        imgs.append(r["image"])
        raw_img = r["raw_image"] if raw_img is None else raw_img + r["raw_image"]
        tot = r["raw_totals"] if tot is None else tot + r["raw_totals"]
        steps += r["steps"]
    imgs = np.stack(imgs)
    total = imgs.sum(axis=0)
    var = batches * imgs.var(axis=0, ddof=1)
    return dict(image=total, var=var, raw_image=raw_img, raw_totals=tot, steps=steps)
