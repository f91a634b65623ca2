"""Checkpoint / resume of long runs, and a JSON-lines run log.

Photon i draws its random numbers from the Philox counter (seed, i, event),
and every tally is an integer sum, so a run of photons [0, N) split into
chunks [0, k), [k, N) gives the same tallies bit for bit as one launch,
whatever happens between the chunks. A checkpoint is therefore small: a key
of the configuration, the photons done, the raw int64 tallies, and the
chunks' per-photon images summed in squares (batch means: the statistical
error of every image bin).
"""
import hashlib
import json
import os
import time

import numpy as np

from . import _native as N

FORMAT = 2   # 2: with the batch-means sums of squares


def config_key(engine, medium, n_photons, seed, run_kw):
    """Hash of everything that decides a run's tallies: medium (coefficients,
    phase function, table contents), geometry, camera, photon count, seed and
    the run parameters."""
    h = hashlib.sha256()
    desc = dict(format=FORMAT, mu_s=float(medium.mu_s), mu_a=float(medium.mu_a), phase=medium.phase,
                hg_g=float(medium.hg_g), geometry=vars(engine.geometry), camera=vars(engine.camera),
                n_photons=int(n_photons), seed=int(seed), run={k: run_kw[k] for k in sorted(run_kw)})
    h.update(json.dumps(desc, sort_keys=True, default=float).encode())
    if medium.table is not None:
        h.update(np.ascontiguousarray(medium.table.blob).tobytes())
    return h.hexdigest()


def _load(path, key):
    with np.load(path) as z:
        if str(z["key"]) != key:
            raise ValueError("checkpoint %s belongs to another configuration" % path)
        return int(z["done"]), z["image"], z["radial"], z["totals"], z["sumsq"], int(z["chunks"])


def _save(path, key, done, engine, sumsq, chunks):
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, key=np.array(key), done=np.array(done, dtype=np.int64),
                 image=engine.image.cpu().numpy(), radial=engine.radial.cpu().numpy(),
                 totals=engine.totals.cpu().numpy(), sumsq=sumsq, chunks=np.array(chunks, dtype=np.int64))
    os.replace(tmp, path)   # a checkpoint is either the old one or the new one


def image_sigma(image, sumsq, n_photons, chunks):
    """Statistical error of each image bin (same units as `image`, the sum
    over n_photons) from batch means: chunk c of n_c photons has per-photon
    image x_c; with sumsq = sum_c n_c x_c^2 and xbar = image / N, the mean's
    variance is (sumsq - N xbar^2) / ((chunks - 1) N), so sigma(image) =
    sqrt(N (sumsq - N xbar^2) / (chunks - 1)). None with fewer than 2 chunks."""
    if chunks < 2 or n_photons <= 0:
        return None
    xbar = image / n_photons
    return np.sqrt(np.maximum(n_photons * (sumsq - n_photons * xbar * xbar), 0.0) / (chunks - 1))


def run_resumable(engine, medium, n_photons, path, chunk=100_000_000, seed=1, stop_after=None, log=None,
                  stream=None, **run_kw):
    """Run photons [0, n_photons) in chunks of `chunk`, saving a checkpoint to
    `path` after each. If `path` holds a checkpoint of the same configuration
    the run resumes after its last chunk (one of another configuration raises
    ValueError). stop_after: chunks to run in this call (None: all). log: a
    JSON-lines file receiving run_record() of each chunk (with the median
    relative error of the image bins from the second chunk on). Returns
    engine.result() of the tallies so far, with 'photons_done' and
    'image_sigma' (per-bin statistical error by batch means over the chunks;
    None before two chunks)."""
    torch = __import__("torch")
    for k in ("photon_offset", "accumulate", "n_photons"):
        if k in run_kw:
            raise ValueError("%s is set by run_resumable" % k)
    if not run_kw.get("image_frac_bits"):
        # the chunks accumulate into one image: one F, from the whole budget
        from .engine import auto_frac_bits
        run_kw = dict(run_kw, image_frac_bits=auto_frac_bits(n_photons))
    key = config_key(engine, medium, n_photons, seed, run_kw)
    done, n_chunks = 0, 0
    sumsq = np.zeros(tuple(engine.image.shape), dtype=np.float64)
    if os.path.exists(path):
        done, img, rad, tot, sumsq, n_chunks = _load(path, key)
        engine.image.copy_(torch.from_numpy(img))
        engine.radial.copy_(torch.from_numpy(rad))
        engine.totals.copy_(torch.from_numpy(tot))
    else:
        engine.image.zero_()
        engine.radial.zero_()
        engine.totals.zero_()
    engine.image_frac_bits = int(run_kw["image_frac_bits"])
    scale = 2.0 ** -engine.image_frac_bits
    prev = engine.image.cpu().numpy().copy()
    chunks = 0
    while done < n_photons and (stop_after is None or chunks < stop_after):
        c = min(int(chunk), n_photons - done)
        steps0 = int(engine.totals[N.TOT_STEPS].item())
        t0 = time.perf_counter()
        engine.run(medium, c, seed=seed, photon_offset=done, accumulate=True, stream=stream, **run_kw)
        engine.check(stream)
        dt = time.perf_counter() - t0
        done += c
        chunks += 1
        n_chunks += 1
        now = engine.image.cpu().numpy().copy()
        x = (now - prev).astype(np.float64) * scale / c       # this chunk's image per photon (exact difference)
        sumsq += c * x * x
        prev = now
        _save(path, key, done, engine, sumsq, n_chunks)
        if log is not None:
            rec = run_record(engine, medium, c, dt, steps=int(engine.totals[N.TOT_STEPS].item()) - steps0,
                             photons_done=done, photons_total=int(n_photons), seed=int(seed), chunks=n_chunks)
            sig = image_sigma(now.astype(np.float64) * scale, sumsq, done, n_chunks)
            if sig is not None:
                img = now.astype(np.float64) * scale
                hit = img > 0
                rec["image_rel_sigma_median"] = float(np.median(sig[hit] / img[hit])) if hit.any() else None
            append_jsonl(log, rec)
    r = engine.result()
    r["photons_done"] = done
    r["image_sigma"] = image_sigma(r["image"], sumsq, done, n_chunks)
    return r


def run_record(engine, medium, n_photons, seconds, steps=None, **extra):
    """One JSON-serialisable record of a run: configuration, photons,
    photon-steps, wall time and rate, the weight totals of the engine's
    tallies (R, T far, T side, A, roulette, truncated, ballistic; weight
    units) and the error word the engine's last check() read (the flags
    raised by the runs it covered; check() raises when any is set, so a run
    recorded after a passing check logs 0)."""
    tot = engine.totals.cpu().numpy()
    w = tot[:7].astype(np.float64) * 2.0 ** -N.WEIGHT_FRAC_BITS
    steps = int(tot[N.TOT_STEPS]) if steps is None else int(steps)
    rec = dict(time=time.time(), medium=dict(mu_s=medium.mu_s, mu_a=medium.mu_a, phase=medium.phase,
                                             hg_g=medium.hg_g),
               geometry=vars(engine.geometry), camera=vars(engine.camera), photons=int(n_photons),
               photon_steps=steps, seconds=float(seconds),
               photon_steps_per_s=steps / seconds if seconds > 0 else None,
               totals=dict(zip(("reflect", "far", "side", "absorbed", "roulette", "truncated", "ballistic"),
                               map(float, w))),
               error=int(getattr(engine, "last_error", 0)))
    rec.update(extra)
    return rec


def append_jsonl(path, record):
    with open(path, "a") as f:
        f.write(json.dumps(record, sort_keys=True, default=float) + "\n")
