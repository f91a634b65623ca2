"""Launch-shape autotuner for the batched walk.

Times candidate (threads per CTA, photons a warp takes per grab) pairs on a
scaled-down copy of the batch (every medium keeps its optical properties,
photon budgets are divided by `scale`), picks the fastest, and caches the
choice in a JSON file keyed by GPU name and a hash of the configuration.
Results do not depend on the choice (integer tallies), only the time does.
"""
import hashlib
import json
import os

CACHE_ENV = "MCMIE_AUTOTUNE_CACHE"
BLOCKS = (256, 512, 1024)
ITEMS = (32, 64, 128, 256, 512)


def cache_path():
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache", "mcmie",
                                                     "autotune.json")


def _key(gpu_name, camera, media, n_photons):
    h = hashlib.sha256()
    h.update(repr((gpu_name, camera.nx, camera.nz, camera.n_radial)).encode())
    for m, n in zip(media, n_photons):
        h.update(repr((round(m.mu_s, 9), round(m.mu_a, 9), m.phase, round(m.hg_g, 9),
                       m.table.params["diameter_um"] if m.table is not None else None, int(n))).encode())
    return h.hexdigest()[:24]


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def tune_batch(batch, media, n_photons, seeds=1, scale=8, reps=2, use_cache=True):
    """Return dict(block_size=..., item_photons=..., ms=...) for this batch."""
    import torch
    from .engine import Batch
    name = torch.cuda.get_device_name(batch.device)
    key = _key(name, batch.camera, media, n_photons)
    db = _load() if use_cache else {}
    if key in db:
        return dict(db[key], cached=True)
    small = [max(1, int(n) // scale) for n in n_photons]
    trial = Batch(len(media), batch.camera, batch.geometry, batch.device)
    best = None
    for block in BLOCKS:
        for item in ITEMS:
            try:
                trial.run(media, small, seeds, 0, item_photons=item, block_size=block)
            except Exception:
                continue   # shape not launchable for this camera (e.g. band needs 1024)
            torch.cuda.synchronize()
            t = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                trial.run(media, small, seeds, 0, item_photons=item, block_size=block)
                b.record()
                b.synchronize()
                t.append(a.elapsed_time(b))
            ms = min(t)
            if best is None or ms < best["ms"]:
                best = dict(block_size=block, item_photons=item, ms=ms)
    if best is None:
        raise RuntimeError("no launchable configuration")
    db[key] = best
    if use_cache:
        _store(db)
    return dict(best, cached=False)
