"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

They stand in for the paper's simulations of 5 um polystyrene spheres in
water at 532 nm in a cuvette imaged by a 90-degree side camera (Sec. 4,
Sec. 5.2: 3e8 photons at optical depths 5-12.5); the paper's experimental
images are not used.

  small       10x10x45 mm cuvette, tau = 1, 1e6 photons, 64x64 image, Mie and H-G
  sweep       tau in {1, 2, 5, 10, 20}, Mie and H-G, 1e8 photons,
              256x256 image + 128-bin radial profile (headline: tau = 5, Mie)
  batched     64 media: d log-uniform in [1, 10] um, tau uniform in [0.5, 20],
              photon budgets log-uniform in [1e6, 1e8], 128x128 images; the
              list is recorded in batched_media.json (python -m
              paper_2507_23189_gb300.workloads --write-batched)
  adjoint     tau = 5, Mie, 1e7 photons, 128x128; target at 0.9 mu_s0, mu_a = 0.01
  plume       256^3 voxel grid over the cuvette: a Gaussian plume (sigma 5 mm,
              centred at x = 22.5 mm on the beam axis) of polystyrene spheres
              with log-normal diameters (median 5 um, sigma_ln 0.3) in 16
              equal-number quantile bins; peak optical depth 30 along the
              beam; 1e9 photons, 512x512 image
"""
import os
from dataclasses import dataclass, field

import numpy as np

CUVETTE_MM = (45.0, 10.0, 10.0)   # beam axis x, then y (camera side), z
N_MEDIUM = 1.33
N_PARTICLE = complex(1.59, 0.0)
DIAMETER_UM = 5.0
WAVELENGTH_NM = 532.0
N_BINS = 4096
RR_THRESHOLD = 1e-4
RR_SURVIVAL = 0.1
R_MAX = 5.0 * 2 ** 0.5            # radial profile covers the far face's half-diagonal


@dataclass
class Case:
    name: str
    tau: float
    phase: str                    # "mie" or "hg" (H-G with g from the Mie table)
    n_photons: int
    nx: int
    nz: int
    n_radial: int = 128
    seed: int = 1
    diameter_um: float = DIAMETER_UM
    extra: dict = field(default_factory=dict)


def small():
    return [Case("small-%s" % p, 1.0, p, 1_000_000, 64, 64) for p in ("mie", "hg")]


def sweep(taus=(1.0, 2.0, 5.0, 10.0, 20.0), n_photons=100_000_000):
    return [Case("sweep-tau%g-%s" % (t, p), t, p, n_photons, 256, 256)
            for t in taus for p in ("mie", "hg")]


def headline(n_photons=100_000_000):
    """The optical-depth sweep's tau = 5 Mie point."""
    return Case("sweep-tau5-mie", 5.0, "mie", n_photons, 256, 256)


def batched_draw(n=64, seed=2026):
    """Instance parameters from numpy's Philox (a 64-bit counter-based stream).
    The uniforms are the same on every platform; numpy's exp and log may not
    be, in the last bit."""
    rng = np.random.Generator(np.random.Philox(seed))
    d = np.exp(rng.uniform(np.log(1.0), np.log(10.0), n))
    tau = rng.uniform(0.5, 20.0, n)
    nph = np.exp(rng.uniform(np.log(1e6), np.log(1e8), n)).astype(np.int64)
    return [Case("batched-%02d" % i, float(tau[i]), "mie", int(nph[i]), 128, 128, seed=1,
                 diameter_um=float(d[i])) for i in range(n)]


def batched(n=64, seed=2026):
    """The batched media. The default 64 (seed 2026) are the recorded list in
    batched_media.json, so every machine runs exactly the same media; other
    arguments draw afresh (batched_draw)."""
    if (n, seed) == (64, 2026) and os.path.exists(BATCHED_RECORD):
        import json
        with open(BATCHED_RECORD) as f:
            rec = json.load(f)
        return [Case(m["name"], float(m["tau"]), "mie", int(m["n_photons"]), rec["image"][0], rec["image"][1],
                     seed=int(rec["photon_seed"]), diameter_um=float(m["diameter_um"])) for m in rec["media"]]
    return batched_draw(n, seed)


BATCHED_RECORD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batched_media.json")


def batched_record(cases=None):
    """The 64 media as a JSON-ready dict (by default a fresh draw)."""
    cases = batched_draw() if cases is None else cases
    return {"generator": "numpy.random.Philox(2026): 64 draws each of ln d ~ U[ln 1, ln 10] (um), "
                         "tau ~ U[0.5, 20], ln N ~ U[ln 1e6, ln 1e8] (N truncated to an integer), in that order",
            "image": [128, 128], "photon_seed": 1,
            "media": [{"name": c.name, "diameter_um": c.diameter_um, "tau": c.tau, "n_photons": c.n_photons}
                      for c in cases]}


def write_batched_record(path=BATCHED_RECORD):
    import json
    with open(path, "w") as f:
        json.dump(batched_record(), f, indent=1)
        f.write("\n")


def adjoint():
    return Case("adjoint-tau5-mie", 5.0, "mie", 10_000_000, 128, 128,
                extra=dict(mu_s_factor=0.9, mu_a=0.01))


@dataclass
class Plume:
    shape: tuple = (256, 256, 256)          # (gz, gy, gx)
    sigma_mm: float = 5.0
    center_x_mm: float = 22.5
    tau_peak: float = 30.0                  # optical depth along the beam through the plume
    median_um: float = 5.0
    sigma_ln: float = 0.3
    n_size_bins: int = 16
    n_photons: int = 1_000_000_000
    nx: int = 512
    nz: int = 512
    block: tuple = (32, 256, 256)           # majorant cells, voxels (bx, by, bz): 8 slabs along the beam
    seed: int = 1


def plume():
    return Plume()


def size_bins(median_um=5.0, sigma_ln=0.3, n=16):
    """Diameters at the centres (in probability) of n equal-number quantile
    bins of a log-normal distribution, with their number fractions."""
    from scipy.special import ndtri
    q = (np.arange(n) + 0.5) / n
    return median_um * np.exp(sigma_ln * ndtri(q)), np.full(n, 1.0 / n)


def plume_shape(shape=(256, 256, 256), cuvette=CUVETTE_MM, sigma_mm=5.0, center_x_mm=22.5):
    """Relative density (peak 1) of a Gaussian plume at the voxel centres,
    float32 [gz, gy, gx], the beam axis at y = z = 0."""
    gz, gy, gx = shape
    lx, ly, lz = cuvette
    x = (np.arange(gx) + 0.5) * lx / gx - center_x_mm
    y = (np.arange(gy) + 0.5) * ly / gy - ly / 2
    z = (np.arange(gz) + 0.5) * lz / gz - lz / 2
    e = lambda v: np.exp(-0.5 * (v / sigma_mm) ** 2)
    return (e(z)[:, None, None] * e(y)[None, :, None] * e(x)[None, None, :]).astype(np.float32)


def rough_grid(shape, seed, mean=1.0, spread=0.6):
    """Seeded log-normal voxel field (a test input without structure)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return (mean * np.exp(spread * rng.standard_normal(shape))).astype(np.float32)


if __name__ == "__main__":
    import sys
    if sys.argv[1:] == ["--write-batched"]:
        write_batched_record()
        print(BATCHED_RECORD)
    else:
        raise SystemExit("usage: python -m paper_2507_23189_gb300.workloads --write-batched")
