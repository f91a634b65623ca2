"""Image comparison metrics (TEST INFRASTRUCTURE: the oracle of the engine's
mc_image_metrics; only the tests and the benchmark's CPU legs may import it).

Sec. 3.1.4 normalises every image the same way before comparing; Table 3
compares images by root-mean-square error and correlation coefficient;
Table 4 compares radial intensity profiles (angular averages) in three
zones named for scattering angles below 30 deg, 30-120 deg and above
120 deg, plus the correlation of the profiles and the share of radii where
one model is closer to the reference. The paper gives no formulas; the
readings taken here are:
  * normalisation: min-max to [0, 1] (an image with max == min maps to 0);
  * RMSE, r: over all pixels of the two normalised images, r = Pearson's
    (0 when either image is constant);
  * radial profile: polar coordinates about the image centre, pixel (ix, iz)
    at (ix + 1/2 - nx/2, iz + 1/2 - nz/2) in pixel units, n_r rings of equal
    width on [0, rho_max], rho_max the half-diagonal (rho = rho_max goes to
    the last ring); the profile is the mean normalised value over a ring;
    rings without pixels are left out of every profile statistic;
  * ring b stands for the angle 180 deg (b + 1/2) / n_r: forward zone below
    30 deg, intermediate 30-120 deg inclusive, edge above 120 deg; a zone's
    error is the RMSE of the two profiles over its rings;
  * "better": the share of rings where |p_a - p_ref| < |p_b - p_ref|.
Plain numpy, double precision, no blocking or reordering.
"""
import numpy as np

N_OUT_FIXED = 13


def normalise(img):
    a = np.asarray(img).astype(np.float64)
    mn, mx = a.min(), a.max()
    if mx == mn:
        return np.zeros_like(a)
    return (a - mn) / (mx - mn)


def rmse(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)))


def pearson(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    da, db = a - a.mean(), b - b.mean()
    saa, sbb = float(np.sum(da * da)), float(np.sum(db * db))
    if saa == 0.0 or sbb == 0.0:
        return 0.0
    return float(np.sum(da * db) / np.sqrt(saa * sbb))


def ring_index(nz, nx, n_r):
    """Ring of every pixel, shape (nz, nx)."""
    iz, ix = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    dx = ix + 0.5 - nx / 2.0
    dz = iz + 0.5 - nz / 2.0
    rho = np.sqrt(dx * dx + dz * dz)
    rho_max = np.sqrt((nx / 2.0) ** 2 + (nz / 2.0) ** 2)
    return np.minimum(np.floor(rho / rho_max * n_r).astype(np.int64), n_r - 1)


def radial_profile(norm_img, n_r):
    """(profile, count): mean normalised value per ring and pixels per ring."""
    nz, nx = norm_img.shape
    ring = ring_index(nz, nx, n_r)
    prof = np.zeros(n_r)
    cnt = np.zeros(n_r, dtype=np.int64)
    for b in range(n_r):
        sel = ring == b
        cnt[b] = int(sel.sum())
        if cnt[b]:
            prof[b] = float(norm_img[sel].sum()) / cnt[b]
    return prof, cnt


def zone_of_ring(n_r):
    ang = 180.0 * (np.arange(n_r) + 0.5) / n_r
    return np.where(ang < 30.0, 0, np.where(ang <= 120.0, 1, 2))


def _pair(nr, pr, na, pa, cnt, zones):
    ok = cnt > 0
    z = []
    for k in range(3):
        sel = ok & (zones == k)
        z.append(float(np.sqrt(np.mean((pa[sel] - pr[sel]) ** 2))) if sel.any() else 0.0)
    return [rmse(na, nr), pearson(na, nr)] + z + [pearson(pa[ok], pr[ok])]


def compare(ref, a, b=None, n_r=32):
    """Metrics of a (and b) against ref, laid out as mc_image_metrics writes
    them: [rmse, r, zone rmse x3, radial r] for a, the same for b (zeros
    without b), the share of rings where a is closer than b, then the
    profiles of ref, a, b."""
    nr = normalise(ref)
    na = normalise(a)
    pr, cnt = radial_profile(nr, n_r)
    pa, _ = radial_profile(na, n_r)
    zones = zone_of_ring(n_r)
    out = _pair(nr, pr, na, pa, cnt, zones)
    ok = cnt > 0
    if b is not None:
        nb = normalise(b)
        pb, _ = radial_profile(nb, n_r)
        out += _pair(nr, pr, nb, pb, cnt, zones)
        closer = np.abs(pa - pr) < np.abs(pb - pr)
        out.append(float(np.count_nonzero(closer & ok)) / max(int(ok.sum()), 1))
    else:
        pb = np.zeros(n_r)
        out += [0.0] * 7
    return np.array(out + list(pr) + list(pa) + list(pb))
