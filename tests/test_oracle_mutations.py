"""Planted mistakes in the oracle: each entry changes one expression of a
copy of oracle/ the way a plausible slip would (a dropped term, a wrong sign,
index, factor or constant) and runs the oracle's pins against that copy. Every
mistake must make a pin fail, and the unchanged copy must pass the same pins,
so the pins are shown to fix the oracle rather than only to agree with it.
Nothing here touches the oracle in the tree; copies live in pytest's tmp_path."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WALK = ["test_oracle_walk.py"]
MIE = ["test_oracle_mie.py"]
TABLE = ["test_oracle_table.py"]
PHILOX = ["test_oracle_philox.py"]
ADJ = ["test_oracle_adjoint.py"]
GRID = ["test_oracle_grid.py"]
GADJ = ["test_oracle_grid_adjoint.py"]
PAPER = ["test_oracle_paper.py"]
METRICS = ["test_oracle_metrics.py"]
WEIGHTS = ["test_oracle_phase_weights.py"]
W32 = ["test_oracle_walk32.py"]

# (file, text, replacement, pin files, the mistake)
MUTATIONS = [
    # Mie series (Sec. 2.2 Eq. 3-9)
    ("mie.c", "double complex ta = D[n] / m + (double)n / x;", "double complex ta = D[n] * m + (double)n / x;",
     MIE, "a_n built with m D_n (a_n and b_n confused)"),
    ("mie.c", "double tau_n = n * mu * pi_n - (n + 1.0) * pi_nm1;", "double tau_n = n * mu * pi_n - n * pi_nm1;",
     MIE, "tau_n recurrence off by one"),
    ("mie.c", "se += (2.0 * n + 1.0) * creal(a[n] + b[n]);", "se += (2.0 * n + 1.0) * creal(a[n] - b[n]);",
     MIE, "sign of b_n in Q_ext"),
    ("mie.c", "        sg += (2.0 * n + 1.0) / ((double)n * (n + 1.0)) * creal(a[n] * conj(b[n]));\n", "",
     MIE, "g series without its a_n b_n* term"),
    ("mie.c", "double lambda_um = (lambda0_nm * 1e-3) / n_medium;", "double lambda_um = (lambda0_nm * 1e-3);",
     MIE, "size parameter with the vacuum wavelength"),
    ("mie.c", "return (int)ceil(x + 4.0 * cbrt(x) + 2.0);", "return (int)ceil(x + 2.0);",
     MIE, "Mie series truncated early"),
    # phase table (Sec. 3.1.2, Eq. 10)
    ("table.c", "cum[p + 1] = cum[p] + h / 3.0 * (F[j] + 4.0 * F[j + 1] + F[j + 2]);",
     "cum[p + 1] = cum[p] + h / 3.0 * (F[j] + 2.0 * F[j + 1] + F[j + 2]);", TABLE, "Simpson weights"),
    ("table.c", "F[j] *= 0.5 * sin((double)(n_fine - j) * h);", "F[j] *= 0.5;", TABLE,
     "solid-angle factor sin(theta) dropped"),
    ("table.c", "double theta = (double)(n_fine - j) * h - s;", "double theta = (double)(n_fine - j) * h + s;",
     TABLE, "panel inversion measured from the wrong end"),
    ("table.c", "pdf[i] = (1.0 / n_bins) / (t_omu[i] - t_omu[i + 1]);", "pdf[i] = (1.0 / n_bins) / (t_omu[i] + t_omu[i + 1]);",
     TABLE, "bin density"),
    ("table.c", "double target = Z * ((double)i / n_bins);", "double target = Z * ((double)(i - 1) / n_bins);",
     TABLE, "inversion levels shifted by one"),
    ("table.c", "F[j] += (w[i] / wsum) * G[j] / Z;", "F[j] += (w[i] / wsum) * G[j];", GRID,
     "mixture of unnormalised components"),
    ("table.c", "cdf[i + 1] = cdf[i] + 0.5 * h * (F[i] + F[i + 1]);", "cdf[i + 1] = cdf[i] + h * F[i];", PAPER,
     "paper CDF by rectangles"),
    ("table.c", "F[i] *= 0.5 * sin(i * h);", "F[i] *= 0.5;", PAPER, "paper CDF without sin(theta)"),
    # Philox4x32-10 and the uniforms
    ("philox.c", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;", PHILOX, "Weyl constant"),
    ("philox.c", "uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;", "uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k1;",
     PHILOX, "round key word"),
    ("philox.c", "return (double)(r >> 9) * 0x1p-23 + 0x1p-24;", "return (double)(r >> 9) * 0x1p-23;", PHILOX,
     "uniform not centred (can be 0)"),
    # the walk (Sec. 3.1.3 Eq. 15-16, the camera of Sec. 4.3)
    ("walk.c", "double s = mu_ext > 0.0 ? -log(u0) / mu_ext : INFINITY;",
     "double s = mu_ext > 0.0 ? -log(u0) * mu_ext : INFINITY;", WALK, "free path in the wrong units (Eq. 15)"),
    ("walk.c", "w = w * (1.0 - mua_here / mu_here);", "w = w * (1.0 - 0.5 * mua_here / mu_here);", WALK,
     "albedo (Eq. 16)"),
    ("walk.c", "double nee = w * psr * exp(-od);", "double nee = w * psr * exp(-0.5 * od);", WALK,
     "camera transmittance"),
    ("walk.c", "psr = pdf / (2.0 * M_PI);", "psr = pdf / (4.0 * M_PI);", WALK, "table density per steradian"),
    ("walk.c", "return (1.0 - g * g) / (4.0 * M_PI * t * sqrt(t));", "return (1.0 - g * g) / (4.0 * M_PI * t);",
     WALK, "H-G density (Eq. 11)"),
    ("walk.c", "double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);", "double q = (1.0 - g * g) / (1.0 + g + 2.0 * g * xi);",
     WALK, "H-G inverse distribution (Eq. 11)"),
    ("walk.c", "int lo = 0, hi = n; /* icdf", "int lo = 0, hi = n - 1; /* icdf", WALK,
     "camera density never from the last table bin"),
    ("walk.c", "double fx = r[0] / c->lx * c->nx;", "double fx = r[0] / c->lz * c->nx;", WALK, "image column scale"),
    ("walk.c", "double fz = (r[2] - lo[2]) / c->lz * c->nz;", "double fz = (r[2] + lo[2]) / c->lz * c->nz;", WALK,
     "image row sign"),
    ("walk.c", "double phi = 2.0 * M_PI * u2;", "double phi = M_PI * u2;", WALK, "azimuth on [0, pi)"),
    ("walk.c", "    double b = d[0] * d[1] * a;\n            double e1[3]",
     "    double b = d[0] * d[2] * a;\n            double e1[3]", WALK, "basis vector index"),
    ("walk.c", "double wn = w / c->rr_survival;", "double wn = w;", WALK, "roulette survivor not reweighted"),
    ("walk.c", "if (face == 0 && d[0] < 0.0) {", "if (face == 0 && d[0] > 0.0) {", WALK,
     "reflection and transmission faces swapped"),
    ("walk.c", "omu = c->omu[i] + f * (c->omu[i + 1] - c->omu[i]);", "omu = c->omu[i];", WALK,
     "table sample without interpolation"),
    ("walk.c", "nbin = table_bin(c->icdf, c->n_bins, muc);", "nbin = table_bin(c->icdf, c->n_bins, -muc);", WALK,
     "camera cosine sign"),
    ("walk.c", "double rho = c->beam_radius * sqrt(oracle_uniform(o[0]));",
     "double rho = c->beam_radius * oracle_uniform(o[0]);", WALK, "beam entry radius not uniform over the disc"),
    ("walk.c", "uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u};",
     "uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};", WALK,
     "beam entry drawn from the first flight's numbers"),
    ("walk.c", "double fr = rho / c->r_max * c->n_radial;", "double fr = rho * rho / c->r_max * c->n_radial;",
     WALK, "radial bin of rho squared"),
    ("walk.c", "rbin = (int)floor(fr);", "rbin = (int)ceil(fr);", WALK, "radial bin rounded up"),
    ("walk.c", "rec->nee = nee;", "rec->nee = w * psr;", WALK, "traced camera term without its transmittance"),
    ("walk.c", "rec->pix = pix;", "rec->pix = ix;", WALK, "traced pixel without its row"),
    # delta tracking (heterogeneous media)
    ("walk.c", "if (mu > *q)\n                        *q = mu;", "if (mu < *q)\n                        *q = mu;", GRID,
     "majorant from the thinnest voxel"),
    ("walk.c", "const double s = tau / mb;", "const double s = tau * mb;", GRID, "tentative flight length"),
    ("walk.c", "tau -= mb * t;", "tau -= t;", GRID, "optical depth spent in a cell"),
    ("walk.c", "for (int j = iy + 1; j < c->gy; ++j)\n        od +=", "for (int j = iy; j < c->gy; ++j)\n        od +=",
     GRID, "camera column counts its own voxel twice"),
    ("walk.c", "const double top = (iy == c->gy - 1) ? hi[1] : lo[1] + (iy + 1) * vy;",
     "const double top = (iy == c->gy - 1) ? hi[1] : lo[1] + iy * vy;", GRID, "top of the collision voxel"),
    ("walk.c", "const double acc = mu_here / mubar;", "const double acc = 0.5 * (1.0 + mu_here / mubar);", GRID,
     "acceptance probability"),
    ("walk.c", "u3 = u3 / acc;  /* uniform", "u3 = u3;  /* uniform", GRID, "roulette number not rescaled"),
    # the paper's sampler (Sec. 3.1.2)
    ("walk.c", "double th = (i + f) * (M_PI / n);", "double th = (i + 0.5) * (M_PI / n);", PAPER,
     "no interpolation inside the angle interval"),
    ("walk.c", "psr = stc > 0.0 ? pth / stc / (2.0 * M_PI) : 0.0;", "psr = pth / (2.0 * M_PI);", PAPER,
     "camera density per radian, not per unit cosine"),
    # image comparison (Sec. 3.1.4, Tables 3-4)
    ("metrics.py", "return (a - mn) / (mx - mn)", "return (a - mn) / mx", METRICS, "min-max normalisation"),
    ("metrics.py", "return float(np.sqrt(np.mean((a - b) ** 2)))", "return float(np.mean(np.abs(a - b)))", METRICS,
     "mean absolute instead of root-mean-square error"),
    ("metrics.py", "return float(np.sum(da * db) / np.sqrt(saa * sbb))", "return float(np.sum(da * db) / (saa * sbb))",
     METRICS, "correlation not normalised"),
    ("metrics.py", "dx = ix + 0.5 - nx / 2.0", "dx = ix - nx / 2.0", METRICS, "ring centre off by half a pixel"),
    ("metrics.py", "rho_max = np.sqrt((nx / 2.0) ** 2 + (nz / 2.0) ** 2)", "rho_max = max(nx, nz) / 2.0", METRICS,
     "ring range"),
    ("metrics.py", "return np.where(ang < 30.0, 0,", "return np.where(ang < 60.0, 0,", METRICS, "forward zone limit"),
    ("metrics.py", "/ max(int(ok.sum()), 1))", "/ n_r)", METRICS, "share counts rings without pixels"),
    # the adjoint (gradients of Eq. 15-16)
    ("adjoint.c", "double t = fabs(mu - (-1.0 + k * h)) / h;", "double t = fabs(mu - (-1.0 + k * h)) / (2.0 * h);",
     ADJ, "hat twice as wide"),
    ("adjoint.c", "s += pdf * hat_integral(n_w, k, a, b);", "s += hat_integral(n_w, k, a, b);", ADJ,
     "hat integrals without the phase density"),
    ("adjoint.c", "S += 1.0 / mu_ext - s;", "S += 1.0 / mu_ext + s;", ADJ, "sign of the flight score"),
    ("adjoint.c", "pg[0] += A * (R.S[j] + jj * (1.0 / c->mu_s - 1.0 / mu_ext) - R.l[j]);",
     "pg[0] += A * (R.S[j] + jj * (1.0 / c->mu_s - 1.0 / mu_ext));", ADJ, "transport term dropped"),
    ("adjoint.c", "pg[1] += A * (R.S[j] - jj / mu_ext - R.l[j]);", "pg[1] += A * (R.S[j] + jj / mu_ext - R.l[j]);",
     ADJ, "sign of the albedo term"),
    ("adjoint.c", "double t = oracle_hat(J->n_w, q, R.muc[j]) / h_w(J->n_w, J->w, R.muc[j]) - jj * J->z[q];",
     "double t = oracle_hat(J->n_w, q, R.muc[j]) / h_w(J->n_w, J->w, R.muc[j]) - J->z[q];", ADJ,
     "normalisation counted once"),
    ("adjoint.c", "for (int i = 0; i < j; ++i)\n                    t +=", "for (int i = 1; i < j; ++i)\n                    t +=",
     ADJ, "range of the sampled-angle sum"),
    # phase weights at w != 1: the reweighted table and its scores
    ("table.c", "cum[j + 1] = cum[j] + p[j] * hw_integral(n_w, w, omu_base[j], omu_base[j + 1]);",
     "cum[j + 1] = cum[j] + hw_integral(n_w, w, omu_base[j], omu_base[j + 1]);", WEIGHTS,
     "reweighted bin masses without the table density"),
    ("table.c", "return w[k] * oracle_hat(n_w, k, mu) + w[k + 1] * oracle_hat(n_w, k + 1, mu);",
     "return w[k] * oracle_hat(n_w, k, mu) + w[k] * oracle_hat(n_w, k + 1, mu);", WEIGHTS,
     "weight interpolant takes one node's weight"),
    ("adjoint.c", "double t = oracle_hat(J->n_w, q, R.muc[j]) / h_w(J->n_w, J->w, R.muc[j]) - jj * J->z[q];",
     "double t = oracle_hat(J->n_w, q, R.muc[j]) - jj * J->z[q];", WEIGHTS,
     "camera-density score without 1/h_w"),
    ("adjoint.c", "t += oracle_hat(J->n_w, q, R.mus[i]) / h_w(J->n_w, J->w, R.mus[i]);",
     "t += oracle_hat(J->n_w, q, R.mus[i]);", WEIGHTS, "sampled-angle score without 1/h_w"),
    ("adjoint.c", "        for (int k = 0; k < n_w; ++k)\n            z[k] /= zw;\n", "", WEIGHTS,
     "hat integrals not divided by Z(w)"),
    ("adjoint.c", "oracle_hat_integrals(base_omu ? base_omu : c->omu, c->n_bins, n_w, z);",
     "oracle_hat_integrals(c->omu, c->n_bins, n_w, z);", WEIGHTS,
     "hat integrals of the reweighted table instead of the unweighted one"),
    ("adjoint.c", "{\n        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u}, o[4];",
     "{\n        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u}, o[4];", ADJ,
     "replayed beam entry from the first flight's numbers"),
    ("adjoint.c", "{\n                uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u}, o[4];",
     "{\n                uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u}, o[4];", GADJ,
     "gradient's beam entry from the first flight's numbers"),
    ("adjoint.c", "r[1] = rho * cos(psi);", "r[1] = -rho * cos(psi);", ADJ, "replayed beam entry point"),
    ("adjoint.c", "r0[1] = rho * cos(psi);", "r0[1] = 0.0;", GADJ, "first flight starts on the axis"),
    ("adjoint.c", "m[i] = a[i] + 0.5 * (t0 + t1) * d[i];", "m[i] = a[i] + t0 * d[i];", GADJ,
     "flight piece given to the voxel at its start"),
    ("adjoint.c", "coef * (t1 - t0) * len;", "coef * (t1 - t0);", GADJ, "flight pieces without their length"),
    ("adjoint.c", "for (int j = v[1] + 1; j < c->gy; ++j)", "for (int j = v[1]; j < c->gy; ++j)", GADJ,
     "camera column counts the collision voxel twice"),
    ("adjoint.c", "grad[vi] += B * c->k_ext / mu;", "grad[vi] += B / mu;", GADJ, "collision point term"),
    ("adjoint.c", "grad[vi] -= Ai * c->k_ext * (top - ry);", "grad[vi] -= Ai * c->k_ext * (top + ry);",
     GADJ, "camera column inside the collision voxel"),
    ("adjoint.c", "segment_voxels(c, lo, prev, ri, -B * c->k_ext, grad, ts, ts_cap);",
     "segment_voxels(c, lo, prev, ri, B * c->k_ext, grad, ts, ts_cap);", GADJ, "sign of the flight transmission"),
    # null-collision scores of the density gradient
    ("adjoint.c", "grad[(size_t)r->pix] -= B * c->k_ext / (r->nee - r->w);",
     "grad[(size_t)r->pix] += B * c->k_ext / (r->nee - r->w);", GADJ, "sign of the null-collision score"),
    ("adjoint.c", "grad[(size_t)r->pix] -= B * c->k_ext / (r->nee - r->w);",
     "grad[(size_t)r->pix] -= B * c->k_ext / r->nee;", GADJ, "null score with the majorant alone"),
    ("adjoint.c", "grad[(size_t)r->pix] -= B * c->k_ext / (r->nee - r->w);",
     "grad[(size_t)r->pix] -= P * c->k_ext / (r->nee - r->w);", GADJ,
     "null score weighted by all the photon's camera terms"),
    ("walk.c", "maj[i] *= c->majorant_scale;", "maj[i] *= 1.0;", GADJ, "majorant scale ignored"),
    # the single-precision mode
    ("walk32.c", "const float s = -logf(u0) / mu_ext;", "const float s = -logf(u0) * mu_ext;", W32,
     "FP32 free path times mu_ext"),
    ("walk32.c", "const float albedo = (float)(c->mu_s / (c->mu_s + c->mu_a));",
     "const float albedo = (float)(c->mu_a / (c->mu_s + c->mu_a));", W32, "FP32 albedo from the absorption"),
    ("walk32.c", "om = 2.0f * (1.0f - g) * (1.0f - g) * (1.0f - u1) * fmaf(g, u1, 1.0f) / (D * D);",
     "om = 2.0f * (1.0f - g) * (1.0f - g) * fmaf(g, u1, 1.0f) / (D * D);", W32, "FP32 H-G inverse without (1 - xi)"),
    ("walk32.c", "op = 2.0f * (1.0f + g) * (1.0f + g) * u1 * fmaf(g, u1, 1.0f - g) / (D * D);",
     "op = 2.0f * (1.0f + g) * (1.0f + g) * (1.0f - u1) * fmaf(g, u1, 1.0f - g) / (D * D);", W32,
     "FP32 H-G 1 + cos(theta)"),
    ("walk32.c", "op = 2.0f * (1.0f + g) * (1.0f + g) * u1 * fmaf(g, u1, 1.0f - g) / (D * D);",
     "op = 2.0f - om;", W32, "FP32 H-G 1 + cos(theta) from 2 - om (its accuracy lost near pi)"),
    ("walk32.c", "om = fmaf(f, omu[i + 1] - omu[i], omu[i]);", "om = fmaf(f, omu[i + 1] - omu[i], omu[i + 1]);", W32,
     "FP32 table interpolation from the wrong level"),
    ("walk32.c", "const float e2[3] = {b, fmaf(d[1] * d[1], a, sg), -d[1]};",
     "const float e2[3] = {b, fmaf(d[1] * d[1], a, sg), d[1]};", W32, "FP32 sign in the Duff basis"),
    ("walk32.c", "sincosf(2.0f * PI_F * u2, &sp, &cp);", "sincosf(PI_F * u2, &sp, &cp);", W32,
     "FP32 azimuth over half the circle"),
    ("walk32.c", "expf(-mu_ext * (hy - r[1]))", "expf(-mu_ext * (hy + r[1]))", W32,
     "FP32 camera path length from the wrong face"),
    ("walk32.c", "psr = pdf[nbin] / (2.0f * PI_F);", "psr = pdf[nbin + 1] / (2.0f * PI_F);", W32,
     "FP32 camera density of the next bin"),
    ("walk32.c", "w = w / surv;", "w = w * surv;", W32, "FP32 roulette survivor weight"),
    ("walk32.c", "const double fz = (double)r[2] / c->lz * c->nz + 0.5 * c->nz;",
     "const double fz = ((double)r[2] + hz) / c->lz * c->nz;", W32,
     "FP32 camera row from the float half-height (z = 0 off row nz/2)"),
]


def _copy(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))


def _pins(root, files, basetemp):
    """Run the pin files against the oracle copy under `root` (it comes first
    on the import path: the working directory of the child)."""
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + ROOT)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
           "--basetemp", basetemp] + [os.path.join(ROOT, "tests", f) for f in files]
    p = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=900)
    return p.returncode, p.stdout[-1500:] + p.stderr[-1500:]


def _compiles(root):
    src = [os.path.join(root, "oracle", s) for s in ("mie.c", "table.c", "philox.c", "walk.c", "walk32.c",
                                                      "adjoint.c")]
    p = subprocess.run(["gcc", "-std=c11", "-D_GNU_SOURCE", "-fsyntax-only", "-Wall"] + src,
                       capture_output=True, text=True)
    return p.returncode == 0, p.stderr[-800:]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    return tmp_path_factory.mktemp("mut")


def test_every_planted_mistake_applies_once():
    for fname, old, new, _, what in MUTATIONS:
        text = open(os.path.join(ROOT, "oracle", fname)).read()
        assert text.count(old) == 1, (fname, what)
        assert old != new


def _pool():
    return ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1)))


def test_unchanged_copy_passes_the_pins(workdir):
    root = str(workdir / "control")
    _copy(root)
    files = sorted({f for m in MUTATIONS for f in m[3]})
    subprocess.run([sys.executable, os.path.join(root, "oracle", "build.py")], check=True, capture_output=True)
    # a child started like the pin runs imports the copy, not the oracle in the tree
    p = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=root,
                       env=dict(os.environ, PYTHONPATH=root + os.pathsep + ROOT), capture_output=True, text=True)
    assert os.path.dirname(p.stdout.strip()) == os.path.join(root, "oracle"), p.stdout + p.stderr
    with _pool() as ex:   # one child per pin file, all on the copy built above
        results = list(ex.map(lambda f: (f, _pins(root, [f], str(workdir / ("control_bt_" + f[:-3])))), files))
    for f, (rc, out) in results:
        assert rc == 0, (f, out)


def test_every_planted_mistake_fails_a_pin(workdir):
    def one(k):
        fname, old, new, files, what = MUTATIONS[k]
        root = str(workdir / ("m%02d" % k))
        _copy(root)
        path = os.path.join(root, "oracle", fname)
        text = open(path).read()
        open(path, "w").write(text.replace(old, new, 1))
        ok, err = _compiles(root)
        if not ok:
            return k, "does not compile: " + err
        rc, out = _pins(root, files, str(workdir / ("m%02d_bt" % k)))
        # exit status 1: tests ran and at least one failed
        return k, None if rc == 1 and "failed" in out else "not caught (exit %d): %s" % (rc, out[-600:])

    with _pool() as ex:
        results = list(ex.map(one, range(len(MUTATIONS))))
    missed = ["%s: %s -> %s" % (MUTATIONS[k][0], MUTATIONS[k][4], why) for k, why in results if why]
    assert not missed, "\n".join(missed)
