"""mc_run_static, the entry point for callers that cannot allocate device
memory: a host application that owns all device memory and hands a plug-in
only the buffers it reads and writes, or a latency-critical thread where an
allocation could synchronise the device. It keeps its scratch in a fixed
array inside the library instead of a caller workspace.

Checked through the C ABI against mc_run on the same inputs, for two calls in
a row (the shared scratch must not carry anything from one call to the next).
This file sorts last so that, when it fails, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0


def _static_run(gpu, med, cam, geo, rp):
    import torch
    from paper_2507_23189_gb300 import _native as N
    image = torch.zeros((cam.nz, cam.nx), dtype=torch.int64, device="cuda")
    radial = torch.zeros(cam.n_radial, dtype=torch.int64, device="cuda")
    totals = torch.zeros(N.N_TOTALS, dtype=torch.int64, device="cuda")
    error = torch.zeros(1, dtype=torch.int32, device="cuda")
    m, keep = med.as_c()
    st = N.lib().mc_run_static(C.byref(m), C.byref(geo.as_c()), C.byref(cam.as_c()), C.byref(rp),
                               C.c_void_p(image.data_ptr()), C.c_void_p(radial.data_ptr()),
                               C.c_void_p(totals.data_ptr()), C.c_void_p(error.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, N.STATUS.get(st)
    N.check("mc_check", N.lib().mc_check(C.c_void_p(error.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return image.cpu().numpy(), radial.cpu().numpy(), totals.cpu().numpy()


@pytest.mark.parametrize("phase,nx", [("table", 64), ("table", 256), ("hg", 128)])
def test_static_scratch_entry_matches_mc_run(gpu, phase, nx):
    t = gpu.PhaseTable()
    med = gpu.Medium(5 / LX, 0.001, phase, t.info["g"], t)
    cam, geo = gpu.Camera(nx, nx, 128, 5 * 2 ** 0.5), gpu.Geometry(LX, LY, LZ)
    for call, seed in enumerate((1, 2)):
        rp = gpu.run_params(400_000, seed=seed)
        img, rad, tot = _static_run(gpu, med, cam, geo, rp)
        e = gpu.Engine(cam, geo)
        e.run(med, 400_000, seed=seed)
        e.check()
        r = e.result()
        # integer tallies of the same photons: identical, not merely close
        np.testing.assert_array_equal(img, r["raw_image"], err_msg="call %d" % call)
        np.testing.assert_array_equal(tot, r["raw_totals"], err_msg="call %d" % call)
        np.testing.assert_array_equal(rad, e.radial.cpu().numpy(), err_msg="call %d" % call)
        assert tot[7] > 400_000
