"""Failure detection on the GPU without a fault: the kernels' bounded wait
gives up on a phase that cannot complete and reports MC_ERR_TIMEOUT with the
context still usable; the host watchdog returns while work still runs; and a
run checkpointed, interrupted and resumed equals one launch bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0


def test_bounded_wait_gives_up_and_context_survives(gpu, ps_table):
    assert gpu.wait_selftest(tries=2048) == -4     # MC_ERR_TIMEOUT
    med = gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table)
    out = []
    for _ in range(2):
        e = gpu.Engine(gpu.Camera(64, 64), gpu.Geometry(LX, LY, LZ))
        e.run(med, 200_000, seed=3)
        e.check()
        out.append(e.result()["raw_image"])
        assert gpu.wait_selftest(tries=16) == -4
    np.testing.assert_array_equal(out[0], out[1])


def test_watchdog_returns_while_work_runs(gpu, ps_table):
    med = gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table)
    e = gpu.Engine(gpu.Camera(256, 256), gpu.Geometry(LX, LY, LZ))
    e.run(med, 400_000_000, seed=1)          # about 20 ms of work
    assert e.check_within(0.0) is False       # still running: the watchdog gives up, nothing is lost
    assert e.check_within(60_000.0) is True
    e.run(med, 1000, seed=1)
    assert e.check_within(60_000.0) is True


def test_resumed_run_is_bit_identical(gpu, ps_table, tmp_path):
    med = gpu.Medium(5 / LX, 0.002, "table", 0.0, ps_table)
    cam, geo = gpu.Camera(128, 128), gpu.Geometry(LX, LY, LZ)
    n = 10_000_000
    ref = gpu.Engine(cam, geo)
    ref.run(med, n, seed=7)
    ref.check()
    r_ref = ref.result()
    path = str(tmp_path / "ck.npz")
    r = gpu.run_resumable(gpu.Engine(cam, geo), med, n, path, chunk=3_000_000, seed=7, stop_after=2)
    assert r["photons_done"] == 6_000_000
    log = str(tmp_path / "log.jsonl")
    r = gpu.run_resumable(gpu.Engine(cam, geo), med, n, path, chunk=3_000_000, seed=7, log=log)
    assert r["photons_done"] == n
    np.testing.assert_array_equal(r["raw_image"], r_ref["raw_image"])
    np.testing.assert_array_equal(r["raw_totals"], r_ref["raw_totals"])
    np.testing.assert_array_equal(r["radial"], r_ref["radial"])
    assert sum(1 for _ in open(log)) == 2
