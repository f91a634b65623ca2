"""Host-side pieces of the Python binding that need no GPU: the trace record
decoder (the layout include/mcmie.h documents for mc_trace) and the medium
argument checks."""
import numpy as np
import pytest

import paper_2507_23189_gb300 as gpu


def test_decode_trace_reads_the_documented_record():
    rec = np.zeros((2, 3, 12), dtype=np.int32)
    f = rec.view(np.float32)
    rec[0, 0, 0] = 0                                   # collision
    f[0, 0, 1:4] = (1.5, -2.25, 3.0)                   # position after the flight
    f[0, 0, 4:7] = (0.6, 0.0, -0.8)                    # direction after the event
    f[0, 0, 7] = 0.875                                 # weight
    f[0, 0, 8] = 1.25e-3                               # camera contribution
    rec[0, 0, 9:12] = (4099, 17, -1)                   # pixel, camera table bin, radial bin
    rec[0, 1, 0] = 2                                   # far-face exit
    rec[0, 1, 11] = 63
    rec[1, :, 0] = -1                                  # no event recorded
    t = gpu.decode_trace(rec)
    assert t["status"].tolist() == [[0, 2, 0], [-1, -1, -1]]
    np.testing.assert_array_equal(t["r"][0, 0], [1.5, -2.25, 3.0])
    np.testing.assert_array_equal(t["d"][0, 0], [0.6000000238418579, 0.0, -0.800000011920929])
    assert t["w"][0, 0] == 0.875 and t["nee"][0, 0] == np.float32(1.25e-3)
    assert (t["pix"][0, 0], t["nee_bin"][0, 0], t["rad_bin"][0, 0]) == (4099, 17, -1)
    assert t["rad_bin"][0, 1] == 63
    assert t["r"].dtype == np.float64 and t["pix"].dtype == np.int32


def test_medium_phase_checks():
    m = gpu.Medium(0.1, 0.0, "paper", 0.0, None)
    with pytest.raises(ValueError):
        m.as_c()                                       # the paper scheme needs a PaperTable
    with pytest.raises(ValueError):
        gpu.Medium(0.1, 0.0, "isotropic", 0.0, None).as_c()
    c, keep = gpu.Medium(0.2, 0.01, "hg", 0.85, None).as_c()
    assert keep is None and (c.mu_s, c.mu_a, c.hg_g) == pytest.approx((0.2, 0.01, 0.85))


def test_run_params_carry_every_field():
    rp = gpu.run_params(123, seed=7, photon_offset=5, rr_threshold=1e-3, rr_survival=0.0, max_events=99,
                        max_scatter=2, image_frac_bits=24, accumulate=True, block_size=512, blocks_per_sm=1,
                        image_mode=2)
    assert (rp.n_photons, rp.photon_offset, rp.seed, rp.max_events, rp.max_scatter, rp.image_frac_bits,
            rp.accumulate, rp.block_size, rp.blocks_per_sm, rp.image_mode) == (123, 5, 7, 99, 2, 24, 1, 512,
                                                                              1, 2)
    assert (rp.rr_threshold, rp.rr_survival) == (1e-3, 0.0)


def test_check_reports_then_clears_the_flags_on_the_checked_stream(monkeypatch):
    """Engine.check: mc_check's status is raised as McError, and the error
    word is cleared afterwards on the stream that was checked (also when it
    raises), so the next check reports only new flags and no run pays a
    device operation for it. check_within clears only once the work is done."""
    import contextlib
    import types

    import torch

    from paper_2507_23189_gb300 import _native as N
    from paper_2507_23189_gb300 import engine as eng_mod
    log = []

    @contextlib.contextmanager
    def stream_ctx(s):
        log.append(("enter", s))
        yield
        log.append(("exit", s))

    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        stream=stream_ctx, current_stream=lambda dev=None: ("current", str(dev))))
    monkeypatch.setattr(eng_mod, "_torch", lambda: fake_torch)
    monkeypatch.setattr(eng_mod, "_stream_handle", lambda s: s)

    class Word:
        device = torch.device("cpu")

        def __init__(self, v):
            self.v = v

        def data_ptr(self):
            return 1234

        def zero_(self):
            log.append(("zero",))
            self.v = 0

        def cpu(self):
            return types.SimpleNamespace(numpy=lambda: np.array([self.v], dtype=np.int32))

    status = {"check": 0, "within": 0}
    fake_lib = types.SimpleNamespace(
        mc_check=lambda ptr, st: (log.append(("mc_check", st)), status["check"])[1],
        mc_check_within=lambda ptr, st, ms: (log.append(("mc_check_within", st)), status["within"])[1])
    monkeypatch.setattr(N, "lib", lambda: fake_lib)

    e = object.__new__(gpu.Engine)
    e.error = Word(0)
    e.check("s1")
    assert log == [("mc_check", "s1"), ("enter", "s1"), ("zero",), ("exit", "s1")]

    log.clear()
    e.error = Word(N.EFLAG_EVENTS)
    status["check"] = -7
    with pytest.raises(N.McError) as err:
        e.check(None)
    assert err.value.status == -7 and e.error.v == 0
    assert e.last_error == N.EFLAG_EVENTS          # the word read before it was cleared
    assert log[1] == ("enter", ("current", "cpu")) and ("zero",) in log

    log.clear()
    e.error = Word(N.EFLAG_TIMEOUT)
    status["within"] = N.MC_NOT_READY
    assert e.check_within(5.0, "s2") is False
    assert e.error.v == N.EFLAG_TIMEOUT and ("zero",) not in log     # still running: nothing cleared
    status["within"] = 0
    assert e.check_within(5.0, "s2") is True and e.error.v == 0
