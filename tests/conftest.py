import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Everything the tests write (pytest's tmp_path, tempfile, the rendezvous files
# of torchrun children) stays inside the working tree, under .tmp/.
TMP = os.path.join(ROOT, ".tmp")
os.makedirs(TMP, exist_ok=True)
os.environ["TMPDIR"] = TMP
tempfile.tempdir = TMP


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built engine")
    if config.option.basetemp is None:
        config.option.basetemp = os.path.join(TMP, "pytest")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """The engine, built in-tree and loaded, on a CUDA device."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device (run with -m 'not gpu')")
    from paper_2507_23189_gb300 import build
    build.build()
    import paper_2507_23189_gb300 as E
    E.lib()
    return E


@pytest.fixture(scope="session")
def ps_table(gpu):
    """Engine table for 5 um polystyrene in water at 532 nm, 4096 bins."""
    return gpu.PhaseTable(diameter_um=5.0, n_particle=1.59, n_medium=1.33, wavelength_nm=532.0)


@pytest.fixture(scope="session")
def ps_oracle_table(oracle_mod):
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    return oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x)
