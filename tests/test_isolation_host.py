"""The product and the oracle stay apart: importing and using the engine's
Python package loads nothing from oracle/, no product source names the
oracle, and the engine library fails loudly instead of falling back when it
has not been built."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2507_23189_gb300")


def _product_sources():
    for d, _, files in os.walk(PKG):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                yield os.path.join(d, f)
    yield os.path.join(ROOT, "include", "mcmie.h")


def test_no_product_source_refers_to_the_oracle():
    for path in _product_sources():
        text = open(path).read()
        assert not re.search(r"\boracle\b", text, flags=re.I), path


def test_importing_the_package_loads_no_oracle_module():
    code = ("import sys; import paper_2507_23189_gb300 as E; "
            "from paper_2507_23189_gb300 import engine, checkpoint, autotune, workloads, build; "
            "E.PhaseTable(); "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "print(bad); sys.exit(1 if bad else 0)")
    from paper_2507_23189_gb300 import build
    build.build()
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr


def test_missing_engine_library_raises(monkeypatch, tmp_path):
    from paper_2507_23189_gb300 import _native as N
    monkeypatch.delenv("MC_CHECKED", raising=False)
    monkeypatch.setattr(N, "_lib", None)
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "absent.so"))
    try:
        N.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("lib() loaded something although the library is absent")
