"""Every ncu summary under profiles/ gives the command that made it, and
that command runs committed code: bench.py with options bench.py accepts."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_options():
    src = open(os.path.join(ROOT, "bench.py")).read()
    return set(re.findall(r'add_argument\("(--[a-z0-9-]+)"', src))


def test_profiles_name_their_commands_and_use_existing_options():
    opts = _bench_options()
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")))
    assert files
    for path in files:
        text = open(path).read()
        assert "ncu " in text and "--clock-control none" in text, path
        for line in text.splitlines():
            if "bench.py" not in line:
                continue
            tail = line.split("bench.py", 1)[1]
            for flag in re.findall(r"(--[a-z0-9-]+)", tail):
                assert flag in opts, (os.path.basename(path), flag)
        for line in text.splitlines():
            if line.strip().startswith("ncu "):      # every ncu command leaves the clocks alone
                assert "--clock-control none" in line, (path, line)
