"""The ctypes binding agrees with include/mcmie.h: every struct's size and
field offsets, and every status, flag, phase and totals constant, as a C
compiler lays them out from the header itself."""
import ctypes
import json
import os
import re
import shutil
import subprocess

import pytest

from paper_2507_23189_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# header struct name -> ctypes class (field names are the same on both sides)
STRUCTS = {"mie_params": N.MieParams, "mie_info": N.MieInfo, "mc_medium": N.Medium,
           "mc_geometry": N.Geometry, "mc_camera": N.Camera, "mc_run_params": N.RunParams,
           "mc_tallies": N.Tallies, "mc_instance": N.Instance, "mc_grid": N.Grid}

CONSTANTS = {"MC_NOT_READY": N.MC_NOT_READY, "MC_OK": N.MC_OK,
             **{name: code for code, name in N.STATUS.items()},
             "MC_EFLAG_EVENTS": N.EFLAG_EVENTS, "MC_EFLAG_TIMEOUT": N.EFLAG_TIMEOUT,
             "MC_EFLAG_NUMERIC": N.EFLAG_NUMERIC, "MC_EFLAG_OVERFLOW": N.EFLAG_OVERFLOW,
             "MC_EFLAG_TABLE": N.EFLAG_TABLE, "MC_EFLAG_BOUNDS": N.EFLAG_BOUNDS,
             "MC_PHASE_TABLE": N.PHASE_TABLE, "MC_PHASE_HG": N.PHASE_HG, "MC_PHASE_PAPER": N.PHASE_PAPER,
             "MC_TOT_REFLECT": N.TOT_REFLECT, "MC_TOT_FAR": N.TOT_FAR, "MC_TOT_SIDE": N.TOT_SIDE,
             "MC_TOT_ABSORB": N.TOT_ABSORB, "MC_TOT_ROULETTE": N.TOT_ROULETTE, "MC_TOT_TRUNC": N.TOT_TRUNC,
             "MC_TOT_BALLISTIC": N.TOT_BALLISTIC, "MC_TOT_STEPS": N.TOT_STEPS,
             "MC_N_TOTALS": N.N_TOTALS, "MC_WEIGHT_FRAC_BITS": N.WEIGHT_FRAC_BITS}


def _probe_source():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcmie.h"', "int main(void) {",
             '    printf("{\\"structs\\": {");']
    for i, (cname, cls) in enumerate(STRUCTS.items()):
        sep = "," if i else ""
        lines.append('    printf("%s\\"%s\\": {\\"size\\": %%zu, \\"offsets\\": {", sizeof(%s));' % (sep, cname, cname))
        for j, (f, _) in enumerate(cls._fields_):
            fsep = "," if j else ""
            lines.append('    printf("%s\\"%s\\": %%zu", offsetof(%s, %s));' % (fsep, f, cname, f))
        lines.append('    printf("}}");')
    lines.append('    printf("}, \\"constants\\": {");')
    for i, name in enumerate(CONSTANTS):
        sep = "," if i else ""
        lines.append('    printf("%s\\"%s\\": %%lld", (long long)(%s));' % (sep, name, name))
    lines += ['    printf("}}\\n");', "    return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def header_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text(_probe_source())
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(header_layout, cname):
    cls = STRUCTS[cname]
    got = header_layout["structs"][cname]
    assert ctypes.sizeof(cls) == got["size"], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == got["offsets"][f], (cname, f)


def test_constants_match_header(header_layout):
    assert header_layout["constants"] == CONSTANTS


def test_every_status_in_the_header_is_in_the_binding():
    text = open(os.path.join(ROOT, "include", "mcmie.h")).read()
    enum = text[text.index("typedef enum"):text.index("} mc_status;")]
    names = set(re.findall(r"\b(MC_(?:OK|NOT_READY|ERR_[A-Z]+))\s*=", enum))
    assert names == set(N.STATUS.values())
