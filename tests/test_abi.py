"""The C-ABI library loads and exports every entry point that include/*.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            if m.group(1) not in ("if", "while", "sizeof", "defined"):
                names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("spamm_tree_build", "spamm_multiply", "spamm_multiply_batched", "sp2_solve",
                 "spamm_task_list", "spamm_to_dense", "spamm_norms", "spamm_free", "spamm_strerror",
                 "spamm_autotune_batched", "spamm_release_scratch", "spamm_cull_noalloc"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1403_7458_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_1403_7458_gb300 import spamm
    lib = spamm.load()
    assert lib.spamm_strerror(0) == b"ok"
    assert lib.spamm_strerror(-6).startswith(b"SP2")
    assert lib.spamm_strerror(-99) == b"unknown status"


def test_binding_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal the C structs of
    include/spamm.h (compiled here with the host C compiler)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    from paper_1403_7458_gb300 import spamm
    structs = {"spamm_opts_t": spamm._Opts, "spamm_stats_t": spamm._Stats, "sp2_opts_t": spamm._Sp2Opts,
               "sp2_report_t": spamm._Sp2Report, "spamm_tune_t": spamm._Tune}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "spamm.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, cls in structs.items():
        assert int(got["%s size" % cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, precision modes, flags, SP2 rules, stop reasons and
    history columns of the binding equal the values include/spamm.h defines
    (printed by a program compiled here with the host C compiler)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    from paper_1403_7458_gb300 import spamm
    pairs = {
        "SPAMM_OK": spamm.OK, "SPAMM_E_INVAL": spamm.E_INVAL, "SPAMM_E_NOMEM": spamm.E_NOMEM,
        "SPAMM_E_CUDA": spamm.E_CUDA, "SPAMM_E_CAPACITY": spamm.E_CAPACITY, "SPAMM_E_TIMEOUT": spamm.E_TIMEOUT,
        "SPAMM_E_NOCONV": spamm.E_NOCONV, "SPAMM_E_NOTSUP": spamm.E_NOTSUP,
        "SPAMM_FP64": spamm.FP64, "SPAMM_OZAKI_BF16": spamm.OZAKI_BF16, "SPAMM_BF16": spamm.BF16,
        "SPAMM_BF16X3": spamm.BF16X3, "SPAMM_TF32": spamm.TF32, "SPAMM_TF32X3": spamm.TF32X3,
        "SPAMM_F_TIMING": spamm.F_TIMING, "SPAMM_F_NOSYM": spamm.F_NOSYM, "SPAMM_F_HEAVIEST": spamm.F_HEAVIEST,
        "SPAMM_F_NOGRAPH": spamm.F_NOGRAPH, "SPAMM_TUNE_MAX": spamm.TUNE_MAX,
        "SP2_RULE_TRACE_DISTANCE": spamm.RULE_TRACE_DISTANCE, "SP2_RULE_TRACE_ABOVE": spamm.RULE_TRACE_ABOVE,
        "SP2_STOP_CONVERGED": spamm.STOP_CONVERGED, "SP2_STOP_STAGNATED": spamm.STOP_STAGNATED,
        "SP2_STOP_FIXED": spamm.STOP_FIXED, "SP2_STOP_MAXITER": spamm.STOP_MAXITER,
        "SP2_H_FILL": spamm.H_FILL, "SP2_H_COLS": spamm.H_COLS,
    }
    lines = ["#include <stdio.h>", '#include "spamm.h"', "int main(void) {"]
    for cname in pairs:
        lines.append('printf("%s %%d\\n", (int)(%s));' % (cname, cname))
    lines += ["return 0; }"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {k: int(v) for k, v in (line.split() for line in out if line)}
    for cname, value in pairs.items():
        assert got[cname] == value, (cname, got[cname], value)
