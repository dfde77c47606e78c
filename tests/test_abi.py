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
    for must in ("spamm_tree_build", "spamm_multiply", "sp2_solve", "spamm_task_list",
                 "spamm_to_dense", "spamm_norms", "spamm_free", "spamm_strerror"):
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
