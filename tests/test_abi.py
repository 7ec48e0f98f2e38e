"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/tsunami.h (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess
import sys

from paper_1901_06798_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "tsunami.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tsu_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 19
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(binding.SYMBOLS) == syms


def test_config_struct_matches_header_field_order():
    txt = open(os.path.join(ROOT, "include", "tsunami.h")).read()
    body = txt[txt.index("typedef struct tsu_config {"):txt.index("} tsu_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_0-9]+)(?:\[[A-Z_0-9]+\])*(?:\[\d+\])?\s*[;,]", body)
    fields = [f[0] for f in binding.tsu_config._fields_]
    assert names == fields


def test_stats_struct_matches_header_field_order():
    txt = open(os.path.join(ROOT, "include", "tsunami.h")).read()
    body = txt[txt.index("typedef struct tsu_stats {"):txt.index("} tsu_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_0-9]+)(?:\[[A-Z_0-9]+\])*(?:\[\d+\])?\s*[;,]", body)
    fields = [f[0] for f in binding.tsu_stats._fields_]
    assert names == fields


def test_product_never_reaches_the_oracle():
    """The product path has no CPU fallback: no module of the package imports
    the oracle, and no CUDA or C++ source includes its headers."""
    pkg = os.path.join(ROOT, "paper_1901_06798_gb300")
    py = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert not py.search(open(path).read()), path
            elif f.endswith((".cu", ".cuh", ".cpp", ".h")):
                assert "oracle" not in "".join(re.findall(r'#include\s+"[^"]+"', open(path).read())), path


def test_binding_fails_loudly_without_its_library():
    """Pointed at a library that does not exist, the binding raises instead
    of falling back to anything."""
    code = ("from paper_1901_06798_gb300 import binding\n"
            "try:\n"
            "    binding.load('/nonexistent/libtsunami.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("raised"), (r.stdout, r.stderr[-1000:])
