"""The oracle and the product share no code: the package (Python binding
and CUDA sources) never imports, includes or loads anything under oracle/,
and the oracle never imports the package or includes its sources.  The
seeded input generators (synth.py) hold none of the method's arithmetic and
are the one module both sides' callers use."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2603_15447_gb300")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s+[\"<][^\">]*oracle)", re.M)
    for p in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
        text = open(p, encoding="utf-8").read()
        assert not pat.search(text), p
        assert "oracle/" not in text and "liboracle" not in text, p


def test_oracle_does_not_use_the_package():
    pat = re.compile(r"^\s*(import\s+paper_2603_15447_gb300|from\s+paper_2603_15447_gb300|#\s*include\s+[\"<][^\">]*"
                     r"(csrc|bez\.h|curve_eval|common\.cuh))", re.M)
    for p in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(p, encoding="utf-8").read()
        assert not pat.search(text), p
        assert "libbez" not in text, p


def test_synth_holds_no_curve_arithmetic():
    # the generators draw numbers; no Bernstein, Horner, de Casteljau or hash-to-parameter evaluation
    text = open(os.path.join(PKG, "synth.py"), encoding="utf-8").read()
    for word in ("bernstein", "casteljau", "horner", "seiler", "def bezier"):
        assert word not in text.lower(), word
