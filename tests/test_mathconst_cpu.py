"""The committed constants header of the kernels' exp and erfcx
(csrc/lskum_mathconst.h) is exactly what the committed generator writes:
regenerating it (mpmath, about ten seconds, including the generator's own
checks of the interpolants and of the fixed-point integer steps against
exact arithmetic) reproduces the file byte for byte."""
import importlib.util
import os
import tempfile

import pytest

pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2406_07441_gb300", "csrc")


def test_header_equals_the_generators_output():
    spec = importlib.util.spec_from_file_location("gen_mathconst", os.path.join(CSRC, "gen_mathconst.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "lskum_mathconst.h")
        gen.main(out)
        with open(out) as f:
            fresh = f.read()
    with open(os.path.join(CSRC, "lskum_mathconst.h")) as f:
        committed = f.read()
    assert fresh == committed
