"""The readings the paper leaves open (backtracking and trust-region
constants) are defined twice, independently: in the kernels' header and in
the oracle.  Parity means something only while both use the same values and
the public header documents them; this test reads the three sources."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def constants(path, pattern):
    text = open(os.path.join(ROOT, path)).read()
    return {name: float(value) for name, value in re.findall(pattern, text)}


def test_kernel_and_oracle_constants_agree():
    kern = constants("paper_2403_16341_gb300/csrc/nls_common.cuh",
                     r"constexpr (?:double|int) ((?:LS|TR)_[A-Z0-9_]+) = ([0-9.e+-]+);")
    orac = constants("oracle/nls_oracle.c",
                     r"static const (?:double|int) ((?:LS|TR)_[A-Z0-9_]+) = ([0-9.e+-]+);")
    assert len(kern) == 10 and kern == orac, (kern, orac)


def test_public_header_documents_the_values():
    text = open(os.path.join(ROOT, "include", "nls.h")).read()
    kern = constants("paper_2403_16341_gb300/csrc/nls_common.cuh",
                     r"constexpr (?:double|int) ((?:LS|TR)_[A-Z0-9_]+) = ([0-9.e+-]+);")
    assert kern["LS_C1"] == 1e-4 and "c1 = 1e-4" in text
    assert kern["LS_RHO"] == 0.5 and "step factor 1/2" in text
    assert kern["LS_MAX_TRIALS"] == 30 and "at most 30 trials" in text
    assert kern["TR_DELTA0"] == 1.0 and "Delta_0 = 1" in text
    assert kern["TR_GROW"] == 2.0 and kern["TR_DELTA_MAX"] == 1e3 and "x2 (cap 1e3)" in text
    assert kern["TR_ETA_EXPAND"] == 0.75 and "rho > 0.75" in text
    assert kern["TR_SHRINK"] == 0.25 and "shrink x1/4" in text
    assert kern["TR_MAX_REJECTIONS"] == 32 and "32 rejections" in text
    assert kern["TR_NW_ETA"] == 1e-4 and "rho > 1e-4" in text
