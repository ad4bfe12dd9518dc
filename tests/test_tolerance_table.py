"""The measured-bounds table of the parity tests follows its own rule: every
entry is the error measured on GB300 (the comment beside it) times 1.1,
rounded up to two significant digits, and no entry reaches below the
stated bound it replaces.  A bound widened by hand without a measurement
fails here."""
import math
import os
import re

import pytest

import tolerances as T

HERE = os.path.dirname(os.path.abspath(__file__))
ENTRY = re.compile(r'^\s*"([\w.]+)":\s*([0-9.eE+-]+),\s*#\s*([0-9.eE+-]+)\s*$')
CASE = re.compile(r'^\s*"([\w]+)":\s*\{\s*$')


def _ceil2(x):
    """x rounded up to two significant digits."""
    e = math.floor(math.log10(x)) - 1
    q = 10.0 ** e
    return math.ceil(x / q - 1e-9) * q


def _entries():
    """(case, tensor, bound, measured) for every entry of MEASURED, read from
    the source so that the measured value in each comment is checked too."""
    out, case, inside = [], None, False
    with open(os.path.join(HERE, "tolerances.py")) as f:
        for line in f:
            if line.startswith("MEASURED = {"):
                inside = True
                continue
            if inside and line.startswith("}"):
                break
            if not inside:
                continue
            m = CASE.match(line)
            if m:
                case = m.group(1)
                continue
            m = ENTRY.match(line)
            if m:
                out.append((case, m.group(1), float(m.group(2)), float(m.group(3))))
    return out


def test_every_entry_has_its_measurement():
    ents = _entries()
    n = sum(len(v) for v in T.MEASURED.values())
    assert len(ents) == n and n > 0
    for case, name, bound, _ in ents:
        assert T.MEASURED[case][name] == bound, (case, name)


def _half_ulp(text_value):
    """Half a unit in the last printed digit of the comment's value."""
    v = float(text_value)
    digits = len(re.sub(r"[^0-9]", "", ("%.3g" % v)).lstrip("0"))
    return 0.5 * 10.0 ** (math.floor(math.log10(v)) - digits + 1)


@pytest.mark.parametrize("case,name,bound,measured", _entries())
def test_bound_is_measured_plus_ten_percent(case, name, bound, measured):
    # the comment prints the measurement to three significant digits; the
    # bound was taken from the unrounded value, so it lies between the rule
    # applied to the two ends of the interval that rounds to the comment
    h = _half_ulp(measured)
    lo, hi = _ceil2((measured - h) * 1.1), _ceil2((measured + h) * 1.1)
    assert lo - 1e-12 <= bound <= hi + 1e-12, (case, name, bound, measured, lo, hi)
    stated = T.FP32_GRAD_TOL if "fp32" in case else T.BF16_GRAD_TOL
    assert bound > stated, (case, name, "a measured bound replaces only a stated bound it exceeds")
