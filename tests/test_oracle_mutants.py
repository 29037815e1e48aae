"""Planted mistakes in the oracle (on the CPU): each mutant must fail at least one pin.

Every mutation below is a plausible slip in writing the definition (a dropped term, a wrong sign, a
wrong row or index, a transposed operand, an off-by-one bound, a wrong constant). The test compiles a
mutated copy of the oracle source, points the oracle module at it and runs the pin set of
`test_oracle_pins.py`; a mutant that passes every pin would mean the pins cannot tell it apart.
"""
from __future__ import annotations

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = [
    ("dropped translation term", "std::fma(M[0], X, M[3])", "std::fma(M[0], X, 0.0)"),
    ("transposed matrix operand", "std::fma(M[4], X, M[7])", "std::fma(M[1], X, M[7])"),
    ("clip z row used as depth", "std::fma(M[12], X, M[15])", "std::fma(M[8], X, M[11])"),
    ("wrong sign in y mapping", "std::fmaf(fcy / fw, 0.5f, 0.5f)", "std::fmaf(fcy / fw, -0.5f, 0.5f)"),
    ("transposed pixel index", "(int64_t)py * v.W + px", "(int64_t)px * v.H + py"),
    ("alpha leaks into key", "(uint64_t)(rgba & 0xFFFFFFu)", "(uint64_t)(rgba & 0xFFFFFFFFu)"),
    ("wrong key shift", "f.key = (q << 24)", "f.key = (q << 23)"),
    ("far plane inclusive", "w < v.far_)) return f;", "w <= v.far_)) return f;"),
    ("right edge inclusive", "fx < (float)v.W", "fx <= (float)v.W"),
    ("wrong linear scale", "1099511627776.0 / (v.far_ - v.near_)", "549755813888.0 / (v.far_ - v.near_)"),
    ("near added instead of subtracted", "const double d = w - v.near_;", "const double d = w + v.near_;"),
    ("depth cap off by one", "(1ull << 40) - 2;", "(1ull << 40) - 1;"),
    ("max instead of min", "f.key < fb[f.pixel]) fb[f.pixel] = f.key;", "f.key > fb[f.pixel]) fb[f.pixel] = f.key;"),
    ("exclusive HQ band", "<= (uint64_t)eps_num * (qmin + Nq)", "< (uint64_t)eps_num * (qmin + Nq)"),
    ("HQ band without near offset", "(uint64_t)eps_num * (qmin + Nq)", "(uint64_t)eps_num * (qmin)"),
    ("HQ average truncates", "(uint32_t)((sum_r[i] + c / 2) / c)", "(uint32_t)(sum_r[i] / c)"),
    ("paper's clear value as empty", "kEmpty = 0xFFFFFFFFFFFFFFFFull", "kEmpty = 0xFFFFFFFFFF000000ull"),
    ("piecewise range offset dropped", "base += std::ceil(", "base += 0.0 * std::ceil("),
    ("metric scale ignored", "t = w * v.metric_scale;", "t = w * 1024.0;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    oracle.use_library(lib)
    failed = []
    try:
        for check in pins.PINS:
            try:
                check()
            except AssertionError:
                failed.append(check.__name__)
            except ValueError:
                failed.append(check.__name__)
    finally:
        oracle.use_library(None)
    assert failed, f"no pin catches the planted mistake: {name}"
