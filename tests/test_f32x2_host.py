"""Host check of the pair-of-FP32 arithmetic used by the QMC_FP32X2 form, and
of the digit slicing that lets the tensor cores contract pairs exactly.

The header paper_2506_09743_gb300/csrc/f32x2.cuh is compiled as plain C++ (no
FMA contraction) together with tests/f32x2_check.cpp, which compares every
operation with long-double references over random operands.  The bounds are
those of double-float arithmetic: about 2^-47 per operation (2^-44 for the
64-term dot products, relative to sum |a_k b_k|), far below the FP32 level
2^-24 that the FP32-AO forms stop at.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

BOUNDS = {
    "exp": 3e-14,     # relative, results above 2^-100
    "mul": 3e-14,
    "add": 3e-14,     # relative to the larger operand
    "div": 5e-14,
    "sqrt": 3e-14,
    "rsqrt": 5e-14,
    "dot": 2e-13,     # relative to sum |a_k b_k|, 64 terms
    "norm": 2.0 ** -24 * 1.001,  # |lo| <= ulp(hi) / 2 after normalisation
    # digit-sliced contraction: dropped digit classes and digit residuals,
    # at most 2^-46 per term of K 2^(e + f)
    "oz_contraction": 2.0 ** -46,
}


def test_digit_class_sums_stay_exact(results):
    """Every class sum of digit products stays below 2^24 (exact in FP32
    accumulation) and every digit is an integer of magnitude <= 256 (exact
    in BF16)."""
    assert results["oz_max_class_log2"] < 24.0
    assert results["oz_bad_digits"] == 0


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("f32x2") / "f32x2_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "f32x2_check.cpp")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


@pytest.mark.parametrize("op", sorted(BOUNDS))
def test_pair_arithmetic_accuracy(results, op):
    assert results[op] <= BOUNDS[op], (op, results[op])


def test_exp_results_are_normalised(results):
    assert results["exp_unnormalised"] == 0
