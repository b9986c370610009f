"""The double-float arithmetic behind the FP32-mixed CG scalars
(csrc/dfloat.cuh), compiled for the host and compared with long double (no
GPU): TwoSum and FastTwoSum are exact, products and quotients carry about
2⁻⁴⁶ relative error, differences about 2⁻⁴⁸ of the larger operand, and the
Chronopoulos–Gear denominator δ − β·c keeps nine correct digits where δ and
β·c agree to 1e-4, where plain FP32 keeps two or three."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("dfloat") / "dfloat_check")
    subprocess.run([gxx, "-O2", "-std=c++17", os.path.join(HERE, "dfloat_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


def test_error_free_sums_are_exact(errors):
    assert errors["two_sum_err"] == 0.0
    assert errors["fast_two_sum_err"] == 0.0


def test_products_and_quotients(errors):
    assert errors["mul_rel"] <= 2.0 ** -45
    assert errors["div_rel"] <= 2.0 ** -45


def test_differences_relative_to_operands(errors):
    assert errors["sub_rel_to_operand"] <= 2.0 ** -47


def test_cg_denominator_survives_cancellation(errors):
    # δ − β·c with δ = β·c·(1 + O(1e-4)): the inputs are exact pairs, so
    # the only errors are those of ff_mul and ff_sub, amplified by 1e4
    assert errors["cg_denominator_rel"] <= 1e-9
    # the plain FP32 evaluation keeps only two or three digits of it
    assert errors["cg_denominator_rel_fp32"] >= 1e-4
