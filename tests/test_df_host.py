"""The FP64 step's hybrid arithmetic, built for the host from the same header the CUDA
kernel compiles (lbm_df.cuh, lbm_collide_df.cuh), against long-double references:

- the exact 64-bit fixed-point conversion of a double (2^-58 units, round half away); the
  six-instruction one for 2^-6 <= d < 16, which must flag every other input; and the one
  that scales through the exponent field and rounds on the FP64 pipe (ties to even), ties
  included;
- the fixed-point and FP64 to double-float conversions (relative error below 2^-47);
- the double-float to double conversion (the nearest double, every case);
- the LBGK + Guo collision of Eq. 2, 3, 7 (agreement with long double per population,
  and mass, over random states with |u| up to 0.17, 2 % non-equilibrium, tau 0.51..2;
  some of them with populations below 2^-6, whose moments take the fallback conversion);
- its form for a force along x (the terms of F_y, F_z left out) against the general form,
  bit for bit;
- the equilibrium closures of inlet nodes (f^eq(rho, u_in)) and outlet nodes
  (f^eq(rho_out, u)) in the same arithmetic;
- the collision's form for the incompressible equilibrium (Eq. 4, 6).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def measured(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dfhost") / "df_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(ROOT, "tests", "df_host_check.cpp")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_fixed_point_conversion_is_exact(measured):
    assert measured["fix_mismatches"] == 0


def test_fast_fixed_point_conversion_flags_every_input_outside_its_range(measured):
    # 2^-6 <= d < 16: the same integer as the exact conversion; anything else is flagged
    assert measured["fix_fast_mismatches"] == 0
    assert measured["fix_fast_flag_errors"] == 0


def test_fixed_point_conversion_on_the_fp64_pipe_rounds_to_nearest_even(measured):
    assert measured["fix_cvt_mismatches"] == 0


def test_pair_conversions_within_2_pow_minus_47(measured):
    assert measured["df_from_fix_rel"] <= 2.0 ** -47
    assert measured["df_from_double_rel"] <= 2.0 ** -47


def test_pair_to_double_rounds_to_nearest(measured):
    assert measured["to_double_mismatches"] == 0


def test_hybrid_collision_matches_long_double(measured):
    # about 2^-48 relative per double-float operation: 4.1e-14 of w_i measured
    assert measured["collide_abs_over_w"] <= 1e-13
    assert measured["collide_mass_rel"] <= 5e-14
    # the random states include nodes whose moments take the FP64-pipe conversion
    assert measured["collide_fallback_states"] > 1000


def test_incompressible_form_matches_long_double(measured):
    assert measured["collide_inc_abs_over_w"] <= 1e-13


def test_equilibrium_closures_match_long_double(measured):
    # inlet rho * kin_i (two FP64 roundings) and outlet in double-float: ~1e-15 of w_i
    assert measured["closure_abs_over_w"] <= 1e-13


def test_force_along_x_form_equals_the_general_form(measured):
    assert measured["collide_xf_mismatches"] == 0
