"""The oracle (oracle/elm_oracle.cpp) built under AddressSanitizer and
UndefinedBehaviorSanitizer runs a cross-section of its own pins: mesh and
location, P1 / P2 interpolation, the departure point and trace continuation,
the transpose and forward-mode derivative, mass and stiffness, the diffusion
step and the blended annulus.  Every parity claim rests on the oracle, so
undefined behaviour or an out-of-bounds access in it would undermine them; the
sanitizers stop the run at the first finding.  The pins themselves run as in
tests/test_oracle_pins.py, in a child process with the sanitizer runtime
preloaded (the Python interpreter is not instrumented).  Test infrastructure;
no GPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = " or ".join([
    "test_refinement_is_bey", "test_locate_brute_force", "test_locate_near_macro_interfaces",
    "test_p2_reproduction_interpolation", "test_p1_interpolation_brute_force",
    "test_rk4_linear_velocity_closed_form", "test_time_interpolation_direction", "test_trace_continuation_exact",
    "test_transpose_dot_product", "test_jvp_linear_fields_match_finite_differences", "test_p1_transpose_dot_product",
    "test_p2_mass_matrix_textbook", "test_p2_stiffness_reference_triangle_textbook",
    "test_diffusion_step_reproduces_fields_in_the_space", "test_blended_annulus_geometry",
    "test_blended_identity_and_constants"])

RUNNER = """
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
oracle.build = lambda force=False: {lib!r}
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", "-k", {pins!r}, {pin_file!r}]))
"""


def test_oracle_pins_under_sanitizers(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    asan = subprocess.run([gxx, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run([gxx, "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.isabs(ubsan)):
        pytest.skip("sanitizer runtimes not found")
    lib = str(tmp_path / "liboracle_sanitized.so")
    b = subprocess.run([gxx, "-O1", "-g", "-std=c++17", "-shared", "-fPIC", "-pthread", "-fno-omit-frame-pointer",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        os.path.join(ROOT, "oracle", "elm_oracle.cpp"), "-o", lib], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr
    runner = tmp_path / "run_pins.py"
    runner.write_text(RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, pins=PINS,
                                    pin_file=os.path.join(ROOT, "tests", "test_oracle_pins.py")))
    env = dict(os.environ, LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([sys.executable, str(runner)], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "passed" in r.stdout and "runtime error" not in r.stdout + r.stderr
