"""The warp kernels compute 2048 * floor(sx) + q in one fma + floor for coordinates in
[0, 4094) (the per-tile fast path); this checks that form against the definition of the
11-bit weight for every fp32 value of the range (about 1.1e8 values, ~2 s of C)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fast_weight_form_is_exact_on_its_range(tmp_path):
    exe = tmp_path / "fast_weight_identity"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-o", str(exe),
                           os.path.join(HERE, "fast_weight_identity.c"), "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 bad" in r.stdout
