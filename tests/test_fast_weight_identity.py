"""The warp kernels' per-tile fast path (coordinates in [0, 4094)) computes 2048 * floor(sx)
+ q with one fma rounded toward minus infinity (u8), and floor(sx) and the fp32 weight with
one rounded-down add and two exact subtractions (f32); this checks both forms against the
definitions for every fp32 value of the range (about 1.1e8 values, a few seconds of C)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fast_weight_form_is_exact_on_its_range(tmp_path):
    exe = tmp_path / "fast_weight_identity"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-frounding-math", "-o", str(exe),
                           os.path.join(HERE, "fast_weight_identity.c"), "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 bad" in r.stdout
