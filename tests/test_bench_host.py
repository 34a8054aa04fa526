"""Host-side pieces of the benchmark (no GPU): the algorithmic byte count of the feature kernel
and the code digest that keys the stored DRAM traffic figures."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1504_01883_gb300 import synth  # noqa: E402


def test_algorithmic_bytes_count_in_frame_pixels_and_outputs():
    r = np.zeros(3, synth.RECT_DTYPE)
    r[0] = (0, 10, 20, 100, 50)      # inside: 5000 px
    r[1] = (0, -30, -10, 50, 40)     # clipped to 20 x 30 = 600 px
    r[2] = (1, 600, 400, 200, 200)   # clipped to 40 x 80 = 3200 px
    crop, dim, k_pad = 64, 16 * 59, 1024
    got = bench.algorithmic_bytes_k1(r, 480, 640, crop, 2, k_pad, dim)
    grey = 5000 + 600 + 3200
    depth = 2 * (min(5000, 4096) + 600 + 3200)   # depth sampled at most crop^2 times
    out = 3 * (2 * dim + 2 * k_pad + 4)
    assert got == grey + depth + out


def test_code_digest_ignores_comments_and_blank_space(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\nint f(int x) {\n    return x + 1;  // add one\n}\n")
    b.write_text("/* another\n   header */\nint f(int x)\n{ return x + 1; }\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_stored_traffic_needs_the_captured_layout():
    for stage, (fname, digest, key, nbytes) in bench.MEASURED_TRAFFIC.items():
        assert bench.measured_traffic(stage, key + "/other") is None
        path = os.path.join(ROOT, "paper_1504_01883_gb300", "csrc", fname)
        want = nbytes if bench.code_digest(path) == digest else None
        assert bench.measured_traffic(stage, key) == want
