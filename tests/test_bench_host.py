"""Host-side logic of bench.py that needs no GPU: the algorithmic operation counts behind the ALU
roofline and the source hash that guards the committed DRAM traffic figures."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fft_operation_counts():
    """Counts of the unnormalised double-float forms (add 8, multiply 4, complex multiply 32):
    a 512-point radix-8 FFT is 3 stages of 64 butterflies (432 operations each) with 7 twiddle
    products (224) in the first two; per real point of a 1024-point DCT that is 109, plus the
    Hermitian split and quarter-wave twiddle (168 per 4 points forward, 160 inverse)."""
    assert bench.fft_ops(512, "df") == 3 * 64 * 432 + 2 * 64 * 224
    assert bench.fft_ops(512, "df") / 1024 == 109.0
    assert bench.line_ops_per_real("dct2", 1024, "df") == 109.0 + 42.0
    assert bench.line_ops_per_real("dct3", 1024, "df") == 109.0 + 40.0
    # FP32: complex add 2, complex multiply 4 (FMUL + FFMA per component)
    assert bench.fft_ops(8, "f32") == 2 * 8 * 2 + 4 + 4 + 8 * 2


def test_code_hash_ignores_comments_only():
    src = "int f(int a) { return a + 1; }  // add one\n/* block\n comment */\n"
    same = "// header\nint f(int a)   {\n  return a + 1;\n}\n"
    other = "int f(int a) { return a + 2; }\n"
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)


def test_committed_traffic_is_for_the_bench_workload():
    with open(os.path.join(ROOT, "profiles", "dram_traffic_solve_f64.json")) as fh:
        d = json.load(fh)
    assert d["bc"] == bench.BC
    assert set(d["per_launch_bytes_at_1024"]) == {"x-forward", "y-forward", "z-solve", "y-inverse", "x-inverse"}
    # every line kernel moves at least its algorithmic 2 x 8.59 GB at 1024^3 (read and write the
    # spectral spill); the checkpointed z sweeps move 3 + 2/8 spill values per value of the 2
    alg = 2 * 8 * 1024 ** 3
    for stage, v in d["per_launch_bytes_at_1024"].items():
        if stage == "z-solve":
            assert 1.5 * alg < v < 1.75 * alg
        else:
            assert v > 0.9 * alg
