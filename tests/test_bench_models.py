"""The work models bench.py divides by, against counts fixed elsewhere.

- Products: Thm 5.2 counts 16mnsp real multiplications and 8m(n-1)sp + 8mnsp additions for the
  per-frequency products, 32mnsp - 8msp in all. bench.py reports the round 32mnsp: 8msp more, a
  relative excess of at most 1/(4n - 1).
- Transforms: a radix-2 FFT of length p = 2^r has (p/2) r butterflies of 10 real flops (one complex
  multiplication, two complex additions). That is 5 p log2 p, counted here by running the butterfly
  recursion. A quaternion tube is two complex tubes, and a product transforms A, B forward and C
  back.
- Per-workload totals: the paper-derived figures for the colour-video and 1024^3 x 128 workloads
  (37.7 + 0.81 and 4398 + 28.2 GFLOP).
"""
import math

import pytest

import bench


def radix2_flops(p):
    """Real flops of an iterative radix-2 FFT of length p, by walking its stages and butterflies."""
    flops, half = 0, 1
    while half < p:
        for _start in range(0, p, 2 * half):
            for _j in range(half):
                flops += 6 + 2 + 2      # twiddle product (4 mul + 2 add), then a + t and a - t
        half *= 2
    return flops


@pytest.mark.parametrize("m,n,s,p", [(240, 320, 240, 64), (1024, 1024, 1024, 128), (128, 64, 128, 32),
                                     (8, 8, 8, 16), (3, 5, 7, 2)])
def test_products_bound_the_theorem_count(m, n, s, p):
    thm52 = 16 * m * n * s * p + 8 * m * (n - 1) * s * p + 8 * m * n * s * p
    ffts = 10.0 * p * math.log2(p) * (m * n + n * s + m * s)
    gemm = bench.effective_flops(m, n, s, p) - ffts
    assert gemm - thm52 == pytest.approx(8 * m * s * p, rel=1e-12)     # the 8msp of the rounding
    assert (gemm - thm52) / thm52 <= 1 / (4 * n - 1) + 1e-15


@pytest.mark.parametrize("p", [2, 4, 8, 16, 32, 64, 128, 1024])
def test_transform_count_is_the_radix2_butterfly_count(p):
    m, n, s = 3, 4, 5
    tubes = m * n + n * s + m * s
    ffts = bench.effective_flops(m, n, s, p) - 32.0 * m * n * s * p
    assert ffts == pytest.approx(2 * tubes * radix2_flops(p), rel=1e-12)


def test_backward_is_two_products_and_five_transforms():
    m, n, s, p = 128, 64, 128, 32
    per_tube = radix2_flops(p)
    # forward transforms of A, B, dC; inverse of dA (m x n) and dB (n x s); two complex tubes each
    tubes = 2 * (m * n + n * s + m * s + m * n + n * s)
    assert bench.backward_flops(m, n, s, p) == pytest.approx(2 * 32.0 * m * n * s * p + tubes * per_tube, rel=1e-12)


def test_workload_totals():
    video = bench.effective_flops(240, 320, 240, 64)
    assert video == pytest.approx(37.75e9 + 0.811e9, rel=1e-3)
    big = bench.effective_flops(1024, 1024, 1024, 128)
    assert big == pytest.approx(4398.0e9 + 28.2e9, rel=1e-3)


def test_tsvd_work_count():
    """Per frequency pair {f, -f} (p // 2 + 1 of them) the thin SVD of a 2 max(m, n) x 2 min(m, n)
    complex matrix, 4 (6 R C^2 + 20 C^3) real flops."""
    m, n, p = 128, 64, 32
    R, C = 256, 128
    assert bench.tsvd_flops(m, n, p) == 17 * 4 * (6 * R * C * C + 20 * C ** 3)
    assert bench.tsvd_flops(n, m, p) == bench.tsvd_flops(m, n, p)
    assert bench.tsvd_flops(m, n, 31) == 16 * 4 * (6 * R * C * C + 20 * C ** 3)
