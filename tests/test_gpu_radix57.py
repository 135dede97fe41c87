"""Line lengths with factors 5 and 7 (radix-5 and radix-7 butterflies of the run-time-length
kernels) against the oracle, for every transform kind: real DFT and complex columns (periodic),
DCT/DST types II/III (Neumann / Dirichlet pairs) and types IV (mixed faces)."""
import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests.gpu_common import gpu_solve, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


CASES = [((6, 10, 14), "NNDDNN"),    # M = 7 along x, 5 along y
         ((5, 20, 28), "PPDNND"),    # periodic x (M = 14), DST-IV along y (M = 10)
         ((4, 70, 50), "DNPPDD"),    # DST-IV x (M = 25 = 5 x 5), C2C columns of 70 (= 2 x 5 x 7)
         ((7, 14, 40), "NDNNPP"),    # DCT-IV x (M = 20), periodic z
         ((3, 98, 30), "PPPPNN"),    # R2C x (M = 15), C2C y (98 = 2 x 7 x 7)
         ((4, 56, 2), "NNPPDD"),     # y periodic only: R2C columns of 56
         ((3, 6, 2940), "DDNNDD")]   # long x line: M = 1470 = 2 x 3 x 5 x 7 x 7


@pytest.mark.parametrize("shape,bc", CASES)
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("mixed_f64io", 1e-6)])
def test_radix57_parity(oracle, shape, bc, dtype, tol):
    sp = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
    f = workloads.uniform_source(shape, seed=sum(shape))
    ref = oracle.solve(f, bc, sp)
    assert rel_l2(gpu_solve(f, bc, sp, dtype), ref) <= tol
