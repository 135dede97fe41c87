"""Prototype tensor-core DFT stage (pp_proto_tc_gemm_check, pp_proto_dft32_tc), not used by the
solver: the operand-layout self-check of the tcgen05 descriptors against an integer matrix product,
and the 32-point DFTs against the CPU oracle's line transform and numpy's FFT."""
import ctypes

import numpy as np
import pytest

from paper_1909_05423_gb300 import _lib
from tests.gpu_common import need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


def _bf16_bits(a):
    return (np.asarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def test_descriptor_layout_self_check():
    """Integer-valued bf16 operands (|entries| <= 64): A B^T is exact in the FP32 accumulators, so
    the descriptor order the kernels use (leading offset = K groups 128 bytes apart, stride offset =
    row groups 1024 bytes apart) must reproduce it exactly; the swapped order must not."""
    lib = _lib.load()
    rng = np.random.default_rng(41)
    A = rng.integers(-64, 65, size=(128, 64)).astype(np.float32)
    B = rng.integers(-64, 65, size=(64, 64)).astype(np.float32)
    ref = (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64)
    a = torch.from_numpy(_bf16_bits(A).astype(np.int16)).cuda()
    b = torch.from_numpy(_bf16_bits(B).astype(np.int16)).cuda()
    out = {}
    for swap in (0, 1):
        d = torch.full((128, 64), float("nan"), dtype=torch.float32, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        _lib.check(lib.pp_proto_tc_gemm_check(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                              ctypes.c_void_p(d.data_ptr()), swap, ctypes.c_void_p(err.data_ptr()),
                                              None))
        torch.cuda.synchronize()
        assert int(err.item()) == 0, swap
        out[swap] = d.double().cpu().numpy()
    assert np.array_equal(out[0], ref)
    assert not np.array_equal(out[1], ref)


def _dft32(re, im):
    lib = _lib.load()
    lines = re.shape[0]
    r = torch.from_numpy(np.ascontiguousarray(re)).cuda()
    i = torch.from_numpy(np.ascontiguousarray(im)).cuda()
    orr = torch.full_like(r, float("nan"))
    oi = torch.full_like(i, float("nan"))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.check(lib.pp_proto_dft32_tc(ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(i.data_ptr()),
                                     ctypes.c_void_p(orr.data_ptr()), ctypes.c_void_p(oi.data_ptr()), lines,
                                     ctypes.c_void_p(err.data_ptr()), None))
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return orr.cpu().numpy() + 1j * oi.cpu().numpy()


@pytest.mark.parametrize("lines", [1, 127, 128, 1000, 152 * 128 * 2 + 5])
def test_dft32_matches_oracle(oracle, lines):
    """Ragged and multi-tile line counts (more tiles than SMs: the persistent loop), lines of very
    different magnitudes (the per-line power-of-two scaling), against numpy's FFT on every line and
    the oracle's naive DFT on a sample of lines, relative L2 per line <= 1e-13."""
    rng = np.random.default_rng(lines)
    z = rng.uniform(-1, 1, size=(lines, 32)) + 1j * rng.uniform(-1, 1, size=(lines, 32))
    z *= 10.0 ** rng.uniform(-30, 30, size=(lines, 1))
    y = _dft32(z.real, z.imag)
    ref = np.fft.fft(z, axis=1)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-13, err.max()
    for li in rng.choice(lines, size=min(lines, 16), replace=False):
        ro = oracle.line_forward(0, z[li])
        assert np.linalg.norm(y[li] - ro) <= 1e-13 * np.linalg.norm(ro)


def test_dft32_special_lines(oracle):
    """A zero line, a single impulse (flat spectrum), a pure tone (one bin), and a line with one
    huge and many tiny values (the small ones lie below the slices' reach: norm-wise accuracy)."""
    z = np.zeros((4, 32), dtype=complex)
    z[1, 5] = 1.0 - 2.0j
    n = np.arange(32)
    z[2] = np.exp(2j * np.pi * 7 * n / 32)
    z[3] = 1e-20
    z[3, 0] = 1.0
    y = _dft32(z.real, z.imag)
    assert np.all(y[0] == 0)
    ref = np.fft.fft(z, axis=1)
    for i in range(1, 4):
        assert np.linalg.norm(y[i] - ref[i]) <= 1e-13 * np.linalg.norm(ref[i]), i
    assert abs(y[2, 7] - 32) <= 1e-12 and np.abs(np.delete(y[2], 7)).max() <= 1e-12
