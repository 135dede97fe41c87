"""pp_solve_refined_noalloc: the refined mixed-precision solve for callers that cannot allocate
device memory when they solve (allocation-free time loops, memory owned by the host application).
It must give the same result as pp_solve_refined, call after call, through the C ABI.

This file is collected last on purpose: it also checks that the library's shared scratch array
works after every other test has used the library in this process."""
import ctypes

import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests.gpu_common import need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu


def _call(lib, fn, plan, f, u):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()), st)


@pytest.mark.parametrize("bc", ["NNNNNN", "NNDDNN", "PPPPPP"])
def test_noalloc_matches_refined_two_calls(bc):
    need_gpu()
    import paper_1909_05423_gb300 as pp
    from paper_1909_05423_gb300 import _lib
    lib = _lib.load()
    shape = (24, 48, 96)
    sp = (1.0 / 96, 1.0 / 48, 1.0 / 24)
    plan = pp.Plan(shape, bc, sp, "mixed_f64io")
    for call in range(2):
        f = torch.from_numpy(workloads.uniform_source(shape, seed=40 + call, remove_mean=False)).cuda()
        u_ref = torch.empty_like(f)
        u_new = torch.full_like(f, float("nan"))
        assert _call(lib, lib.pp_solve_refined, plan, f, u_ref) == 0
        assert _call(lib, lib.pp_solve_refined_noalloc, plan, f, u_new) == 0, lib.pp_last_error_string()
        torch.cuda.synchronize()
        assert rel_l2(u_new.cpu().numpy(), u_ref.cpu().numpy()) <= 1e-12
    plan.close()


def test_noalloc_rejects_oversize_grid():
    need_gpu()
    import paper_1909_05423_gb300 as pp
    from paper_1909_05423_gb300 import _lib
    lib = _lib.load()
    shape = (160, 128, 128)  # 2,621,440 cells > 2,097,152
    plan = pp.Plan(shape, "NNDDNN", (1.0, 1.0, 1.0), "mixed_f64io")
    f = torch.zeros(shape, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    assert _call(lib, lib.pp_solve_refined_noalloc, plan, f, u) == 2
    assert b"exceeds" in lib.pp_last_error_string()
    plan.close()
