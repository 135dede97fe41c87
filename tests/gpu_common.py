"""Shared helpers for the GPU tests (parity against the CPU oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_solve(f, bc, sp, dtype="f64", how="solve", options=None):
    import paper_1909_05423_gb300 as pp
    plan = pp.Plan(f.shape, bc, sp, dtype, options=options)
    io = torch.float32 if dtype == "mixed_f32io" else torch.float64
    ft = torch.from_numpy(np.ascontiguousarray(f)).to(device="cuda", dtype=io)
    u = getattr(plan, how)(ft)
    torch.cuda.synchronize()
    plan.status()
    out = u.double().cpu().numpy()
    plan.close()
    return out
