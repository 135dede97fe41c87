"""GPU path vs the CPU oracle, element by element (relative L2), FP64-class path.
Sizes span several CTAs, ragged last CTAs and odd nz; edge sizes (2, 6) and every per-axis
boundary kind are covered."""
import itertools
import math

import numpy as np
import pytest

from paper_1909_05423_gb300 import workloads
from tests import helpers
from tests.gpu_common import gpu_solve, need_gpu, rel_l2, torch

pytestmark = pytest.mark.gpu
TOL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _setup(oracle):
    need_gpu()


@pytest.mark.parametrize("bc", ["PPPPDD", "NNDDNN", "PPPPPP", "NNNNNN", "DDDDDD", "DNNDPP", "NDPPDN",
                                "PPNNDD", "DDPPNN", "NNPPND"])
@pytest.mark.parametrize("shape", [(37, 48, 96), (11, 72, 54), (8, 18, 144)])
def test_parity_f64(oracle, bc, shape):
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.3 / nz)
    f = workloads.uniform_source(shape, seed=7, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    u = gpu_solve(f, bc, sp)
    assert rel_l2(u, ref) <= TOL_F64, rel_l2(u, ref)


@pytest.mark.parametrize("shape", [(5, 6, 4), (3, 2, 6), (2, 4, 2)])
def test_tiny_all_axis_kinds(oracle, shape):
    """Every per-axis boundary kind (5^3 combinations) on tiny uneven grids, incl. length-2 axes."""
    rng = np.random.default_rng(3)
    sp = (0.7, 1.3, 0.9)
    for kinds in itertools.product(helpers.AXIS_KINDS, repeat=3):
        bc = "".join(kinds)
        if bc[4] == "P" and shape[0] < 3:
            continue
        f = rng.uniform(-1, 1, size=shape)
        ref = oracle.solve(f, bc, sp)
        u = gpu_solve(f, bc, sp)
        assert rel_l2(u, ref) <= TOL_F64, (bc, rel_l2(u, ref))


@pytest.mark.parametrize("shape", [(5, 16, 32), (6, 32, 64), (4, 64, 16), (3, 8, 16)])
@pytest.mark.parametrize("bc", ["NNDDNN", "PPPPDD", "DNNDPP", "PPNDDN", "NNPPND"])
def test_short_power_of_two_lines(oracle, shape, bc):
    """FFT lengths 4..32 (kernels compiled for 8, 16, 32; shorter ones at run time), every kind."""
    nz, ny, nx = shape
    if bc[4] == "P" and nz < 3:
        pytest.skip("periodic z needs nz >= 3")
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=sum(shape))
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in (("f64", TOL_F64), ("mixed_f64io", 1e-6)):
        assert rel_l2(gpu_solve(f, bc, sp, dtype), ref) <= tol, dtype


@pytest.mark.parametrize("shape", [(5, 48, 96), (4, 96, 48), (3, 192, 384), (3, 768, 24), (4, 36, 1536)])
@pytest.mark.parametrize("bc", ["NNDDNN", "PPPPDD", "DNNDPP", "PPNDDN"])
def test_three_times_power_of_two_lines(oracle, shape, bc):
    """FFT lengths 3 x 2^k (kernels compiled for 24..768, radix-3 last stage), every kind."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=sum(shape) + 1)
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in (("f64", TOL_F64), ("mixed_f64io", 1e-6)):
        assert rel_l2(gpu_solve(f, bc, sp, dtype), ref) <= tol, dtype


def test_config1_manufactured_32(oracle):
    """32^3, periodic x/y, Dirichlet z, u* = sin 2pi x sin 2pi y sin pi z: GPU RMS error equals the
    closed form 1.042987e-03 and the GPU matches the oracle."""
    n = 32
    sp = (1.0 / n,) * 3
    u_star, f = workloads.manufactured((n, n, n), sp, [(1.0, ("sin", 2 * math.pi), ("sin", 2 * math.pi),
                                                        ("sin", math.pi))])
    u = gpu_solve(f, "PPPPDD", sp)
    err = math.sqrt(((u - u_star) ** 2).mean())
    assert abs(err - 1.042987e-03) <= 1e-6 * 1.042987e-03
    assert rel_l2(u, oracle.solve(f, "PPPPDD", sp)) <= TOL_F64


def test_exact_discrete_eigenfunction():
    """A sampled eigenfunction product is returned scaled by -sum k^2 / sum lambda_d (exact discrete
    solution) element by element, at 96^3 with the NN-NN-DD mode of Table tb4."""
    n = 96
    sp = (1.0 / n,) * 3
    kap = [math.pi, 2 * math.pi, 3 * math.pi]
    u_star, f = workloads.manufactured((n, n, n), sp, [(1.0, ("cos", kap[0]), ("cos", kap[1]), ("sin", kap[2]))])
    u = gpu_solve(f, "NNNNDD", sp)
    ratio = helpers.discrete_solution_ratio(kap, [1.0 / n] * 3)
    assert rel_l2(u, u_star * ratio) <= TOL_F64


@pytest.mark.parametrize("shape,bc", [((1024, 4, 6), "DDNNPP"), ((700, 8, 16), "PPPPPP"), ((512, 6, 4), "NNNNPP")])
def test_periodic_z_long_lines(oracle, shape, bc):
    """Cyclic z solves of long lines, where the first row of the inverse (the Sherman-Morrison q
    vector) decays slowly for the low modes and is stored only up to 2^-64 of its first entry."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=13, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    assert rel_l2(gpu_solve(f, bc, sp), ref) <= TOL_F64
    assert rel_l2(gpu_solve(f, bc, sp, "mixed_f64io"), ref) <= 1e-6


@pytest.mark.parametrize("shape", [(1024, 8, 16), (768, 12, 10), (2048, 4, 6)])
@pytest.mark.parametrize("bc", ["NNDDNN", "NNNNDD", "DNDNND"])
def test_thomas_z_long_lines(oracle, shape, bc):
    """Long non-periodic z lines on a random source, element by element against the oracle.  The
    low (kx, ky) modes are the weakly dominant ones: their Thomas multipliers approach the fixed
    point slowly, so the stored prefix is long and the switch to the converged multiplier (and, in
    the FP32-spill sweeps, the converged-batch fast path) is exercised far into the line."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=17, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    assert rel_l2(gpu_solve(f, bc, sp), ref) <= TOL_F64
    assert rel_l2(gpu_solve(f, bc, sp, "mixed_f64io"), ref) <= 1e-6
    assert rel_l2(gpu_solve(f, bc, sp, "mixed_f32io"), ref) <= 1e-6
    # a z-only source puts all of its energy into the (0,0)-neighbourhood modes, the slowest to converge
    fz = np.broadcast_to(np.random.default_rng(18).uniform(-1, 1, size=(nz, 1, 1)), shape).copy()
    fz[:, 0, 0] += 0.25
    refz = oracle.solve(fz, bc, sp)
    assert rel_l2(gpu_solve(fz, bc, sp), refz) <= TOL_F64


@pytest.mark.parametrize("shape", [(4095, 8, 8), (2047, 4, 6)])
@pytest.mark.parametrize("bc", ["DDNNDD", "NNDDNN", "DDDDDN"])
def test_weak_modes_long_lines(oracle, shape, bc):
    """Long z lines on few, coarse x-y modes: with dz much below dx and dy every mode is weakly
    dominant, its converged multiplier within a few 1e-3 of -1.  Stored as 1 + w those multipliers
    keep their FP64 values; a plain double-float w would carry a relative error of 2^-48 / (1 + w)
    into every row alike (1.6e-12 against the oracle at 8 x 8 x 4095, Dirichlet z)."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=19, remove_mean=False)
    ref = oracle.solve(f, bc, sp)
    assert rel_l2(gpu_solve(f, bc, sp), ref) <= TOL_F64
    assert rel_l2(gpu_solve(f, bc, sp, "mixed_f64io"), ref) <= 1e-6


@pytest.mark.parametrize("shape,bc,sp", [((1024, 8, 8), "NNNNNN", None), ((2048, 8, 8), "PPPPPP", None),
                                         ((300, 12, 16), "NNNNNN", (0.1, 0.2, 0.3)), ((1024, 6, 4), "PPNNNN", None)])
def test_singular_long_lines_source_mean(oracle, shape, bc, sp):
    """Singular problems on long z lines with a source of non-zero mean: the (0,0) mode's right-hand
    side is the plane sums, a large constant plus fluctuations.  The pinned solve needs its exact
    zero mean (a remainder c grows like c k^2 / 2), which takes a second pass over the residuals
    (one double-float pass left 1.1e-11 against the oracle at 8 x 8 x 1024)."""
    nz, ny, nx = shape
    sp = sp or (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = np.random.default_rng(25).uniform(0, 1, size=shape)
    ref = oracle.solve(f, bc, sp)
    u = gpu_solve(f, bc, sp)
    assert abs(u.mean()) <= 1e-13 * np.abs(u).max()
    assert rel_l2(u, ref) <= TOL_F64


def test_singular_zero_mean(oracle):
    shape = (16, 24, 36)
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 1, size=shape)  # non-zero mean: solved as f - mean(f)
    for bc in ("NNNNNN", "PPPPPP", "PPNNNN", "NNPPPP"):
        u = gpu_solve(f, bc, (0.1, 0.2, 0.3))
        assert abs(u.mean()) <= 1e-13 * np.abs(u).max()
        assert rel_l2(u, oracle.solve(f, bc, (0.1, 0.2, 0.3))) <= TOL_F64


def test_residual_invariant_256(oracle):
    """256^3, config-2 boundary set (Neumann x, Dirichlet y, Neumann z): ||A u - f|| / ||f|| < 1e-12 with
    the oracle's stencil, plus sampled elementwise parity against a full oracle solve."""
    n = 256
    shape = (n, n, n)
    sp = (1.0 / n,) * 3
    f = workloads.uniform_source(shape, seed=2, remove_mean=True)
    u = gpu_solve(f, "NNDDNN", sp)
    r = oracle.laplacian(u, "NNDDNN", sp) - f
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12


def test_deterministic(oracle):
    shape = (9, 24, 48)
    f = workloads.uniform_source(shape, seed=9)
    a = gpu_solve(f, "DNPPNN", (1, 1, 1))
    b = gpu_solve(f, "DNPPNN", (1, 1, 1))
    assert np.array_equal(a, b)


def test_aliasing_in_place(oracle):
    import paper_1909_05423_gb300 as pp
    shape = (10, 12, 18)
    f = workloads.uniform_source(shape, seed=4)
    plan = pp.Plan(shape, "DDNNPP", (1, 1, 1), "f64")
    t = torch.from_numpy(f).cuda()
    plan.solve(t, out=t)
    torch.cuda.synchronize()
    assert rel_l2(t.cpu().numpy(), oracle.solve(f, "DDNNPP")) <= TOL_F64
    plan.close()


def test_host_buffers(oracle):
    import paper_1909_05423_gb300 as pp
    shape = (14, 18, 24)
    f = workloads.uniform_source(shape, seed=6)
    plan = pp.Plan(shape, "NDDNPP", (1, 1, 1), "f64")
    fh = torch.from_numpy(f).pin_memory()
    u = plan.solve_host(fh)
    assert rel_l2(u.numpy(), oracle.solve(f, "NDDNPP")) <= TOL_F64
    plan.close()


@pytest.mark.parametrize("shape,bc,dtype,tol", [((13, 12, 16), "NNDDPP", "f64", TOL_F64),     # 8 uneven plane chunks
                                                 ((5, 8, 24), "DDPPNN", "f64", TOL_F64),       # fewer planes than chunks
                                                 ((2, 6, 8), "PPNNDD", "mixed_f64io", 1e-6),
                                                 ((11, 16, 12), "DNNDND", "mixed_f32io", 1e-5)])
def test_host_buffers_chunked(oracle, shape, bc, dtype, tol):
    """Host-buffer solves copy and transform in plane chunks; every chunk size and dtype."""
    import paper_1909_05423_gb300 as pp
    f = workloads.uniform_source(shape, seed=16)
    plan = pp.Plan(shape, bc, (1, 1, 1), dtype)
    fh = torch.from_numpy(f).to(plan.io_dtype).pin_memory()
    ref = oracle.solve(fh.double().numpy(), bc)
    for _ in range(2):  # the second call reuses the staging buffers and streams
        u = plan.solve_host(fh)
        assert rel_l2(u.double().numpy(), ref) <= tol
    plan.close()


def test_batched_uneven(oracle):
    """Uneven sizes and boundary sets in one batched call (each against its own oracle solve)."""
    import paper_1909_05423_gb300 as pp
    grids = workloads.batched_grids(seed=4, count=6, sides=(6, 12, 18, 24, 32, 48))
    plans, fs, refs = [], [], []
    for i, (shape, bc) in enumerate(grids):
        if bc[4] == "P" and shape[0] < 3:
            continue
        f = workloads.uniform_source(shape, seed=100 + i)
        plans.append(pp.Plan(shape, bc, (1.0, 1.0, 1.0), "f64"))
        fs.append(torch.from_numpy(f).cuda())
        refs.append(oracle.solve(f, bc))
    outs = pp.solve_batched(plans, fs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert rel_l2(o.cpu().numpy(), r) <= TOL_F64
    for p in plans:
        p.close()


def test_batched_graph_replay_and_shared_plan(oracle):
    """The batch is one cached CUDA graph: a second call with the same lists replays it (new data in
    the same buffers), a member that reuses a plan shares its workspace and still comes out right."""
    import paper_1909_05423_gb300 as pp
    shapes = [((8, 12, 18), "PPNNDD"), ((6, 18, 12), "DNPPNN"), ((10, 6, 24), "NNNNNN")]
    plans = [pp.Plan(s, bc, (1.0, 1.0, 1.0), "f64") for s, bc in shapes]
    plans.append(plans[0])  # the same plan twice: one branch, in order
    shapes.append(shapes[0])
    fs = [torch.empty(s, dtype=torch.float64, device="cuda") for s, _ in shapes]
    us = [torch.empty_like(f) for f in fs]
    for rep in range(2):
        host = [workloads.uniform_source(s, seed=300 + 10 * rep + i) for i, (s, _) in enumerate(shapes)]
        for f, h in zip(fs, host):
            f.copy_(torch.from_numpy(h))
        pp.solve_batched(plans, fs, us)
        torch.cuda.synchronize()
        for (s, bc), h, u in zip(shapes, host, us):
            assert rel_l2(u.cpu().numpy(), oracle.solve(h, bc)) <= TOL_F64
    for p in plans[:3]:
        p.close()


@pytest.mark.parametrize("dtype", ["f64", "mixed_f32io"])
def test_batched_config4_shaped(oracle, dtype):
    """Config-4 shaped batch (sides drawn per axis, boundary sets drawn per axis/face), scaled down
    to sides {12..48} so the oracle stays fast; 24 grids in one graph launch."""
    import paper_1909_05423_gb300 as pp
    grids = [g for g in workloads.batched_grids(seed=4, count=24, sides=(12, 18, 24, 32, 36, 48))]
    io = torch.float32 if dtype == "mixed_f32io" else torch.float64
    plans, fs, refs = [], [], []
    for i, (shape, bc) in enumerate(grids):
        f = workloads.uniform_source(shape, seed=500 + i)
        plans.append(pp.Plan(shape, bc, (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0]), dtype))
        fs.append(torch.from_numpy(f).to(device="cuda", dtype=io))
        refs.append(oracle.solve(f.astype(np.float32).astype(np.float64) if dtype == "mixed_f32io" else f, bc,
                                 (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])))
    outs = pp.solve_batched(plans, fs)
    torch.cuda.synchronize()
    tol = TOL_F64 if dtype == "f64" else 1e-6
    for o, r in zip(outs, refs):
        assert rel_l2(o.double().cpu().numpy(), r) <= tol
    for p in plans:
        p.close()


@pytest.mark.parametrize("dtype", ["f64", "mixed_f32io"])
def test_batched_autotuned_members(oracle, dtype):
    """A batch whose members were autotuned: its first call times the graph with the members' own
    settings and with the shared-GPU settings, and keeps the faster.  Every member still matches the
    oracle (first call and replay with new data), a member may appear twice and beside a plan with
    default settings, and the plans' own launch shapes and z split are unchanged afterwards, for
    their lone solves."""
    import paper_1909_05423_gb300 as pp
    grids = [g for g in workloads.batched_grids(seed=7, count=10, sides=(12, 18, 24, 32, 36, 48))]
    io = torch.float32 if dtype == "mixed_f32io" else torch.float64
    tol = TOL_F64 if dtype == "f64" else 1e-6
    sps = [(1.0 / s[2], 1.0 / s[1], 1.0 / s[0]) for s, _ in grids]
    plans = [pp.Plan(s, bc, sp, dtype, options={"autotune": 1} if i else None)
             for i, ((s, bc), sp) in enumerate(zip(grids, sps))]
    plans.append(plans[3])
    grids.append(grids[3])
    sps.append(sps[3])
    before = [(p.launch_shapes(), p.z_split()) for p in plans]
    fs = [torch.empty(s, dtype=io, device="cuda") for s, _ in grids]
    us = [torch.empty_like(f) for f in fs]
    for rep in range(2):
        host = [workloads.uniform_source(s, seed=700 + 20 * rep + i) for i, (s, _) in enumerate(grids)]
        for f, h in zip(fs, host):
            f.copy_(torch.from_numpy(h))
        pp.solve_batched(plans, fs, us)
        torch.cuda.synchronize()
        for (s, bc), sp, h, u in zip(grids, sps, host, us):
            ref = oracle.solve(h.astype(np.float32).astype(np.float64) if dtype == "mixed_f32io" else h, bc, sp)
            assert rel_l2(u.double().cpu().numpy(), ref) <= tol
    assert [(p.launch_shapes(), p.z_split()) for p in plans] == before
    # a lone solve after the batch runs with the plan's own settings
    s, bc = grids[1]
    h = workloads.uniform_source(s, seed=799)
    u = plans[1].solve(torch.from_numpy(h).to(device="cuda", dtype=io))
    torch.cuda.synchronize()
    ref = oracle.solve(h.astype(np.float32).astype(np.float64) if dtype == "mixed_f32io" else h, bc, sps[1])
    assert rel_l2(u.double().cpu().numpy(), ref) <= tol
    for p in plans[:-1]:
        p.close()


def test_autotuned_plan_matches_oracle(oracle):
    """A plan created with autotune=1 (launch shapes timed and chosen at creation, then cached)
    gives the same parity as the default shapes."""
    shape = (20, 36, 64)
    sp = (1.0 / 64, 1.0 / 36, 1.0 / 20)
    f = workloads.uniform_source(shape, seed=21)
    ref = oracle.solve(f, "NDPPDD", sp)
    for _ in range(2):  # second creation hits the cache
        u = gpu_solve(f, "NDPPDD", sp, options={"autotune": 1})
        assert rel_l2(u, ref) <= TOL_F64


def test_launch_shapes_and_overrides():
    """Reported launch shapes obey the capacity rule (lines x FFT length <= 8 x threads), and
    per-direction overrides reach the inverse kernels only."""
    import paper_1909_05423_gb300 as pp
    shape = (8, 48, 64)  # x: NN -> M = 32, y: DD -> M = 24
    plan = pp.Plan(shape, "NNDDPP", (1, 1, 1), "f64", options={"threads_x_inv": 256, "lines_x_inv": 3})
    sh = plan.launch_shapes()
    M = {"x-forward": 32, "x-inverse": 32, "y-forward": 24, "y-inverse": 24}
    for k, (t, l) in sh.items():
        assert t % 32 == 0 and 32 <= t <= 512 and l >= 1 and l * M[k] <= 8 * t, (k, t, l)
    assert sh["x-inverse"] == (256, 3)
    assert sh["x-forward"][0] == 128  # the default CTA size
    plan.close()


def test_fault_injection_graph(oracle, monkeypatch):
    """An injected graph-instantiation failure surfaces as PP_ERR_CUDA from pp_solve_batched; the
    plans stay usable and the next batch (injection off) is correct."""
    import paper_1909_05423_gb300 as pp
    shape = (6, 12, 18)
    f = workloads.uniform_source(shape, seed=77)
    plans = [pp.Plan(shape, "DDNNPP", (1.0, 1.0, 1.0), "f64")]
    fs = [torch.from_numpy(f).cuda()]
    us = [torch.empty_like(fs[0])]
    monkeypatch.setenv("PP_FAULT_INJECT", "graph")
    with pytest.raises(pp.PPError) as ei:
        pp.solve_batched(plans, fs, us)
    assert ei.value.status == 5
    monkeypatch.delenv("PP_FAULT_INJECT")
    pp.solve_batched(plans, fs, us)
    torch.cuda.synchronize()
    assert rel_l2(us[0].cpu().numpy(), oracle.solve(f, "DDNNPP")) <= TOL_F64
    plans[0].close()


@pytest.mark.parametrize("shape,bc", [((2, 2, 4096), "DNNNDD"), ((3, 4096, 2), "PPPPNN"), ((3, 4096, 4), "NNDNPP"),
                                      ((3, 6, 3456), "PPDDNN")])
def test_maximum_line_lengths(oracle, shape, bc):
    """The longest supported lines (4096 = the size limit, and the 3-smooth 3456), which run the
    run-time-length kernels with one or two lines per CTA."""
    sp = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
    f = workloads.uniform_source(shape, seed=31)
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in (("f64", TOL_F64), ("mixed_f64io", 1e-6)):
        u = gpu_solve(f, bc, sp, dtype)
        assert rel_l2(u, ref) <= tol, (dtype, rel_l2(u, ref))


@pytest.mark.parametrize("shape", [(3, 1024, 8), (3, 512, 16), (3, 256, 10), (4, 128, 12)])
@pytest.mark.parametrize("bc", ["NNDDNN", "DDNNPP", "PPNNDD", "NNDDPP"])
@pytest.mark.parametrize("shape_opt", [None, dict(threads_y=256, cols_y=8, threads_y_inv=256, cols_y_inv=8)])
def test_y_power_of_two_tiles(oracle, shape, bc, shape_opt):
    """y lines of 128..1024 reals (compile-time FFT lengths 64..512) in full tiles, where each thread
    takes a fixed set of items per tile, and in partial last tiles (nx = 10, 12), which take the
    general loop; forward (DST-II / DCT-II) and inverse (DST-III / DCT-III) kinds, FP64 and mixed."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=41)
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in (("f64", TOL_F64), ("mixed_f64io", 1e-6)):
        u = gpu_solve(f, bc, sp, dtype, options=shape_opt)
        assert rel_l2(u, ref) <= tol, (dtype, rel_l2(u, ref))


@pytest.mark.parametrize("shape", [(3, 8, 1024), (3, 16, 512), (3, 10, 256), (3, 14, 128)])
@pytest.mark.parametrize("bc", ["NNDDNN", "DDNNPP", "NDNDDD"])
@pytest.mark.parametrize("shape_opt", [None, dict(threads_x=256, lines_x=4, threads_x_inv=256, lines_x_inv=4),
                                       dict(threads_x=128, lines_x=2, threads_x_inv=128, lines_x_inv=2)])
def test_x_power_of_two_tiles(oracle, shape, bc, shape_opt):
    """x lines of 128..1024 reals (compile-time FFT lengths 64..512) in full tiles, where each line's
    team of threads takes a fixed set of items, and in tiles whose last one is partial (ny nz not a
    multiple of the lines per CTA); DCT-II/DST-II forward, DCT-III/DST-III inverse, type IV for the
    mixed faces, FP64 and mixed."""
    nz, ny, nx = shape
    sp = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    f = workloads.uniform_source(shape, seed=43)
    ref = oracle.solve(f, bc, sp)
    for dtype, tol in (("f64", TOL_F64), ("mixed_f64io", 1e-6)):
        u = gpu_solve(f, bc, sp, dtype, options=shape_opt)
        assert rel_l2(u, ref) <= tol, (dtype, rel_l2(u, ref))


@pytest.mark.parametrize("scale", [1e-20, 1e25])
def test_magnitude_range(oracle, scale):
    """The double-float path has FP32's exponent range; sources scaled to 1e-20 and 1e25 (inside
    the range the header states) keep FP64-class accuracy.  The problem is linear, so the
    oracle's solution of the unscaled source, scaled, is the reference."""
    shape = (12, 64, 256)
    sp = (1.0 / 256, 1.0 / 64, 1.0 / 12)
    f = workloads.uniform_source(shape, seed=47)
    ref = oracle.solve(f, "NNDDNN", sp) * scale
    assert rel_l2(gpu_solve(f * scale, "NNDDNN", sp), ref) <= TOL_F64


def test_plans_on_two_devices(oracle):
    """Plans created and solved on two devices of one process (the >48 KB shared-memory opt-in of the
    line kernels is kept per device); skipped where fewer than two GPUs are visible."""
    import paper_1909_05423_gb300 as pp
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    shape = (16, 64, 128)
    sp = (1.0 / 128, 1.0 / 64, 1.0 / 16)
    f = workloads.uniform_source(shape, seed=71)
    ref = oracle.solve(f, "NNDDNN", sp)
    for dev in (0, 1, 0):
        with torch.cuda.device(dev):
            plan = pp.Plan(shape, "NNDDNN", sp, "f64")
            u = plan.solve(torch.from_numpy(f).cuda(dev))
            torch.cuda.synchronize(dev)
            plan.status()
            assert rel_l2(u.cpu().numpy(), ref) <= TOL_F64, dev
            plan.close()
