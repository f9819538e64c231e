"""Differentiable fitness and gBest polish on the GPU.

* psso_fitness_forward against the oracle's FP64 fitness at the same (float)
  points; psso_fitness_backward against FP64 central differences of the oracle
  (h = 1e-6) on 64 random particles and against torch's FP64 autograd of the
  textbook definitions (CPU).
* psso_polish never raises the gBest fitness, keeps the swarm state
  consistent (pBest row, pBest fitness, gBest row), and with zero steps leaves
  the run on the oracle's trajectory.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workload

pytestmark = pytest.mark.gpu

ALL_FNS = ["sphere", "ellipsoid", "rastrigin", "rosenbrock", "ackley", "rot_ellipsoid",
           "rot_rastrigin", "rot_ackley"]


def _f32_problem(fn, D, seed):
    """Problem data rounded to float32 (the FP32 kernels read float32 copies),
    returned as float64 arrays that hold exactly those floats."""
    p = workload.problem(fn, 4, D, seed=seed, lattice="f32")
    r = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)
    return p, r(p["o"]), r(p["w"]), r(p["M"])


def _points(fn, N, D, seed):
    lb, ub = workload.BOUNDS[fn]
    rng = np.random.default_rng(seed)
    return rng.uniform(lb, ub, size=(N, D)).astype(np.float32).astype(np.float64)


def _dev(a):
    return None if a is None else torch.tensor(a, dtype=torch.float32, device="cuda")


def _forward_backward(lib, fn, X, o, w, M, grad_f=None, impl="warp"):
    """impl "warp": psso_fitness_forward / _backward (CUDA cores); "tc": the
    *_ws calls (rotated products on the tensor cores, device workspace)."""
    N, D = X.shape
    Xd, od, wd, Md = _dev(X), _dev(o), _dev(w), _dev(M)
    f = torch.empty(N, dtype=torch.float32, device="cuda")
    gX = torch.empty((N, D), dtype=torch.float32, device="cuda")
    gf = torch.ones(N, dtype=torch.float32, device="cuda") if grad_f is None else _dev(grad_f)
    ptr = lambda t: None if t is None else t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    if impl == "warp":
        lib.psso_fitness_forward(fn, N, D, Xd.data_ptr(), od.data_ptr(), ptr(wd), ptr(Md),
                                 f.data_ptr(), s)
        lib.psso_fitness_backward(fn, N, D, Xd.data_ptr(), od.data_ptr(), ptr(wd), ptr(Md),
                                  gf.data_ptr(), gX.data_ptr(), s)
    else:
        nws = lib.psso_fitness_workspace_size(fn, N, D)
        ws = torch.empty(max(nws, 1), dtype=torch.uint8, device="cuda")
        lib.psso_fitness_forward_ws(fn, N, D, Xd.data_ptr(), od.data_ptr(), ptr(wd), ptr(Md),
                                    f.data_ptr(), ws.data_ptr(), nws, s)
        lib.psso_fitness_backward_ws(fn, N, D, Xd.data_ptr(), od.data_ptr(), ptr(wd), ptr(Md),
                                     gf.data_ptr(), gX.data_ptr(), ws.data_ptr(), nws, s)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.float64), gX.cpu().numpy().astype(np.float64)


IMPLS = ["warp", "tc"]


def _plain_torch(fn, X, o, w, M):
    """Textbook definitions (shifted, optionally rotated), FP64 on the CPU."""
    z = X - o
    if fn.startswith("rot_"):
        z = z @ M.T
    base = fn.replace("rot_", "")
    D = X.shape[1]
    if base == "sphere":
        return (z * z).sum(1)
    if base == "ellipsoid":
        return (w * z * z).sum(1)
    if base == "rastrigin":
        return 10 * D + (z * z - 10 * torch.cos(2 * math.pi * z)).sum(1)
    if base == "rosenbrock":
        a = z + 1
        return (100 * (a[:, 1:] - a[:, :-1] ** 2) ** 2 + (a[:, :-1] - 1) ** 2).sum(1)
    return (-20 * torch.exp(-0.2 * torch.sqrt((z * z).mean(1))) -
            torch.exp(torch.cos(2 * math.pi * z).mean(1)) + 20 + math.e)


def _rot_tol(fn, rot_tol, tol):
    return rot_tol if fn.startswith("rot_") else tol


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("fn", ALL_FNS)
@pytest.mark.parametrize("D", [1, 37, 256, 1024])
def test_forward_matches_oracle(lib, fn, D, impl):
    p, o, w, M = _f32_problem(fn, D, 5 + D)
    X = _points(fn, 70, D, 100 + D)
    f, _ = _forward_backward(lib, fn, X, o, w, M, impl=impl)
    ref = np.array([oracle.fitness(fn, x, o, w, M) for x in X])
    rel = np.abs(f - ref) / np.maximum(np.abs(ref), 1e-30)
    assert np.all(np.isfinite(f))
    assert rel.max() <= _rot_tol(fn, 1e-3, 2e-5), rel.max()


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("fn", ALL_FNS)
def test_gradient_central_differences(lib, fn, impl):
    """df/dx against FP64 central differences (h = 1e-6) of the oracle's
    fitness, 64 random particles, D = 256."""
    if impl == "tc" and not fn.startswith("rot_"):
        pytest.skip("the *_ws calls run the warp kernels for unrotated functions")
    D, N, h = 256, 64, 1e-6
    p, o, w, M = _f32_problem(fn, D, 77)
    X = _points(fn, N, D, 78)
    _, g = _forward_backward(lib, fn, X, o, w, M, impl=impl)
    worst = 0.0
    for i in range(N):
        fd = np.empty(D)
        for j in range(D):
            xp = X[i].copy()
            xm = X[i].copy()
            xp[j] += h
            xm[j] -= h
            fd[j] = (oracle.fitness(fn, xp, o, w, M) - oracle.fitness(fn, xm, o, w, M)) / (2 * h)
        err = np.abs(g[i] - fd).max() / np.abs(fd).max()
        worst = max(worst, err)
    assert worst <= _rot_tol(fn, 2e-3, 1e-4), worst


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("fn", ALL_FNS)
@pytest.mark.parametrize("D", [1, 5, 131, 1024])
def test_gradient_torch_autograd(lib, fn, D, impl):
    """df/dx against torch's FP64 autograd of the textbook definition."""
    p, o, w, M = _f32_problem(fn, D, 9 + D)
    X = _points(fn, 33, D, 10 + D)
    gf = np.random.default_rng(D).uniform(-2, 2, size=33).astype(np.float32).astype(np.float64)
    _, g = _forward_backward(lib, fn, X, o, w, M, grad_f=gf, impl=impl)
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    tw = None if w is None else torch.tensor(w)
    tM = None if M is None else torch.tensor(M)
    f = _plain_torch(fn, Xt, torch.tensor(o), tw, tM)
    (f * torch.tensor(gf)).sum().backward()
    ref = Xt.grad.numpy()
    scale = np.maximum(np.abs(ref).max(1, keepdims=True), 1e-30)
    err = (np.abs(g - ref) / scale).max()
    assert err <= _rot_tol(fn, 2e-3, 1e-4), err


@pytest.mark.parametrize("impl", IMPLS)
def test_gradient_at_optimum_is_zero(lib, impl):
    for fn in ALL_FNS:
        p, o, w, M = _f32_problem(fn, 64, 12)
        f, g = _forward_backward(lib, fn, o[None, :].copy(), o, w, M, impl=impl)
        assert f[0] == 0.0, fn
        assert np.all(g == 0.0), fn


def test_autograd_function(lib):
    from paper_2110_01470_gb300.autograd import fitness
    p, o, w, M = _f32_problem("rot_rastrigin", 100, 21)
    X = torch.tensor(_points("rot_rastrigin", 40, 100, 22), dtype=torch.float32, device="cuda")
    X.requires_grad_(True)
    c = torch.linspace(-1, 2, 40, device="cuda")
    f = fitness(X, "rot_rastrigin", _dev(o), rotation=_dev(M))
    (f * c).sum().backward()
    f2, g = _forward_backward(lib, "rot_rastrigin", X.detach().cpu().numpy().astype(np.float64),
                              o, None, M, grad_f=c.cpu().numpy().astype(np.float64), impl="tc")
    assert np.array_equal(f.detach().cpu().numpy(), f2.astype(np.float32))
    assert np.array_equal(X.grad.cpu().numpy(), g.astype(np.float32))


def test_fitness_arguments_rejected(lib):
    X = torch.zeros((4, 8), device="cuda")
    f = torch.empty(4, device="cuda")
    o = torch.zeros(8, device="cuda")
    with pytest.raises(lib.PssoError):
        lib.psso_fitness_forward("sphere", 4, 0, X.data_ptr(), o.data_ptr(), None, None, f.data_ptr())
    with pytest.raises(lib.PssoError):
        lib.psso_fitness_forward("sphere", 4, 2000, X.data_ptr(), o.data_ptr(), None, None,
                                 f.data_ptr())
    with pytest.raises(lib.PssoError):
        lib.psso_fitness_forward("ellipsoid", 4, 8, X.data_ptr(), o.data_ptr(), None, None,
                                 f.data_ptr())
    with pytest.raises(lib.PssoError):
        lib.psso_fitness_forward("rot_ackley", 4, 8, X.data_ptr(), o.data_ptr(), None, None,
                                 f.data_ptr())
    with pytest.raises(lib.PssoError):
        lib.psso_fitness_backward("sphere", 4, 8, X.data_ptr(), o.data_ptr(), None, None, None,
                                  X.data_ptr())


# ---------------------------------------------------------------------------
# gBest polish

def _check_consistent(lib, h, k, p, exact_pF=True):
    """gBest row = pBest row of the gBest particle; the gBest value is that
    row's FP64 fitness and the lowest-index minimum over all pBests (FP64
    fitness recomputed by the oracle).  With FP32 fitness the library's pF
    holds FP64 values only where it needed them, so it is compared loosely."""
    v, b, row = lib.psso_best(h, k, p["D"])
    X, P, pF = lib.psso_get_state(h, k, p["N"], p["D"])
    true = np.array([oracle.fitness(p["fn"], r, p["o"], p["w"], p["M"]) for r in P])
    assert np.array_equal(P[b], row)
    assert v == true[b]
    assert b == int(np.argmin(true))
    if exact_pF:
        assert np.array_equal(pF, true)
    else:
        assert np.all(np.abs(pF - true) <= 1e-4 * np.abs(true))
    lb, ub = p["lb"], p["ub"]
    assert np.all(row >= lb) and np.all(row <= ub)
    return v, b


POLISH_CFGS = [dict(), dict(single_block_max=-1, max_blocks=3), dict(single_block_max=-1, pipeline=2)]


@pytest.mark.parametrize("cfg", POLISH_CFGS)
@pytest.mark.parametrize("fn,lattice,precision,lr", [("sphere", "f64", "f64", 1e-3),
                                                     ("rosenbrock", "f32", "f32", 1e-4),
                                                     ("rot_ackley", "f32", "f32", 1e-1),
                                                     ("ellipsoid", "f64", "f64", 1e-7)])
def test_polish_improves_and_stays_consistent(lib, fn, lattice, precision, lr, cfg):
    p = workload.problem(fn, 300, 64, seed=31, lattice=lattice)
    h = lib.psso_create_ex([p], precision, **cfg)
    try:
        ex = precision == "f64"
        lib.psso_run(h, 40)
        improved_any = False
        for _ in range(4):
            before, _ = _check_consistent(lib, h, 0, p, ex)
            improved = lib.psso_polish(h, 0, 20, lr)
            after, b = _check_consistent(lib, h, 0, p, ex)
            assert after <= before
            assert improved == (after < before)
            improved_any |= improved
            lib.psso_run(h, 10)
            later, _ = _check_consistent(lib, h, 0, p, ex)
            assert later <= after
        assert improved_any
        log = lib.psso_get_log(h, 0)
        assert np.all(np.diff(log["value"]) <= 0)
    finally:
        lib.psso_destroy(h)


def test_polish_never_worsens(lib):
    """A step far too long for Rastrigin: the polished row is worse and is
    rejected, leaving the state bit-identical."""
    p = workload.problem("rastrigin", 200, 40, seed=8, lattice="f64")
    h = lib.psso_create_ex([p], "f64")
    try:
        lib.psso_run(h, 30)
        X0, P0, pF0 = lib.psso_get_state(h, 0, p["N"], p["D"])
        best0 = lib.psso_best(h, 0, p["D"])
        assert not lib.psso_polish(h, 0, 5, 10.0)
        X1, P1, pF1 = lib.psso_get_state(h, 0, p["N"], p["D"])
        best1 = lib.psso_best(h, 0, p["D"])
        assert np.array_equal(P0, P1) and np.array_equal(pF0, pF1) and np.array_equal(X0, X1)
        assert best0[0] == best1[0] and best0[1] == best1[1]
        assert np.array_equal(best0[2], best1[2])
    finally:
        lib.psso_destroy(h)


@pytest.mark.parametrize("cfg", [dict(), dict(single_block_max=-1, max_blocks=2)])
def test_polish_zero_steps_keeps_oracle_trajectory(lib, cfg):
    """Zero steps leave the row as it is, so nothing is replaced and the run
    stays bit-identical to the oracle's."""
    p = workload.problem("rosenbrock", 150, 33, seed=4, lattice="f64")
    t1, t2 = 25, 25
    h = lib.psso_create_ex([p], "f64", log_stride=1, log_capacity=t1 + t2 + 1, **cfg)
    try:
        lib.psso_run(h, t1)
        assert not lib.psso_polish(h, 0, 0, 1e-3)
        assert not lib.psso_polish(h, 0, 20, 0.0)
        lib.psso_run(h, t2)
        X, P, pF = lib.psso_get_state(h, 0, p["N"], p["D"])
        v, b, row = lib.psso_best(h, 0, p["D"])
    finally:
        lib.psso_destroy(h)
    r = oracle.run_problem(p, t1 + t2)
    assert np.array_equal(X, r["X"]) and np.array_equal(P, r["P"]) and np.array_equal(pF, r["pF"])
    assert v == r["log_v"][-1] and b == r["log_b"][-1] and np.array_equal(row, r["G"])


def test_polish_one_instance_of_a_batch(lib):
    ps = [workload.problem(fn, 64, 20, seed=50 + k, lattice="f64")
          for k, fn in enumerate(["sphere", "rosenbrock", "sphere"])]
    h = lib.psso_create_ex(ps, "f64")
    try:
        lib.psso_run(h, 20)
        before = [lib.psso_get_state(h, k, 64, 20) for k in range(3)]
        assert lib.psso_polish(h, 1, 20, 1e-4)
        after = [lib.psso_get_state(h, k, 64, 20) for k in range(3)]
        for k in (0, 2):
            assert all(np.array_equal(a, b) for a, b in zip(before[k], after[k]))
        _check_consistent(lib, h, 1, ps[1])
    finally:
        lib.psso_destroy(h)


def test_polish_arguments_rejected(lib):
    p = workload.problem("sphere", 16, 4, seed=1)
    h = lib.psso_create_ex([p], "f64")
    try:
        for args in ((1, 1, 1e-3), (0, -1, 1e-3), (0, 1, float("nan")), (0, 1, -1.0),
                     (0, 1, float("inf"))):
            with pytest.raises(lib.PssoError):
                lib.psso_polish(h, *args)
    finally:
        lib.psso_destroy(h)


@pytest.mark.parametrize("fn", ["rot_ellipsoid", "rot_rastrigin", "rot_ackley"])
@pytest.mark.parametrize("N,D", [(1, 16), (129, 100), (300, 257), (4096, 256)])
def test_tensor_core_gradient_matches_warp_kernels(lib, fn, N, D):
    """The tensor-core forward / backward against the CUDA-core kernels on the
    same rows: both FP32, so they agree to the GEMM's split-BF16 accuracy."""
    p, o, w, M = _f32_problem(fn, D, 40 + D)
    X = _points(fn, N, D, 41 + D)
    gf = np.random.default_rng(N).uniform(-2, 2, size=N).astype(np.float32).astype(np.float64)
    fw, gw = _forward_backward(lib, fn, X, o, w, M, grad_f=gf, impl="warp")
    ft, gt = _forward_backward(lib, fn, X, o, w, M, grad_f=gf, impl="tc")
    assert np.all(np.isfinite(ft)) and np.all(np.isfinite(gt))
    assert np.max(np.abs(ft - fw) / np.maximum(np.abs(fw), 1e-30)) <= 2e-4
    scale = np.maximum(np.abs(gw).max(1, keepdims=True), 1e-30)
    assert (np.abs(gt - gw) / scale).max() <= 2e-4


def test_tensor_core_workspace_checked(lib):
    X = torch.zeros((4, 64), device="cuda")
    o = torch.zeros(64, device="cuda")
    M = torch.eye(64, device="cuda")
    f = torch.empty(4, device="cuda")
    n = lib.psso_fitness_workspace_size("rot_rastrigin", 4, 64)
    assert n > 0 and lib.psso_fitness_workspace_size("rastrigin", 4, 64) == 0
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.PssoError) as e:
        lib.psso_fitness_forward_ws("rot_rastrigin", 4, 64, X.data_ptr(), o.data_ptr(), None,
                                    M.data_ptr(), f.data_ptr(), ws.data_ptr(), n - 1)
    assert e.value.status == lib.PSSO_ERR_ARG
