"""psso_evaluate_noalloc: the allocation-free batched fitness.

Some callers cannot allocate device memory (another allocator owns it, or
cudaMalloc / cudaFree must not synchronise the device inside their loop).
This entry point takes device buffers and keeps its scratch in a static device
array; here its results are compared with psso_evaluate's on the same rows,
for two calls in a row that share that array -- once with a synchronisation
between the calls and once with both calls queued on one stream."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

CASES = (("ellipsoid", 300, 257), ("rastrigin", 77, 31))


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _enqueue(lib, torch, fn, X, o, w, precision):
    """Queues one call on the current stream; returns the device buffers."""
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    od = torch.from_numpy(o).to(dev) if o is not None else None
    wd = torch.from_numpy(w).to(dev) if w is not None else None
    f = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device=dev)
    e = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib.psso_evaluate_noalloc(fn, X.shape[0], X.shape[1], Xd.data_ptr(),
                              od.data_ptr() if od is not None else None,
                              wd.data_ptr() if wd is not None else None, precision,
                              f.data_ptr(), e.data_ptr(), stream.cuda_stream)
    return (Xd, od, wd, f, e)


def _call(lib, torch, fn, X, o, w, precision):
    bufs = _enqueue(lib, torch, fn, X, o, w, precision)
    torch.cuda.synchronize()
    return bufs[3].cpu().numpy(), bufs[4].cpu().numpy()


def _inputs(rng, fn, N, D, precision):
    lb, ub = workload.BOUNDS[fn]
    lat = "f32" if precision == "f32" else "f64"
    o = workload.shift(D, 0.8 * lb, 0.8 * ub, N, lattice=lat)
    w = workload.ellipsoid_weights(D) if fn == "ellipsoid" else None
    X = rng.uniform(lb, ub, (N, D))
    if precision == "f32":
        X = X.astype(np.float32).astype(np.float64)
    return X, o, w


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_matches_evaluate_two_calls(lib, precision):
    torch = _torch()
    rng = np.random.default_rng(17)
    # two calls in a row with different functions, sizes and shifts: the second
    # must not see anything the first left in the shared scratch array
    for fn, N, D in CASES:
        X, o, w = _inputs(rng, fn, N, D, precision)
        f_ref, e_ref = lib.psso_evaluate(fn, X, o, w, precision=precision)
        f, e = _call(lib, torch, fn, X, o, w, precision)
        assert np.array_equal(f, f_ref), fn
        if precision == "f32":
            assert np.array_equal(e, e_ref), fn


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_two_calls_queued_on_one_stream(lib, precision):
    """Both calls are queued back to back on one stream, each with its own
    output buffers, and the stream is synchronised once: stream order alone
    keeps the second call's scratch writes after the first call's reads."""
    torch = _torch()
    rng = np.random.default_rng(23)
    inputs = [_inputs(rng, fn, N, D, precision) for fn, N, D in CASES]
    refs = [lib.psso_evaluate(fn, X, o, w, precision=precision)
            for (fn, _, _), (X, o, w) in zip(CASES, inputs)]
    bufs = [_enqueue(lib, torch, fn, X, o, w, precision)
            for (fn, _, _), (X, o, w) in zip(CASES, inputs)]
    torch.cuda.synchronize()
    for (fn, _, _), b, (f_ref, e_ref) in zip(CASES, bufs, refs):
        assert np.array_equal(b[3].cpu().numpy(), f_ref), fn
        if precision == "f32":
            assert np.array_equal(b[4].cpu().numpy(), e_ref), fn


def test_noalloc_fp32_needs_float_inputs(lib):
    """FP32 mode: a row holding a value that is not a float gets NaN in f and
    err; a shift value that is not a float makes every row NaN (its terms would
    belong to another problem, so the bound would not hold)."""
    torch = _torch()
    rng = np.random.default_rng(29)
    X, o, w = _inputs(rng, "rastrigin", 40, 37, "f32")
    X[5, 3] = 0.1                       # not a float
    f, e = _call(lib, torch, "rastrigin", X, o, w, "f32")
    assert np.isnan(f[5]) and np.isnan(e[5])
    keep = np.arange(40) != 5
    f_ref, e_ref = lib.psso_evaluate("rastrigin", X[keep], o, w, precision="f32")
    assert np.array_equal(f[keep], f_ref) and np.array_equal(e[keep], e_ref)
    o2 = o.copy()
    o2[7] = 0.1                         # not a float
    f, e = _call(lib, torch, "rastrigin", X[keep], o2, w, "f32")
    assert np.all(np.isnan(f)) and np.all(np.isnan(e))
    # the same call in FP64 is valid
    f64, _ = _call(lib, torch, "rastrigin", X[keep], o2, w, "f64")
    ref64, _ = lib.psso_evaluate("rastrigin", X[keep], o2, w, precision="f64")
    assert np.array_equal(f64, ref64)


def test_noalloc_rejects_oversized_rows(lib):
    _torch()
    with pytest.raises(lib.PssoError) as exc:
        lib.psso_evaluate_noalloc("sphere", 4, 1025, 1, None, None, "f64", 1, None, None)
    assert exc.value.status == lib.PSSO_ERR_ARG
