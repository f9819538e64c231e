"""psso_evaluate_noalloc: the allocation-free batched fitness.

Some callers cannot allocate device memory (another allocator owns it, or
cudaMalloc / cudaFree must not synchronise the device inside their loop).
This entry point takes device buffers and keeps its scratch in a static device
array; here its results are compared with psso_evaluate's on the same rows,
for two calls in a row that share that array."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


def _call(lib, torch, fn, X, o, w, precision):
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
    torch.cuda.synchronize(dev)
    return f.cpu().numpy(), e.cpu().numpy()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_matches_evaluate_two_calls(lib, precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(17)
    # two calls in a row with different functions, sizes and shifts: the second
    # must not see anything the first left in the shared scratch array
    for fn, N, D in (("ellipsoid", 300, 257), ("rastrigin", 77, 31)):
        lb, ub = workload.BOUNDS[fn]
        lat = "f32" if precision == "f32" else "f64"
        o = workload.shift(D, 0.8 * lb, 0.8 * ub, N, lattice=lat)
        w = workload.ellipsoid_weights(D) if fn == "ellipsoid" else None
        X = rng.uniform(lb, ub, (N, D))
        if precision == "f32":
            X = X.astype(np.float32).astype(np.float64)
        f_ref, e_ref = lib.psso_evaluate(fn, X, o, w, precision=precision)
        f, e = _call(lib, torch, fn, X, o, w, precision)
        assert np.array_equal(f, f_ref), fn
        if precision == "f32":
            assert np.array_equal(e, e_ref), fn


def test_noalloc_rejects_oversized_rows(lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(lib.PssoError) as exc:
        lib.psso_evaluate_noalloc("sphere", 4, 1025, 1, None, None, "f64", 1, None, None)
    assert exc.value.status == lib.PSSO_ERR_ARG
