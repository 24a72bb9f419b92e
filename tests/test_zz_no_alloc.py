"""pmcmc_scan_noalloc: the diagonal scan for callers that cannot allocate device memory (code
running under stream capture, fixed-budget hosts, plugins under another framework's allocator).
It must give the same result as the allocating pmcmc_scan, on consecutive calls that reuse its
static scratch.  Collected last on purpose, so a failure here comes after every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_scan_matches_allocating_scan_twice(precision):
    import paper_2508_18413_gb300 as P
    dt = torch.float64 if precision == "f64" else torch.float32
    tol = 1e-12 if precision == "f64" else 2e-5
    rng = np.random.default_rng(7)
    for call, (T, D) in enumerate([(50_003, 3), (20_011, 25)]):   # two calls in a row
        a = torch.tensor(rng.uniform(-0.95, 0.95, (T, D)), dtype=dt, device="cuda")
        b = torch.tensor(rng.standard_normal((T, D)), dtype=dt, device="cuda")
        s = torch.tensor(rng.standard_normal((T, D)), dtype=dt, device="cuda")
        ref = P.pmcmc_scan("diag", precision, a, b, s.clone())
        got = P.pmcmc_scan_noalloc(precision, a, b, s.clone())
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=tol, atol=tol * 10)


@pytest.mark.gpu
def test_noalloc_scan_rejects_sizes_beyond_its_static_scratch():
    """A scan whose look-back scratch would exceed the static 8 MiB is refused up front (the
    size check runs before any memory is touched, so small buffers suffice here)."""
    import ctypes as C
    from paper_2508_18413_gb300 import _lib as L
    import paper_2508_18413_gb300 as P
    P.pmcmc_create()
    buf = torch.zeros(16, device="cuda")
    ptr = C.c_void_p(buf.data_ptr())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.load().pmcmc_scan_noalloc(L.PRECISIONS["f32"], 4_000_000, 200, ptr, ptr, ptr, stream)
    assert st == L.PMCMC_EUNSUPPORTED
    st = L.load().pmcmc_scan_noalloc(L.PRECISIONS["f32"], 10, 300, ptr, ptr, ptr, stream)
    assert st == L.PMCMC_EUNSUPPORTED            # D beyond the scan's channel limit
    torch.cuda.synchronize()
