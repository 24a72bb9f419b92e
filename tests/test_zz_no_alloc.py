"""pmcmc_scan_noalloc: the diagonal scan for callers that cannot allocate device memory (code
running under stream capture, fixed-budget hosts, plugins under another framework's allocator).
It must give the same result as the allocating pmcmc_scan, on consecutive calls that reuse its
static scratch, whichever scan kernel the size (or PMCMC_SCAN_KERNEL / PMCMC_PIPE_CTAS /
PMCMC_SCAN_CLUSTER) selects.
Collected last on purpose, so a failure here comes after every other test."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _pair(precision, T, D, rng):
    sd = torch.float64 if precision == "f64" else torch.float32
    ad = torch.bfloat16 if precision == "f32_scan_bf16" else sd
    a = torch.tensor(rng.uniform(-0.95, 0.95, (T, D)), dtype=sd, device="cuda").to(ad)
    b = torch.tensor(rng.standard_normal((T, D)), dtype=sd, device="cuda").to(ad)
    s = torch.tensor(rng.standard_normal((T, D)), dtype=sd, device="cuda")
    return a, b, s


def _compare_twice(precision, shapes, env=None):
    import paper_2508_18413_gb300 as P
    tol = 1e-12 if precision == "f64" else 2e-5
    rng = np.random.default_rng(7)
    saved = {k: os.environ.get(k) for k in (env or {})}
    try:
        os.environ.update(env or {})
        for T, D in shapes:                      # consecutive calls share the static scratch
            a, b, s = _pair(precision, T, D, rng)
            ref = P.pmcmc_scan("diag", precision, a, b, s.clone())
            got = P.pmcmc_scan_noalloc(precision, a, b, s.clone())
            torch.cuda.synchronize()
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=tol,
                                       atol=tol * 10)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_scan_matches_allocating_scan_twice(precision):
    """Register-resident row kernel sizes (below 2^21 elements)."""
    _compare_twice(precision, [(50_003, 3), (20_011, 25)])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f32", "f32_scan_bf16"])
def test_noalloc_scan_pipelined_kernel_twice(precision):
    """About 4M elements at D = 8: the pipelined bulk-copy kernel (the default there), whose
    smaller tiles size the static scratch."""
    _compare_twice(precision, [(500_009, 8), (500_009, 8)])


@pytest.mark.gpu
def test_noalloc_scan_pipelined_two_ctas_per_sm_twice():
    _compare_twice("f32", [(500_009, 8), (300_007, 8)], env={"PMCMC_PIPE_CTAS": "2"})


@pytest.mark.gpu
def test_noalloc_scan_staged_kernel_twice():
    _compare_twice("f32", [(200_003, 8), (150_001, 4)], env={"PMCMC_SCAN_KERNEL": "staged"})


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f32", "f32_scan_bf16"])
def test_noalloc_scan_cluster_kernel_twice(precision):
    """The thread-block cluster kernel (FP32 iterates), clusters of 8 and of 4."""
    _compare_twice(precision, [(500_009, 8), (300_007, 25)], env={"PMCMC_SCAN_KERNEL": "cluster"})
    _compare_twice(precision, [(200_003, 3)], env={"PMCMC_SCAN_KERNEL": "cluster", "PMCMC_SCAN_CLUSTER": "4"})


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["f32", "f64", "f32_scan_bf16"])
def test_noalloc_scan_wide_state_twice(precision):
    """D = 64 and D = 256: the shared-memory staged kernel for D > 32."""
    _compare_twice(precision, [(30_011, 64), (4_099, 256)])


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
    z = torch.zeros((8, 300), device="cuda")
    with pytest.raises(P.PmcmcError, match="EUNSUPPORTED"):   # the binding names the status
        P.pmcmc_scan_noalloc("f32", z, z.clone(), z.clone())
    torch.cuda.synchronize()
