"""Every diagonal-scan kernel (D <= 32) against the oracle's plain linear recursion.

The kernel is chosen per launch by PMCMC_SCAN_KERNEL (rows: the register-resident kernels, with
D fixed at compile time for the powers of two unless PMCMC_SCAN_DCONST=0,
staged: bulk copies into shared memory, pipe: persistent and double-buffered, cluster: tiles
shared by a thread-block cluster, FP32 iterates only; FP64 falls back to the row kernels there,
so those cases check the fallback).  Shapes span one
tile to tens of tiles per CTA, ragged last tiles (including tails shorter than a 16-byte bulk
copy), lane groups of every width 32 / D, and the non-finite reset.  Bar: FP64 to 1e-12, FP32
(and bf16 storage, compared with the rounded a, b the kernel reads) to 2e-5 relative."""
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P

DEV = "cuda:0"
KERNELS = ["rows", "rows_generic", "staged", "pipe", "pipe2", "cluster", "cluster4"]
_ENV = {  # kernel variant -> environment
    # the row kernels; D a power of two runs the instance with D fixed at compile time
    "rows": {"PMCMC_SCAN_KERNEL": "rows"},
    # the row kernels with D a run-time value for every D
    "rows_generic": {"PMCMC_SCAN_KERNEL": "rows", "PMCMC_SCAN_DCONST": "0"},
    "staged": {"PMCMC_SCAN_KERNEL": "staged"},
    "pipe": {"PMCMC_SCAN_KERNEL": "pipe", "PMCMC_PIPE_CTAS": "1"},
    "pipe2": {"PMCMC_SCAN_KERNEL": "pipe", "PMCMC_PIPE_CTAS": "2"},
    # clusters of 8 CTAs, 4 slots, carries 2 tiles after pass 1 (the defaults)
    "cluster": {"PMCMC_SCAN_KERNEL": "cluster", "PMCMC_SCAN_CLUSTER": "8", "PMCMC_SCAN_SLOTS": "4",
                "PMCMC_SCAN_LAG": "2"},
    # clusters of 4 CTAs, 8 slots, carries 5 tiles later
    "cluster4": {"PMCMC_SCAN_KERNEL": "cluster", "PMCMC_SCAN_CLUSTER": "4", "PMCMC_SCAN_SLOTS": "8",
                 "PMCMC_SCAN_LAG": "5"},
}


@pytest.fixture
def kernel(request):
    """rows, rows_generic, staged, pipe (one CTA per SM), pipe2 (two CTAs per SM, smaller
    tiles), cluster or cluster4 (two cluster shapes)."""
    keys = {k for v in _ENV.values() for k in v}
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ.pop(k, None)
    os.environ.update(_ENV[request.param])
    yield request.param
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def _run(precision, a, b, s):
    sd = torch.float64 if precision == "f64" else torch.float32
    ad = torch.bfloat16 if precision == "f32_scan_bf16" else sd
    ag = torch.tensor(a, dtype=ad, device=DEV)
    bg = torch.tensor(b, dtype=ad, device=DEV)
    sg = torch.tensor(s, dtype=sd, device=DEV)
    s_in = sg.double().cpu().numpy()
    P.pmcmc_scan("diag", precision, ag, bg, sg)
    return (ag.double().cpu().numpy(), bg.double().cpu().numpy(), s_in,
            sg.double().cpu().numpy())


@pytest.mark.parametrize("kernel", KERNELS, indirect=True)
@pytest.mark.parametrize("precision", ["f64", "f32", "f32_scan_bf16"])
@pytest.mark.parametrize("T,D", [(1, 1), (3, 8), (97, 32), (1001, 3), (4099, 16), (100003, 8),
                                 (16384, 25), (60001, 1), (33335, 5), (524288, 8)])
def test_scan_kernel_matches_linear_recursion(kernel, precision, T, D):
    rng = np.random.default_rng(T * 7 + D)
    a = rng.uniform(-0.98, 0.98, (T, D))
    b = rng.standard_normal((T, D))
    s = rng.standard_normal((T, D))
    a_used, b_used, s_in, out = _run(precision, a, b, s)
    delta = O.linear_recursion(a_used, b_used, dense=False)
    tol = 1e-12 if precision == "f64" else 2e-5
    np.testing.assert_allclose(out - s_in, delta, rtol=tol, atol=tol * 10)


@pytest.mark.parametrize("kernel", KERNELS, indirect=True)
@pytest.mark.parametrize("T,D", [(20000, 8), (3000, 25)])
def test_scan_kernel_resets_non_finite(kernel, T, D):
    """An infinite b at (t0, d0) makes delta infinite from t0 on in channel d0: those states are
    reset (to 0 without a reset state); every other channel is untouched."""
    rng = np.random.default_rng(D)
    a = rng.uniform(0.1, 0.9, (T, D))
    b = rng.standard_normal((T, D))
    s = rng.standard_normal((T, D))
    t0, d0 = T // 3 + 1, D // 2
    b[t0, d0] = np.inf
    _, _, s_in, out = _run("f32", a, b, s)
    assert np.all(out[t0:, d0] == 0.0)
    b2 = b.copy()
    b2[:, d0] = 0.0
    delta = O.linear_recursion(a.astype(np.float32).astype(np.float64),
                               b2.astype(np.float32).astype(np.float64), dense=False)
    keep = np.ones(D, bool)
    keep[d0] = False
    np.testing.assert_allclose((out - s_in)[:, keep], delta[:, keep], rtol=2e-5, atol=2e-4)
    np.testing.assert_allclose((out - s_in)[:t0, d0],
                               O.linear_recursion(a[:t0, d0:d0 + 1].astype(np.float32).astype(np.float64),
                                                  b[:t0, d0:d0 + 1].astype(np.float32).astype(np.float64),
                                                  dense=False)[:, 0], rtol=2e-5, atol=2e-4)


@pytest.mark.parametrize("kernel", KERNELS, indirect=True)
def test_scan_kernel_repeated_launches(kernel):
    """The tickets, flags and epochs of one launch leave the control block ready for the next:
    twenty launches on the same inputs all match the recursion (the carries may associate
    differently from launch to launch, so the bar is the FP32 tolerance, not equal bits)."""
    T, D = 300007, 8
    rng = np.random.default_rng(11)
    a = rng.uniform(-0.9, 0.9, (T, D)).astype(np.float32)
    b = rng.standard_normal((T, D)).astype(np.float32)
    s0 = rng.standard_normal((T, D)).astype(np.float32)
    delta = O.linear_recursion(a.astype(np.float64), b.astype(np.float64), dense=False)
    ag, bg, sg0 = (torch.tensor(x, device=DEV) for x in (a, b, s0))
    for _ in range(20):
        s = sg0.clone()
        P.pmcmc_scan("diag", "f32", ag, bg, s)
        np.testing.assert_allclose(s.double().cpu().numpy() - s0.astype(np.float64), delta,
                                   rtol=2e-5, atol=2e-4)


@pytest.mark.parametrize("shape", ["8,2", "8,3", "8,6", "8,32", "16,5", "16,16"])
@pytest.mark.parametrize("precision", ["f64", "f32", "f32_scan_bf16"])
@pytest.mark.parametrize("T,D", [(100003, 8), (40001, 3), (65536, 32)])
def test_row_kernel_shapes_match_linear_recursion(shape, precision, T, D):
    """The row kernel with several sub-chunks per warp (PMCMC_SCAN_SHAPE = "rows,sub-chunks"
    fixes the shape), including counts that are not powers of two and tiles of every size from
    a few per CTA to a single ragged one."""
    saved = {k: os.environ.get(k) for k in ("PMCMC_SCAN_KERNEL", "PMCMC_SCAN_SHAPE")}
    os.environ["PMCMC_SCAN_KERNEL"] = "rows"
    os.environ["PMCMC_SCAN_SHAPE"] = shape
    try:
        rng = np.random.default_rng(T + D + len(shape))
        a = rng.uniform(-0.98, 0.98, (T, D))
        b = rng.standard_normal((T, D))
        s = rng.standard_normal((T, D))
        a_used, b_used, s_in, out = _run(precision, a, b, s)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    delta = O.linear_recursion(a_used, b_used, dense=False)
    tol = 1e-12 if precision == "f64" else 2e-5
    np.testing.assert_allclose(out - s_in, delta, rtol=tol, atol=tol * 10)


@pytest.mark.parametrize("precision", ["f32", "f32_scan_bf16"])
@pytest.mark.parametrize("T,D", [((1 << 20) // 8 - 1, 8), ((1 << 20) // 8, 8), ((1 << 22) // 8, 8),
                                 ((1 << 22) // 8 + 3, 8), ((3 << 21) // 8, 8), ((3 << 21) // 8 + 5, 8),
                                 ((1 << 20) // 2 + 7, 2), ((1 << 22) // 32, 32)])
def test_default_kernel_choice_boundaries(precision, T, D):
    """With no kernel forced, sizes on either side of the boundaries where the default switches
    between the row kernel (D fixed at compile time) and the pipelined kernel: the result is the
    recursion, whichever kernel the size picks."""
    keys = ("PMCMC_SCAN_KERNEL", "PMCMC_SCAN_SHAPE", "PMCMC_SCAN_DCONST", "PMCMC_PIPE_CTAS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ.pop(k, None)
    try:
        rng = np.random.default_rng(T * 3 + D)
        a = rng.uniform(-0.98, 0.98, (T, D))
        b = rng.standard_normal((T, D))
        s = rng.standard_normal((T, D))
        a_used, b_used, s_in, out = _run(precision, a, b, s)
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v
    delta = O.linear_recursion(a_used, b_used, dense=False)
    np.testing.assert_allclose(out - s_in, delta, rtol=2e-5, atol=2e-4)
