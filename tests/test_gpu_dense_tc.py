"""Dense scan with the compositions on the tensor cores (tcgen05 kind::f16, bfloat16 operands,
FP32 accumulation; four 32-row chunks per M = 128 tile, block-diagonal A operand), the dense
path of the F32_SCAN_BF16 precision.

Bars.  With signed permutation matrices every product is exact in bfloat16, so the scan must
equal the oracle's plain recursion to FP32 rounding: no worse than twice the error of the plain
FP32 recursion delta_t = fl(J_t delta_{t-1} + b_t) run in order (at T = 20011 that error is
already 1e-5 to 2.4e-5 relative, from the growth of |delta| like sqrt(t)).  This checks the
operand layouts, the block-diagonal packing, the transposed write-back, the chunk and tile
carries and the ragged tails.  With general contracting matrices the carry passes through
bfloat16 products: each chunk product P_i = J_i bf16(P_{i-1}) rounds its right factor (relative
2^-9) 31 times.  A CPU model of that rounding (products rounded to bfloat16 before each step,
FP32 elsewhere) sets the bar: the kernel's distance from the oracle, in maximum and in mean,
stays within 1.5 times the model's (the model is 3.6e-2 (1 + |delta|) away at most on this
input), and within 5e-2 (1 + |delta|).  The two are not compared element by element: the tensor
core's accumulation truncates, so a product near a bfloat16 rounding boundary can round the
other way and the difference then propagates through the chunk.  In a Newton
solve the residual is formed in FP32, so the solve still reaches the oracle's trace within the
FP32 bar.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2508_18413_gb300 as P

DEV = "cuda:0"


def _scan(a, b, s):
    ag = torch.tensor(a, dtype=torch.bfloat16, device=DEV)
    bg = torch.tensor(b, dtype=torch.bfloat16, device=DEV)
    sg = torch.tensor(s, dtype=torch.float32, device=DEV)
    P.pmcmc_scan("dense", "f32_scan_bf16", ag, bg, sg)
    torch.cuda.synchronize()
    return ag.double().cpu().numpy(), bg.double().cpu().numpy(), sg.double().cpu().numpy()


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _bf16(x):
    return torch.tensor(x, dtype=torch.float32).bfloat16().double().numpy()


def _seq_f32(a, b):
    """delta_t = fl32(J_t delta_{t-1} + b_t), in timestep order."""
    d = np.zeros(a.shape[1], dtype=np.float32)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    out = np.zeros(b.shape)
    for t in range(len(b)):
        d = a32[t] @ d + b32[t]
        out[t] = d
    return out


def _chunk_model(a, b, C):
    """The chunked recursion with each chunk's transfer product rounded to bfloat16 before every
    multiplication (the tensor-core operand), FP32 elsewhere."""
    T, D = b.shape
    out = np.zeros((T, D))
    c = np.zeros(D)
    for k in range(0, T, C):
        P, bl = a[k], b[k].copy()
        for t in range(k + 1, k + C):
            J, bt = (a[t], b[t]) if t < T else (np.eye(D), np.zeros(D))
            P, bl = _f32(J @ _bf16(P)), _f32(J @ bl + bt)
        dl = c.copy()
        for t in range(k, min(k + C, T)):
            dl = _f32(a[t] @ dl + b[t])
            out[t] = dl
        c = _f32(P @ c + bl)
    return out


def _signed_perms(T, D, rng):
    a = np.zeros((T, D, D))
    for t in range(T):
        p = rng.permutation(D)
        a[t, np.arange(D), p] = rng.choice([-1.0, 1.0], size=D)
    return a


@pytest.mark.parametrize("D", [5, 16, 25, 32])
@pytest.mark.parametrize("T", [1, 37, 128, 129, 1000, 20011])
def test_dense_tc_scan_exact_products(D, T):
    rng = np.random.default_rng(D * 1000 + T)
    a = _signed_perms(T, D, rng)
    b = rng.standard_normal((T, D))
    s = rng.standard_normal((T, D))
    a32, b32, out = _scan(a, b, s)
    want = s.astype(np.float32).astype(np.float64) + O.linear_recursion(a32, b32, dense=True)
    err = np.abs(out - want) / (1 + np.abs(want))
    d64 = want - _f32(s)
    seq = _seq_f32(a32, b32)
    bar = max(1e-5, 2.0 * (np.abs(seq - d64) / (1 + np.abs(d64))).max())
    assert err.max() <= bar, (err.max(), bar, np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("D", [16, 25])
def test_dense_tc_scan_contracting(D):
    rng = np.random.default_rng(7)
    T = 5000
    a = 0.95 * np.eye(D) + rng.standard_normal((T, D, D)) * (0.04 / np.sqrt(D))
    b = rng.standard_normal((T, D))
    s = np.zeros((T, D))
    a32, b32, out = _scan(a, b, s)
    want = O.linear_recursion(a32, b32, dense=True)
    err = np.abs(out - want) / (1 + np.abs(want))
    assert err.max() <= 5e-2, err.max()
    # the kernel's chunk length: ceil(T / (4 chunks x 152 SMs)), clamped to [8, 256]
    model = _chunk_model(a32, b32, min(256, max(8, -(-T // (4 * 152)))))
    err_model = np.abs(model - want) / (1 + np.abs(want))
    assert err.max() <= 1.5 * err_model.max() and err.mean() <= 1.5 * err_model.mean(), \
        (err.max(), err_model.max(), err.mean(), err_model.mean())


@pytest.mark.parametrize("kind,D,sampler,L", [("gaussian", 16, "mala", 0), ("gaussian", 32, "hmc", 4),
                                              ("logreg", 25, "mala", 0)])
def test_dense_newton_with_tc_compositions_reaches_oracle(kind, D, sampler, L):
    T = 3000
    if kind == "gaussian":
        _, prec, _ = W.random_spd(D, seed=D)
        mu = np.random.default_rng(D).standard_normal(D) * 0.3
        ot = O.Target("gaussian", D, mu=mu, P=prec)
        gt = P.Target("gaussian", D, mean=torch.tensor(mu, dtype=torch.float32, device=DEV),
                      prec=torch.tensor(prec, dtype=torch.float32, device=DEV))
        eps = 0.1 if sampler == "mala" else 0.05
    else:
        X, y, _ = W.blr_data(300, D, seed=3)
        ot = O.Target("logreg", D, X=X, y=y, sigma_p=1.0)
        gt = P.Target("logreg", D, X=torch.tensor(X, dtype=torch.float32, device=DEV),
                      y=torch.tensor(y, dtype=torch.float32, device=DEV))
        eps = 0.002
    xi, u = W.noise(T, D, seed=11)
    xi = xi.astype(np.float32).astype(np.float64)
    ref, ell, acc = O.chain(O.Problem(ot, sampler, eps, xi=xi, u=u, L=L), T, np.zeros(D))
    opt = P.Options(sampler=sampler, step=eps, leapfrog_L=L, jac="dense", precision="f32_scan_bf16",
                    atol=1e-6, rtol=1e-6, gate_grad=0)
    s, res = P.pmcmc_solve(gt, opt, T, torch.zeros(D, dtype=torch.float32, device=DEV),
                           xi=torch.tensor(xi, dtype=torch.float32, device=DEV),
                           u=torch.tensor(u, device=DEV))
    assert res["status"] == "OK", res
    s = s.cpu().double().numpy()
    margin = np.abs(np.minimum(ell, 0.0) - np.log(u))
    near = np.nonzero(margin < 1e-4)[0]
    upto = near[0] if len(near) else T
    err = np.abs(s[:upto] - ref[:upto]) / (1 + np.abs(ref[:upto]))
    assert upto > 500 and err.max() <= 1e-4, (upto, err.max())
