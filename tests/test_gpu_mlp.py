"""The surrogate network's GPU kernels (BF16 tensor-core forward, backward,
through the C ABI test hooks) against the FP64 numpy reference.

Two comparisons on BF16-representable inputs and weights:
1. against the reference that stores activations and back-propagated
   gradients in BF16 at the same points as the GPU design (mlp.py, bf16=True):
   only FP32-versus-FP64 accumulation order differs -> 1e-3 relative
   (Frobenius) for the outputs, the loss and every gradient tensor;
2. against the plain FP64 reference: outputs and loss within 1e-2, and, for
   training-size batches (>= 4096 rows), every gradient tensor within 2e-2.
   Smaller batches are not compared here: a ReLU mask that BF16 rounding
   flips near zero (~1e-3 of the units) changes that unit's whole gradient
   term, which dominates the gradient of a handful of rows (15 % for one
   row) and averages out over a training batch."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


def _case(n, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init(seed) + rng.normal(scale=0.02, size=mlp.n_params())
    off = 0
    for i, o in mlp.LAYERS:           # weights BF16-representable, biases FP32
        p[off:off + i * o] = mlp.bf16_round(p[off:off + i * o])
        off += i * o + o
    x = np.zeros((n, 16))
    x[:, :5] = mlp.bf16_round(rng.uniform(-1, 1, size=(n, 5)))
    t = rng.normal(scale=0.5, size=(n, 4))
    return p, x, t


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [1, 37, 1000, 4096, 20000, 65536])
def test_forward_loss_and_gradients_match_fp64(n):
    from paper_1812_05902_gb300 import pivbos as P
    assert P.MLP_PARAMS == mlp.n_params()
    p, x, t = _case(n, 3 + n)
    y = P.pivbos_mlp_forward(p, x)
    loss, g = P.pivbos_mlp_loss_grad(p, x, t)
    errs, bad = {}, []
    for bf16, tol_y, tol_g in ((True, 1e-3, 1e-3), (False, 1e-2, 2e-2 if n >= 4096 else np.inf)):
        y_ref, _ = mlp.forward(p, x, bf16)
        loss_ref, g_ref = mlp.loss_and_grad(p, x, t, bf16)
        checks = [("y", _rel(y, y_ref), tol_y), ("loss", abs(loss - loss_ref) / loss_ref, tol_y)]
        off = 0
        for li, (i, o) in enumerate(mlp.LAYERS):
            for name, size in (("W%d" % li, i * o), ("b%d" % li, o)):
                checks.append((name, _rel(g[off:off + size], g_ref[off:off + size]), tol_g))
                off += size
        for name, e, tol in checks:
            errs["%s/%s" % ("bf16" if bf16 else "fp64", name)] = e
            if not e < tol:
                bad.append((bf16, name, e, tol))
    assert not bad, (bad, errs)
