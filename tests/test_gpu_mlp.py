"""The surrogate network's GPU kernels against the FP64 reference
(oracle/mlp.py), element by element, through the testing library's hooks
(include/pivbos_testing.h): the tcgen05 inference forward, the tcgen05
training step (forward, loss, backward chain and weight gradients), the Adam
step, and the network kernel of the surrogate render itself (biases carried
through the tensor core).

Inputs and weights are BF16-representable.  The reference that stores the
hidden activations and back-propagated gradients in BF16 at the same points
as the GPU (mlp.py with bf16=True) differs from the kernels only in FP32
versus FP64 accumulation.  Errors are measured per element as

    e = |gpu - ref| / (|ref| + rms(ref over the tensor)).

Outputs: 99 % of the elements within 1e-4 (the FP32 accumulation level; an
FP32 emulation on the CPU gives a 99th percentile of ~1e-7) and every
element within 2.5e-2.  The second bound covers the rare element where a
pre-activation lies within an FP32 rounding of a BF16 rounding boundary, so
that the two sides store one hidden unit one BF16 ulp (2^-8 relative) apart
and the following layers carry the difference to the output: the same FP32
emulation shows such elements at ~1e-3 of the outputs of a 65,536-row batch
with a worst case of 8e-3.  Gradients (sums over the rows) every element
within 2e-3.  The plain FP64 reference (no BF16 storage) is compared on
training-size batches, where a ReLU mask flipped by BF16 rounding near zero
averages out: outputs 1e-2 and gradients 2e-2 relative to the tensor's
norm."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

RTOL = 2e-3          # gradients, every element
OUT_RTOL = 1e-4      # outputs, 99 % of the elements
OUT_FLIP = 2.5e-2    # outputs, every element


def _case(n, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init(seed) + rng.normal(scale=0.02, size=mlp.n_params())
    off = 0
    for i, o in mlp.LAYERS:           # weights BF16-representable, biases FP32
        p[off:off + i * o] = mlp.bf16_round(p[off:off + i * o])
        p[off + i * o:off + i * o + o] = np.float32(p[off + i * o:off + i * o + o])
        off += i * o + o
    x = np.zeros((n, 16))
    x[:, :5] = mlp.bf16_round(rng.uniform(-1, 1, size=(n, 5)))
    t = rng.normal(scale=0.5, size=(n, 4))
    return p, x, t


def _per_element(got, ref, rtol, label, flip_tol=None):
    """Per-element error |got - ref| / (|ref| + rms(ref)).  Every element
    within rtol; with flip_tol, every element within flip_tol and 99 % of
    them within rtol (see the module docstring).  Returns (worst, 99th
    percentile)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    err = np.abs(got - ref) / (np.abs(ref) + max(scale, 1e-30))
    worst = float(err.max()) if err.size else 0.0
    p99 = float(np.quantile(err, 0.99)) if err.size else 0.0
    if flip_tol is None:
        assert worst <= rtol, (label, worst, rtol, int(np.argmax(err)))
    else:
        assert worst <= flip_tol, (label, worst, flip_tol, int(np.argmax(err)))
        assert p99 <= rtol, (label, p99, rtol)
    return worst, p99


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _split_bias_params(p):
    """The network the inference kernels evaluate: each bias as a BF16 leading
    part plus a BF16 remainder (the pair rides through the tensor core)."""
    q = np.array(p, dtype=np.float64)
    off = 0
    for i, o in mlp.LAYERS:
        b = np.float32(q[off + i * o:off + i * o + o])
        lead = mlp.bf16_round(b)
        rest = mlp.bf16_round(np.float32(b - np.float32(lead)))
        q[off + i * o:off + i * o + o] = lead + rest
        off += i * o + o
    return q


@pytest.mark.parametrize("n", [1, 37, 1000, 4096, 20000, 65536])
def test_forward_loss_and_gradients_per_element(n):
    from paper_1812_05902_gb300 import pivbos as P
    assert P.MLP_PARAMS == mlp.n_params()
    p, x, t = _case(n, 3 + n)
    y_inf = P.pivbos_mlp_forward(p, x)
    y_tr = P.pivbos_mlp_train_forward(p, x)
    loss, g = P.pivbos_mlp_loss_grad(p, x, t)
    # both forwards carry each bias through the tensor core as a BF16
    # leading part and remainder: the network they evaluate has those biases
    ps = _split_bias_params(p)
    y_ref, _ = mlp.forward(ps, x, bf16=True)
    loss_ref, g_ref = mlp.loss_and_grad(ps, x, t, bf16=True)
    errs = {"y_inference": _per_element(y_inf, y_ref, OUT_RTOL, "inference forward", OUT_FLIP),
            "y_training": _per_element(y_tr, y_ref, OUT_RTOL, "training forward", OUT_FLIP),
            "loss": abs(loss - loss_ref) / loss_ref}
    assert errs["loss"] <= 1e-4, errs
    off = 0
    for li, (i, o) in enumerate(mlp.LAYERS):
        for name, size in (("W%d" % li, i * o), ("b%d" % li, o)):
            errs[name] = _per_element(g[off:off + size], g_ref[off:off + size], RTOL, name)
            off += size
    print(n, errs)


@pytest.mark.parametrize("n", [4096, 65536])
def test_against_the_plain_fp64_network(n):
    """No BF16 storage in the reference: the GPU network is the FP64 network
    to within what BF16 activations cost."""
    from paper_1812_05902_gb300 import pivbos as P
    p, x, t = _case(n, 11 + n)
    y = P.pivbos_mlp_forward(p, x)
    loss, g = P.pivbos_mlp_loss_grad(p, x, t)
    y_ref, _ = mlp.forward(p, x, bf16=False)
    loss_ref, g_ref = mlp.loss_and_grad(p, x, t, bf16=False)
    assert _rel(y, y_ref) < 1e-2
    assert abs(loss - loss_ref) / loss_ref < 1e-2
    off = 0
    for i, o in mlp.LAYERS:
        for size in (i * o, o):
            assert _rel(g[off:off + size], g_ref[off:off + size]) < 2e-2
            off += size


def test_adam_steps_per_element():
    """Five Adam steps of the training kernel (FP32 master weights, moments)
    against mlp.adam in FP64, element by element; the BF16 weight copy the
    kernel writes is the FP32 weight rounded to nearest even, bit for bit."""
    from paper_1812_05902_gb300 import pivbos as P
    rng = np.random.default_rng(21)
    p0 = np.float32(mlp.init(4) + rng.normal(scale=0.02, size=mlp.n_params()))
    m0 = np.float32(rng.normal(scale=1e-3, size=mlp.n_params()))
    v0 = np.float32(np.abs(rng.normal(scale=1e-6, size=mlp.n_params())))
    grads = np.float32(rng.normal(scale=1e-2, size=(5, mlp.n_params())) *
                       rng.uniform(0.0, 2.0, size=mlp.n_params()))
    lrs = np.float32([3e-3, 2.5e-3, 2e-3, 1e-3, 5e-4])
    t0 = 3
    p_g, m_g, v_g, wbf = P.pivbos_mlp_adam_steps(p0, m0, v0, grads, t0, lrs)
    p_r, m_r, v_r = p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
    for q in range(5):
        p_r, m_r, v_r = mlp.adam(p_r, grads[q].astype(np.float64), m_r, v_r, t0 + q, float(lrs[q]))
    # moments: FP32 against FP64 (m can cancel to near zero: a floor at its RMS)
    _per_element(m_g, m_r, 1e-5, "adam m")
    assert np.max(np.abs(v_g - v_r) / np.abs(v_r)) < 1e-5
    # FP32 rounding of p at every step (half an ulp each) and of each step's
    # quotient (a few FP32 roundings of the step's size)
    steps = np.zeros_like(p_r)
    pp, mm, vv = p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
    for q in range(5):
        pn, mm, vv = mlp.adam(pp, grads[q].astype(np.float64), mm, vv, t0 + q, float(lrs[q]))
        steps += np.abs(pn - pp)
        pp = pn
    dp = np.abs(p_g.astype(np.float64) - p_r)
    bound = 2.0 ** -24 * 5 * np.maximum(np.abs(p_r), np.abs(p0)) + 1e-6 * steps
    assert np.all(dp <= bound), float(np.max(dp / bound))
    # the BF16 copy of the weights (biases excluded), bit for bit
    bits = p_g.view(np.uint32)
    rne = ((bits + ((bits >> 16) & 1) + np.uint32(0x7FFF)) >> 16).astype(np.uint16)
    off, woff = 0, 0
    for i, o in mlp.LAYERS:
        assert np.array_equal(wbf[woff:woff + i * o], rne[off:off + i * o])
        off += i * o + o
        woff += i * o


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 70001])
def test_surrogate_network_kernel_per_element(n):
    """The render's network kernel (persistent CTAs, two warpgroups, tcgen05
    with TMEM accumulators) over n served rows: r = b + MLP(x) * t_scale,
    against the FP64 network with the kernel's two-part BF16 biases, every
    element of every row (partial last tile included)."""
    from paper_1812_05902_gb300 import pivbos as P
    p, x, _ = _case(n, 29 + n)
    rng = np.random.default_rng(n)
    b = np.float32(rng.normal(scale=1e-4, size=(n, 4)))
    ts = np.float32([2e-5, 3e-5, 1e-4, 5e-5])
    r = P.pivbos_surrogate_net_apply(p, x, b, ts)
    y_ref, _ = mlp.forward(_split_bias_params(p), x, bf16=True)
    corr = (r.astype(np.float64) - b.astype(np.float64)) / ts.astype(np.float64)
    # r is rounded to FP32 after the addition: one ulp of |b| + |y| * t_scale
    ulp = 2.0 ** -23 * (np.abs(b) + np.abs(y_ref) * ts) / ts
    err = np.maximum(np.abs(corr - y_ref) - 2.0 * ulp, 0.0)
    scale = np.sqrt(np.mean(y_ref * y_ref))
    e = err / (np.abs(y_ref) + scale)
    worst, p99 = float(np.max(e)), float(np.quantile(e, 0.99))
    print(n, worst, p99)
    assert worst <= OUT_FLIP, worst
    assert p99 <= OUT_RTOL, p99
