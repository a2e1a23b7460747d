"""Pin of the FP64 proposal-network oracle: analytic gradients against
central finite differences (CPU)."""
import numpy as np

from oracle import mlp_oracle as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = M.init_params(1).astype(np.float64) * 0.5
    # non-zero biases so every bias gradient is exercised
    k = 0
    for i, o in M.DIMS:
        k += i * o
        p[k:k + o] = rng.normal(0, 0.1, o)
        k += o
    X = rng.normal(0, 1, (4, 1536))
    lab = rng.integers(0, 4096, 4)
    loss, g = M.loss_and_grad(p, X, lab)
    assert np.isfinite(loss) and g.shape == p.shape
    # parameters from every tensor, including the largest-gradient ones
    offs, k = [], 0
    for i, o in M.DIMS:
        offs.append((k, i * o))
        k += i * o
        offs.append((k, o))
        k += o
    idx = []
    for start, size in offs:
        seg = np.abs(g[start:start + size])
        idx += list(start + rng.choice(size, 3, replace=False))
        idx.append(start + int(np.argmax(seg)))
    h = 1e-6
    for j in idx:
        q = p.copy()
        q[j] += h
        lp, _ = M.loss_and_grad(q, X, lab)
        q[j] -= 2 * h
        lm, _ = M.loss_and_grad(q, X, lab)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j])) + 1e-8, (j, fd, g[j])


def test_loss_closed_form_at_zero_weights():
    """All-zero parameters give uniform logits: loss = log 4096, and the only
    nonzero gradient is the output bias, (1/4096 - onehot) / B."""
    p = np.zeros(M.num_params())
    X = np.ones((3, 1536))
    lab = np.array([0, 5, 4095])
    loss, g = M.loss_and_grad(p, X, lab)
    assert abs(loss - np.log(4096)) < 1e-12
    gb4 = g[-4096:]
    expect = np.full(4096, 1 / 4096)
    for l in lab:
        expect[l] -= 1 / 3
    np.testing.assert_allclose(gb4, expect, rtol=0, atol=1e-15)
    assert np.all(g[:-4096] == 0)
