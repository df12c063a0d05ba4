"""Pins of the surrogate oracle (no GPU): scipy's wrap-boundary correlation for
the forward pass, central finite differences for both gradients and for the
whole network, closed forms of Adam and of BF16 rounding."""
import numpy as np
import pytest

from oracle import surrogate as S

signal = pytest.importorskip("scipy.signal")


def test_forward_matches_scipy_correlate2d():
    g = np.random.default_rng(0)
    x = g.normal(size=(2, 8, 16, 3))
    w = g.normal(size=(4, 9, 3))
    b = g.normal(size=4)
    y = S.conv_forward(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = np.full((8, 16), b[co])
            for ci in range(3):
                k = w[co, :, ci].reshape(3, 3)
                ref += signal.correlate2d(x[n, :, :, ci], k, mode="same", boundary="wrap")
            assert np.allclose(y[n, :, :, co], ref, atol=1e-12)


def _fd(f, a, idx, h=1e-6):
    a = a.copy()
    a[idx] += h
    fp = f(a)
    a[idx] -= 2 * h
    fm = f(a)
    return (fp - fm) / (2 * h)


def test_backward_data_and_weight_finite_differences():
    g = np.random.default_rng(1)
    x = g.normal(size=(2, 8, 16, 5))
    w = g.normal(size=(3, 9, 5))
    b = g.normal(size=3)
    c = g.normal(size=(2, 8, 16, 3))      # L = sum(c * y)
    L = lambda xx=x, ww=w, bb=b: float((c * S.conv_forward(xx, ww, bb)).sum())
    dx = S.conv_backward_data(c, w)
    dw, db = S.conv_backward_weight(x, c)
    for idx in [(0, 0, 0, 0), (1, 7, 15, 4), (0, 3, 9, 2), (1, 0, 15, 1)]:
        assert abs(_fd(lambda a: L(xx=a), x, idx) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0), (2, 8, 4), (1, 4, 2)]:
        assert abs(_fd(lambda a: L(ww=a), w, idx) - dw[idx]) < 1e-6
    for k in range(3):
        assert abs(_fd(lambda a: L(bb=a), b, k) - db[k]) < 1e-6


def test_network_gradient_finite_differences():
    g = np.random.default_rng(2)
    n = sum(co * 9 * ci + co for ci, co in S.LAYERS)
    params = g.normal(size=n) * 0.2
    # keep the padding at zero like the library
    layers = S.unpack(params.copy())
    layers[0][0][:, :, 4:] = 0
    layers[3][0][3:] = 0
    layers[3][1][3:] = 0
    params = S.pack(layers)
    fields = np.abs(g.normal(size=(2, 3, 8, 16))) + 1.0
    target = fields + 0.1 * g.normal(size=fields.shape)
    st, x0 = S.normalise(fields, [0.35, 0.45], 2.0, 0.4, 0.1)
    tg, _ = S.normalise(target, [0.35, 0.45], 2.0, 0.4, 0.1)
    loss, grad = S.loss_and_grad(params, st, x0, tg)
    f = lambda p: S.loss_and_grad(p, st, x0, tg)[0]
    nz = np.nonzero(grad)[0]
    for i in np.random.default_rng(3).choice(nz, 12, replace=False):
        assert abs(_fd(f, params, i, 1e-6) - grad[i]) < 1e-7 + 1e-5 * abs(grad[i])
    # padded weights get no gradient
    gl = S.unpack(grad)
    assert not gl[0][0][:, :, 4:].any() and not gl[3][0][3:].any() and not gl[3][1][3:].any()


def test_adam_first_step_closed_form():
    """First Adam step moves every parameter by lr * sign(grad) (bias-corrected)."""
    p = np.array([1.0, -2.0, 0.5])
    gr = np.array([0.3, -4.0, 1e-3])
    p1, m, v = S.adam(p, gr, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(gr), atol=1e-15)


def test_adam_constant_gradient_every_step():
    """A constant gradient g gives bias-corrected moments m^ = g and v^ = g^2 at
    every step t, so each step moves a parameter by exactly lr g / (|g| + eps).
    A moment that is not carried over between steps, or a bias correction with
    the wrong t, breaks this from t = 2 on."""
    p = np.array([1.0, -2.0, 0.5, 3.0])
    gr = np.array([0.3, -4.0, 1e-3, 2.5e-6])
    lr, eps = 0.01, 1e-8
    m = v = np.zeros(4)
    for t in range(1, 8):
        p_new, m, v = S.adam(p, gr, m, v, t, lr=lr, eps=eps)
        assert np.allclose(p_new - p, -lr * gr / (np.abs(gr) + eps), rtol=1e-10, atol=1e-16), t
        p = p_new


def test_adam_alternating_gradient_closed_form():
    """g_t = (-1)^t c: the first moment is the geometric sum
    m_t = (1 - b1) c (-1)^t (1 - (-b1)^t) / (1 + b1) and the second
    v_t = (1 - b2^t) c^2, so the step is known in closed form for every t."""
    c, lr, b1, b2, eps = np.array([0.7, -1.3]), 0.05, 0.9, 0.999, 1e-8
    p = np.array([0.2, 0.4])
    m = v = np.zeros(2)
    for t in range(1, 9):
        g = (-1.0) ** t * c
        p_new, m, v = S.adam(p, g, m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        mt = (1 - b1) * c * (-1.0) ** t * (1 - (-b1) ** t) / (1 + b1)
        vt = (1 - b2 ** t) * c * c
        assert np.allclose(m, mt, rtol=1e-12) and np.allclose(v, vt, rtol=1e-12)
        step = lr * (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
        assert np.allclose(p - p_new, step, rtol=1e-10), t
        p = p_new


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.0e-5, 65280.0, 1.0 + 2 ** -9])
    r = S.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert r[5] == 1.0   # tie to even
    assert np.array_equal(S.from_bf16_bits(S.bf16_bits(vals)), r)


@pytest.mark.parametrize("conserve", [1, 2, 3])
def test_conserving_network_keeps_means_and_gradient(conserve):
    """With the projection P the conserved channels keep their per-sample grid
    mean exactly over an application (the total particle number for the
    density), and the gradient still matches central finite differences."""
    g = np.random.default_rng(5)
    n = sum(co * 9 * ci + co for ci, co in S.LAYERS)
    layers = S.unpack(g.normal(size=n) * 0.2)
    layers[0][0][:, :, 4:] = 0
    layers[3][0][3:] = 0
    layers[3][1][3:] = 0
    params = S.pack(layers)
    fields = np.abs(g.normal(size=(2, 3, 8, 16))) + 1.0
    target = fields + 0.1 * g.normal(size=fields.shape)
    st, x0 = S.normalise(fields, [0.3, 0.5], 2.0, 0.4, 0.1)
    tg, _ = S.normalise(target, [0.3, 0.5], 2.0, 0.4, 0.1)
    out, _ = S.forward(params, st, x0, conserve=conserve)
    free, _ = S.forward(params, st, x0, conserve=0)
    for c in range(3):
        kept = c in S.conserved_channels(conserve)
        same = np.allclose(out[..., c].mean(axis=(1, 2)), st[..., c].mean(axis=(1, 2)), rtol=0, atol=1e-12)
        assert same == kept or (not kept and np.allclose(out[..., c], free[..., c]))
    loss, grad = S.loss_and_grad(params, st, x0, tg, conserve=conserve)
    f = lambda p: S.loss_and_grad(p, st, x0, tg, conserve=conserve)[0]
    nz = np.nonzero(grad)[0]
    for i in np.random.default_rng(6).choice(nz, 12, replace=False):
        assert abs(_fd(f, params, i, 1e-6) - grad[i]) < 1e-7 + 1e-5 * abs(grad[i])
