"""BF16 surrogate kernels vs the FP64 surrogate oracle, and training on fields
produced by the particle simulation (CUDA path; needs a GB300).

Tolerances: the kernels round operands and outputs to BF16 (8 significant
bits, relative spacing 2^-8) and accumulate in FP32, so a BF16 output must be
within 2^-8 |ref| + 2e-3 max|ref| of the oracle fed the same BF16 operands,
and an FP32 weight gradient within 1e-4 max|ref|."""
import numpy as np
import pytest

import paper_2211_15630_gb300 as A
from oracle import surrogate as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15630_gb300 import build

    build.build()
    return A.load()


def _dev_bf16(a):
    bits = S.bf16_bits(a)
    return torch.from_numpy(bits.view(np.int16).copy()).cuda()


def _host_bf16(t):
    return S.from_bf16_bits(t.cpu().numpy().view(np.uint16))


def _dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _close_bf16(got, ref):
    tol = 2.0 ** -8 * np.abs(ref) + 2e-3 * np.abs(ref).max()
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{bad.sum()} of {bad.size} out of tolerance, worst {np.abs(got - ref).max():.3g}"


@pytest.mark.parametrize("cin,cout,relu", [(16, 32, 1), (32, 32, 1), (32, 8, 0), (32, 32, 0)])
def test_conv_forward(lib, cin, cout, relu):
    g = np.random.default_rng(cin + cout + relu)
    B, H, W = 2, 16, 32
    x = S.bf16_round(g.normal(size=(B, H, W, cin)))
    w = S.bf16_round(g.normal(size=(cout, 9, cin)) * 0.2)
    b = g.normal(size=cout).astype(np.float32).astype(np.float64)
    y = torch.zeros(B * H * W * cout, dtype=torch.int16, device="cuda")
    # keep every device tensor referenced until the kernel has run: a freed
    # temporary's memory would be handed to the next allocation
    xd, wd, bd = _dev_bf16(x), _dev_bf16(w.transpose(1, 0, 2)), _dev_f32(b)
    A.aap_conv3x3_forward(xd.data_ptr(), B, H, W, cin, cout, wd.data_ptr(), bd.data_ptr(), relu, y.data_ptr())
    torch.cuda.synchronize()
    ref = S.conv_forward(x, w, b)
    if relu:
        ref = np.maximum(ref, 0)
    _close_bf16(_host_bf16(y).reshape(ref.shape), ref)


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 16)])
def test_conv_backward_data(lib, cin, cout):
    """cout is the channel count of dy (16: the padded output gradient of the
    last layer)."""
    g = np.random.default_rng(7 + cout)
    B, H, W = 2, 16, 32
    dy = S.bf16_round(g.normal(size=(B, H, W, cout)))
    w = S.bf16_round(g.normal(size=(cout, 9, cin)) * 0.2)       # forward weights of the layer
    mask = S.bf16_round(g.normal(size=(B, H, W, cin)))
    wt_t = np.zeros((9, cin, cout))
    for tap in range(9):
        wt_t[tap] = w[:, 8 - tap, :].T
    dx = torch.zeros(B * H * W * cin, dtype=torch.int16, device="cuda")
    dyd, wtd, md = _dev_bf16(dy), _dev_bf16(wt_t), _dev_bf16(mask)
    A.aap_conv3x3_backward_data(dyd.data_ptr(), B, H, W, cin, cout, wtd.data_ptr(), md.data_ptr(), dx.data_ptr())
    torch.cuda.synchronize()
    ref = S.conv_backward_data(dy, w) * (mask > 0)
    _close_bf16(_host_bf16(dx).reshape(ref.shape), ref)


@pytest.mark.parametrize("cin,cout,stride", [(32, 32, 32), (16, 32, 32), (32, 8, 16)])
def test_conv_backward_weight(lib, cin, cout, stride):
    g = np.random.default_rng(11 + cin + cout)
    B, H, W = 3, 16, 32
    x = S.bf16_round(g.normal(size=(B, H, W, cin)))
    dyf = S.bf16_round(g.normal(size=(B, H, W, stride)))
    parts = (H // 4) * B * (cout * 9 * cin + cout)
    part = torch.zeros(parts, dtype=torch.float32, device="cuda")
    dw = torch.zeros(cout * 9 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    xd, dyd = _dev_bf16(x), _dev_bf16(dyf)
    A.aap_conv3x3_backward_weight(xd.data_ptr(), dyd.data_ptr(), stride, B, H, W, cin, cout, part.data_ptr(),
                                  parts, dw.data_ptr(), db.data_ptr())
    torch.cuda.synchronize()
    rdw, rdb = S.conv_backward_weight(x, dyf[..., :cout])
    gdw = dw.cpu().numpy().reshape(rdw.shape)
    assert np.abs(gdw - rdw).max() <= 1e-4 * np.abs(rdw).max()
    assert np.abs(db.cpu().numpy() - rdb).max() <= 1e-4 * np.abs(rdb).max()
    # deterministic: a second call gives the same bits
    dw2 = torch.zeros_like(dw)
    A.aap_conv3x3_backward_weight(xd.data_ptr(), dyd.data_ptr(), stride, B, H, W, cin, cout, part.data_ptr(),
                                  parts, dw2.data_ptr(), db.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(dw, dw2)


# The convolution runs persistent blocks (at most 4 per SM, 608 on a GB300)
# over tiles of 16 x 8 pixels with two halo buffers, two TMEM accumulators and
# two mbarriers whose wait parity flips every second tile of a block.  At
# 128 x 128 and batch 20 there are 2560 tiles, so every block runs at least
# four of them: both buffers and both parities of each mbarrier, the path
# every full-size call of the surrogate (128 x 128 fields) takes.
FULL_B, FULL_H, FULL_W = 20, 128, 128


@pytest.mark.parametrize("cin,cout,relu", [(16, 32, 1), (32, 32, 1), (32, 8, 0)])
def test_conv_forward_full_size(lib, cin, cout, relu):
    g = np.random.default_rng(100 + cin + cout + relu)
    B, H, W = FULL_B, FULL_H, FULL_W
    assert (H // 16) * (W // 8) * B >= 4 * 608
    x = S.bf16_round(g.normal(size=(B, H, W, cin)))
    w = S.bf16_round(g.normal(size=(cout, 9, cin)) * 0.2)
    b = g.normal(size=cout).astype(np.float32).astype(np.float64)
    y = torch.zeros(B * H * W * cout, dtype=torch.int16, device="cuda")
    xd, wd, bd = _dev_bf16(x), _dev_bf16(w.transpose(1, 0, 2)), _dev_f32(b)
    A.aap_conv3x3_forward(xd.data_ptr(), B, H, W, cin, cout, wd.data_ptr(), bd.data_ptr(), relu, y.data_ptr())
    torch.cuda.synchronize()
    ref = S.conv_forward(x, w, b)
    if relu:
        ref = np.maximum(ref, 0)
    _close_bf16(_host_bf16(y).reshape(ref.shape), ref)


def test_conv_backward_data_full_size(lib):
    cin, cout = 32, 32
    g = np.random.default_rng(207)
    B, H, W = FULL_B, FULL_H, FULL_W
    dy = S.bf16_round(g.normal(size=(B, H, W, cout)))
    w = S.bf16_round(g.normal(size=(cout, 9, cin)) * 0.2)
    mask = S.bf16_round(g.normal(size=(B, H, W, cin)))
    wt_t = np.zeros((9, cin, cout))
    for tap in range(9):
        wt_t[tap] = w[:, 8 - tap, :].T
    dx = torch.zeros(B * H * W * cin, dtype=torch.int16, device="cuda")
    dyd, wtd, md = _dev_bf16(dy), _dev_bf16(wt_t), _dev_bf16(mask)
    A.aap_conv3x3_backward_data(dyd.data_ptr(), B, H, W, cin, cout, wtd.data_ptr(), md.data_ptr(), dx.data_ptr())
    torch.cuda.synchronize()
    ref = S.conv_backward_data(dy, w) * (mask > 0)
    _close_bf16(_host_bf16(dx).reshape(ref.shape), ref)


def _random_params(n, seed):
    g = np.random.default_rng(seed)
    layers = S.unpack(g.normal(size=n) * 0.1)
    layers[0][0][:, :, 4:] = 0
    layers[3][0][3:] = 0
    layers[3][1][3:] = 0
    return S.pack(layers).astype(np.float32)


@pytest.mark.parametrize("conserve", [0, 3])
def test_network_loss_and_gradient(lib, conserve):
    """One train step's loss and parameter gradient against the oracle network
    (BF16-rounded weights, input and activations, FP64 arithmetic), without and
    with the projection that keeps the grid means."""
    B, H, W = 2, 16, 32
    sp = A.aap_sur_params_default(nbx=W, nby=H, max_batch=B, conserve=conserve)
    s = A.aap_sur_create(sp)
    try:
        n = A.aap_sur_param_count(s)
        params = _random_params(n, 5)
        A.aap_sur_set_params(s, params)
        g = np.random.default_rng(9)
        fields = np.abs(g.normal(size=(B, 3, H, W))) + 1.0
        fields[:, 1:] -= 1.5
        target = fields + 0.2 * g.normal(size=fields.shape)
        eta = np.array([0.33, 0.47])
        fd, td, ed = _dev_f32(fields), _dev_f32(target), _dev_f32(eta)
        loss = A.aap_sur_train_step(s, fd.data_ptr(), td.data_ptr(), ed.data_ptr(), B)
        grad = A.aap_sur_get_grads(s).astype(np.float64)
        st, x0 = S.normalise(fields.astype(np.float32), eta.astype(np.float32), 2.0, 0.4, 0.1)
        tg, _ = S.normalise(target.astype(np.float32), eta.astype(np.float32), 2.0, 0.4, 0.1)
        pw = S.pack([(S.bf16_round(w), b) for w, b in S.unpack(params.astype(np.float64))])
        rloss, rgrad = S.loss_and_grad(pw, st, S.bf16_round(x0), tg, round_act=S.bf16_round, conserve=conserve)
        assert abs(loss - rloss) <= 1e-2 * rloss
        rel = np.linalg.norm(grad - rgrad) / np.linalg.norm(rgrad)
        cos = grad @ rgrad / (np.linalg.norm(grad) * np.linalg.norm(rgrad))
        assert rel < 3e-2 and cos > 0.999, (rel, cos)
        # after the step the parameters moved by the Adam rule
        p1 = A.aap_sur_get_params(s).astype(np.float64)
        e1, _, _ = S.adam(params.astype(np.float64), grad, np.zeros(n), np.zeros(n), 1)
        assert np.abs(p1 - e1).max() < 1e-6
    finally:
        A.aap_sur_destroy(s)


def test_network_gradient_full_size(lib):
    """One train step at the surrogate's own field size (128 x 128) and batch
    20: every convolution of the forward and backward pass runs its blocks
    over several tiles.  Loss and gradient against the oracle network."""
    B, H, W = FULL_B, FULL_H, FULL_W
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B))
    try:
        n = A.aap_sur_param_count(s)
        params = _random_params(n, 41)
        A.aap_sur_set_params(s, params)
        g = np.random.default_rng(42)
        fields = np.abs(g.normal(size=(B, 3, H, W))) + 1.0
        fields[:, 1:] -= 1.5
        target = fields + 0.2 * g.normal(size=fields.shape)
        eta = g.uniform(0.3, 0.5, B)
        fd, td, ed = _dev_f32(fields), _dev_f32(target), _dev_f32(eta)
        loss = A.aap_sur_train_step(s, fd.data_ptr(), td.data_ptr(), ed.data_ptr(), B)
        grad = A.aap_sur_get_grads(s).astype(np.float64)
        st, x0 = S.normalise(fields.astype(np.float32), eta.astype(np.float32), 2.0, 0.4, 0.1)
        tg, _ = S.normalise(target.astype(np.float32), eta.astype(np.float32), 2.0, 0.4, 0.1)
        pw = S.pack([(S.bf16_round(w), b) for w, b in S.unpack(params.astype(np.float64))])
        rloss, rgrad = S.loss_and_grad(pw, st, S.bf16_round(x0), tg, round_act=S.bf16_round)
        assert abs(loss - rloss) <= 1e-2 * rloss
        rel = np.linalg.norm(grad - rgrad) / np.linalg.norm(rgrad)
        cos = grad @ rgrad / (np.linalg.norm(grad) * np.linalg.norm(rgrad))
        assert rel < 3e-2 and cos > 0.999, (rel, cos)
    finally:
        A.aap_sur_destroy(s)


def test_adam_over_several_steps(lib):
    """Five train steps on one batch: after each, the parameters equal the
    oracle's Adam recursion fed the library's own gradients, with the moments
    carried over and the bias correction of step t (a one-step check cannot
    tell a moment that restarts every step from one that is kept)."""
    B, H, W = 2, 16, 32
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B, lr=1e-3))
    try:
        n = A.aap_sur_param_count(s)
        params = _random_params(n, 51)
        A.aap_sur_set_params(s, params)
        g = np.random.default_rng(52)
        fields = np.abs(g.normal(size=(B, 3, H, W))) + 1.0
        target = fields + 0.2 * g.normal(size=fields.shape)
        fd, td, ed = _dev_f32(fields), _dev_f32(target), _dev_f32([0.35, 0.45])
        p_ref = params.astype(np.float64)
        m = np.zeros(n)
        v = np.zeros(n)
        for t in range(1, 6):
            A.aap_sur_train_step(s, fd.data_ptr(), td.data_ptr(), ed.data_ptr(), B)
            grad = A.aap_sur_get_grads(s).astype(np.float64)
            p_ref, m, v = S.adam(p_ref, grad, m, v, t, lr=1e-3)
            got = A.aap_sur_get_params(s).astype(np.float64)
            assert np.abs(got - p_ref).max() < 2e-6, (t, np.abs(got - p_ref).max())
            p_ref = got                      # the next step starts from the library's FP32 weights
    finally:
        A.aap_sur_destroy(s)


def test_predict_zero_and_one_application(lib):
    B, H, W = 2, 16, 16
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B, seed=3))
    try:
        g = np.random.default_rng(4)
        f = np.abs(g.normal(size=(B, 3, H, W))).astype(np.float32) + 1
        fin, eta = _dev_f32(f), _dev_f32([0.4, 0.45])
        out = torch.zeros_like(fin)
        A.aap_sur_predict(s, fin.data_ptr(), eta.data_ptr(), B, 0, out.data_ptr())
        torch.cuda.synchronize()
        assert np.allclose(out.cpu().numpy(), f, rtol=1e-6, atol=1e-6)
        A.aap_sur_predict(s, fin.data_ptr(), eta.data_ptr(), B, 1, out.data_ptr())
        torch.cuda.synchronize()
        params = A.aap_sur_get_params(s).astype(np.float64)
        st, x0 = S.normalise(f, np.array([0.4, 0.45], np.float32), 2.0, 0.4, 0.1)
        pw = S.pack([(S.bf16_round(w), b) for w, b in S.unpack(params)])
        ref, _ = S.forward(pw, st, S.bf16_round(x0), round_act=S.bf16_round)
        got = out.cpu().numpy()
        rf = S.denormalise(ref, 2.0)
        assert np.abs(got - rf).max() < 2e-2 * np.abs(rf).max()
    finally:
        A.aap_sur_destroy(s)


def _trajectory_frames(eta, seed, n, L, bins, warm, frames, every):
    p = A.aap_params_default(n=n, lx=L, ly=L, eta=eta, v=0.5, seed=seed)
    h = A.aap_create(p)
    out = torch.zeros(frames, 3 * bins * bins, dtype=torch.float32, device="cuda")
    try:
        A.aap_step(h, warm)
        for k in range(frames):
            A.aap_coarse_grain(h, bins, bins, out[k].data_ptr())
            A.aap_step(h, every)
        A.aap_sync(h)
    finally:
        A.aap_destroy(h)
    return out.view(frames, 3, bins, bins)


def test_trained_surrogate_beats_persistence(lib):
    """Train on fields of the particle simulation (N = 2^17, L = 256, 64 x 64
    bins of 4 x 4, 10 steps per application) and compare with the method
    without the network -- keeping the fields unchanged -- on a held-out
    trajectory: the network's mean squared error must be clearly lower."""
    n, L, bins = 1 << 17, 256.0, 64
    train = []
    for k, eta in enumerate((0.3, 0.35, 0.4, 0.45, 0.5)):
        fr = _trajectory_frames(eta, 10000 + k, n, L, bins, 100, 41, 10)
        train.append((eta, fr))
    held = _trajectory_frames(0.42, 20000, n, L, bins, 100, 21, 10)
    B = 16
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=bins, nby=bins, max_batch=B, lr=2e-3, seed=7))
    g = np.random.default_rng(0)
    try:
        xin = torch.zeros(B, 3, bins, bins, device="cuda")
        xtg = torch.zeros_like(xin)
        eta_t = torch.zeros(B, device="cuda")
        for it in range(500):
            for b in range(B):
                j = g.integers(len(train))
                t = g.integers(40)
                xin[b] = train[j][1][t]
                xtg[b] = train[j][1][t + 1]
                eta_t[b] = train[j][0]
            A.aap_sur_train_step(s, xin.data_ptr(), xtg.data_ptr(), eta_t.data_ptr(), B)
        # held-out one-application error vs persistence (normalised units)
        hb = min(B, 20)
        fin = held[:hb].contiguous()
        tgt = held[1:hb + 1].contiguous()
        eta_h = torch.full((hb,), 0.42, device="cuda")
        pred = torch.zeros_like(fin)
        A.aap_sur_predict(s, fin.data_ptr(), eta_h.data_ptr(), hb, 1, pred.data_ptr())
        torch.cuda.synchronize()
        mse_net = float(((pred - tgt) ** 2).mean())
        mse_keep = float(((fin - tgt) ** 2).mean())
        assert mse_net < 0.85 * mse_keep, (mse_net, mse_keep)
    finally:
        A.aap_sur_destroy(s)


def test_conserving_predict_keeps_grid_means(lib):
    """With conserve = 3, ten applications keep every sample's total density
    (particle number) and total polarisation; without, they drift."""
    B, H, W = 2, 16, 32
    g = np.random.default_rng(12)
    f = (np.abs(g.normal(size=(B, 3, H, W))) + 1.0).astype(np.float32)
    f[:, 1:] -= 1.2
    fin, eta = _dev_f32(f), _dev_f32([0.35, 0.45])
    sums = {}
    for conserve in (0, 3):
        s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B, seed=8, conserve=conserve))
        try:
            A.aap_sur_set_params(s, _random_params(A.aap_sur_param_count(s), 13))
            out = torch.zeros_like(fin)
            A.aap_sur_predict(s, fin.data_ptr(), eta.data_ptr(), B, 10, out.data_ptr())
            torch.cuda.synchronize()
            sums[conserve] = out.cpu().numpy().astype(np.float64).sum(axis=(2, 3))
        finally:
            A.aap_sur_destroy(s)
    ref = f.astype(np.float64).sum(axis=(2, 3))
    assert np.allclose(sums[3], ref, rtol=1e-4, atol=1e-3 * H * W)
    assert not np.allclose(sums[0], ref, rtol=1e-4, atol=1e-3 * H * W)


def test_predict_replays_its_graph(lib):
    """A predict call is captured as a CUDA graph and replayed while its buffers,
    batch and number of applications stay the same: the replay gives the same
    fields bit for bit, and six applications in one call match six chained
    one-application calls (which re-normalise the fields in between)."""
    B, H, W = 2, 16, 32
    s = A.aap_sur_create(A.aap_sur_params_default(nbx=W, nby=H, max_batch=B, seed=21))
    try:
        A.aap_sur_set_params(s, _random_params(A.aap_sur_param_count(s), 22))
        g = np.random.default_rng(23)
        f = (np.abs(g.normal(size=(B, 3, H, W))) + 1.0).astype(np.float32)
        fin, eta = _dev_f32(f), _dev_f32([0.38, 0.46])
        out1, out2 = torch.zeros_like(fin), torch.zeros_like(fin)
        A.aap_sur_predict(s, fin.data_ptr(), eta.data_ptr(), B, 6, out1.data_ptr())
        torch.cuda.synchronize()
        first = out1.clone()
        out1.zero_()
        A.aap_sur_predict(s, fin.data_ptr(), eta.data_ptr(), B, 6, out1.data_ptr())   # replay
        torch.cuda.synchronize()
        assert torch.equal(first, out1)
        x, y = fin.clone(), out2
        for _ in range(6):
            A.aap_sur_predict(s, x.data_ptr(), eta.data_ptr(), B, 1, y.data_ptr())
            torch.cuda.synchronize()
            x, y = y, x
        assert np.allclose(x.cpu().numpy(), first.cpu().numpy(), rtol=1e-4, atol=1e-4)
    finally:
        A.aap_sur_destroy(s)
