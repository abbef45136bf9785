"""Pins of the FP64 reference network (oracle/unet.py): gradients against
central differences, closed forms of the convolution and of the first Adam
step, and the exact parameter count."""
import numpy as np

from oracle import unet


def test_parameter_count():
    # 27 (2*16 + 16*32 + 32*64 + 64*128 + 192*64 + 96*32 + 48*16) + 16*1 weights + biases
    assert unet.param_count() == 27 * 26912 + 16 + (16 + 32 + 64 + 128 + 64 + 32 + 16 + 1)


def test_conv_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 5, 6, 3))
    # only the centre tap: a per-voxel matrix product
    w = np.zeros((27, 2, 3))
    w[13] = rng.standard_normal((2, 3))
    b = np.array([0.5, -1.0])
    assert np.allclose(unet.conv(x, w, b), x @ w[13].T + b, atol=1e-14)
    # all-ones kernel on a constant field: 27 * Cin * c inside, fewer taps at the zero-padded faces
    ones = np.ones((27, 1, 3))
    y = unet.conv(np.full((4, 5, 6, 3), 2.0), ones, np.zeros(1))
    assert np.allclose(y[1:-1, 1:-1, 1:-1, 0], 27 * 3 * 2.0)
    assert np.allclose(y[0, 0, 0, 0], 8 * 3 * 2.0)           # corner: 2x2x2 neighbours
    # a tap moves the field by one cell: tap (dz,dy,dx) = (0,0,+1) reads x[.., i+1]
    w = np.zeros((27, 3, 3))
    w[(0 + 1) * 9 + (0 + 1) * 3 + (1 + 1)] = np.eye(3)
    y = unet.conv(x, w, np.zeros(3))
    assert np.allclose(y[:, :, :-1], x[:, :, 1:]) and np.allclose(y[:, :, -1], 0.0)


def test_pool_up_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((4, 4, 4, 2))
    b = rng.standard_normal((2, 2, 2, 2))
    # <pool(a), b> = <a, pool^T(b)> and <up(b), a> = <b, up^T(a)>
    assert np.isclose(np.sum(unet.pool(a) * b), np.sum(a * unet.pool_backward(b)))
    assert np.isclose(np.sum(unet.up(b) * a), np.sum(b * unet.up_backward(a)))


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    P = unet.init_params(3)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal((8, 8, 8, 2))
    t = rng.standard_normal((8, 8, 8, 1))
    y, c = unet.forward(P, x)
    G = unet.backward(P, c, y, t)
    h = 1e-6
    checked = 0
    for k in sorted(P):
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = unet.loss(unet.forward(P, x)[0], t)
            flat[idx] = old - h
            lm = unet.loss(unet.forward(P, x)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            g = G[k].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(abs(fd), abs(g)) + 1e-10, (k, idx, fd, g)
            checked += 1
    assert checked >= 60


def test_first_adam_step_closed_form():
    P = {"w": np.array([1.0, -2.0, 3.0])}
    G = {"w": np.array([0.5, -4.0, 0.0])}
    st = {}
    unet.adam_step(P, G, st, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)
    assert np.allclose(P["w"], [1.0 - 0.01 * 0.5 / (0.5 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8), 3.0])


def test_adam_bias_correction_with_a_constant_gradient():
    """Kingma and Ba's bias correction makes both moment estimates of a
    constant gradient exact at every step (m_hat = g, v_hat = g^2), so each of
    many steps moves a parameter by exactly -lr g / (|g| + eps); a correction
    with the wrong power of beta1 or beta2 after the first step would not."""
    g = np.array([0.5, -4.0, 2.0e-3])
    P = {"w": np.array([1.0, -2.0, 3.0])}
    st = {}
    want = P["w"].copy()
    for _ in range(12):
        unet.adam_step(P, {"w": g}, st, lr=0.01)
        want = want - 0.01 * g / (np.abs(g) + 1e-8)
        assert np.allclose(P["w"], want, rtol=0, atol=1e-13)


def test_bf16_round_ties_and_bounds():
    e = 2.0 ** -8          # half the bfloat16 spacing at 1
    vals = np.array([1.0, 3.0, 1 + e, 1 + 3 * e, 1 + e + 2.0 ** -20, -(1 + e), 2.0 ** -130, 65504.0])
    want = np.array([1.0, 3.0, 1.0, 1 + 4 * e, 1 + 2 * e, -1.0, 2.0 ** -130, 65536.0])
    assert np.array_equal(unet.bf16_round(vals), want)
    # relative rounding error at most half a unit in the 8th bit, and idempotent
    x = np.random.default_rng(4).standard_normal(10000) * 10.0 ** np.random.default_rng(5).uniform(-5, 5, 10000)
    r = unet.bf16_round(x)
    assert np.all(np.abs(r - np.float32(x)) <= 2.0 ** -8 * np.abs(np.float32(x)))
    assert np.array_equal(unet.bf16_round(r), r)


def test_bf16_round_matches_torch():
    torch = __import__("pytest").importorskip("torch")
    x = np.random.default_rng(6).standard_normal(4096).astype(np.float32)
    ours = unet.bf16_round(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, lib)


def test_storage_rounding_is_a_bounded_perturbation():
    """With every stored array rounded to bfloat16 the output stays within a
    few bfloat16 units of the FP64 network, and store=None is the FP64 path."""
    rng = np.random.default_rng(8)
    P = unet.init_params(9)
    x = rng.standard_normal((8, 8, 16, 2))
    y64, c64 = unet.forward(P, x)
    y_id, _ = unet.forward(P, x, store=lambda a: a)
    assert np.array_equal(y64, y_id)
    y16, _ = unet.forward(P, x, store=unet.bf16_round)
    e = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-4 < e < 2e-2


def test_seeded_initial_parameters_match_the_layer_table():
    """The input module's initial parameters (the GPU network's seeded input)
    are the reference network's He-normal initialisation in the flat order."""
    from paper_2412_16843_gb300 import inputs
    assert tuple(inputs.UNET_LAYERS) == tuple(unet.LAYERS)
    P = unet.init_params(5)
    flat = np.concatenate([np.concatenate([P[n + ".w"].ravel(), P[n + ".b"]]) for n, _, _, _ in unet.LAYERS])
    assert np.array_equal(inputs.unet_initial_params(5), flat)
    x, t = inputs.unet_pair(np.array([3.0, -4.0]), np.array([1.0, 2.0]), np.array([1.0, 0.0]), 2.0, 1.0, 0.5)
    # rms(f) = sqrt(12.5); rho = (2, 1) / 2; p / (rms * 2 * 0.25)
    assert np.allclose(x, [[3 / 12.5 ** 0.5, 1.0], [-4 / 12.5 ** 0.5, 0.5]])
    assert np.allclose(t, np.array([1.0, 2.0]) / (12.5 ** 0.5 * 0.5))


def test_parity_bounds_catch_a_wrong_tap_or_channel():
    """The bounds the GPU network tests use (forward 2e-3 relative L2, 1e-2
    per voxel; gradients 5e-2 relative L2, 1e-1 per entry, per layer) are
    below what a plausible indexing mistake does to the FP64 network: a
    mirrored tap (x+1 read as x-1) or two swapped input channels in one layer
    move the output by more than 10x the forward bound (18x to 600x here),
    and that layer's weight gradient by more than 1.5x the gradient bound."""
    rng = np.random.default_rng(5)
    shape = (8, 8, 8)
    P = unet.init_params(3)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal(shape + (2,))
    t = rng.standard_normal(shape + (1,))
    y, c = unet.forward(P, x)
    G = unet.backward(P, c, y, t)

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    tp, tm = 1 * 9 + 1 * 3 + 2, 1 * 9 + 1 * 3 + 0      # taps (0, 0, +1) and (0, 0, -1)
    for layer, kind in (("e1", "tap"), ("d0", "tap"), ("e0", "channel"), ("d1", "channel")):
        Pm = {k: v.copy() for k, v in P.items()}
        w = Pm[layer + ".w"]
        if kind == "tap":
            w[[tp, tm]] = w[[tm, tp]]
        else:
            w[:, :, [0, 1]] = w[:, :, [1, 0]]
        ym, cm = unet.forward(Pm, x)
        Gm = unet.backward(Pm, cm, ym, t)
        assert rel(ym, y) > 10 * 2e-3, (layer, kind, rel(ym, y))
        assert rel(Gm[layer + ".w"], G[layer + ".w"]) > 1.5 * 5e-2, (layer, kind)
