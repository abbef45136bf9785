"""GPU tests of the warm-start U-Net (BF16 tensor-core convolutions, FP32
accumulation): forward pass and gradients against the FP64 reference network,
Adam's first step, training on pressure solves of a 3D drop, and the
prediction as the multigrid first guess (same converged tolerance, fewer
V-cycles than a zero start)."""
import numpy as np
import pytest

from oracle import unet as ref
from paper_2412_16843_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_16843_gb300 import build
    build.build()
    cdi.load()


def flat(P):
    return np.concatenate([np.concatenate([P[n + ".w"].ravel(), P[n + ".b"]]) for n, _, _, _ in ref.LAYERS])


def unflat(v):
    P, o = {}, 0
    for n, ci, co, t in ref.LAYERS:
        P[n + ".w"] = v[o:o + t * co * ci].reshape(t, co, ci)
        o += t * co * ci
        P[n + ".b"] = v[o:o + co].copy()
        o += co
    assert o == v.size
    return P


def relnorm(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def as_stored(P):
    """The parameters as the tensor cores see them: BF16 weights, FP32 biases."""
    return {k: (ref.bf16_round(v) if k.endswith(".w") else np.float32(v).astype(np.float64)) for k, v in P.items()}


def random_case(shape, seed):
    rng = np.random.default_rng(seed)
    P = ref.init_params(seed)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal(shape + (2,))
    t = rng.standard_normal(shape + (1,))
    return P, x, t


@pytest.mark.parametrize("n", [(8, 8, 8), (24, 16, 8)], ids=["8^3", "24x16x8"])
def test_forward_matches_fp64_reference(n):
    """BF16 weights and activations, FP32 accumulation: output within 2e-2
    relative (L2) of the FP64 network on the same parameters and input, and
    within 2e-3 of the FP64 network that stores its arrays in BF16 (the
    remaining difference is FP32 against FP64 accumulation)."""
    shape = (n[2], n[1], n[0])
    P, x, _ = random_case(shape, 7)
    net = cdi.Unet(n)
    assert net.nparams == ref.param_count() == 726993
    net.set_params(flat(P))
    back = net.get_params()
    assert np.abs(back - flat(P)).max() <= 1e-6 * np.abs(flat(P)).max()   # FP32 master copy
    y = net.forward(x)
    y_ref, _ = ref.forward(P, x)
    e = relnorm(y, y_ref[..., 0])
    y_st, _ = ref.forward(as_stored(P), x, store=ref.bf16_round)
    e_st = relnorm(y, y_st[..., 0])
    m_st = np.abs(y - y_st[..., 0]).max() / np.abs(y_st).max()
    print("forward rel L2 error %.3e (FP64), %.3e (BF16 storage); max per voxel %.3e" % (e, e_st, m_st))
    assert e < 2e-2
    assert e_st < 2e-3
    # element by element: every output voxel within 1e-2 of the largest output
    assert m_st < 1e-2


def test_gradients_match_fp64_reference():
    """Gradients of the mean squared error, layer by layer.  The gradient of a
    ReLU network jumps where a pre-activation changes sign, so it is compared
    with the FP64 network that stores its arrays, and takes its ReLU
    decisions, in BF16 like the kernels (BF16 weights, FP32 biases): within
    5e-2 relative (L2).  Against the plain FP64 network the rounding of
    weights and activations alone moves these gradients by up to about 7e-2
    on this small grid (a numpy emulation of the storage points gives the same
    figure); that difference is bounded at 1e-1.  The loss is within 2e-2."""
    n = (16, 8, 8)
    shape = (n[2], n[1], n[0])
    P, x, t = random_case(shape, 11)
    net = cdi.Unet(n)
    net.set_params(flat(P))
    loss, g = net.train_step(x, t[..., 0], lr=0.0, want_grads=True)
    y_ref, cache = ref.forward(P, x)
    G = ref.backward(P, cache, y_ref, t)
    Ps = as_stored(P)
    y_st, cache_st = ref.forward(Ps, x, store=ref.bf16_round)
    G_st = ref.backward(Ps, cache_st, y_st, t, store=ref.bf16_round)
    assert abs(loss - ref.loss(y_ref, t)) <= 2e-2 * ref.loss(y_ref, t)
    Gg = unflat(g)
    for name, _, _, _ in ref.LAYERS:
        for part in (".w", ".b"):
            e_st = relnorm(Gg[name + part], G_st[name + part])
            e = relnorm(Gg[name + part], G[name + part])
            m_st = np.abs(Gg[name + part] - G_st[name + part]).max() / np.abs(G_st[name + part]).max()
            print("%-7s rel L2 error %.3e (BF16 storage), %.3e (FP64); max per entry %.3e"
                  % (name + part, e_st, e, m_st))
            assert e_st < 5e-2, (name + part, e_st)
            assert e < 1e-1, (name + part, e)
            # element by element: every gradient entry within 1e-1 of the layer's largest
            assert m_st < 1e-1, (name + part, m_st)
    # lr = 0 leaves the parameters untouched
    assert np.array_equal(net.get_params(), np.float32(flat(P)).astype(np.float64))


def test_first_adam_step():
    """First Adam step: m_hat = g and v_hat = g^2, so every parameter moves by
    lr * g / (|g| + 1e-8): at most lr, and exactly -lr sign(g) where the FP64
    gradient is large."""
    n = (8, 8, 8)
    shape = (n[2], n[1], n[0])
    P, x, t = random_case(shape, 13)
    net = cdi.Unet(n)
    net.set_params(flat(P))
    p0 = net.get_params()
    lr = 1e-3
    net.train_step(x, t[..., 0], lr=lr)
    d = net.get_params() - p0
    assert np.abs(d).max() <= lr * (1 + 3e-4)   # FP32 rounding of w - lr
    y_ref, cache = ref.forward(P, x)
    g = flat(ref.backward(P, cache, y_ref, t))
    big = np.abs(g) > 0.2 * np.abs(g).max()
    assert big.sum() > 10
    assert np.allclose(d[big], -lr * np.sign(g[big]), rtol=3e-4, atol=0)   # FP32 rounding of w - lr


def _pairs(s, wl, nsteps, dt):
    """Normalised (input, target) pairs from the last pressure solve of each step."""
    X, T = [], []
    for _ in range(nsteps):
        s.step(dt, 1)
        f, p = s.last_pressure()
        x, t = inputs.unet_pair(f, p, s.get_fields()[0], wl.rho1, wl.rho2, wl.h)
        X.append(x)
        T.append(t)
    return X, T


def test_training_and_warm_start_on_3d_drop():
    """Train (1600 Adam steps) on the pressure solves of the first 40 steps of
    a 32^3 drop, then continue the run with the network as the first guess:
    every solve still reaches the 1e-8 tolerance, the state agrees with a
    zero-start run to the solver tolerance, and the solves need fewer V-cycles
    than from zero (6 against 8 per solve when this was written; the previous
    step's pressure needs about 4)."""
    n = 32
    wl = inputs.drop_3d(n)
    dt = inputs.stable_dt(wl)
    s = cdi.from_workload(wl, tol=1e-8)
    X, T = _pairs(s, wl, 40, dt)
    phi, vel, _ = s.get_fields()

    net = cdi.Unet((n, n, n))
    net.set_params(inputs.unet_initial_params(0))
    losses = []
    for it in range(1600):
        i = it % len(X)
        losses.append(net.train_step(X[i], T[i], lr=1e-3 if it < 1000 else 3e-4))
    first, last = np.mean(losses[:40]), np.mean(losses[-40:])
    print("training loss %.3e -> %.3e" % (first, last))
    assert np.isfinite(last) and last < 0.2 * first

    def run(warm):
        r = cdi.from_workload(wl, tol=1e-8)
        r.set_exec(cdi.EXEC_KERNELS)
        r.set_solver(1e-8, 100, warm)
        if warm == cdi.WARM_UNET:
            r.set_warm_unet(net)
        r.set_state(phi, vel)
        cyc = 0
        for _ in range(8):
            r.step(dt, 1)
            st = r.last_stats()
            assert st["resid"] <= 1e-8
            cyc += st["total_cycles_call"]
        return cyc, r.get_fields()

    c_zero, f_zero = run(cdi.WARM_ZERO)
    c_unet, f_unet = run(cdi.WARM_UNET)
    c_prev, _ = run(cdi.WARM_PREV)
    print("V-cycles over 8 steps: zero %d, network %d, previous %d" % (c_zero, c_unet, c_prev))
    assert c_unet < c_zero
    umax = max(np.abs(f_zero[1][a]).max() for a in range(3))
    for a in range(3):
        assert np.abs(f_unet[1][a] - f_zero[1][a]).max() <= 1e-5 * umax
    assert np.abs(f_unet[0] - f_zero[0]).max() <= 1e-8


def test_warm_unet_needs_a_network():
    wl = inputs.drop_3d(16)
    s = cdi.from_workload(wl, tol=1e-8)
    s.set_solver(1e-8, 100, cdi.WARM_UNET)
    with pytest.raises(cdi.CdiError) as e:
        s.step(1e-5, 1)
    assert e.value.status == 2


@pytest.mark.parametrize("n", [(8, 8, 8), (24, 40, 16)], ids=["8^3", "24x40x16"])
def test_tensor_core_and_warp_mma_convolutions_agree(n):
    """The tcgen05 convolution (default) and the mma.sync one compute the same
    FP32 sums over the same BF16 operands: forward outputs and gradients agree
    to accumulation-order round-off (relative 1e-3; ReLU masks can flip where a
    BF16 rounding tie breaks differently)."""
    shape = (n[2], n[1], n[0])
    P, x, t = random_case(shape, 21)
    nets = []
    for tc in (True, False):
        net = cdi.Unet(n)
        net.set_conv_kernel(tc)
        net.set_params(flat(P))
        nets.append(net)
    y_tc, y_mma = nets[0].forward(x), nets[1].forward(x)
    assert relnorm(y_tc, y_mma) < 1e-3
    _, g_tc = nets[0].train_step(x, t[..., 0], lr=0.0, want_grads=True)
    _, g_mma = nets[1].train_step(x, t[..., 0], lr=0.0, want_grads=True)
    assert relnorm(g_tc, g_mma) < 1e-2


@pytest.mark.parametrize("n", [(16, 8, 8), (24, 40, 16)], ids=["16x8x8", "24x40x16"])
def test_tcgen05_weight_gradients_match_mma_sync(n):
    """The same forward pass (tcgen05 convolutions) with the weight and bias
    gradients of every layer from the tcgen05 voxel-reduction GEMM (row of
    ones for the bias, fixed-order split sums) or from the mma.sync kernel
    with FP32 atomics: both sum the same BF16 products in FP32, so every
    entry agrees to accumulation-order round-off, 1e-4 of the layer's
    largest entry.  The 24x40x16 grid's coarse levels (3x5x2 voxels at the
    bottleneck) have extents that are not multiples of 8."""
    shape = (n[2], n[1], n[0])
    P, x, t = random_case(shape, 5)
    grads = []
    for mode in (1, 2):
        net = cdi.Unet(n)
        net.set_conv_kernel(mode)
        net.set_params(flat(P))
        _, g = net.train_step(x, t[..., 0], lr=0.0, want_grads=True)
        grads.append(unflat(g))
    g_tc, g_mma = grads
    for name, _, _, _ in ref.LAYERS:
        for part in (".w", ".b"):
            a, b = g_tc[name + part], g_mma[name + part]
            m = np.abs(a - b).max() / np.abs(b).max()
            print("%-7s max diff / max %.3e" % (name + part, m))
            assert m < 1e-4, (name + part, m)


def test_fused_decoder_inputs_match_stored_ones():
    """Inference gathers the decoder inputs [up(coarser), skip] while staging
    the convolution tiles; training stores them.  Both feed the same BF16
    values to the same MMAs, so the outputs are identical."""
    torch = pytest.importorskip("torch")
    n = (16, 24, 16)
    shape = (n[2], n[1], n[0])
    P, x, t = random_case(shape, 31)
    net = cdi.Unet(n)
    net.set_params(flat(P))
    y_host = net.forward(x)                       # fused gather
    xd = torch.tensor(x.reshape(-1), dtype=torch.float32, device="cuda")
    yd = torch.empty(x.size // 2, dtype=torch.float32, device="cuda")
    net.forward_device(xd, yd)                    # fused gather, FP32 input
    torch.cuda.synchronize()
    y_ref, _ = ref.forward(as_stored(P), x, store=ref.bf16_round)
    assert relnorm(yd.cpu().numpy().reshape(shape), y_ref[..., 0]) < 2e-3
    loss, _ = net.train_step(x, t[..., 0], lr=0.0, want_grads=True)   # stored concatenations
    assert abs(loss - float(np.mean((y_host - t[..., 0]) ** 2))) <= 1e-6 * loss
