"""Pins of the FP64 oracle of the learned mu proposal network (no GPU)."""
import numpy as np

from oracle import mlp


def _theta(seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=mlp.N_PARAMS) * 0.2


def test_param_layout():
    assert mlp.N_PARAMS == 21378
    p = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=float))
    assert p["W1"].shape == (128, 35) and p["b3"].shape == (2,)
    assert p["W1"][0, 1] == 1 and p["b1"][0] == 128 * 35


def test_forward_hand_example():
    # one active path: x0 -> hidden unit 0 -> hidden unit 0 -> outputs
    th = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(th)
    p["W1"][0, 0] = 2.0
    p["b1"][0] = -1.0
    p["W2"][0, 0] = 3.0
    p["W3"][0, 0] = 0.5
    p["W3"][1, 0] = -1.0
    p["b3"][:] = [0.25, 0.125]
    X = np.zeros((2, 35))
    X[0, 0], X[1, 0] = 1.5, 0.2  # second sample: 2*0.2-1 < 0 -> ReLU cuts it
    out, _ = mlp.forward(th, X)
    assert np.allclose(out[0], [0.5 * 3 * 2.0 + 0.25, -3 * 2.0 + 0.125])
    assert np.allclose(out[1], [0.25, 0.125])


def test_loss_pieces():
    out = np.array([[0.3, np.log(0.5)], [2.0, np.log(0.1)]])
    L, _ = mlp.loss_and_dout(out, np.array([0.1, 0.0]), np.array([1.0, 1.0]))
    # sample 0: d = 0.2 (quadratic), w = 0.5, covered: 0.02 + 0.005
    # sample 1: d = 2 (linear), w = 0.1, missed: 1.5 + 1.9 + 0.001
    assert abs(L - ((0.02 + 0.005) + (1.5 + 1.9 + 0.001)) / 2) < 1e-12


def test_backward_matches_central_differences():
    th = _theta(1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(6, 35))
    xs = rng.normal(size=6) * 0.3
    sc = rng.uniform(0.5, 2.0, size=6)

    def L(t):
        o, _ = mlp.forward(t, X)
        return mlp.loss_and_dout(o, xs, sc)[0]

    out, cache = mlp.forward(th, X)
    _, dout = mlp.loss_and_dout(out, xs, sc)
    g = mlp.backward(th, cache, dout)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2, 0]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (L(th + e) - L(th - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_is_signed_lr():
    th = _theta(3)
    g = np.random.default_rng(4).normal(size=th.shape)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t1, m1, v1 = mlp.adam_step(th, g, m, v, 1, lr=1e-3)
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_features():
    f = mlp.features(np.arange(40.0), 10, -8.0, 9.0, 5.0)
    assert f.shape == (35,) and f[31] == 3.1 and f[32] == -0.8 and f[33] == 0.9 and f[34] == 0.5


def test_splitmix64_published_sequence():
    # the first three outputs of SplitMix64 from state 0 (state advances by the
    # golden-ratio increment each call)
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        states = np.array([0, g, g + g], dtype=np.uint64)
    out = [int(v) for v in mlp.splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_xavier_init_range_and_variance():
    th = mlp.xavier_init(3).astype(np.float64)
    p = mlp.unpack(th)
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        W = p[w]
        a = np.sqrt(6.0 / (W.shape[0] + W.shape[1]))
        assert np.all(p[b] == 0.0) and np.all(np.abs(W) < a)
        # U(-a, a): mean 0, variance a^2/3 = 2/(fan_in + fan_out)
        n = W.size
        assert abs(W.mean()) < 4 * a / np.sqrt(3 * n)
        assert abs(W.var() / (a * a / 3) - 1) < 4 * np.sqrt(0.8 / n)
    assert not np.array_equal(th, mlp.xavier_init(4))
    assert np.array_equal(th, mlp.xavier_init(3).astype(np.float64))
