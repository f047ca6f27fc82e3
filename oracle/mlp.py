"""FP64 oracle of the learned mu proposal network -- TEST INFRASTRUCTURE ONLY.

Not in the paper: a small multilayer perceptron maps low-order Chebyshev moments
of the scaled Hamiltonian, its spectral bounds and the filling N_e/N to a guess
of the scaled Fermi level and a log half-width of a bracket around it, so that
the plain bisection (Sec. "Fermi Operator Expansion") can be judged on one
expansion carrying 4 mu accumulators instead of two expansions.

Architecture: 35 -> 128 -> 128 -> 2, ReLU after the two hidden layers.
Parameters are one flat vector in the order W1[128,35], b1[128], W2[128,128],
b2[128], W3[2,128], b3[2] (row-major weights, y = W x + b).

Loss per sample, with d = (xhat - xstar)/s, w = exp(z)/s, s = sigma*kT (the
target's scale in units of the smearing):
    L = huber(d) + relu(|d| - w) + 0.01 * w
(huber with delta 1: d^2/2 for |d| <= 1, |d| - 1/2 otherwise).  The batch loss
is the mean.  Adam: lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.
"""

from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 35, 128, 2
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state x (Steele, Lea and Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014): add the golden-ratio
    increment, then two xor-shift-multiply rounds and a final xor-shift."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def xavier_init(seed: int) -> np.ndarray:
    """Xavier-uniform weights W ~ U(-a, a), a = sqrt(6 / (fan_in + fan_out)),
    zero biases, as FP32.  Parameter i draws u = (top 24 bits of
    splitmix64((seed * 0xD1B54A32D192ED03) xor i) + 1/2) / 2^24 and takes
    a (2u - 1) in float64, rounded once to float32."""
    i = np.arange(N_PARAMS, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0xD1B54A32D192ED03)) ^ i
    u = ((splitmix64(ctr) >> np.uint64(40)).astype(np.float64) + 0.5) / 16777216.0
    theta = np.zeros(N_PARAMS, dtype=np.float64)
    o = 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        if name.startswith("W"):
            a = np.sqrt(6.0 / (shp[0] + shp[1]))
            theta[o:o + n] = a * (2.0 * u[o:o + n] - 1.0)
        o += n
    return theta.astype(np.float32)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns (out [B,2], cache) with cache = (X, a1, h1, a2, h2)."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (X, a1, h1, a2, h2)


def loss_and_dout(out: np.ndarray, xstar: np.ndarray, scale: np.ndarray):
    """Mean loss over the batch and dL/dout [B,2]."""
    B = out.shape[0]
    d = (out[:, 0] - xstar) / scale
    w = np.exp(out[:, 1]) / scale
    ad = np.abs(d)
    hub = np.where(ad <= 1.0, 0.5 * d * d, ad - 0.5)
    miss = ad > w
    L = hub + np.where(miss, ad - w, 0.0) + 0.01 * w
    dhub = np.where(ad <= 1.0, d, np.sign(d))
    dd = dhub + np.where(miss, np.sign(d), 0.0)
    dout = np.zeros_like(out)
    dout[:, 0] = dd / scale / B
    dout[:, 1] = (np.where(miss, -1.0, 0.0) + 0.01) * w / B
    return float(L.mean()), dout


def backward(theta: np.ndarray, cache, dout: np.ndarray) -> np.ndarray:
    """Gradient of sum(dout * out) with respect to theta (flat)."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    X, a1, h1, a2, h2 = cache
    g = {}
    g["W3"] = dout.T @ h2
    g["b3"] = dout.sum(axis=0)
    dh2 = dout @ p["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])


def adam_step(theta, grad, m, v, t: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(t_moments: np.ndarray, n_rows: int, emin: float, emax: float, N_e: float) -> np.ndarray:
    """The 35 inputs: Tr T_k / N for k < 32, emin/10, emax/10 (Ha), N_e/N."""
    f = np.zeros(N_IN)
    f[:32] = np.asarray(t_moments[:32], dtype=np.float64) / n_rows
    f[32] = emin / 10.0
    f[33] = emax / 10.0
    f[34] = N_e / n_rows
    return f
