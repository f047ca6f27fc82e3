"""Reference Hilbert order of points in a periodic box (test infrastructure):
a plain restatement of Skilling's transpose form of the 3-D Hilbert index
(J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707, 381 (2004))
on cells floor(1024 frac(x / box)), sorted with ties by point index."""
import numpy as np

BITS = 10


def hilbert_keys_ref(xyz: np.ndarray, box: float) -> np.ndarray:
    """Skilling's transpose form of the 3-D Hilbert index, then bit interleaving
    from the most significant bit, axis 0 first; cells floor(1024 frac(x/box))."""
    u = xyz / box
    u = u - np.floor(u)
    X = np.minimum(np.maximum((u * (1 << BITS)).astype(np.int64), 0), (1 << BITS) - 1).T.copy()
    M = 1 << (BITS - 1)
    Q = M
    while Q > 1:
        P = Q - 1
        for i in range(3):
            # bit Q of axis i set: invert the low bits of axis 0; else exchange
            # the low bits of axes 0 and i
            hit = (X[i] & Q) != 0
            t = (X[0] ^ X[i]) & P
            x0 = np.where(hit, X[0] ^ P, X[0] ^ t)
            if i != 0:
                X[i] = np.where(hit, X[i], X[i] ^ t)
            X[0] = x0
        Q >>= 1
    X[1] ^= X[0]
    X[2] ^= X[1]
    t = np.zeros_like(X[0])
    Q = M
    while Q > 1:
        t = np.where((X[2] & Q) != 0, t ^ (Q - 1), t)
        Q >>= 1
    for i in range(3):
        X[i] ^= t
    key = np.zeros(xyz.shape[0], dtype=np.int64)
    for b in range(BITS - 1, -1, -1):
        for i in range(3):
            key = (key << 1) | ((X[i] >> b) & 1)
    return key


def order_ref(xyz: np.ndarray, box: float) -> np.ndarray:
    key = hilbert_keys_ref(xyz, box)
    return np.lexsort((np.arange(len(key)), key))
