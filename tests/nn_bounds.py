"""Rounding-error bounds of the neural decoder variants, shared by the oracle pins and the GPU tests."""
import numpy as np

import oracle as O


def e4m3_first_order_bound(lat, R, P, idx, e):
    """First-order bound on |E4M3 decode - FP64 decode| per output: u = 2^-4 relative per E4M3
    rounding (plus half a subnormal step, 2^-10, in the scaled units), 2^-9 relative for the FP16
    stages of layer 1, propagated through |W| with the FP64 activations."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(a, np.float64) for a in O.nn_split(np.asarray(P, np.float64))]
    W1, W2, W3 = W1.reshape(64, 24), W2.reshape(64, 64), W3.reshape(8, 64)
    s1, s2, s3 = 2.0 ** e[0], 2.0 ** e[1], 2.0 ** e[2]
    u, sub = 2.0 ** -4, 2.0 ** -10
    out = []
    for t in idx:
        x = O.nn_features(lat, R, int(t) & 0xffff, int(t) >> 16)
        z1 = W1 @ x + b1
        h1 = np.maximum(z1, 0)
        h2 = np.maximum(W2 @ h1 + b2, 0)
        e1 = u * h1 + sub / s1 + 2.0 ** -9 * (np.abs(W1) @ np.abs(x) + np.abs(b1))
        e2 = (np.abs(W2) @ e1 + (u * np.abs(W2) + sub / s2) @ h1 + u ** 3 * np.abs(b2)) * (1 + u) + u * h2 + sub / (s1 * s2)
        out.append(np.abs(W3) @ e2 + (u * np.abs(W3) + sub / s3) @ h2 + u ** 3 * np.abs(b3))
    return np.array(out)
