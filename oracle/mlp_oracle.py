"""TEST INFRASTRUCTURE ONLY: plain FP64 NumPy reference of the learned
controller's network (MLP 16 -> 64 -> 64 -> 2 with GELU hidden layers), its
weighted squared-error loss, the backward pass written out by the chain rule,
and one Adam step (Kingma & Ba, bias-corrected).  Used by the tests to check
the CUDA kernels; the product path never imports it.

Parameter layout (flat, row-major out x in): W1[64][16], b1[64], W2[64][64],
b2[64], W3[2][64], b3[2].  GELU(z) = z * Phi(z) with the standard normal CDF
Phi(z) = (1 + erf(z / sqrt 2)) / 2 (scipy's erf as the library primitive).
"""
import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 16, 64, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_prime(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(theta, X):
    """Y[B][2] and the intermediate values of every sample."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}


def wmse(Y, T, w=None):
    """L = sum_s w_s |y_s - t_s|^2 / sum_s w_s and dL/dY."""
    Y = np.asarray(Y, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    w = np.ones(Y.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    sw = w.sum() if w.sum() > 0 else 1.0
    E = Y - T
    return float((w[:, None] * E * E).sum() / sw), 2.0 * w[:, None] * E / sw


def backward(theta, cache, dY):
    """dL/dtheta (flat) for the given dL/dY, by the chain rule layer by layer."""
    p = unpack(theta)
    dY = np.asarray(dY, dtype=np.float64)
    g = {"W3": dY.T @ cache["H2"], "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * gelu_prime(cache["Z2"])
    g["W2"] = dZ2.T @ cache["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_prime(cache["Z1"])
    g["W1"] = dZ1.T @ cache["X"]
    g["b1"] = dZ1.sum(axis=0)
    return pack(g)


def loss_of(theta, X, T, w=None):
    return wmse(forward(theta, X)[0], T, w)[0]


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam step; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
