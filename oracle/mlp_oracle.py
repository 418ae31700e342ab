"""FP64 reference of the troubled-cell flag network -- TEST INFRASTRUCTURE ONLY.

A plain numpy restatement of the network the library trains and runs in FP32 CUDA kernels:
in (22) -> 32 (ReLU) -> 32 (ReLU) -> 1 (sigmoid), parameters packed as
W1[32][22], b1[32], W2[32][32], b2[32], w3[32], b3 (1825 floats), and its training loss, the
binary cross-entropy with a positive-class weight pw averaged over the batch:
    L = mean( -pw y log(sig(z)) - (1 - y) log(1 - sig(z)) ).
Gradients are written out by the chain rule; tests pin them with finite differences.  Used only
by tests (gradient check of the CUDA kernels) -- the library never imports it.
"""
import numpy as np

NIN, NH = 22, 32
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init(seed):
    """He-style initialisation (the same recipe the training driver uses)."""
    rng = np.random.default_rng(seed)
    return pack({"W1": rng.normal(0, np.sqrt(2 / NIN), (NH, NIN)), "b1": np.zeros(NH),
                 "W2": rng.normal(0, np.sqrt(2 / NH), (NH, NH)), "b2": np.zeros(NH),
                 "w3": rng.normal(0, np.sqrt(1 / NH), NH), "b3": np.zeros(1)})


def forward(theta, X):
    p = unpack(np.asarray(theta, dtype=np.float64))
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    return z1, h1, z2, h2, z3


def prob(theta, X):
    return 1.0 / (1.0 + np.exp(-forward(theta, X)[-1]))


def loss(theta, X, y, pw):
    z3 = forward(theta, X)[-1]
    # log(sig(z)) = -log1p(exp(-z)), log(1 - sig(z)) = -z - log1p(exp(-z)), written stably
    lsig = -np.logaddexp(0.0, -z3)
    l1sig = -np.logaddexp(0.0, z3)
    return float(np.mean(-pw * y * lsig - (1.0 - y) * l1sig))


def grad(theta, X, y, pw):
    p = unpack(np.asarray(theta, dtype=np.float64))
    z1, h1, z2, h2, z3 = forward(theta, X)
    n = X.shape[0]
    s = 1.0 / (1.0 + np.exp(-z3))
    dz3 = (-pw * y * (1.0 - s) + (1.0 - y) * s) / n      # dL/dz3 per sample
    g = {"w3": h2.T @ dz3, "b3": np.array([dz3.sum()])}
    dh2 = np.outer(dz3, p["w3"]) * (z2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = dh1.T @ X, dh1.sum(axis=0)
    return pack(g)


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, bias-corrected), step counted from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
