"""Rank-prediction MLP: plain NumPy FP64 reference of the learned-rank form.

Not in the paper: the paper grows the sample width adaptively (Theorem 1
needs k + p samples).  The learned form predicts each front's largest HSS
rank before sampling, from six features of the front, and starts the
adaptive loop at the predicted width.  This file is the definition the GPU
kernels are checked against:

  features x (6): log(1 + |B|), tree level, kappa * h, p, mean and variance of
                  c over the box's elements
  standardisation: xh = (x - mu) / sd per feature, th = (t - tmu) / tsd, with
                  mu, sd, tmu, tsd the mean and population standard deviation
                  of the training data (sd = 1 where it is zero)
  network:        h1 = relu(W1 xh + b1), h2 = relu(W2 h1 + b2),
                  h3 = relu(W3 h2 + b3), y = W4 h3 + b4  (64 hidden units)
  loss:           mean over samples of (y - th)^2
  target:         t = log(1 + k), k the front's largest node rank
  Adam:           m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
                  w -= lr * (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps)

Parameter vector layout (8,833 values): W1 (64 x 6, row j = unit j), b1 (64),
W2 (64 x 64), b2 (64), W3 (64 x 64), b3 (64), W4 (64), b4 (1).

THIS FILE IS TEST INFRASTRUCTURE (see the package docstring).
"""
import numpy as np

NF, NH = 6, 64
SHAPES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NH,)), ("b4", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def standardisation(X, t):
    """Mean and population standard deviation of the features and targets."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    tmu = t.mean()
    tsd = t.std() if t.std() > 0 else 1.0
    return mu, sd, tmu, tsd


def forward(theta, X, norm):
    """Network output y (standardised target units) and the activations."""
    P = unpack(theta)
    mu, sd = norm[0], norm[1]
    Xh = (np.asarray(X, dtype=np.float64) - mu) / sd
    z1 = Xh @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ P["W4"] + P["b4"][0]
    return y, dict(Xh=Xh, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss_grad(theta, X, t, norm):
    """Mean squared error against the standardised targets and its gradient
    with respect to the parameter vector (backpropagation by the chain rule)."""
    P = unpack(theta)
    tmu, tsd = norm[2], norm[3]
    th = (np.asarray(t, dtype=np.float64) - tmu) / tsd
    y, a = forward(theta, X, norm)
    n = y.shape[0]
    r = y - th
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["W4"] = a["h3"].T @ dy
    g["b4"] = np.array([dy.sum()])
    d3 = np.outer(dy, P["W4"]) * (a["z3"] > 0)
    g["W3"] = d3.T @ a["h2"]
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ P["W3"]) * (a["z2"] > 0)
    g["W2"] = d2.T @ a["h1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (a["z1"] > 0)
    g["W1"] = d1.T @ a["Xh"]
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns theta, m, v."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round to the nearest bfloat16 (8-bit significand), ties to even,
    returned as float64: the float32 bit pattern with the low 16 bits rounded
    off."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X, norm):
    """The network with weights, standardised features and activations
    rounded to bfloat16 (inference form); sums in FP64.  Returns log(1 + k)."""
    P = {k: bf16_round(v) for k, v in unpack(theta).items()}
    mu, sd = np.asarray(norm[0], dtype=np.float32), np.asarray(norm[1], dtype=np.float32)
    Xh = bf16_round((np.asarray(X, dtype=np.float32) - mu) / sd)
    h1 = bf16_round(np.maximum(Xh @ P["W1"].T + P["b1"], 0.0))
    h2 = bf16_round(np.maximum(h1 @ P["W2"].T + P["b2"], 0.0))
    h3 = bf16_round(np.maximum(h2 @ P["W3"].T + P["b3"], 0.0))
    y = h3 @ P["W4"] + P["b4"][0]
    return norm[2] + norm[3] * y


def predicted_rank(theta, X, norm):
    """k = exp(tmu + tsd * y) - 1, the predicted largest rank (real-valued)."""
    y, _ = forward(theta, X, norm)
    return np.expm1(norm[2] + norm[3] * y)
