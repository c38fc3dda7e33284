"""Line-local MLP Newton predictor (oracle; test infrastructure).

Not in the paper. For every line of reference direction 1 (each node lies
on exactly one) the features are the nodal states of three time levels
and nine metric terms; a 69 -> 128 -> 128 -> 128 -> 20 MLP with GELU
predicts the line's correction to the linear extrapolation 2 U^n - U^{n-1}
of the next level.

Feature order (69 = 3 * (p+1) * n_c + 9 for p = 3, n_c = 5):
  [ u^n, u^n - u^{n-1}, u^{n-1} - u^{n-2} ]  each over the line's nodes t
  (outer) and components c (inner), i.e. index (level (p+1) + t) n_c + c;
  then the 3x3 deformation gradient G = dx/dX averaged over the line's
  nodes and divided by h = J^{1/D} averaged likewise, row-major.
The differences are a linear re-parametrisation of [u^n, u^{n-1}, u^{n-2}].
Inputs are standardised with per-feature (mean, std); outputs are the
correction divided by a per-component scale.

Parameters in one flat FP64 vector, in this order: W1 [in][128], b1 [128],
W2 [128][128], b2, W3 [128][128], b3, W4 [128][out], b4 [out].
GELU is the tanh form of Hendrycks and Gimpel:
  gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
The loss is the mean of squared errors over all outputs of the batch.
Adam follows Kingma and Ba with bias correction.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 128
C_GELU = math.sqrt(2.0 / math.pi)


def layer_shapes(n_in, n_out, hidden=HIDDEN):
    return [(n_in, hidden), (hidden, hidden), (hidden, hidden), (hidden, n_out)]


def n_params(n_in, n_out, hidden=HIDDEN):
    return sum(a * b + b for a, b in layer_shapes(n_in, n_out, hidden))


def unpack(theta, n_in, n_out, hidden=HIDDEN):
    out, o = [], 0
    for a, b in layer_shapes(n_in, n_out, hidden):
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bb = theta[o:o + b]
        o += b
        out.append((W, bb))
    return out


def init_params(n_in, n_out, seed=0, hidden=HIDDEN):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; the
    last layer scaled by 0.1 so the initial correction is small."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = layer_shapes(n_in, n_out, hidden)
    for li, (a, b) in enumerate(shapes):
        lim = 1.0 / math.sqrt(a)
        W = rng.uniform(-lim, lim, size=(a, b))
        if li == len(shapes) - 1:
            W *= 0.1
        parts += [W.ravel(), np.zeros(b)]
    return np.concatenate(parts)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + 0.044715 * x ** 3)))


def gelu_prime(x):
    t = np.tanh(C_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * x * x)


def forward(theta, X, n_out, hidden=HIDDEN):
    """Y = MLP(X); returns Y and the pre-activations for the backward pass."""
    layers = unpack(theta, X.shape[1], n_out, hidden)
    h = X
    zs, hs = [], [X]
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        zs.append(z)
        if li < len(layers) - 1:
            h = gelu(z)
            hs.append(h)
        else:
            h = z
    return h, (zs, hs)


def loss_and_grad(theta, X, T, hidden=HIDDEN):
    """Mean squared error over all outputs and its gradient (backprop)."""
    n_out = T.shape[1]
    Y, (zs, hs) = forward(theta, X, n_out, hidden)
    M = X.shape[0]
    loss = np.mean((Y - T) ** 2)
    layers = unpack(theta, X.shape[1], n_out, hidden)
    g = 2.0 * (Y - T) / (M * n_out)
    grads = [None] * len(layers)
    for li in reversed(range(len(layers))):
        W, _ = layers[li]
        gW = hs[li].T @ g
        gb = g.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            g = (g @ W.T) * gelu_prime(zs[li - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_update(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# line features
# ---------------------------------------------------------------------------
def line_metric_features(mesh, rules):
    """Per direction-1 line: G (3x3, row-major) averaged over the line's nodes
    divided by h = mean of J^{1/D} over the same nodes. [E * nl, D*D]."""
    from .mesh import from_lines, to_lines
    D, p = mesh["D"], mesh["p"]
    X = mesh["nodes"]
    E = X.shape[0]
    Gn = np.zeros((E, (p + 1) ** D, D, D))
    for b in range(D):
        for a in range(D):
            dl = np.einsum("ij,elj->eli", rules.Dn, to_lines(X[..., a], D, p, b))
            Gn[:, :, a, b] = from_lines(dl, D, p, b)
    J = np.linalg.det(Gn)
    h = J ** (1.0 / D)
    Gl = np.stack([to_lines(Gn[..., a, b], D, p, 0) for a in range(D) for b in range(D)], axis=-1)
    hl = to_lines(h, D, p, 0)                        # [E, nl, p+1]
    feats = Gl.mean(axis=2) / hl.mean(axis=2)[..., None]
    return feats.reshape(E * (p + 1) ** (D - 1), D * D)


def line_state_features(Un, Unm1, Unm2, D, p):
    """[u^n, u^n - u^{n-1}, u^{n-1} - u^{n-2}] per direction-1 line, feature
    index (level (p+1) + t) n_c + c. [E * nl, 3 (p+1) n_c]."""
    from .mesh import to_lines
    E, nc, _ = Un.shape
    levels = [Un, Un - Unm1, Unm1 - Unm2]
    out = []
    for A in levels:
        L = to_lines(A, D, p, 0)                      # [E, nc, nl, p+1]
        L = np.transpose(L, (0, 2, 3, 1))             # [E, nl, p+1, nc]
        out.append(L.reshape(E * L.shape[1], (p + 1) * nc))
    return np.concatenate(out, axis=1)


def line_targets(Unext, Un, Unm1, D, p):
    """Correction to linear extrapolation per direction-1 line, [E*nl, (p+1) n_c]."""
    from .mesh import to_lines
    C = Unext - (2.0 * Un - Unm1)
    L = np.transpose(to_lines(C, D, p, 0), (0, 2, 3, 1))
    return L.reshape(L.shape[0] * L.shape[1], -1)


def scatter_correction(Yc, Un, Unm1, D, p):
    """U0 = 2 U^n - U^{n-1} + correction scattered back to the nodes."""
    from .mesh import from_lines
    E, nc, _ = Un.shape
    nl = (p + 1) ** (D - 1)
    C = Yc.reshape(E, nl, p + 1, nc).transpose(0, 3, 1, 2)   # [E, nc, nl, p+1]
    return 2.0 * Un - Unm1 + from_lines(C, D, p, 0)
