"""CPU oracle for the block router's MLP (test infrastructure only).

The router is a 16-32-32-1 perceptron with tanh hidden units that maps the
standardised features of a quartet tile to a predicted log10 magnitude of
its largest gradient contribution.  Training minimises the expectile loss
  L = mean_s w_s r_s^2,  r_s = y_s - yhat_s,  w_s = q if r_s > 0 else 1 - q,
which for q > 1/2 biases predictions upward (under-prediction is the costly
error when routing to fp32).  This module writes forward and backward out in
fp64 numpy with the textbook chain rule, so the GPU kernels' gradients can be
compared with it.  Parameter layout (flat, fp32 on the device):
W1[32][16], b1[32], W2[32][32], b2[32], w3[32], b3.
"""
import numpy as np

NIN, NH = 16, 32
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(theta):
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = t[o:o + NH]; o += NH
    W2 = t[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = t[o:o + NH]; o += NH
    w3 = t[o:o + NH]; o += NH
    b3 = t[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, X):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, (X, h1, h2)


def loss_and_grad(theta, X, y, q):
    """Expectile loss and its gradient with respect to theta (fp64)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    yhat, (X, h1, h2) = forward(theta, X)
    r = np.asarray(y, dtype=np.float64) - yhat
    w = np.where(r > 0, q, 1.0 - q)
    n = len(r)
    L = float(np.sum(w * r * r) / n)
    dy = -2.0 * w * r / n                      # dL/dyhat
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    da2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(0)
    da1 = (da2 @ W2) * (1.0 - h1 * h1)
    gW1 = da1.T @ X
    gb1 = da1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return L, g
