"""POD basis and the small MLP of the learned warm start (oracle, FP64, test infrastructure).

Not part of the paper: the warm start supplies the initial guess of each new frequency solve
from solutions the method has already computed (the adaptive sampling of Sec. 3 solves one new
frequency at a time).  Definitions written out plainly:

* POD: the r leading left singular vectors Phi (N x r) of the snapshot matrix X = [x(s_1) ..
  x(s_J)] (library SVD); r is the smallest rank whose discarded energy sum_{k>r} sigma_k^2 is at
  most energy_tol * sum_k sigma_k^2 (at most r_max); coefficients c_j = Phi^H x(s_j).
* Targets: the network predicts only the direction of the coefficient vector: c_j / |c_j| turned
  by the phase that makes its first (leading-mode) entry real and non-negative, as
  [Re, Im] pairs.  Magnitude and phase are fixed at solve time (below).
* MLP: u = (Re s / Omega, Im s / Omega) -> h1 = g(W1 u + b1) -> h2 = g(W2 h1 + b2)
  -> y = W3 h2 + b3 (y = [Re c, Im c] / scale), widths 2 -> 128 -> 128 -> 2r, with the tanh form
  of GELU, g(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks and Gimpel).
* Loss: L = (1 / (2 B)) sum_batch |y - y_target|^2; gradients by the chain rule.
* Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
* Warm start: the direction x^(s) = Phi c(s), c from the network output (or the stored solution
  at the nearest stored frequency), scaled by the complex alpha that minimises |b - alpha A x^|:
  alpha = (A x^)^H b / |A x^|^2 (a one-dimensional least-squares problem), x0 = alpha x^.
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)


def pod(X, r_max=32, energy_tol=1e-10):
    """X: (N, J) complex snapshots -> Phi (N, r)."""
    U, S, _ = np.linalg.svd(X, full_matrices=False)
    e = S ** 2
    tail = np.concatenate([np.cumsum(e[::-1])[::-1][1:], [0.0]])   # sum_{k > r} sigma_k^2
    r = int(np.argmax(tail <= energy_tol * e.sum())) + 1
    return U[:, :min(r, r_max)]


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * x * x)


def init_params(n_out, hidden=128, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and zero biases (seeded)."""
    rng = np.random.default_rng(seed)

    def lin(fi, fo):
        a = 1.0 / math.sqrt(fi)
        return rng.uniform(-a, a, size=(fo, fi)), np.zeros(fo)

    W1, b1 = lin(2, hidden)
    W2, b2 = lin(hidden, hidden)
    W3, b3 = lin(hidden, n_out)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def forward(p, U):
    """U: (B, 2) inputs -> outputs (B, n_out) and the cache for backward."""
    z1 = U @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (U, z1, h1, z2, h2)


def loss_and_grads(p, U, Y):
    y, (U, z1, h1, z2, h2) = forward(p, U)
    B = U.shape[0]
    d = (y - Y) / B
    loss = 0.5 * np.sum((y - Y) ** 2) / B
    g = {}
    g["W3"] = d.T @ h2
    g["b3"] = d.sum(axis=0)
    dh2 = d @ p["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ U
    g["b1"] = dz1.sum(axis=0)
    return loss, g


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * grads[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * grads[k] ** 2
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)


def features(s, omega):
    s = np.asarray(s)
    return np.stack([s.real / omega, s.imag / omega], axis=1)


def targets(Phi, X):
    """[Re c~, Im c~] per snapshot column of X, c~ = c / |c| * conj(c_1) / |c_1|, c = Phi^H x."""
    C = Phi.conj().T @ X                     # (r, J)
    nrm = np.linalg.norm(C, axis=0)
    nrm = np.where(nrm > 0, nrm, 1.0)
    ph = np.where(np.abs(C[0]) > 0, np.conj(C[0]) / np.where(np.abs(C[0]) > 0, np.abs(C[0]), 1.0), 1.0)
    C = C / nrm * ph
    return np.concatenate([C.real, C.imag], axis=0).T


def direction(p, Phi, s, omega):
    """Predicted warm-start directions Phi c(s), (len(s), N)."""
    y, _ = forward(p, features(s, omega))
    r = Phi.shape[1]
    return (y[:, :r] + 1j * y[:, r:]) @ Phi.T


def min_residual_scale(A, b, xh):
    """x0 = alpha xh with alpha = (A xh)^H b / |A xh|^2 (alpha = 0 when A xh = 0)."""
    y = A @ xh
    d = np.vdot(y, y).real
    return (np.vdot(y, b) / d if d > 0 else 0.0) * xh
