"""Exact references for the tests, independent of the oracle and of the CUDA path.

* :func:`phi` — phi_k(z) of eq 3 by its Taylor series (|z| < 1) or the recurrence
  phi_k(z) = (phi_{k-1}(z) - 1/(k-1)!) / z (|z| >= 1), itself pinned to quadrature of eq 3.
* :func:`augmented` — the matrix A~ and vector v of Theorem 1 (eq 13), built from its definition.
* :func:`exact_dense` — top N entries of scipy.linalg.expm(tau A~) v (Theorem 1, eq 14).
* :func:`exact_dst_1d` / :func:`exact_dst_2d` / :func:`exact_dst_3d` — closed forms for Dirichlet Laplacians
  (+ constant shift)
  through the orthonormal DST-I eigenbasis, w = sum_k S diag(tau^k phi_k(tau lambda)) S^T b_k.
"""
from math import factorial

import numpy as np
import scipy.fft
import scipy.linalg


def phi(k: int, z):
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    s = np.zeros_like(zs)
    term = np.full_like(zs, 1.0 / factorial(k))
    for i in range(60):
        s += term
        term = term * zs / (i + k + 1)
    out[small] = s
    zl = z[~small]
    f = np.exp(zl)
    for kk in range(1, k + 1):
        f = (f - 1.0 / factorial(kk - 1)) / zl
    out[~small] = f
    return out


def augmented(a: np.ndarray, b: np.ndarray):
    """A~ = [[A, B], [0, K]], B = [b_p, ..., b_1], K = upper shift, v = [b_0; e_p] (eq 13)."""
    p = b.shape[0] - 1
    n = a.shape[0]
    at = np.zeros((n + p, n + p))
    at[:n, :n] = a
    for c in range(p):
        at[:n, n + c] = b[p - c]
    for i in range(p - 1):
        at[n + i, n + i + 1] = 1.0
    v = np.zeros(n + p)
    v[:n] = b[0]
    if p >= 1:
        v[n + p - 1] = 1.0
    return at, v


def exact_dense(a: np.ndarray, b: np.ndarray, tau: float, full: bool = False):
    at, v = augmented(a, b)
    y = scipy.linalg.expm(tau * at) @ v
    return y if full else y[: a.shape[0]]


def _dst(x, axes):
    return scipy.fft.dstn(x, type=1, norm="ortho", axes=axes)


def exact_dst_1d(n: int, coeff: float, b: np.ndarray, tau: float, shift: float = 0.0):
    h = 1.0 / (n + 1)
    kk = np.arange(1, n + 1)
    lam = coeff * (-4.0 / h**2) * np.sin(kk * np.pi * h / 2) ** 2 + shift
    w = np.zeros(n)
    for k in range(b.shape[0]):
        w += _dst(tau**k * phi(k, tau * lam) * _dst(b[k], axes=[0]), axes=[0])
    return w


def exact_dst_2d(n: int, diff: float, shift: float, b: np.ndarray, tau: float):
    h = 1.0 / (n + 1)
    kk = np.arange(1, n + 1)
    l1 = diff * (-4.0 / h**2) * np.sin(kk * np.pi * h / 2) ** 2
    lam = l1[:, None] + l1[None, :] + shift
    w = np.zeros((n, n))
    for k in range(b.shape[0]):
        bk = b[k].reshape(n, n)
        w += _dst(tau**k * phi(k, tau * lam) * _dst(bk, axes=[0, 1]), axes=[0, 1])
    return w.reshape(-1)


def exact_dst_3d(n: int, diff: float, shift: float, b: np.ndarray, tau: float):
    h = 1.0 / (n + 1)
    kk = np.arange(1, n + 1)
    l1 = diff * (-4.0 / h**2) * np.sin(kk * np.pi * h / 2) ** 2
    lam = l1[:, None, None] + l1[None, :, None] + l1[None, None, :] + shift
    w = np.zeros((n, n, n))
    for k in range(b.shape[0]):
        bk = b[k].reshape(n, n, n)
        w += _dst(tau**k * phi(k, tau * lam) * _dst(bk, axes=[0, 1, 2]), axes=[0, 1, 2])
    return w.reshape(-1)
