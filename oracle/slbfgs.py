"""Stochastic limited-memory BFGS (Alg. 2) in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Only the test-suite may import this module; the
product path (paper_2102_00755_b300.slbfgs) never does.

Alg. 2 minimises J(u) given only an estimator g(u, theta, n) -> (F, G) of the
energy and its gradient, where n fixes the stochastic approximation (the same n
gives the same approximation at different u).  Per iteration i it evaluates the
estimator twice with the same n: at u and at u + nu z with z = -H G_u; the pair
(nu z, G_z - G_u) enters the history buffers, the step is z - H G_z, and the
result is projected onto [u_min, u_max].  The energy estimate is min(F_u, F_z);
after its first increase the iterates are averaged with weights w(i).

Readings where Alg. 2 leaves a choice:
* H_0 = h0 I with h0 = s'y / y'y of the newest pair (the usual L-BFGS scaling)
  when h0 is None, else the given constant.
* A pair with s'y <= 0 (no positive curvature) is not stored, which keeps H
  positive definite; Alg. 2 stores every pair.
* No line search (do_linesearch = false; the paper's runs use a fixed step).
* The trial point u + nu z is projected onto the bounds as well, and the stored
  pair is (u_trial - u, G_z - G_u): the bounds exist to keep the wave simulation
  stable, which the trial evaluation needs too.  With inactive bounds this is
  Alg. 2 as printed.
"""
from __future__ import annotations

import numpy as np


def two_loop(g, S, Y, h0):
    """H g by the two-loop recursion over the stored pairs (oldest first in S, Y),
    H_0 = h0 I."""
    q = np.array(g, dtype=np.float64, copy=True)
    saved = []
    for s, y in zip(reversed(S), reversed(Y)):          # newest to oldest
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        q -= a * y
        saved.append((rho, a, s, y))
    r = h0 * q
    for rho, a, s, y in reversed(saved):                # oldest to newest
        b = rho * float(y @ r)
        r += (a - b) * s
    return r


def push_pair(S, Y, s, y, m):
    """Append (s, y) to the history (at most m pairs), unless s'y <= 0."""
    if float(s @ y) <= 0.0:
        return False
    S.append(np.array(s, dtype=np.float64))
    Y.append(np.array(y, dtype=np.float64))
    if len(S) > m:
        S.pop(0)
        Y.pop(0)
    return True


def scaling(S, Y, h0):
    if h0 is not None:
        return h0
    if not S:
        return 1.0
    s, y = S[-1], Y[-1]
    return float(s @ y) / float(y @ y)


def slbfgs(u, estimator, nu, n_evl, m=64, h0=None, weight=lambda i: float(i) ** 3,
           u_min=-np.inf, u_max=np.inf, theta=lambda i: 0.0):
    """Alg. 2 without line search.  estimator(u, theta, n) -> (F, G).
    Returns (u_hat, energy estimates per iteration, iterates u per iteration)."""
    u = np.array(u, dtype=np.float64, copy=True)
    u_bar = np.zeros_like(u)
    w_bar = 0.0
    J_prev = np.inf
    S, Y = [], []
    averaging = False
    i = 0
    evl = 0
    u_hat = u.copy()
    Js, us = [], []
    while evl < n_evl:
        i += 1
        F_u, G_u = estimator(u, theta(i), i)
        evl += 1
        z = -two_loop(G_u, S, Y, scaling(S, Y, h0))
        u_trial = np.clip(u + nu * z, u_min, u_max)
        F_z, G_z = estimator(u_trial, theta(i), i)
        evl += 1
        push_pair(S, Y, u_trial - u, G_z - G_u, m)
        z = z - two_loop(G_z, S, Y, scaling(S, Y, h0))
        u = np.clip(u + nu * z, u_min, u_max)
        J = min(F_u, F_z)
        if averaging:
            u_bar += weight(i) * u
            w_bar += weight(i)
            u_hat = u_bar / w_bar
        else:
            if J > J_prev:
                averaging = True
            u_hat = u.copy()
        J_prev = J
        Js.append(J)
        us.append(u.copy())
    return u_hat, Js, us
