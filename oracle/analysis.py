"""Two-level convergence analysis of Sec. 3.3 (FP64 CPU oracle; test infrastructure only).

* ``lemma31_cpoint_error``: the C-point error after one two-level FCF iteration, evaluated from
  the closed form of Lemma 3.1 with the actual (time-dependent) propagators.
* ``tub_bound``: the right-hand side of Theorem 3.1 / Eq. (3.11),
      max_w (lam+_w)^m |(lam+_w)^m - mu++_w| (1 - (mu*_w)^{N_c-1}) / (1 - mu*_w),
  lam+ = max_j |lambda_w^(j)|, mu++ = min_j mu_w^(j), mu* = max_j |mu_w^(j)|, with the
  eigenvalues of Eq. (3.7).

Parity status: ``lemma31_cpoint_error`` is pinned against one iteration of ``oracle.mgrit``;
``tub_bound`` is evaluated as printed, but the T.U.B. column printed in Tables 5-6 is not
reproduced by it for the tensor-product operator (parity unpinned for those printed digits).
"""
from __future__ import annotations

import numpy as np

from .sfde import SFDE, modal_lambda


def lemma31_cpoint_error(prob: SFDE, E_c, m: int, coarse: str = "cn"):
    """E~_{km} = sum_{i=0}^{k-2} B^{k-2-i}_{Psi^D,k} (B^m_{Psi,(i+2)m} - Psi^D_{i+2})
    B^m_{Psi,(i+1)m} E_{im}, with E~_0 = E~_m = 0 (Lemma 3.1).

    B^l_{Psi,s} = Psi_s Psi_{s-1} ... Psi_{s-l+1}; Psi_n is the fine propagator (Eq. (3.2)),
    Psi^D_k the coarse one with step t_{km} - t_{(k-1)m}.  E_c[k] is the error at C-point km.
    """
    t = prob.t
    Nc = len(E_c) - 1

    def fine_block(s, l, v):  # B^l_{Psi,s} v
        for n in range(s - l + 1, s + 1):
            v = prob.propagate(v, t[n] - t[n - 1], "cn")
        return v

    def coarse_prop(k, v):
        return prob.propagate(v, t[k * m] - t[(k - 1) * m], coarse)

    def coarse_block(s, l, v):  # B^l_{Psi^D,s} v
        for k in range(s - l + 1, s + 1):
            v = coarse_prop(k, v)
        return v

    out = [np.zeros_like(E_c[0]) for _ in range(Nc + 1)]
    for k in range(2, Nc + 1):
        acc = np.zeros_like(E_c[0])
        for i in range(0, k - 1):
            w = fine_block((i + 1) * m, m, E_c[i])
            w = fine_block((i + 2) * m, m, w) - coarse_prop(i + 2, w)
            acc += coarse_block(k, k - 2 - i, w)
        out[k] = acc
    return out


def tub_bound(sigma, t, m: int, coarse: str = "cn"):
    """Theorem 3.1's two-level bound for the fine grid t and coarsening factor m."""
    sig = np.asarray(sigma, dtype=np.float64).reshape(-1)
    dt = np.diff(np.asarray(t, dtype=np.float64))
    tc = np.asarray(t)[::m]
    dtc = np.diff(tc)
    Nc = len(dtc)
    lam_dag = np.zeros_like(sig)
    for d in np.unique(dt):
        lam_dag = np.maximum(lam_dag, np.abs(modal_lambda(sig, d, "cn")))
    mu = np.stack([modal_lambda(sig, d, coarse) for d in np.unique(dtc)])
    mu_ddag = mu.min(axis=0)
    mu_star = np.abs(mu).max(axis=0)
    lm = lam_dag ** m
    geo = np.where(mu_star < 1.0, (1.0 - mu_star ** (Nc - 1)) / np.where(mu_star < 1, 1 - mu_star, 1),
                   float(Nc - 1))
    return float(np.max(lm * np.abs(lm - mu_ddag) * geo))
