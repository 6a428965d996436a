"""Explicit block-Toeplitz matrix A_n^h of Property 1 (test infrastructure only).

Built by the induction of the proof of Property 1, independent of the loop
code in cdv_oracle.c:

* n = 1 (Eq. S1): A_1^h has m + 2p rows and m columns; column c holds
  h(0), ..., h(2p) in rows c, ..., c + 2p.
* n > 1 (Eq. 1 / S10): A_n^h is a block-Toeplitz matrix of
  (m_1 + 2p_1) x m_1 blocks; block (r, c) is A_{n-1}^h(r - c, ...), the
  (n-1)-D matrix of the template slice H[r - c, ...], when 0 <= r - c <= 2p_1,
  and zero otherwise.

Rows and columns follow the vectorisation by row partition (C-order).
"""
from __future__ import annotations

import numpy as np


def dense_A(H, m):
    H = np.asarray(H, dtype=np.float64)
    m = tuple(int(v) for v in m)
    if H.ndim != len(m):
        raise ValueError("H and m disagree on n")
    q1, m1 = H.shape[0], m[0]
    if H.ndim == 1:
        A = np.zeros((m1 + q1 - 1, m1))
        for c in range(m1):
            A[c:c + q1, c] = H
        return A
    blocks = [dense_A(H[j], m[1:]) for j in range(q1)]
    br, bc = blocks[0].shape
    A = np.zeros(((m1 + q1 - 1) * br, m1 * bc))
    for r in range(m1 + q1 - 1):
        for c in range(m1):
            j = r - c
            if 0 <= j < q1:
                A[r * br:(r + 1) * br, c * bc:(c + 1) * bc] = blocks[j]
    return A
