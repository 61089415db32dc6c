"""Eq. "squirmerflow" of Kuron et al. (arXiv:1903.04799), written out for the
tests that compare a computed flow with it.  Plain numpy; neither the oracle
nor the CUDA library is used here.
"""
from itertools import product

import numpy as np


def squirmer_flow(r, e, R, B1, beta):
    """Eq. "squirmerflow": the Stokes flow around a squirmer at displacement r
    (3 x M) from its centre.  The printed field decays at infinity and equals
    v0 e + slip on r = R, so it is the laboratory-frame field of a squirmer
    swimming at v0 = 2 B1 / 3 (Eq. "squirmer-speed")."""
    B2 = beta * B1
    rn = np.linalg.norm(r, axis=0)
    rh = r / rn
    c = e @ rh
    ec = e[:, None]
    return (B1 * (R / rn) ** 3 * (c * rh - ec / 3)
            + B2 * ((R / rn) ** 4 - (R / rn) ** 2) * (1.5 * c * c - 0.5) * rh
            + B2 * (R / rn) ** 4 * c * (c * rh - ec))


def periodic_squirmer_flow(r, e, R, B1, beta, L, K=3):
    """Sec. "Squirmers in Bulk": the periodic images approximated by summing
    Eq. "squirmerflow" over the images inside a sphere of K box lengths."""
    u = np.zeros_like(r)
    for n in product(range(-K, K + 1), repeat=3):
        if n[0] ** 2 + n[1] ** 2 + n[2] ** 2 <= K * K:
            u += squirmer_flow(r + L * np.array(n, float)[:, None], e, R, B1, beta)
    return u
