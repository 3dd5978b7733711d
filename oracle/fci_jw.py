"""Brute-force full CI from Jordan-Wigner operator matrices (test infrastructure).

Independent of the Slater-Condon rules used by both the oracle and the GPU
path: the second-quantised Hamiltonian of Sec. II (one-body h_pq, two-body
(pq|rs) in chemists' notation) is assembled literally from sparse
creation/annihilation matrices on the 2^(2n) Fock space, then restricted to
the (n_alpha, n_beta) sector.  Usable for n <= 6.

Mode order: alpha orbitals 0..n-1, then beta orbitals n..2n-1.  The Fock
basis state with bit m set for each occupied mode equals the determinant
prod_{m ascending} a+_m |0>, so JW basis states and the determinant
convention (alpha block then beta block, ascending) coincide with sign +1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def annihilators(nmodes: int):
    """a_m = Z x ... x Z x sigma^- x I x ... (Z on modes below m)."""
    dim = 1 << nmodes
    states = np.arange(dim, dtype=np.int64)
    ops = []
    for m in range(nmodes):
        occ = (states >> m) & 1
        src = states[occ == 1]
        dst = src ^ (1 << m)
        below = np.array([bin(int(s) & ((1 << m) - 1)).count("1") for s in src])
        sign = np.where(below % 2 == 0, 1.0, -1.0)
        ops.append(sp.csr_matrix((sign, (dst, src)), shape=(dim, dim)))
    return ops


def fock_hamiltonian(h: np.ndarray, eri: np.ndarray, e_core: float = 0.0):
    n = h.shape[0]
    a = annihilators(2 * n)
    ad = [x.T.tocsr() for x in a]
    dim = 1 << (2 * n)
    H = sp.identity(dim, format="csr") * e_core
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    H = H + h[p, q] * (ad[s * n + p] @ a[s * n + q])
    # 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs
    pair = {}
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    P, Q = s * n + p, s * n + q
                    for r in range(n):
                        for w in range(n):
                            v = eri[p, q, r, w]
                            if v == 0.0:
                                continue
                            R, S = t * n + r, t * n + w
                            key = (P, Q)
                            if key not in pair:
                                pair[key] = []
                            pair[key].append((R, S, v))
    for (P, Q), lst in pair.items():
        inner = None
        for R, S, v in lst:
            term = v * (ad[R] @ a[S])
            inner = term if inner is None else inner + term
        H = H + 0.5 * (ad[P] @ inner @ a[Q])
    return H.tocsr()


def sector_states(n: int, nalpha: int, nbeta: int) -> np.ndarray:
    """Fock indices of the (nalpha, nbeta) sector, ordered by (alpha bits, beta bits)."""
    out = []
    for ka in range(1 << n):
        if bin(ka).count("1") != nalpha:
            continue
        for kb in range(1 << n):
            if bin(kb).count("1") != nbeta:
                continue
            out.append((ka, kb))
    return np.array(out, dtype=np.uint64).reshape(-1, 2)


def keys_to_fock(keys: np.ndarray, n: int) -> np.ndarray:
    return (keys[:, 0].astype(np.int64) | (keys[:, 1].astype(np.int64) << n))


def sector_matrix(h, eri, e_core, nalpha, nbeta):
    """(keys, dense H restricted to the sector)."""
    n = h.shape[0]
    H = fock_hamiltonian(h, eri, e_core)
    keys = sector_states(n, nalpha, nbeta)
    idx = keys_to_fock(keys, n)
    return keys, H[idx][:, idx].toarray()


def fci(h, eri, e_core, nalpha, nbeta):
    keys, Hs = sector_matrix(h, eri, e_core, nalpha, nbeta)
    w, v = np.linalg.eigh(Hs)
    return w[0], v[:, 0], keys


def rdm12_jw(n: int, keys: np.ndarray, c: np.ndarray):
    """Spin-summed rdm1[p,q] = sum_s <a+_ps a_qs>,
    rdm2[p,q,r,s] = sum_st <a+_ps a+_rt a_st a_qs> from JW matrices."""
    a = annihilators(2 * n)
    ad = [x.T.tocsr() for x in a]
    dim = 1 << (2 * n)
    psi = np.zeros(dim)
    psi[keys_to_fock(keys, n)] = c
    rdm1 = np.zeros((n, n))
    rdm2 = np.zeros((n, n, n, n))
    for s in range(2):
        for p in range(n):
            for q in range(n):
                rdm1[p, q] += psi @ (ad[s * n + p] @ (a[s * n + q] @ psi))
    for s in range(2):
        for t in range(2):
            for q in range(n):
                x1 = a[s * n + q] @ psi
                for w in range(n):
                    x2 = a[t * n + w] @ x1
                    if not np.any(x2):
                        continue
                    for r in range(n):
                        x3 = ad[t * n + r] @ x2
                        for p in range(n):
                            rdm2[p, q, r, w] += psi @ (ad[s * n + p] @ x3)
    return rdm1, rdm2
