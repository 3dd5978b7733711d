"""Pins of the oracle's screened Epstein-Nesbet correction (Sec. II.B,
Eq. pt_hci) against facts outside the oracle:

* the numerators sum'_i H_ai c_i taken from the Jordan-Wigner FCI matrix
  (fci_jw shares no Slater-Condon rule with the oracle), screened term by
  term, for closed and open shells and several eps2;
* V = the whole sector leaves nothing outside it: E2 = 0;
* E2(eps2) tends to E2(0) as eps2 -> 0 (the paper's exact limit).
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle
from oracle import fci_jw


def _subspace(keys, H, frac, seed):
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(keys), max(2, int(frac * len(keys))), replace=False))
    w, v = np.linalg.eigh(H[np.ix_(sel, sel)])
    return sel, w[0], v[:, 0]


def _pt2_dense(H, sel, c, e0, eps2):
    outside = np.setdiff1d(np.arange(H.shape[0]), sel)
    terms = H[np.ix_(outside, sel)] * c[None, :]
    kept = np.abs(terms) > eps2
    num = np.where(kept, terms, 0.0).sum(axis=1)
    has = kept.any(axis=1)
    den = e0 - np.diag(H)[outside]
    return float(np.sum(num[has] ** 2 / den[has])), int(has.sum())


@pytest.mark.parametrize("norb,na,nb,seed", [(5, 2, 2, 21), (5, 3, 2, 22), (6, 3, 3, 23), (6, 1, 3, 24)])
@pytest.mark.parametrize("eps2", [0.0, 1e-3, 2e-2])
def test_pt2_matches_jordan_wigner(norb, na, nb, seed, eps2):
    inst = hi.random_tiny(norb, na, nb, seed)
    keys, H = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, na, nb)
    sel, e0, c = _subspace(keys, H, 0.3, seed)
    want, n_want = _pt2_dense(H, sel, c, e0, eps2)
    got, n_got = oracle.pt2(inst, keys[sel], c, eps2, e0)
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))
    if eps2 > 0:
        assert n_got == n_want
    assert got <= 0.0


def test_pt2_full_space_is_zero():
    inst = hi.random_tiny(5, 2, 2, 31)
    keys, H = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, 2, 2)
    w, v = np.linalg.eigh(H)
    e2, n = oracle.pt2(inst, keys, v[:, 0], 0.0, w[0])
    assert e2 == 0.0 and n == 0


def test_pt2_small_eps_limit():
    inst = hi.random_tiny(6, 3, 3, 41)
    keys, H = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, 3, 3)
    sel, e0, c = _subspace(keys, H, 0.2, 41)
    e_exact, n_exact = oracle.pt2(inst, keys[sel], c, 0.0, e0)
    e_loose, n_loose = oracle.pt2(inst, keys[sel], c, 1e-2, e0)
    e_tight, n_tight = oracle.pt2(inst, keys[sel], c, 1e-9, e0)
    assert n_loose < n_tight <= n_exact
    assert abs(e_loose - e_exact) > 1e-9
    assert abs(e_tight - e_exact) < 1e-12


def _pt2_rdm_jw(norb, keys, H, sel, c, e0, eps2):
    """Gamma^dd and Gamma^dc from Jordan-Wigner operator matrices: for every
    operator string, its elements between the kept (source, target) pairs
    weighted by c_i d_a, and its diagonal elements on the targets weighted
    by d_a^2 (d_a and the screening taken from the dense sector H)."""
    n = norb
    outside = np.setdiff1d(np.arange(H.shape[0]), sel)
    terms = H[np.ix_(outside, sel)] * c[None, :]
    kept = np.abs(terms) > eps2
    num = np.where(kept, terms, 0.0).sum(axis=1)
    has = kept.any(axis=1)
    d = np.where(has, num / (e0 - np.diag(H)[outside]), 0.0)
    W = (c[:, None] * d[None, :]) * kept.T            # [source, target]
    fock = fci_jw.keys_to_fock(keys, n)
    fs, fo = fock[sel], fock[outside]
    a = fci_jw.annihilators(2 * n)
    ad = [x.T.tocsr() for x in a]
    r1dd, r1dc = np.zeros((n, n)), np.zeros((n, n))
    r2dd, r2dc = np.zeros((n,) * 4), np.zeros((n,) * 4)
    for s in range(2):
        for p in range(n):
            for q in range(n):
                O = (ad[s * n + p] @ a[s * n + q]).tocsr()
                r1dc[p, q] += np.sum(W * O[fs][:, fo].toarray())
                r1dd[p, q] += np.sum(d ** 2 * O[fo, fo].A1)
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for w in range(n):
                            O = (ad[s * n + p] @ ad[t * n + r] @ a[t * n + w] @ a[s * n + q]).tocsr()
                            if O.nnz == 0:
                                continue
                            r2dc[p, q, r, w] += np.sum(W * O[fs][:, fo].toarray())
                            r2dd[p, q, r, w] += np.sum(d ** 2 * O[fo, fo].A1)
    return r1dd, r2dd, r1dc, r2dc


@pytest.mark.parametrize("norb,na,nb,seed,eps2", [(4, 2, 2, 61, -1.0), (4, 2, 1, 62, 5e-3), (5, 2, 2, 63, 1e-3)])
def test_pt2_rdm_matches_jordan_wigner(norb, na, nb, seed, eps2):
    inst = hi.random_tiny(norb, na, nb, seed)
    keys, H = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, na, nb)
    sel, e0, c = _subspace(keys, H, 0.35, seed)
    want = _pt2_rdm_jw(norb, keys, H, sel, c, e0, eps2)
    got = oracle.pt2_rdm(inst, keys[sel], c, eps2, e0)
    for g, w in zip(got, want):
        assert np.abs(g - w).max() < 1e-12 * max(1.0, np.abs(w).max())
    # traces: tr Gamma^dd_1 = N |d|^2 and tr Gamma^dc_1 = N <c|d> = 0 (d lives outside V)
    e2, _ = oracle.pt2(inst, keys[sel], c, eps2, e0)
    N = na + nb
    assert abs(np.trace(got[2])) < 1e-12
    assert abs(np.einsum("pprr->", got[1]) - N * (N - 1) * np.trace(got[0]) / N) < 1e-10
