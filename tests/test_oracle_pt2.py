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
