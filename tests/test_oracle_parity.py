"""Pins of the oracle's spin-parity sector (the singlet and triplet states of
Sec. VI told apart in the S_z = 0 sector by the spin-flip symmetry of the
spin-free Hamiltonian) against the Jordan-Wigner spectrum:

* at eps1 = 0 the whole sector is selected, and the lowest state of parity
  p = +1 (-1) equals the lowest Jordan-Wigner eigenvalue whose eigenvector
  has even (odd) total spin S, from <S^2> = S(S + 1);
* the state has c(beta, alpha) = p c(alpha, beta) and <S^2> of that parity;
* at eps1 > 0 the space is closed under the flip and the energy lies above
  the sector's exact one (variational bound).
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle
from oracle import fci_jw


def _lowest_by_parity(inst, m):
    keys, Hs = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, m, m)
    w, v = np.linalg.eigh(Hs)
    out = {}
    for r in range(len(w)):
        s2 = oracle.spin_square(inst.norb, keys, v[:, r])
        S = int(round(0.5 * (np.sqrt(1.0 + 4.0 * s2) - 1.0)))
        assert abs(S * (S + 1) - s2) < 1e-8
        p = 1 if S % 2 == 0 else -1
        if p not in out:
            out[p] = (w[r], S)
        if len(out) == 2:
            break
    return out


CASES = [
    ("polyene6", lambda: hi.ppp_polyene(6), 3),
    ("tiny6", lambda: hi.random_tiny(6, 3, 3, 71), 3),
    ("tiny5", lambda: hi.random_tiny(5, 2, 2, 72), 2),
]


@pytest.mark.parametrize("name,make,m", CASES)
@pytest.mark.parametrize("parity", [1, -1])
def test_full_sector_matches_jordan_wigner_by_spin(name, make, m, parity):
    inst = make()
    want, S_want = _lowest_by_parity(inst, m)[parity]
    res = oracle.hci_parity(inst, 0.0, parity)
    n = inst.norb
    from math import comb
    assert len(res["keys"]) == comb(n, m) ** 2
    assert abs(res["E"] - want) < 1e-10
    keys, c = res["keys"], res["c"]
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(keys.tolist())}
    flip = np.array([idx[(int(b), int(a))] for a, b in keys.tolist()])
    assert np.abs(c[flip] - parity * c).max() < 1e-12
    s2 = oracle.spin_square(n, keys, c)
    assert abs(s2 - S_want * (S_want + 1)) < 1e-8


@pytest.mark.parametrize("parity", [1, -1])
def test_selected_space_is_flip_closed_and_variational(parity):
    inst = hi.ppp_polyene(6)
    exact = _lowest_by_parity(inst, 3)[parity][0]
    res = oracle.hci_parity(inst, 3e-3, parity)
    keys = res["keys"]
    assert 1 < len(keys) < 400
    closed = oracle.close_under_flip(keys)
    assert np.array_equal(closed, keys)
    assert res["E"] >= exact - 1e-12
    # the sector basis is orthonormal and respects the parity
    B = oracle.parity_basis(keys, parity).toarray()
    assert np.abs(B.T @ B - np.eye(B.shape[1])).max() < 1e-14
    f = oracle.flip_keys(keys)
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(keys.tolist())}
    perm = np.array([idx[(int(a), int(b))] for a, b in f.tolist()])
    assert np.abs(B[perm] - parity * B).max() < 1e-15


def test_parity_needs_equal_spin_counts():
    with pytest.raises(ValueError):
        oracle.hci_parity(hi.random_tiny(5, 3, 2, 1), 1e-3, 1)
