"""Pin of the oracle's <S^2> (spin of a determinant expansion) against S^2
assembled literally from Jordan-Wigner operator matrices,
S^2 = S_- S_+ + S_z^2 + S_z with S_+ = sum_p a+_{p alpha} a_{p beta}, on random
vectors of closed- and open-shell sectors, and against S(S+1) for the
eigenstates of a Hubbard-like chain."""
import numpy as np
import pytest

import hci_inputs as hi
import oracle
from oracle import fci_jw


def _jw_s2(n):
    a = fci_jw.annihilators(2 * n)
    ad = [x.T.tocsr() for x in a]
    sp_ = sum(ad[p] @ a[n + p] for p in range(n))
    sm_ = sp_.T.tocsr()
    nop = [ad[m] @ a[m] for m in range(2 * n)]
    sz = 0.5 * (sum(nop[:n]) - sum(nop[n:]))
    return (sm_ @ sp_ + sz @ sz + sz).tocsr()


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (4, 3, 1), (5, 2, 3), (5, 3, 3)])
def test_spin_square_matches_jordan_wigner(n, na, nb):
    keys = fci_jw.sector_states(n, na, nb)
    c = hi.random_vector(len(keys), seed=10 * n + na)
    psi = np.zeros(1 << (2 * n))
    psi[fci_jw.keys_to_fock(keys, n)] = c
    want = psi @ (_jw_s2(n) @ psi)
    assert abs(oracle.spin_square(n, keys, c) - want) < 1e-12 * max(1.0, abs(want))


def test_spin_square_of_eigenstates_is_s_times_s_plus_one():
    inst = hi.ppp_polyene(4)
    keys, Hs = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, 2, 2)
    w, v = np.linalg.eigh(Hs)
    for r in range(6):
        s2 = oracle.spin_square(4, keys, v[:, r])
        S = 0.5 * (np.sqrt(1.0 + 4.0 * s2) - 1.0)
        assert abs(S - round(S)) < 1e-8, (r, s2)
    assert abs(oracle.spin_square(4, keys, v[:, 0])) < 1e-10      # singlet ground state
