"""Pins of the oracle's bit arithmetic above bit 31 (orbitals 32..63 of the
(44e,44o) and 64-orbital determinant words).

A small problem that the Jordan-Wigner build (fci_jw, no Slater-Condon rule
shared with the oracle) solves exactly is embedded into 5 active orbitals of
a 44- or 64-orbital space, spread over both 32-bit halves, with doubly
occupied core orbitals between them and every other orbital empty.  All
integrals touching a core or empty orbital are zero apart from their
diagonal h, so on the embedded sector

    <D|H|D'> = s(D) s(D') <d|H_small|d'> + delta_DD' (2 sum_core h_kk + e_core),

where d is D with the core removed and the active orbitals relabelled
0..4, and s(D) = (-1)^(sum over core k of the active electrons of the same
spin below k), the sign of moving every core creation operator in front of
the active ones (Sec. II: determinants as ordered products of creation
operators).  The RDMs (Sec. IV) follow from the small problem's and the
fixed core: rdm1_kk = 2, rdm2_kkll = 4, rdm2_kllk = -2 (k != l), rdm2_kkkk = 2,
rdm2_kkPQ = rdm2_PQkk = 2 rdm1_PQ, rdm2_kQPk = rdm2_PkkQ = -rdm1_PQ.
A misplaced shift or mask in the oracle's phases, excitation search or
operator application above bit 31 breaks one of these equalities.
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle
from oracle import fci_jw

LAYOUTS = [
    # (n, active orbitals, core orbitals)
    (44, [30, 33, 38, 40, 43], [0, 5, 31, 34, 39, 41]),
    (64, [5, 31, 32, 47, 63], [0, 6, 33, 48, 62, 40]),
]


def embed(n, act, core, small):
    act = list(act)
    core = sorted(core)
    h = np.zeros((n, n))
    for k in range(n):
        h[k, k] = -1.0 - 0.01 * k if k in core else 0.7 + 0.01 * k
    ix = np.array(act)
    h[np.ix_(ix, ix)] = small.h
    eri = np.zeros((n,) * 4)
    eri[np.ix_(ix, ix, ix, ix)] = small.eri
    na = small.nalpha + len(core)
    nb = small.nbeta + len(core)
    return oracle.Problem(n, na, nb, h, eri, small.e_core)


def big_keys(small_keys, act, core):
    cm = sum(1 << k for k in core)
    out = []
    for ka, kb in np.asarray(small_keys, np.uint64).tolist():
        a = cm | sum(1 << act[i] for i in range(len(act)) if (ka >> i) & 1)
        b = cm | sum(1 << act[i] for i in range(len(act)) if (kb >> i) & 1)
        out.append((a, b))
    return np.array(out, dtype=np.uint64)


def core_sign(big, act, core):
    s = np.ones(len(big))
    for i, (a, b) in enumerate(big.tolist()):
        m = 0
        for k in core:
            for w in (a, b):
                m += sum(1 for p in act if p < k and (w >> p) & 1)
        s[i] = -1.0 if m % 2 else 1.0
    return s


@pytest.mark.parametrize("n,act,core", LAYOUTS)
@pytest.mark.parametrize("na,nb,seed", [(2, 3, 31), (3, 3, 32)])
def test_hamiltonian_above_bit_31_matches_jordan_wigner(n, act, core, na, nb, seed):
    small = hi.random_tiny(5, na, nb, seed)
    ks, Hs = fci_jw.sector_matrix(small.h, small.eri, small.e_core, na, nb)
    P = embed(n, act, core, small)
    kb = big_keys(ks, act, core)
    # the embedding keeps (alpha, beta) order, so kb is sorted like ks
    assert np.all(np.lexsort((kb[:, 1], kb[:, 0])) == np.arange(len(kb)))
    s = core_sign(kb, act, core)
    assert np.any(s < 0) and np.any(s > 0)
    shift = 2.0 * sum(P.h[k, k] for k in core)
    want = s[:, None] * Hs * s[None, :] + shift * np.eye(len(kb))
    Ho = oracle.hamiltonian(P, kb).toarray()
    assert np.abs(Ho - want).max() < 1e-12
    assert np.abs(oracle.diag(P, kb) - np.diag(want)).max() < 1e-12
    # H c row by row (the routine that checks sampled GPU sigma rows)
    c = hi.random_vector(len(kb), seed=seed)
    rows = np.arange(len(kb))
    assert np.abs(oracle.sigma_rows(P, kb, c, rows) - want @ c).max() < 1e-12


@pytest.mark.parametrize("n,act,core", LAYOUTS)
def test_rdm_above_bit_31_matches_jordan_wigner(n, act, core):
    small = hi.random_tiny(5, 3, 2, 41)
    e, cs, ks = fci_jw.fci(small.h, small.eri, small.e_core, 3, 2)
    r1s, r2s = fci_jw.rdm12_jw(5, ks, cs)
    kb = big_keys(ks, act, core)
    s = core_sign(kb, act, core)
    r1, r2 = oracle.rdm12(n, kb, cs * s)
    ix = np.array(act)
    w1 = np.zeros((n, n))
    w2 = np.zeros((n,) * 4)
    w1[np.ix_(ix, ix)] = r1s
    w2[np.ix_(ix, ix, ix, ix)] = r2s
    for k in core:
        w1[k, k] = 2.0
        w2[k, k, k, k] = 2.0
        for l in core:
            if l != k:
                w2[k, k, l, l] = 4.0
                w2[k, l, l, k] = -2.0
        w2[k, k][np.ix_(ix, ix)] = 2.0 * r1s
        w2[np.ix_(ix, ix, [k], [k])] = 2.0 * r1s[:, :, None, None]
        w2[np.ix_([k], ix, ix, [k])] = -r1s.T[None, :, :, None]
        w2[np.ix_(ix, [k], [k], ix)] = -r1s[:, None, None, :]
    assert np.abs(r1 - w1).max() < 1e-12
    assert np.abs(r2 - w2).max() < 1e-12
    P = embed(n, act, core, small)
    shift = 2.0 * sum(P.h[k, k] for k in core)
    assert abs(oracle.energy_from_rdm(P, r1, r2) - (e + shift)) < 1e-11


@pytest.mark.parametrize("n,act,core", LAYOUTS)
@pytest.mark.parametrize("eps1", [0.05, 0.2])
def test_selection_above_bit_31_matches_dense_criterion(n, act, core, eps1):
    """Eq. (criteria): from a part of the embedded sector, the new
    determinants are exactly the rest of the sector with max_i |H_ai c_i| >
    eps1 under the Jordan-Wigner matrix (excitations out of the core or into
    empty orbitals have H_ai = 0 and are never selected at eps1 > 0)."""
    small = hi.random_tiny(5, 3, 2, 51)
    ks, Hs = fci_jw.sector_matrix(small.h, small.eri, small.e_core, 3, 2)
    P = embed(n, act, core, small)
    kb = big_keys(ks, act, core)
    s = core_sign(kb, act, core)
    H = s[:, None] * Hs * s[None, :]
    rng = np.random.default_rng(9)
    inV = np.zeros(len(kb), bool)
    inV[rng.choice(len(kb), 12, replace=False)] = True
    c = hi.random_vector(int(inV.sum()), seed=10)
    f = np.abs(H[~inV][:, inV] * c[None, :]).max(axis=1)
    want = kb[~inV][f > eps1]
    assert 0 < len(want) < len(kb) - 12
    new, _, ties = oracle.select(P, kb[inV], c, eps1)
    assert len(ties) == 0
    assert np.array_equal(new, want)


def test_non_interacting_64_orbitals():
    """No two-electron integrals, diagonal h over 64 orbitals, 40 + 35
    electrons: E = sum of the occupied levels and nothing is selected."""
    n, na, nb = 64, 40, 35
    rng = np.random.default_rng(3)
    eps = np.sort(rng.uniform(-2.0, 2.0, n))
    P = oracle.Problem(n, na, nb, np.diag(eps), np.zeros((n,) * 4), 0.5)
    k0 = oracle.aufbau(na, nb)
    assert int(k0[0, 0]) == (1 << 40) - 1
    assert abs(oracle.diag(P, k0)[0] - (eps[:na].sum() + eps[:nb].sum() + 0.5)) < 1e-13
    new, _, _ = oracle.select(P, k0, [1.0], 1e-14)
    assert len(new) == 0
