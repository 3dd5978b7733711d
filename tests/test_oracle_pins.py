"""Pins of the CPU oracle against facts fixed outside the oracle itself.

* Slater-Condon elements and RDMs vs a Jordan-Wigner operator build (fci_jw),
  which shares no rule with the oracle.
* Closed forms: Hubbard dimer, non-interacting limit.
* HCI(eps1 = 0) = FCI (Sec. II.B: the eps -> 0 limit recovers the full space).
* Selection vs a dense-matrix evaluation of f_HCI (Eq. criteria, Sec. II.A).
* RDM invariants (trace, partial trace, hermiticity, E from RDMs).
* Variational bound, rotation invariance of FCI (Sec. III: CASCI is
  invariant to active-active rotations, HCI is not).
* vHCISCF gradient (Eq. vdedk2) vs central finite differences at fixed V.
"""
import os

import numpy as np
import pytest

import hci_inputs as hi
import oracle
from oracle import fci_jw

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("norb,na,nb,seed", [(4, 2, 2, 1), (4, 2, 1, 2), (5, 3, 2, 3), (5, 1, 3, 4),
                                             (6, 3, 3, 5)])
def test_hamiltonian_matches_jordan_wigner(norb, na, nb, seed):
    inst = hi.random_tiny(norb, na, nb, seed)
    keys, Hj = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, na, nb)
    Ho = oracle.hamiltonian(inst, keys).toarray()
    assert np.abs(Hj - Ho).max() < 1e-12
    # the diagonal routine agrees with the CSR diagonal
    assert np.abs(oracle.diag(inst, keys) - np.diag(Ho)).max() < 1e-12


@pytest.mark.parametrize("norb,na,nb,seed", [(4, 2, 2, 11), (5, 2, 3, 12)])
def test_rdm_matches_jordan_wigner(norb, na, nb, seed):
    inst = hi.random_tiny(norb, na, nb, seed)
    e, c, keys = fci_jw.fci(inst.h, inst.eri, inst.e_core, na, nb)
    r1j, r2j = fci_jw.rdm12_jw(norb, keys, c)
    r1o, r2o = oracle.rdm12(norb, keys, c)
    assert np.abs(r1j - r1o).max() < 1e-12
    assert np.abs(r2j - r2o).max() < 1e-12
    assert abs(oracle.energy_from_rdm(inst, r1o, r2o) - e) < 1e-11


def test_hubbard_dimer_closed_form():
    # two sites, one orbital each, (2e,2o): E = U/2 - sqrt((U/2)^2 + 4 t^2)
    for t, U in [(-1.0, 4.0), (-0.3, 1.7), (0.5, 8.0)]:
        h = np.array([[0.0, t], [t, 0.0]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        P = oracle.Problem(2, 1, 1, h, eri, 0.0)
        res = oracle.hci(P, 0.0)
        exact = U / 2 - np.sqrt((U / 2) ** 2 + 4 * t * t)
        assert len(res["keys"]) == 4
        assert abs(res["E"] - exact) < 1e-12


def test_non_interacting_limit():
    n, na, nb = 6, 3, 2
    eps = np.array([-1.3, -0.9, -0.2, 0.1, 0.4, 1.1])
    P = oracle.Problem(n, na, nb, np.diag(eps), np.zeros((n,) * 4), 0.25)
    res = oracle.hci(P, 1e-6)
    assert len(res["keys"]) == 1
    assert abs(res["E"] - (eps[:na].sum() + eps[:nb].sum() + 0.25)) < 1e-14
    new, f, _ = oracle.select(P, oracle.aufbau(na, nb), [1.0], 1e-12)
    assert len(new) == 0


def test_hci_eps0_is_fci_polyene6_jw():
    inst = hi.ppp_polyene(6)
    e_jw, _, keys = fci_jw.fci(inst.h, inst.eri, inst.e_core, 3, 3)
    res = oracle.hci(inst, 0.0)
    assert len(res["keys"]) == 400
    assert np.array_equal(res["keys"], keys)
    assert abs(res["E"] - e_jw) < 1e-10


def test_hci_eps0_is_fci_polyene8():
    inst = hi.ppp_polyene(8)
    res = oracle.hci(inst, 0.0)
    assert len(res["keys"]) == 4900       # C(8,4)^2
    full = fci_jw.sector_states(8, 4, 4)
    assert np.array_equal(res["keys"], full)
    H = oracle.hamiltonian(inst, full).toarray()
    assert abs(res["E"] - np.linalg.eigvalsh(H)[0]) < 1e-10
    # variational bound at eps1 > 0
    res4 = oracle.hci(inst, 1e-4)
    assert res4["E"] >= res["E"] - 1e-12
    assert len(res4["keys"]) < 4900


def test_selection_matches_dense_criterion():
    # f(D_a) = max_i |H_ai c_i| from the Jordan-Wigner matrix
    inst = hi.random_tiny(5, 2, 2, 21)
    keys, Hj = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, 2, 2)
    rng = np.random.default_rng(5)
    vidx = np.sort(rng.choice(len(keys), 12, replace=False))
    c = hi.random_vector(12, 6, decay=0.3)
    for eps1 in [1e-3, 1e-2, 5e-2]:
        f = np.max(np.abs(Hj[:, vidx] * c[None, :]), axis=1)
        f[vidx] = -1.0
        want = keys[f > eps1]
        got, _, ties = oracle.select(inst, keys[vidx], c, eps1)
        tie_set = {tuple(x) for x in ties.tolist()}
        a = {tuple(x) for x in want.tolist()} - tie_set
        b = {tuple(x) for x in got.tolist()} - tie_set
        assert a == b
    # eps1 <= 0: every single and double of V not in V
    got, _, _ = oracle.select(inst, keys[vidx], c, 0.0)
    conn = np.zeros(len(keys), bool)
    for i in vidx:
        ka = keys[:, 0] ^ keys[i, 0]
        kb = keys[:, 1] ^ keys[i, 1]
        lev = np.array([bin(int(x)).count("1") + bin(int(y)).count("1") for x, y in zip(ka, kb)])
        conn |= (lev <= 4) & (lev > 0)
    conn[vidx] = False
    assert np.array_equal(got, keys[conn])


def _rdm_invariants(norb, nelec, r1, r2, tol):
    assert abs(np.trace(r1) - nelec) < tol
    assert abs(np.einsum("pprr->", r2) - nelec * (nelec - 1)) < tol
    assert np.abs(np.einsum("pqrr->pq", r2) - (nelec - 1) * r1).max() < tol
    assert np.abs(r1 - r1.T).max() < tol
    assert np.abs(r2 - r2.transpose(2, 3, 0, 1)).max() < tol
    assert np.abs(r2 - r2.transpose(1, 0, 3, 2)).max() < tol


def test_rdm_invariants_polyene8_eps4():
    inst = hi.ppp_polyene(8)
    res = oracle.hci(inst, 1e-4)
    r1, r2 = oracle.rdm12(8, res["keys"], res["c"])
    _rdm_invariants(8, 8, r1, r2, 1e-10)
    assert abs(oracle.energy_from_rdm(inst, r1, r2) - res["E"]) < 1e-10


def test_sigma_rows_match_csr():
    inst = hi.random_tiny(6, 3, 3, 31)
    keys = hi.random_det_keys(6, 3, 3, 150, 32)
    c = hi.random_vector(len(keys), 33)
    H = oracle.hamiltonian(inst, keys)
    rows = np.arange(0, len(keys), 7)
    assert np.abs(oracle.sigma_rows(inst, keys, c, rows) - (H @ c)[rows]).max() < 1e-12


def test_phase_rule():
    c = np.array([0.1, -0.7, 0.7, 0.2])
    assert np.array_equal(oracle.fix_phase(c), -c)    # first of the tied maxima
    assert np.array_equal(oracle.fix_phase(-c), -c)


def test_fci_rotation_invariance_and_zero_gradient():
    inst = hi.ppp_polyene(6)
    res = oracle.hci(inst, 0.0)
    kap = hi.random_kappa(6, seed=3, sigma=0.2)
    R, _ = oracle.rotate(inst, kap)
    e_rot, _ = oracle.ground_state(R, res["keys"])
    assert abs(e_rot - res["E"]) < 1e-10
    r1, r2 = oracle.rdm12(6, res["keys"], res["c"])
    g = oracle.gradient(inst, np.zeros((6, 6)), r1, r2)["dkappa"]
    # antisymmetric-direction derivative vanishes at the full-CI limit
    assert np.abs(g - g.T).max() < 1e-9


def test_vhciscf_gradient_matches_finite_differences():
    inst = hi.df_instance(6, 24, seed=99, name="df6")
    res = oracle.hci(inst, 2e-3)
    keys = res["keys"]
    assert 1 < len(keys) < 400      # a genuinely truncated space
    kap = hi.random_kappa(6, seed=1709, sigma=0.05)
    R, _ = oracle.rotate(inst, kap)
    e0, c0 = oracle.ground_state(R, keys)
    r1, r2 = oracle.rdm12(6, keys, c0)
    assert abs(oracle.energy_from_rdm(R, r1, r2) - e0) < 1e-10
    g = oracle.gradient(inst, kap, r1, r2)
    step = 1e-5
    worst = 0.0
    for p, q in [(0, 3), (1, 4), (2, 5), (0, 1), (3, 5)]:
        d = np.zeros((6, 6))
        d[p, q], d[q, p] = step, -step
        ep, _ = oracle.energy_fixed_space(inst, kap + d, keys)
        em, _ = oracle.energy_fixed_space(inst, kap - d, keys)
        fd = (ep - em) / (2 * step)
        an = g["dkappa"][p, q] - g["dkappa"][q, p]
        worst = max(worst, abs(fd - an))
        assert abs(fd - an) < 1e-7 * max(1.0, abs(fd)), (p, q, fd, an)
    # the gradient is not trivially zero at eps1 > 0 (HCI is not rotation invariant)
    assert np.abs(g["dkappa"] - g["dkappa"].T).max() > 1e-6
    # dE/dh: perturb one symmetric pair of h
    hp = inst.h.copy(); hm = inst.h.copy()
    hp[1, 2] += step; hp[2, 1] += step; hm[1, 2] -= step; hm[2, 1] -= step
    Pp = oracle.Problem(6, 3, 3, hp, inst.eri, 0.0)
    Pm = oracle.Problem(6, 3, 3, hm, inst.eri, 0.0)
    fd = (oracle.energy_fixed_space(Pp, kap, keys)[0] - oracle.energy_fixed_space(Pm, kap, keys)[0]) / (2 * step)
    assert abs(fd - (g["dh"][1, 2] + g["dh"][2, 1])) < 1e-7
    # dE/d(pq|rs): perturb the whole 8-fold orbit of (01|23)
    orbit = {(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 0, 1),
             (2, 3, 1, 0), (3, 2, 1, 0)}
    ep_ = inst.eri.copy(); em_ = inst.eri.copy()
    for ix in orbit:
        ep_[ix] += step; em_[ix] -= step
    Pp = oracle.Problem(6, 3, 3, inst.h, ep_, 0.0)
    Pm = oracle.Problem(6, 3, 3, inst.h, em_, 0.0)
    fd = (oracle.energy_fixed_space(Pp, kap, keys)[0] - oracle.energy_fixed_space(Pm, kap, keys)[0]) / (2 * step)
    an = sum(g["deri"][ix] for ix in orbit)
    assert abs(fd - an) < 1e-7


def test_golden_polyene8():
    """Stored values written by tests/golden/make_golden.py (oracle only)."""
    path = os.path.join(GOLDEN, "polyene8.txt")
    vals = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    inst = hi.ppp_polyene(8)
    res = oracle.hci(inst, 1e-4)
    assert len(res["keys"]) == int(vals["nV_eps1e-4"])
    assert abs(res["E"] - vals["E_eps1e-4"]) < 1e-9
    assert abs(oracle.hci(inst, 0.0)["E"] - vals["E_fci"]) < 1e-9


def test_hci_roots_at_eps_zero_is_fci_spectrum():
    """Several roots: HCI(eps1 = 0) reaches the whole sector and its lowest
    states are the lowest Jordan-Wigner FCI eigenvalues."""
    inst = hi.random_tiny(5, 2, 2, 81)
    keys_j, Hj = fci_jw.sector_matrix(inst.h, inst.eri, inst.e_core, 2, 2)
    w = np.linalg.eigvalsh(Hj)
    res = oracle.hci_roots(inst, 0.0, 3)
    assert len(res["keys"]) == len(keys_j)
    assert np.abs(res["E"] - w[:3]).max() < 1e-10
    # the states are orthonormal eigenvectors on the final space
    H = oracle.hamiltonian(inst, res["keys"]).toarray()
    C = res["c"]
    assert np.abs(C @ C.T - np.eye(3)).max() < 1e-10
    assert np.abs(C @ H @ C.T - np.diag(res["E"])).max() < 1e-10
