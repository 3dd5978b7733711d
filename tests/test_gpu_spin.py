"""Spin parity in the S_z = 0 sector (hci_set_spin_parity) against the
oracle: the singlet and triplet states of Sec. VI are the lowest states with
c(beta, alpha) = +c(alpha, beta) (even total spin) and -c(alpha, beta) (odd).

* a selection adds the spin-flip partner of every selected determinant;
* Davidson (one root and several) gives the oracle's sector eigenpairs, with
  flip pairs of exactly equal magnitude;
* whole solves give the oracle's flip-closed space and energy, the state has
  the requested flip parity, and its <S^2> (from its 2-RDM) equals the
  oracle's and lies near an integer S of the requested parity;
* misuse (odd parity without such a state, unequal spin counts, an open
  space, a parity outside {-1, 0, 1}) is refused.
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1708_07544_gb300 import build

    build.build()
    import paper_1708_07544_gb300 as p

    return p


def dev_keys(keys):
    k = np.ascontiguousarray(np.asarray(keys, np.uint64).reshape(-1, 2))
    return torch.from_numpy(k.view(np.int64)).cuda()


def host_keys(t):
    return t.cpu().numpy().view(np.uint64).reshape(-1, 2)


def keyset(a):
    return {(int(x), int(y)) for x, y in np.asarray(a, np.uint64).reshape(-1, 2)}


def solver(pkg, inst, parity):
    s = pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, torch.tensor(inst.h).cuda(),
                      torch.tensor(inst.eri).cuda(), inst.e_core)
    s.set_spin_parity(parity)
    return s


def flip_perm(keys):
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(np.asarray(keys).tolist())}
    return np.array([idx[(int(b), int(a))] for a, b in np.asarray(keys).tolist()])


def closed_space(inst, count, seed):
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, count, seed=seed)
    return oracle.close_under_flip(keys)


@pytest.mark.parametrize("parity", [1, -1])
def test_selection_adds_flip_partners(pkg, parity):
    inst = hi.df_12o()
    keys = closed_space(inst, 600, 3)
    c = hi.random_vector(len(keys), seed=4, decay=6.0 / len(keys))
    perm = flip_perm(keys)
    c = 0.5 * (c + parity * c[perm])
    for eps1 in (1e-3, 1e-4):
        want, _, ties = oracle.select(inst, keys, c, eps1)
        want = oracle.close_under_flip(want) if len(want) else want
        with solver(pkg, inst, parity) as s:
            got = host_keys(s.select(eps1, dev_keys(keys), torch.tensor(c).cuda()))
        t = keyset(ties) | keyset(oracle.flip_keys(ties)) if len(ties) else set()
        assert keyset(got) - t == keyset(want) - t
        assert keyset(got) == keyset(oracle.flip_keys(got))
        assert not (keyset(got) & keyset(keys))


@pytest.mark.parametrize("name,make", [("df12", hi.df_12o), ("polyene8", lambda: hi.ppp_polyene(8))])
@pytest.mark.parametrize("parity", [1, -1])
def test_davidson_in_the_sector_matches_oracle(pkg, name, make, parity):
    inst = make()
    keys = closed_space(inst, 1500 if inst.norb > 8 else 900, 5)
    e_or, c_or = oracle.parity_ground_state(inst, keys, parity)
    with solver(pkg, inst, parity) as s:
        e, c, _ = s.davidson(dev_keys(keys), None, tol=1e-10)
        # two roots of the sector, deflated
        es, cs, _ = s.davidson_roots(dev_keys(keys), 2, tol=1e-10)
    c = c.cpu().numpy()
    assert abs(e - e_or) < 1e-9
    perm = flip_perm(keys)
    assert np.array_equal(c[perm], parity * c)
    assert np.abs(c - c_or).max() < 1e-7
    B = oracle.parity_basis(keys, parity)
    H = oracle.hamiltonian(inst, keys)
    w = np.linalg.eigvalsh((B.T @ H @ B).toarray())
    assert np.abs(np.asarray(es) - w[:2]).max() < 1e-9
    cs = cs.cpu().numpy().reshape(2, -1)
    assert np.abs(cs[:, perm] - parity * cs).max() < 1e-12


@pytest.mark.parametrize("name,make,eps1", [("polyene8", lambda: hi.ppp_polyene(8), 1e-4),
                                            ("df12", hi.df_12o, 5e-3),
                                            ("df12_batch", lambda: hi.df_batch(64)[2], 1e-4)])
@pytest.mark.parametrize("parity", [1, -1])
def test_solve_in_the_sector_matches_oracle(pkg, name, make, eps1, parity):
    inst = make()
    ref = oracle.hci_parity(inst, eps1, parity)
    with solver(pkg, inst, parity) as s:
        out = s.solve(eps1, dav_tol=1e-10)
        r1, r2 = s.rdm12(out["keys"], out["c"])
        s2 = s.spin_square(r2)
    got = host_keys(out["keys"])
    assert keyset(got) == keyset(ref["keys"])
    assert abs(out["E"] - ref["E"]) < 1e-9
    # flip parity exactly; the total spin only near an integer of that
    # parity, since a selected space need not hold every determinant of a
    # spin multiplet
    c = out["c"].cpu().numpy()
    assert np.array_equal(c[flip_perm(got)], parity * c)
    S = 0.5 * (np.sqrt(1.0 + 4.0 * s2) - 1.0)
    assert abs(S - round(S)) < 0.01 and int(round(S)) % 2 == (0 if parity > 0 else 1)
    assert abs(s2 - oracle.spin_square(inst.norb, ref["keys"], ref["c"])) < 1e-7


def test_spin_parity_refusals(pkg):
    inst = hi.ppp_polyene(8)
    with pytest.raises(pkg.HCIError):
        solver(pkg, inst, 2)
    open_inst = hi.Instance("p8o", 8, 5, 3, inst.h, inst.eri, 0.0)
    with pytest.raises(pkg.HCIError):
        solver(pkg, open_inst, 1)
    keys = hi.random_det_keys(8, 4, 4, 200, seed=9)
    assert keyset(keys) != keyset(oracle.flip_keys(keys))
    with solver(pkg, inst, 1) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.davidson(dev_keys(keys), None)
        assert "partner" in str(ei.value)
    # odd parity on the aufbau determinant alone: no such state
    with solver(pkg, inst, -1) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.davidson(dev_keys(oracle.aufbau(4, 4)), None)
        assert "no state" in str(ei.value)
