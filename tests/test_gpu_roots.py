"""Several lowest states: deflated Davidson against the oracle's
eigensolver (energies within 1e-9, orthonormal eigenvectors with
residuals below the tolerance), and the multi-state HCI loop (selection
with max_r |H_ai c_i^(r)|) against the oracle's: the same determinant set
and energies within 1e-9, and the full space at eps1 = 0.
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


def solver(pkg, inst):
    return pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, torch.tensor(inst.h).cuda(),
                         torch.tensor(inst.eri).cuda(), inst.e_core)


@pytest.mark.parametrize("name,make,nv,nroots", [
    ("tiny6", lambda: hi.random_tiny(6, 3, 3, 91), 300, 4),
    ("df12", lambda: hi.df_12o(), 2500, 3),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 600, 3),
])
def test_davidson_roots_match_oracle(pkg, name, make, nv, nroots):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 91)
    w, _ = oracle.lowest_states(inst, keys, nroots)
    H = oracle.hamiltonian(inst, keys)
    with solver(pkg, inst) as s:
        e, c, it = s.davidson_roots(dev_keys(keys), nroots, tol=1e-10)
    C = c.cpu().numpy()
    assert np.abs(e - w).max() < 1e-9
    assert np.abs(C @ C.T - np.eye(nroots)).max() < 1e-9
    for r in range(nroots):
        assert np.linalg.norm(H @ C[r] - e[r] * C[r]) < 1e-9


def test_solve_roots_matches_oracle(pkg):
    inst = hi.ppp_polyene(8)
    ref = oracle.hci_roots(inst, 1e-3, 3)
    with solver(pkg, inst) as s:
        out = s.solve_roots(3, 1e-3, dav_tol=1e-10)
    got = {tuple(x) for x in host_keys(out["keys"]).tolist()}
    want = {tuple(x) for x in np.asarray(ref["keys"]).tolist()}
    assert got == want
    assert np.abs(out["E"] - ref["E"]).max() < 1e-9


@pytest.mark.parametrize("eps1", [1.0, 0.7])
def test_solve_roots_growing_from_fewer_determinants_than_roots(pkg, eps1):
    """The first selection leaves 3 determinants for 4 roots: the loop
    solves for the states V holds until it has grown (eps1 = 1.0 ends with
    exactly 4 determinants, 0.7 with 11)."""
    inst = hi.random_tiny(6, 3, 3, 91)
    ref = oracle.hci_roots(inst, eps1, 4)
    with solver(pkg, inst) as s:
        out = s.solve_roots(4, eps1, dav_tol=1e-10)
    got = {tuple(x) for x in host_keys(out["keys"]).tolist()}
    assert got == {tuple(x) for x in np.asarray(ref["keys"]).tolist()}
    assert np.abs(out["E"] - ref["E"]).max() < 1e-9


def test_solve_roots_eps_zero_is_full_space(pkg):
    inst = hi.random_tiny(6, 3, 2, 93)
    w = np.linalg.eigvalsh(oracle.hamiltonian(inst, oracle.hci(inst, 0.0)["keys"]).toarray())
    with solver(pkg, inst) as s:
        out = s.solve_roots(3, 0.0, dav_tol=1e-10)
    assert out["keys"].shape[0] == 20 * 15
    assert np.abs(out["E"] - w[:3]).max() < 1e-9


@pytest.mark.parametrize("nalpha,nbeta", [(4, 4), (5, 3)])
def test_spin_square_of_roots(pkg, nalpha, nbeta):
    """<S^2> from each root's 2-RDM (hci_spin_square) against the oracle's
    S_+ evaluation on the CI vector; at eps1 = 0 the roots are eigenstates
    of S^2 (integer S), and S_z = 1 leaves S >= 1."""
    p8 = hi.ppp_polyene(8)
    inst = hi.Instance("p8", 8, nalpha, nbeta, p8.h, p8.eri, p8.e_core)
    with solver(pkg, inst) as s:
        out = s.solve_roots(4, 0.0, dav_tol=1e-10)
        keys = out["keys"]
        kh = host_keys(keys)
        for r in range(4):
            cr = out["c"][r].contiguous()
            _, r2 = s.rdm12(keys, cr)
            s2 = s.spin_square(r2)
            want = oracle.spin_square(8, kh, cr.cpu().numpy())
            assert abs(s2 - want) < 1e-8, (r, s2, want)
            S = 0.5 * (np.sqrt(1.0 + 4.0 * s2) - 1.0)
            assert abs(S - round(S)) < 1e-6, (r, s2)
            assert S > 0.5 * (nalpha - nbeta) - 1e-6
