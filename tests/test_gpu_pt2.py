"""GPU screened Epstein-Nesbet correction (Sec. II.B, Eq. pt_hci) against the
oracle, which enumerates every single and double of V:

* E2 to 1e-11 relative and |C(eps2)| exactly, for eps2 > 0, eps2 = 0 (every
  non-zero term) and eps2 < 0 (every term), closed and open shell;
* the result does not depend on how many hash classes the targets are
  split into (max_pairs);
* V = the full space leaves no target (E2 = 0); an empty V gives 0.
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


def close(a, b, rel=1e-11):
    return abs(a - b) <= rel * max(1e-12, abs(b))


@pytest.fixture(scope="module")
def poly8_state(pkg):
    inst = hi.ppp_polyene(8)
    with solver(pkg, inst) as s:
        out = s.solve(1e-3, dav_tol=1e-10)
    return inst, out


@pytest.mark.parametrize("eps2", [1e-5, 1e-7, 0.0, -1.0])
def test_pt2_polyene8_matches_oracle(pkg, poly8_state, eps2):
    inst, out = poly8_state
    keys, c = out["keys"], out["c"]
    with solver(pkg, inst) as s:
        e2, n = s.pt2(keys, c, eps2, out["E"])
    want, n_want = oracle.pt2(inst, host_keys(keys), c.cpu().numpy(), eps2, out["E"])
    assert close(e2, want), (e2, want)
    assert n == n_want
    assert e2 < 0.0


def test_pt2_hash_classes_do_not_matter(pkg, poly8_state):
    inst, out = poly8_state
    with solver(pkg, inst) as s:
        one = s.pt2(out["keys"], out["c"], 1e-6, out["E"])
        many = s.pt2(out["keys"], out["c"], 1e-6, out["E"], max_pairs=500)
    assert close(many[0], one[0], 1e-13) and many[1] == one[1]


@pytest.mark.parametrize("name,make,nv,eps2", [
    ("df12", lambda: hi.df_12o(), 2000, 1e-5),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 400,
     1e-6),
    ("tiny7", lambda: hi.random_tiny(7, 3, 2, 51), 150, 0.0),
])
def test_pt2_random_space_matches_oracle(pkg, name, make, nv, eps2):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 41)
    c = hi.random_vector(len(keys), seed=nv + 42)
    e0 = float(oracle.diag(inst, keys).min()) - 0.5
    with solver(pkg, inst) as s:
        e2, n = s.pt2(dev_keys(keys), torch.tensor(c).cuda(), eps2, e0)
    want, n_want = oracle.pt2(inst, keys, c, eps2, e0)
    assert close(e2, want), (e2, want)
    assert n == n_want


def test_pt2_full_space_and_empty(pkg):
    inst = hi.ppp_polyene(8)
    with solver(pkg, inst) as s:
        out = s.solve(0.0, dav_tol=1e-10)
        assert out["keys"].shape[0] == 4900
        e2, n = s.pt2(out["keys"], out["c"], 0.0, out["E"])
        assert e2 == 0.0 and n == 0
        e2, n = s.pt2(out["keys"][:0], out["c"][:0], 1e-6, out["E"])
        assert e2 == 0.0 and n == 0


def _rdm_close(got, want, rel=1e-10):
    for g, w in zip(got, want):
        g = g.cpu().numpy()
        assert np.abs(g - w).max() <= rel * max(1.0, np.abs(w).max()), np.abs(g - w).max()


@pytest.mark.parametrize("name,make,nv,eps2", [
    ("tiny7_all", lambda: hi.random_tiny(7, 3, 2, 51), 150, -1.0),
    ("tiny7", lambda: hi.random_tiny(7, 3, 2, 51), 150, 1e-4),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 300,
     1e-5),
])
def test_pt2_rdm_random_space_matches_oracle(pkg, name, make, nv, eps2):
    """Gamma^dd and Gamma^dc (Sec. V) against the oracle's definition."""
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 61)
    c = hi.random_vector(len(keys), seed=nv + 62)
    e0 = float(oracle.diag(inst, keys).min()) - 0.5
    with solver(pkg, inst) as s:
        e2, n, rd = s.pt2(dev_keys(keys), torch.tensor(c).cuda(), eps2, e0, rdms=True)
        e2_plain, n_plain = s.pt2(dev_keys(keys), torch.tensor(c).cuda(), eps2, e0)
    assert close(e2, e2_plain, 1e-13) and n == n_plain
    _rdm_close(rd, oracle.pt2_rdm(inst, keys, c, eps2, e0))


def test_pt2_rdm_polyene8_state_and_classes(pkg, poly8_state):
    inst, out = poly8_state
    keys, c = out["keys"], out["c"]
    with solver(pkg, inst) as s:
        _, _, rd = s.pt2(keys, c, 1e-5, out["E"], rdms=True)
        _, _, rdm = s.pt2(keys, c, 1e-5, out["E"], max_pairs=700, rdms=True)
    want = oracle.pt2_rdm(inst, host_keys(keys), c.cpu().numpy(), 1e-5, out["E"])
    _rdm_close(rd, want)
    _rdm_close(rdm, [x.cpu().numpy() for x in rd], 1e-12)
