"""Direct connections (hci_set_sigma_mode): every H c and RDM pass searches
the connections of V again and evaluates their elements instead of reading
the stored graph (Sec. IV generates every single and double between pairs of
V; the stored form keeps them, the direct form regenerates them).

* sigma equals the oracle's H c and the stored form's (rounding order);
* Davidson energies and the RDMs equal the oracle's;
* full solves give the oracle's space and energy;
* HCI_SIGMA_AUTO stores the graph while it fits the budget and falls back
  to the direct form when it does not; HCI_SIGMA_STORED refuses instead.
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


def solver(pkg, inst, mode=None, budget=0):
    s = pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, torch.tensor(inst.h).cuda(),
                      torch.tensor(inst.eri).cuda(), inst.e_core)
    if mode is not None:
        s.set_sigma_mode(mode, budget)
    return s


CASES = [
    ("tiny7", lambda: hi.random_tiny(7, 3, 2, 51), 400),
    ("df12", lambda: hi.df_12o(), 3000),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 900),
]


@pytest.mark.parametrize("name,make,nv", CASES)
def test_direct_sigma_davidson_rdm_match_oracle(pkg, name, make, nv):
    from paper_1708_07544_gb300 import _abi

    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 7)
    c = hi.random_vector(len(keys), seed=nv + 8)
    H = oracle.hamiltonian(inst, keys)
    want = H @ c
    kd, cd = dev_keys(keys), torch.tensor(c).cuda()
    with solver(pkg, inst, _abi.SIGMA_DIRECT) as s, solver(pkg, inst) as t:
        got = s.sigma(kd, cd).cpu().numpy()
        ref = t.sigma(kd, cd).cpu().numpy()
        st_d, st_s = s.stats(), t.stats()
        e, cv, _ = s.davidson(kd, None, tol=1e-10)
        r1, r2 = s.rdm12(kd, cv)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-11 * scale
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert st_d["sigma_direct"] == 1 and st_s["sigma_direct"] == 0
    assert st_d["graph_nnz"] == st_s["graph_nnz"] > 0
    e_or, c_or = oracle.ground_state(inst, keys)
    assert abs(e - e_or) < 1e-9
    w1, w2 = oracle.rdm12(inst.norb, keys, c_or)
    assert np.abs(r1.cpu().numpy() - w1).max() < 1e-8
    assert np.abs(r2.cpu().numpy() - w2).max() < 1e-8


def test_direct_full_solve_matches_oracle(pkg):
    from paper_1708_07544_gb300 import _abi

    inst = hi.ppp_polyene(8)
    ref = oracle.hci(inst, 1e-4)
    with solver(pkg, inst, _abi.SIGMA_DIRECT) as s:
        out = s.solve(1e-4, dav_tol=1e-10)
        assert s.stats()["sigma_direct"] == 1
    got = {tuple(x) for x in host_keys(out["keys"]).tolist()}
    assert got == {tuple(x) for x in np.asarray(ref["keys"]).tolist()}
    assert abs(out["E"] - ref["E"]) < 1e-9


def test_auto_falls_back_under_a_budget(pkg):
    from paper_1708_07544_gb300 import _abi

    inst = hi.df_12o()
    with solver(pkg, inst) as t:
        want = t.solve(1e-3, dav_tol=1e-10)
        r_want = t.rdm12(want["keys"], want["c"])
        assert t.stats()["sigma_direct"] == 0
    # a budget far below the graph: stored until the first build fails, then direct
    with solver(pkg, inst, _abi.SIGMA_AUTO, 4096) as s:
        out = s.solve(1e-3, dav_tol=1e-10)
        r = s.rdm12(out["keys"], out["c"])
        assert s.stats()["sigma_direct"] == 1
    assert torch.equal(out["keys"], want["keys"])
    assert abs(out["E"] - want["E"]) < 1e-10
    for a, b in zip(r, r_want):
        assert (a - b).abs().max().item() < 1e-10
    # a budget the graph fits: stored
    with solver(pkg, inst, _abi.SIGMA_AUTO, 1 << 34) as s:
        s.solve(1e-3, dav_tol=1e-10)
        assert s.stats()["sigma_direct"] == 0
    # stored only: the budget is an error
    with solver(pkg, inst, _abi.SIGMA_STORED, 4096) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.solve(1e-3, dav_tol=1e-10)
        assert ei.value.status == _abi.HCI_ERR_NOMEM
    with solver(pkg, inst) as s:
        with pytest.raises(pkg.HCIError):
            s.set_sigma_mode(7)
        with pytest.raises(pkg.HCIError):
            s.set_sigma_mode(_abi.SIGMA_AUTO, -1)
