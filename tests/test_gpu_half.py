"""One orientation per connected pair (hci_set_sigma_mode HCI_SIGMA_HALF):
each pair of V that differs by a single or double excitation (Sec. IV) is
stored once, in the row of the later-inserted determinant, and every H c
adds the entry to both rows (the second through an FP64 atomic add), so
the graph takes half the memory of the both-orientation form.

* sigma equals the oracle's H c and the both-orientation form's (rounding
  order), with the same connection count, in one pass and as a row-sum
  pass plus a scatter pass (the form for vectors beyond L2);
* Davidson energies and the RDMs (one orientation accumulated, the other as
  its transpose) equal the oracle's;
* a space grown in steps (rows appended, stored rows untouched), including a
  row longer than the row search's scratch, gives the oracle's H c;
* full solves give the oracle's space and energy;
* HCI_SIGMA_AUTO keeps both orientations while they fit the budget, then one
  orientation, then the direct form.
"""
import itertools

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


@pytest.fixture(params=["by_size", "two_passes"])
def passes(request, monkeypatch):
    """The product in one pass (c and sigma fit L2 at these sizes) and, with
    HCI_SIGMA_HALF_PASSES=2, as a row-sum pass plus a scatter pass (the form
    taken when c and sigma exceed half of L2)."""
    if request.param == "two_passes":
        monkeypatch.setenv("HCI_SIGMA_HALF_PASSES", "2")
    return request.param


@pytest.mark.parametrize("name,make,nv", CASES)
def test_half_sigma_davidson_rdm_match_oracle(pkg, name, make, nv, passes):
    from paper_1708_07544_gb300 import _abi

    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 17)
    c = hi.random_vector(len(keys), seed=nv + 18)
    H = oracle.hamiltonian(inst, keys)
    want = H @ c
    kd, cd = dev_keys(keys), torch.tensor(c).cuda()
    with solver(pkg, inst, _abi.SIGMA_HALF) as s, solver(pkg, inst, _abi.SIGMA_STORED) as t:
        got = s.sigma(kd, cd).cpu().numpy()
        ref = t.sigma(kd, cd).cpu().numpy()
        st_h, st_s = s.stats(), t.stats()
        # two vectors in one pass
        c2 = np.stack([c, hi.random_vector(len(keys), seed=nv + 19)])
        got2 = s.sigma(kd, torch.tensor(c2).cuda()).cpu().numpy()
        e, cv, _ = s.davidson(kd, None, tol=1e-10)
        r1, r2 = s.rdm12(kd, cv)
    scale = max(1.0, np.abs(want).max())
    assert np.abs(got - want).max() <= 1e-11 * scale
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert np.abs(got2[1] - H @ c2[1]).max() <= 1e-11 * scale
    assert np.abs(got2[0] - want).max() <= 1e-11 * scale
    assert st_h["graph_half"] == 1 and st_s["graph_half"] == 0
    assert st_h["graph_nnz"] == st_s["graph_nnz"] == H.nnz - len(keys)
    e_or, c_or = oracle.ground_state(inst, keys)
    assert abs(e - e_or) < 1e-9
    w1, w2 = oracle.rdm12(inst.norb, keys, c_or)
    assert np.abs(r1.cpu().numpy() - w1).max() < 1e-8
    assert np.abs(r2.cpu().numpy() - w2).max() < 1e-8


def test_half_grown_space_matches_oracle(pkg, passes):
    from paper_1708_07544_gb300 import _abi

    inst = hi.df_12o()
    full = hi.random_det_keys(12, 6, 6, 4000, seed=41)
    rng = np.random.default_rng(42)
    order = rng.permutation(len(full))
    steps = [np.sort(order[:500]), np.sort(order[:1800]), np.sort(order[:3100]), np.arange(len(full))]
    with solver(pkg, inst, _abi.SIGMA_HALF) as s:
        for idx in steps:
            keys = full[idx]
            c = hi.random_vector(len(keys), seed=len(keys))
            got = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
            want = oracle.hamiltonian(inst, keys) @ c
            assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())
        st = s.stats()
        r1, r2 = s.rdm12(dev_keys(full), torch.tensor(c).cuda())
    assert st["graph_builds"] == 4 and st["graph_half"] == 1
    w1, w2 = oracle.rdm12(12, full, c)
    assert np.abs(r1.cpu().numpy() - w1).max() < 1e-8
    assert np.abs(r2.cpu().numpy() - w2).max() < 1e-8


def test_half_row_beyond_scratch(pkg):
    """The aufbau determinant of (26e,26o) added after all 41067 of its
    single and double excitations: its stored row holds all of them, more
    than the row search's per-warp scratch, and is filled by the second
    search."""
    from paper_1708_07544_gb300 import _abi

    norb, ne = 26, 13
    inst = hi.random_tiny(norb, ne, ne, 31)
    a0 = b0 = (1 << ne) - 1
    occ, vir = range(ne), range(ne, norb)
    singles = [a0 ^ (1 << i) ^ (1 << a) for i in occ for a in vir]
    doubles = [a0 ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << b)
               for i, j in itertools.combinations(occ, 2) for a, b in itertools.combinations(vir, 2)]
    exc = ([(x, b0) for x in singles + doubles] + [(a0, y) for y in singles + doubles]
           + [(x, y) for x in singles for y in singles])
    exc = np.array(sorted(exc), dtype=np.uint64)
    full = np.array(sorted([tuple(r) for r in exc.tolist()] + [(a0, b0)]), dtype=np.uint64)
    c = hi.random_vector(len(full), seed=6)
    i0 = int(np.nonzero((full[:, 0] == a0) & (full[:, 1] == b0))[0][0])
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[i0], rng.choice(len(full), 64, replace=False)]))
    with solver(pkg, inst, _abi.SIGMA_HALF) as s:
        s.sigma(dev_keys(exc), torch.tensor(hi.random_vector(len(exc), seed=7)).cuda())
        got = s.sigma(dev_keys(full), torch.tensor(c).cuda()).cpu().numpy()
        assert s.stats()["rows_refilled"] >= 1
    want = oracle.sigma_rows(inst, full, c, rows)
    assert np.abs(got[rows] - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_half_full_solve_matches_oracle(pkg):
    from paper_1708_07544_gb300 import _abi

    inst = hi.ppp_polyene(8)
    ref = oracle.hci(inst, 1e-4)
    with solver(pkg, inst, _abi.SIGMA_HALF) as s:
        out = s.solve(1e-4, dav_tol=1e-10)
        assert s.stats()["graph_half"] == 1
    got = {tuple(x) for x in host_keys(out["keys"]).tolist()}
    assert got == {tuple(x) for x in np.asarray(ref["keys"]).tolist()}
    assert abs(out["E"] - ref["E"]) < 1e-9


def test_auto_steps_down_from_both_orientations(pkg):
    from paper_1708_07544_gb300 import _abi

    inst = hi.df_12o()
    with solver(pkg, inst, _abi.SIGMA_STORED) as t:
        want = t.solve(1e-3, dav_tol=1e-10)
        r_want = t.rdm12(want["keys"], want["c"])
        nnz = t.stats()["graph_nnz"]
    # one orientation (6 bytes per ordered pair) fits, both (>= 12) do not
    with solver(pkg, inst, _abi.SIGMA_AUTO, 8 * nnz) as s:
        out = s.solve(1e-3, dav_tol=1e-10)
        r = s.rdm12(out["keys"], out["c"])
        st = s.stats()
    assert st["graph_half"] == 1 and st["sigma_direct"] == 0
    assert torch.equal(out["keys"], want["keys"])
    assert abs(out["E"] - want["E"]) < 1e-10
    for a, b in zip(r, r_want):
        assert (a - b).abs().max().item() < 1e-10
    # below one orientation: direct
    with solver(pkg, inst, _abi.SIGMA_AUTO, 4 * nnz) as s:
        s.solve(1e-3, dav_tol=1e-10)
        st = s.stats()
    assert st["sigma_direct"] == 1 and st["graph_half"] == 0
    # one orientation only: the budget is an error
    with solver(pkg, inst, _abi.SIGMA_HALF, 4 * nnz) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.solve(1e-3, dav_tol=1e-10)
        assert ei.value.status == _abi.HCI_ERR_NOMEM
