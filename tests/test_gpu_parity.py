"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bars: selected determinant sets bit-exact apart from the oracle's listed
ties (|f - eps1| <= 1e-12 eps1); energies within 1e-9 Ha; sigma and RDM
elements within 1e-8 (absolute; the FP64 rounding-order differences are
~1e-13); Davidson vectors compared after the phase convention.
"""
import itertools

import numpy as np
import pytest

import hci_inputs as hi
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

E_TOL = 1e-9
RDM_TOL = 1e-8


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


def solver(pkg, inst):
    return pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, torch.tensor(inst.h).cuda(),
                         torch.tensor(inst.eri).cuda(), inst.e_core)


CASES = [
    ("tiny6", lambda: hi.random_tiny(6, 3, 2, 41), 60),
    ("polyene8", lambda: hi.ppp_polyene(8), 700),
    ("df12", lambda: hi.df_12o(), 3000),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 500),
]


@pytest.mark.parametrize("name,make,nv", CASES)
@pytest.mark.parametrize("eps1", [0.0, 1e-4, 3e-3])
def test_select_step_bitexact(pkg, name, make, nv, eps1):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 7)
    c = hi.random_vector(len(keys), seed=nv + 8, decay=8.0 / len(keys))
    want, _, ties = oracle.select(inst, keys, c, eps1)
    with solver(pkg, inst) as s:
        got = host_keys(s.select(eps1, dev_keys(keys), torch.tensor(c).cuda()))
    # sorted, unique, disjoint from V
    assert np.all(np.lexsort((got[:, 1], got[:, 0])) == np.arange(len(got)))
    assert len(keyset(got)) == len(got)
    assert not (keyset(got) & keyset(keys))
    t = keyset(ties)
    assert keyset(got) - t == keyset(want) - t


def test_select_aufbau_and_empty(pkg):
    inst = hi.ppp_polyene(8)
    k0 = oracle.aufbau(4, 4)
    with solver(pkg, inst) as s:
        got = host_keys(s.select(0.0, dev_keys(k0), torch.ones(1, dtype=torch.float64).cuda()))
        # every single and double of the aufbau determinant of (8e,8o)
        want, _, _ = oracle.select(inst, k0, [1.0], 0.0)
        assert keyset(got) == keyset(want)
        # a coefficient of zero generates nothing at eps1 > 0
        got0 = s.select(1e-6, dev_keys(k0), torch.zeros(1, dtype=torch.float64).cuda())
        assert got0.shape[0] == 0


def test_merge(pkg):
    inst = hi.ppp_polyene(8)
    allk = hi.random_det_keys(8, 4, 4, 900, seed=3)
    rng = np.random.default_rng(4)
    m = rng.random(len(allk)) < 0.37
    a, b = allk[~m], allk[m]
    ca = rng.standard_normal(len(a))
    with solver(pkg, inst) as s:
        ok, oc = s.merge(dev_keys(a), torch.tensor(ca).cuda(), dev_keys(b))
    wk, wc = oracle.merge(a, ca, b)
    assert np.array_equal(host_keys(ok), wk)
    assert np.array_equal(oc.cpu().numpy(), wc)


@pytest.mark.parametrize("name,make,nv", CASES)
def test_sigma_matches_oracle(pkg, name, make, nv):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 1)
    c = hi.random_vector(len(keys), seed=nv + 2)
    H = oracle.hamiltonian(inst, keys)
    want = H @ c
    with solver(pkg, inst) as s:
        got = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
        # the graph holds exactly the oracle's off-diagonal non-zero pattern
        nnz_off = H.nnz - len(keys)
        assert s.stats()["graph_nnz"] == nnz_off
        # two vectors at once
        c2 = np.stack([c, hi.random_vector(len(keys), seed=nv + 3)])
        got2 = s.sigma(dev_keys(keys), torch.tensor(c2).cuda()).cpu().numpy()
    assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())
    assert np.abs(got2[1] - H @ c2[1]).max() < 1e-11 * max(1.0, np.abs(want).max())
    # the one- and several-vector kernels add the same terms in different
    # orders: equal up to FP64 rounding
    assert np.abs(got2[0] - got).max() < 1e-13 * max(1.0, np.abs(want).max())


def test_sigma_ragged_and_single(pkg):
    inst = hi.random_tiny(5, 2, 2, 5)
    with solver(pkg, inst) as s:
        for nv in [1, 2, 33, 97]:
            keys = hi.random_det_keys(5, 2, 2, nv, seed=nv)
            c = hi.random_vector(len(keys), seed=nv + 1)
            got = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
            want = oracle.hamiltonian(inst, keys) @ c
            assert np.abs(got - want).max() < 1e-12


def _bits(idx):
    v = 0
    for i in idx:
        v |= 1 << i
    return v


def test_sigma_long_and_empty_rows(pkg):
    """Rows longer than the kernel's whole shared-memory ring (every beta
    string of 12 orbitals on the aufbau alpha string and its 36 single
    excitations: up to ~1600 connections a row) next to determinants with no
    connection at all (alpha and beta strings 3 or more excitations from
    every other determinant's): every row of H c equals the oracle's."""
    norb = 12
    betas = [_bits(x) for x in itertools.combinations(range(norb), 6)]
    a0 = _bits(range(6))
    alphas = [a0] + [(a0 & ~(1 << i)) | (1 << a) for i in range(6) for a in range(6, 12)]
    keys = [(a, b) for a in alphas for b in betas]
    top = _bits(range(6, 12))
    keys += [(top, _bits(range(6))), (top, _bits(range(6, 12))), (top, _bits([0, 1, 2, 9, 10, 11]))]
    keys = np.array(sorted(keys), dtype=np.uint64)
    inst = hi.random_tiny(norb, 6, 6, 19)
    H = oracle.hamiltonian(inst, keys)
    offd = np.diff(H.indptr) - (H.diagonal() != 0)
    assert offd.max() > 4 * 256 and (offd == 0).sum() == 3
    c = hi.random_vector(len(keys), seed=23)
    want = H @ c
    with solver(pkg, inst) as s:
        got = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
        assert s.stats()["graph_nnz"] == H.nnz - len(keys)
    assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("name,make,nv", CASES[:3])
def test_davidson_matches_oracle(pkg, name, make, nv):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 5)
    e_ref, c_ref = oracle.ground_state(inst, keys)
    with solver(pkg, inst) as s:
        e, c, it = s.davidson(dev_keys(keys), None, tol=1e-10)
    assert abs(e - e_ref) < E_TOL
    assert np.abs(c.cpu().numpy() - c_ref).max() < 1e-7


@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (7, 4, 2), (7, 1, 3)])
def test_rdm_matches_oracle_random_vector(pkg, norb, na, nb):
    """Every element of both RDMs for a random vector on a random space,
    closed and open shell (alpha and beta aufbau strings differ)."""
    inst = hi.random_tiny(norb, na, nb, 77)
    keys = hi.random_det_keys(norb, na, nb, 250, seed=78)
    c = hi.random_vector(len(keys), seed=79)
    r1o, r2o = oracle.rdm12(norb, keys, c)
    with solver(pkg, inst) as s:
        r1, r2 = s.rdm12(dev_keys(keys), torch.tensor(c).cuda())
    assert np.abs(r1.cpu().numpy() - r1o).max() < RDM_TOL
    assert np.abs(r2.cpu().numpy() - r2o).max() < RDM_TOL


@pytest.fixture(scope="module")
def poly8_ref():
    inst = hi.ppp_polyene(8)
    return inst, oracle.hci(inst, 1e-4), oracle.hci(inst, 0.0)


def test_solve_polyene8_fci_and_eps(pkg, poly8_ref):
    inst, r4, r0 = poly8_ref
    with solver(pkg, inst) as s:
        out0 = s.solve(0.0)
        out4 = s.solve(1e-4)
    assert out0["keys"].shape[0] == 4900
    assert abs(out0["E"] - r0["E"]) < E_TOL
    assert keyset(host_keys(out4["keys"])) == keyset(r4["keys"])
    assert abs(out4["E"] - r4["E"]) < E_TOL
    assert out4["iters"] == len(r4["history"]) - 1


def test_rdm_on_hci_state_and_invariants(pkg, poly8_ref):
    inst, r4, _ = poly8_ref
    r1o, r2o = oracle.rdm12(8, r4["keys"], r4["c"])
    with solver(pkg, inst) as s:
        r1, r2 = s.rdm12(dev_keys(r4["keys"]), torch.tensor(r4["c"]).cuda())
    r1, r2 = r1.cpu().numpy(), r2.cpu().numpy()
    assert np.abs(r1 - r1o).max() < RDM_TOL
    assert np.abs(r2 - r2o).max() < RDM_TOL
    assert abs(oracle.energy_from_rdm(inst, r1, r2) - r4["E"]) < E_TOL


def test_rotation_matches_oracle(pkg):
    inst = hi.df_instance(9, 30, seed=5, name="df9")
    kap = hi.random_kappa(9, seed=6, sigma=0.3)
    R, U = oracle.rotate(inst, kap)
    Ug, hg, eg = pkg.hci_rotate(torch.tensor(kap).cuda(), torch.tensor(inst.h).cuda(), torch.tensor(inst.eri).cuda())
    assert np.abs(Ug.cpu().numpy() - U).max() < 1e-13
    assert np.abs(hg.cpu().numpy() - R.h).max() < 1e-12
    assert np.abs(eg.cpu().numpy() - R.eri).max() < 1e-12
    # backward against the oracle's chain rule on the oracle RDMs
    res = oracle.hci(R, 3e-3)
    r1, r2 = oracle.rdm12(9, res["keys"], res["c"])
    g = oracle.gradient(inst, kap, r1, r2)
    dh, de, dk = pkg.hci_rotate_backward(torch.tensor(kap).cuda(), torch.tensor(inst.h).cuda(),
                                         torch.tensor(inst.eri).cuda(), torch.tensor(r1).cuda(),
                                         torch.tensor(r2).cuda())
    assert np.abs(dh.cpu().numpy() - g["dh"]).max() < 1e-11
    assert np.abs(de.cpu().numpy() - g["deri"]).max() < 1e-11
    assert np.abs(dk.cpu().numpy() - g["dkappa"]).max() < 1e-9


def test_autograd_gradient_vs_oracle_and_fd(pkg):
    inst = hi.df_instance(8, 32, seed=11, name="df8")
    kap = hi.random_kappa(8, seed=12, sigma=0.05)
    eps1 = 1e-3
    h = torch.tensor(inst.h).cuda()
    eri = torch.tensor(inst.eri).cuda()
    k = torch.tensor(kap).cuda().requires_grad_(True)
    E = pkg.HCIEnergy.apply(h, eri, k, inst.nalpha, inst.nbeta, 0.0, eps1)
    E.backward()
    R, _ = oracle.rotate(inst, kap)
    ref = oracle.hci(R, eps1)
    assert abs(E.item() - ref["E"]) < E_TOL
    r1, r2 = oracle.rdm12(8, ref["keys"], ref["c"])
    g = oracle.gradient(inst, kap, r1, r2)["dkappa"]
    assert np.abs(k.grad.cpu().numpy() - g).max() < 1e-8
    # central finite differences of the GPU energy at fixed V
    keys = dev_keys(ref["keys"])
    step = 1e-5
    for p, q in [(0, 5), (2, 7), (1, 3)]:
        vals = []
        for sgn in (1, -1):
            d = kap.copy()
            d[p, q] += sgn * step
            d[q, p] -= sgn * step
            _, h2, e2 = pkg.hci_rotate(torch.tensor(d).cuda(), h, eri)
            with pkg.HCISolver(8, inst.nalpha, inst.nbeta, h2, e2, 0.0) as s:
                vals.append(s.davidson(keys, None, tol=1e-11)[0])
        fd = (vals[0] - vals[1]) / (2 * step)
        an = k.grad[p, q].item() - k.grad[q, p].item()
        assert abs(fd - an) < 1e-7, (p, q, fd, an)


def test_autograd_backward_twice_and_warm_start(pkg):
    """The backward reuses the forward's context (graph kept, CI vector
    recomputed by a cold Davidson); a second backward through a retained
    graph gives the same gradient from a fresh context.  A Davidson on the
    converged space with the converged start vector finishes at once (its
    kept Ritz vectors span the answer), and from a zero start it starts
    cold and reaches the same energy."""
    inst = hi.df_instance(8, 32, seed=11, name="df8")
    kap = hi.random_kappa(8, seed=12, sigma=0.05)
    h = torch.tensor(inst.h).cuda()
    eri = torch.tensor(inst.eri).cuda()
    k = torch.tensor(kap).cuda().requires_grad_(True)
    E = pkg.HCIEnergy.apply(h, eri, k, inst.nalpha, inst.nbeta, 0.0, 1e-3)
    (g1,) = torch.autograd.grad(E, k, retain_graph=True)
    (g2,) = torch.autograd.grad(E, k)
    assert torch.max(torch.abs(g1 - g2)).item() < 1e-10
    _, h2, e2 = pkg.hci_rotate(k.detach(), h, eri)
    with pkg.HCISolver(8, inst.nalpha, inst.nbeta, h2, e2, 0.0) as s:
        out = s.solve(1e-3, dav_tol=1e-10)
        e_warm, c_warm, it_warm = s.davidson(out["keys"], out["c"], tol=1e-10)
        e_cold, c_cold, it_cold = s.davidson(out["keys"], None, tol=1e-10)
    assert it_warm == 1 and it_cold > 3
    assert abs(e_warm - out["E"]) < 1e-12 and abs(e_cold - out["E"]) < 1e-9
    assert torch.max(torch.abs(c_cold - out["c"])).item() < 1e-7


def test_capacity_error_reports_required_size(pkg):
    inst = hi.ppp_polyene(8)
    k0 = oracle.aufbau(4, 4)
    from paper_1708_07544_gb300 import _abi
    import ctypes

    L = _abi.load()
    with solver(pkg, inst) as s:
        kk = dev_keys(k0)
        c = torch.ones(1, dtype=torch.float64).cuda()
        out = torch.empty((4, 2), dtype=torch.int64).cuda()
        n = ctypes.c_int64(0)
        st = L.hci_select(s.ctx, 0.0, kk.data_ptr(), c.data_ptr(), 1, out.data_ptr(), 4, ctypes.byref(n))
        assert st == _abi.HCI_ERR_CAPACITY
        want, _, _ = oracle.select(inst, k0, [1.0], 0.0)
        assert n.value == len(want)
        # unsorted input is rejected
        bad = dev_keys(np.array([[15, 15], [15, 15]], np.uint64))
        st = L.hci_select(s.ctx, 1e-4, bad.data_ptr(), torch.ones(2, dtype=torch.float64).cuda().data_ptr(), 2,
                          out.data_ptr(), 4, ctypes.byref(n))
        assert st == _abi.HCI_ERR_INVALID


@pytest.mark.parametrize("name,make,nv", [CASES[1], CASES[2]])
def test_incremental_graph_matches_oracle(pkg, name, make, nv):
    """A space that grows by merges reuses the cached graph (new rows only,
    transposes appended to old rows); the product must equal the oracle's
    H c on every space of the chain, and a space that is not a superset
    falls back to a full rebuild."""
    inst = make()
    allk = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 21)
    rng = np.random.default_rng(nv)
    order = rng.permutation(len(allk))
    sizes = [len(allk) // 5, len(allk) // 2, len(allk) - 3, len(allk)]
    with solver(pkg, inst) as s:
        builds0 = s.stats()["graph_builds"]
        for m in sizes:
            sub = allk[np.sort(order[:m])]
            c = hi.random_vector(len(sub), seed=m)
            got = s.sigma(dev_keys(sub), torch.tensor(c).cuda()).cpu().numpy()
            H = oracle.hamiltonian(inst, sub)
            want = H @ c
            assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max()), m
            assert s.stats()["graph_nnz"] == H.nnz - len(sub)
        assert s.stats()["graph_builds"] - builds0 == len(sizes)
        # shrink: not an extension
        sub = allk[np.sort(order[: len(allk) // 3])]
        c = hi.random_vector(len(sub), seed=5)
        got = s.sigma(dev_keys(sub), torch.tensor(c).cuda()).cpu().numpy()
        assert np.abs(got - oracle.hamiltonian(inst, sub) @ c).max() < 1e-11 * max(1.0, np.abs(got).max())


def test_incremental_graph_row_beyond_scratch(pkg):
    """A new row longer than the row search's per-warp scratch (32768
    entries): the aufbau determinant of 26 orbitals with 13 + 13 electrons
    joins a space of all its single and double excitations (41067 of them)
    in an incremental update; its stored row (the connections to every
    earlier determinant) is filled by the second search.  That row of H c
    and sampled others equal the oracle's."""
    norb, ne = 26, 13
    inst = hi.random_tiny(norb, ne, ne, 31)
    a0 = b0 = (1 << ne) - 1
    occ, vir = range(ne), range(ne, norb)
    singles = [a0 ^ (1 << i) ^ (1 << a) for i in occ for a in vir]
    doubles = [a0 ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << b)
               for i, j in itertools.combinations(occ, 2) for a, b in itertools.combinations(vir, 2)]
    exc = ([(x, b0) for x in singles + doubles] + [(a0, y) for y in singles + doubles]
           + [(x, y) for x in singles for y in singles])
    assert len(exc) == 41067
    exc = np.array(sorted(exc), dtype=np.uint64)
    full = np.array(sorted([tuple(r) for r in exc.tolist()] + [(a0, b0)]), dtype=np.uint64)
    rng = np.random.default_rng(5)
    first = exc
    c = hi.random_vector(len(full), seed=6)
    i0 = int(np.nonzero((full[:, 0] == a0) & (full[:, 1] == b0))[0][0])
    rows = np.unique(np.concatenate([[i0], rng.choice(len(full), 64, replace=False)]))
    with solver(pkg, inst) as s:
        s.sigma(dev_keys(first), torch.tensor(hi.random_vector(len(first), seed=7)).cuda())
        got = s.sigma(dev_keys(full), torch.tensor(c).cuda()).cpu().numpy()
        assert s.stats()["rows_refilled"] >= 1
    want = oracle.sigma_rows(inst, full, c, rows)
    assert np.abs(got[rows] - want).max() < 1e-11 * max(1.0, np.abs(want).max())
    # the same space built at once: the aufbau row of the fresh graph takes
    # the second search too
    with solver(pkg, inst) as s:
        got2 = s.sigma(dev_keys(full), torch.tensor(c).cuda()).cpu().numpy()
        assert s.stats()["rows_refilled"] >= 1
    assert np.abs(got2[rows] - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_incremental_solve_matches_fresh_contexts(pkg, poly8_ref):
    """Davidson on each space of an HCI run with one context (incremental
    graphs) equals the oracle's eigenvalue on that space."""
    inst, r4, _ = poly8_ref
    keys = oracle.aufbau(4, 4)
    c = np.array([1.0])
    with solver(pkg, inst) as s:
        for _ in range(4):
            new, _, _ = oracle.select(inst, keys, c, 1e-4)
            if len(new) == 0:
                break
            keys, c = oracle.merge(keys, c, new)
            e, cg, _ = s.davidson(dev_keys(keys), torch.tensor(c).cuda(), tol=1e-10)
            e_ref, c = oracle.ground_state(inst, keys)
            assert abs(e - e_ref) < E_TOL
