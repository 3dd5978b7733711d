"""Selected-set parity at the bench sizes (Sec. II.A, Eq. criteria with the
HCI importance function f(D_a) = max_i |H_ai c_i|).

The variational loop is driven step by step through the C ABI (hci_select,
hci_merge, hci_davidson at a residual of 1e-10), so that every intermediate
space V^mu and vector c^mu is at hand.  At each mu:

* the GPU selection restricted to a source set S (c zeroed outside S: a zero
  coefficient generates nothing at eps1 > 0) must equal, bit for bit, the
  oracle's enumeration of every single and double of the determinants in S
  (``oracle.select(..., sources=S)``), apart from the oracle's listed ties
  (|f - eps1| <= 1e-12 eps1).  S holds the largest |c_i| -- whose heat-bath
  prefixes are long enough to be cut into several walk work items -- plus
  random determinants.  Extras and misses both fail.
* at mu = 0 the source set is the aufbau determinant, i.e. the whole first
  selection (3e5 determinants on the (44e,44o) space) is compared.
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DAV_TOL = 1e-10
N_TOP = 160          # largest |c| sources
N_RAND = 160         # random sources


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


def walk_parity(pkg, inst, kap, eps1, min_final, seed):
    # both sides take the same rotated integrals, made exactly 8-fold
    # symmetric (the solver's input requirement)
    R0, _ = oracle.rotate(inst, kap)
    R = oracle.Problem(inst.norb, inst.nalpha, inst.nbeta, hi.symmetrize_h(R0.h), hi.symmetrize_eri(R0.eri),
                       inst.e_core)
    h = torch.tensor(R.h).cuda()
    eri = torch.tensor(R.eri).cuda()
    rng = np.random.default_rng(seed)
    n_checked = 0
    with pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, h, eri, inst.e_core) as s:
        a0 = (1 << inst.nalpha) - 1
        b0 = (1 << inst.nbeta) - 1
        keys_d = dev_keys(np.array([[a0, b0]], np.uint64))
        c_d = torch.ones(1, dtype=torch.float64).cuda()
        for mu in range(30):
            keys = host_keys(keys_d)
            c = c_d.cpu().numpy()
            nV = len(keys)
            if nV == 1:
                src = np.array([0])
            else:
                top = np.argsort(-np.abs(c), kind="stable")[:N_TOP]
                src = np.unique(np.concatenate([top, rng.choice(nV, min(N_RAND, nV), replace=False)]))
            cm = np.zeros_like(c)
            cm[src] = c[src]
            got = host_keys(s.select(eps1, keys_d, torch.tensor(cm).cuda()))
            want, _, ties = oracle.select(R, keys, c, eps1, sources=src)
            t = keyset(ties)
            gs, ws = keyset(got), keyset(want)
            assert len(gs) == len(got)
            extra, miss = (gs - ws) - t, (ws - gs) - t
            assert not extra and not miss, (mu, nV, len(extra), len(miss))
            if nV == 1:
                assert len(got) > 1000
            n_checked += 1
            # the real step of the solve
            new = s.select(eps1, keys_d, c_d)
            if new.shape[0] == 0:
                break
            keys_d, c0 = s.merge(keys_d, c_d, new)
            _, c_d, _ = s.davidson(keys_d, c0, tol=DAV_TOL)
        assert keys_d.shape[0] > min_final
    return n_checked


def test_df44_bench_configuration_selection_every_mu(pkg):
    """(44e,44o) DF, kappa ~ N(0, 0.01^2) (seed 1709), eps1 = 1e-4: the
    configuration bench.py times."""
    inst = hi.df_44o()
    kap = hi.random_kappa(44, seed=1709, sigma=0.01)
    n = walk_parity(pkg, inst, kap, 1e-4, 1_000_000, seed=5)
    assert n >= 10


def test_pentacene22_selection_every_mu(pkg):
    """PPP pentacene (22e,22o) at eps1 = 5e-5 in the Hueckel MO basis."""
    inst = hi.ppp_pentacene()
    n = walk_parity(pkg, inst, np.zeros((22, 22)), 5e-5, 300_000, seed=6)
    assert n >= 5
