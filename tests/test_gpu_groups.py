"""Parity on spaces whose string groups are large (the shape of the full-size
spaces, where the aufbau alpha string alone owns a large share of V), element
by element against the oracle:

* the variational 1- and 2-RDMs (Sec. IV, Gamma^{c,c}) on a (12e,12o) space
  in which one alpha string carries all C(12,6) = 924 beta strings and one
  beta string all 924 alpha strings, plus random determinants: the diagonal
  part sums group weights over chunks of 256 consecutive members (a group
  spread over several chunks and warps) and occupation sums over 256 slices
  of the groups (every slice non-empty);
* H c on the same space (Sec. II.A / IV) and the RDMs of an incrementally
  grown graph of it.
"""
import itertools

import numpy as np
import pytest

import hci_inputs as hi
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

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


def strings(n, k):
    return [sum(1 << p for p in occ) for occ in itertools.combinations(range(n), k)]


def big_group_space(n, na, nb, extra, seed):
    a0, b0 = (1 << na) - 1, (1 << nb) - 1
    dets = {(a0, b) for b in strings(n, nb)} | {(a, b0) for a in strings(n, na)}
    dets |= {(int(x), int(y)) for x, y in hi.random_det_keys(n, na, nb, extra, seed=seed)}
    return np.array(sorted(dets), dtype=np.uint64)


@pytest.mark.parametrize("na,nb", [(6, 6), (7, 5)])
def test_rdm_and_sigma_with_groups_beyond_one_chunk(pkg, na, nb):
    inst = hi.df_instance(12, 48, seed=77, nelec=na + nb, name="df12g")
    inst = hi.Instance("df12g", 12, na, nb, inst.h, inst.eri, 0.25)
    keys = big_group_space(12, na, nb, 2500, seed=na * 10 + nb)
    # the aufbau alpha group and beta group each span several chunks
    a0 = (1 << na) - 1
    assert np.count_nonzero(keys[:, 0] == a0) > 3 * 256
    c = hi.random_vector(len(keys), seed=19, decay=4.0 / len(keys))
    H = oracle.hamiltonian(inst, keys)
    w1, w2 = oracle.rdm12(12, keys, c)
    with pkg.HCISolver(12, na, nb, torch.tensor(inst.h).cuda(), torch.tensor(inst.eri).cuda(), inst.e_core) as s:
        sig = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
        g1, g2 = s.rdm12(dev_keys(keys), torch.tensor(c).cuda())
    want = H @ c
    assert np.abs(sig - want).max() < 1e-11 * max(1.0, np.abs(want).max())
    assert np.abs(g1.cpu().numpy() - w1).max() < RDM_TOL
    assert np.abs(g2.cpu().numpy() - w2).max() < RDM_TOL


def test_rdm_of_grown_graph_with_large_groups(pkg):
    """The same space reached in two steps (graph extended in place): RDMs
    and H c against the oracle on the grown space."""
    inst = hi.df_instance(12, 48, seed=78, name="df12g2")
    keys = big_group_space(12, 6, 6, 3000, seed=5)
    rng = np.random.default_rng(8)
    part = np.sort(rng.choice(len(keys), len(keys) // 2, replace=False))
    first = keys[part]
    c1 = hi.random_vector(len(first), seed=20)
    c = hi.random_vector(len(keys), seed=21, decay=3.0 / len(keys))
    w1, w2 = oracle.rdm12(12, keys, c)
    want = oracle.hamiltonian(inst, keys) @ c
    with pkg.HCISolver(12, 6, 6, torch.tensor(inst.h).cuda(), torch.tensor(inst.eri).cuda(), 0.0) as s:
        s.sigma(dev_keys(first), torch.tensor(c1).cuda())
        sig = s.sigma(dev_keys(keys), torch.tensor(c).cuda()).cpu().numpy()
        g1, g2 = s.rdm12(dev_keys(keys), torch.tensor(c).cuda())
    assert np.abs(sig - want).max() < 1e-11 * max(1.0, np.abs(want).max())
    assert np.abs(g1.cpu().numpy() - w1).max() < RDM_TOL
    assert np.abs(g2.cpu().numpy() - w2).max() < RDM_TOL
