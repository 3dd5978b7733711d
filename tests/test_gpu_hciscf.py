"""The HCISCF gradient of E_var + E2 (Sec. III.A, Eq. lambda) at a fixed
variational space and a fixed set of perturbative pairs (eps2 < 0: every
single and double of V):

* the z-vector equation against the eigen-expansion of the dense oracle H;
* dE/dkappa from the relaxed density matrices (hci_relaxed_rdm12, then
  hci_rotate_backward) against central finite differences of the oracle's
  E_var + E2 on the rotated integrals.
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


def _space():
    inst = hi.random_tiny(6, 3, 3, 71)
    keys = hi.random_det_keys(6, 3, 3, 150, seed=72)
    return inst, keys


def test_zvector_matches_eigen_expansion(pkg):
    inst, keys = _space()
    H = oracle.hamiltonian(inst, keys).toarray()
    w, U = np.linalg.eigh(H)
    c, e0 = U[:, 0], w[0]
    g = hi.random_vector(len(keys), seed=73)
    want = U[:, 1:] @ ((U[:, 1:].T @ g) / (w[1:] - e0))
    with pkg.HCISolver(6, 3, 3, torch.tensor(inst.h).cuda(), torch.tensor(inst.eri).cuda(), inst.e_core) as s:
        z, it = s.zvector(dev_keys(keys), torch.tensor(c).cuda(), e0, torch.tensor(g).cuda(), tol=1e-12)
    z = z.cpu().numpy()
    assert it > 0
    assert abs(z @ c) < 1e-10
    assert np.abs(z - want).max() < 1e-9 * max(1.0, np.abs(want).max())


def _e_total(inst, keys, kap, eps2):
    R, _ = oracle.rotate(inst, kap)
    e, c = oracle.ground_state(R, keys)
    e2, _ = oracle.pt2(R, keys, c, eps2, e)
    return e + e2


def test_relaxed_gradient_matches_finite_differences(pkg):
    inst, keys = _space()
    eps2 = -1.0
    kap = hi.random_kappa(6, seed=74, sigma=0.05)
    h = torch.tensor(inst.h).cuda()
    eri = torch.tensor(inst.eri).cuda()
    k = torch.tensor(kap).cuda()
    _, h2, e2r = pkg.hci_rotate(k, h, eri)
    with pkg.HCISolver(6, 3, 3, h2, e2r, inst.e_core) as s:
        kd = dev_keys(keys)
        e0, c, _ = s.davidson(kd, None, tol=1e-12)
        e2, r1, r2 = s.relaxed_rdm12(kd, c, e0, eps2, zv_tol=1e-12)
    R, _ = oracle.rotate(inst, kap)
    e_or, c_or = oracle.ground_state(R, keys)
    assert abs(e0 - e_or) < 1e-10
    assert abs(e2 - oracle.pt2(R, keys, c_or, eps2, e_or)[0]) < 1e-10
    _, _, dk = pkg.hci_rotate_backward(k, h, eri, r1, r2)
    dk = dk.cpu().numpy()
    step = 1e-4
    for p, q in [(0, 3), (1, 4), (2, 5), (0, 1)]:
        vals = []
        for sg in (1, -1):
            d = kap.copy()
            d[p, q] += sg * step
            d[q, p] -= sg * step
            vals.append(_e_total(inst, keys, d, eps2))
        fd = (vals[0] - vals[1]) / (2 * step)
        an = dk[p, q] - dk[q, p]
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (p, q, fd, an)
