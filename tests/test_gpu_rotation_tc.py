"""The quarter transforms of the integral rotation (Sec. III.A:
(pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd), U = exp(kappa)) run on the bf16
tensor cores as exact products of 7-bit digits rounded once to FP64.  Their
result must be an FP64-quality product:

* against the oracle's rotation (numpy, FP64) for every padded width of
  the kernel (n <= 16, 32, 48, 64) and ragged last tiles (n^3 not a
  multiple of the 128-row tile), within 1e-13 of max |(pq|rs)|;
* for kappa = 0 (U = I exactly) the integrals come back within 2^-52 of
  each entry's own scale (the entries summed with it);
  (the bound is normwise, against the largest entry of each summed row
  and of U's column, where an FP64 dot product's is componentwise: an
  entry far below the rest of its row carries an absolute error of about
  2^-55 of that row's largest entry);
* the backward (dE/d(pq|rs) = the 2-RDM back-transformed by the same
  kernel) matches the oracle's chain rule at n = 44.
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


def _rotate(pkg, inst, kap):
    U, h2, e2 = pkg.hci_rotate(torch.tensor(kap).cuda(), torch.tensor(inst.h).cuda(), torch.tensor(inst.eri).cuda())
    return U.cpu().numpy(), h2.cpu().numpy(), e2.cpu().numpy()


@pytest.mark.parametrize("n", [3, 5, 9, 16, 17, 31, 44, 49])
def test_rotation_matches_oracle_every_width(pkg, n):
    inst = hi.df_instance(n, 2 * n, seed=100 + n, name=f"df{n}")
    kap = hi.random_kappa(n, seed=200 + n, sigma=0.3)
    R, U = oracle.rotate(inst, kap)
    Ug, hg, eg = _rotate(pkg, inst, kap)
    scale = np.abs(R.eri).max()
    assert np.abs(Ug - U).max() < 1e-13
    assert np.abs(hg - R.h).max() < 1e-12
    assert np.abs(eg - R.eri).max() < 1e-13 * scale
    # exact 8-fold symmetry of the result
    assert np.array_equal(eg, eg.transpose(1, 0, 2, 3))
    assert np.array_equal(eg, eg.transpose(2, 3, 0, 1))


def test_identity_rotation_returns_the_integrals(pkg):
    n = 44
    inst = hi.df_instance(n, 4 * n, seed=7, name="df44i")
    Ug, hg, eg = _rotate(pkg, inst, np.zeros((n, n)))
    assert np.array_equal(Ug, np.eye(n))
    assert np.array_equal(hg, inst.h)
    # each entry within 2^-52 of the largest |(ab|cd)| sharing three of its
    # indices (the rows the four transforms sum over)
    E = np.abs(inst.eri)
    s = np.maximum.reduce([np.broadcast_to(E.max(axis=k, keepdims=True), E.shape) for k in range(4)])
    assert np.all(np.abs(eg - inst.eri) <= 2.0 ** -52 * s)


def test_backward_at_44_orbitals_matches_oracle(pkg):
    n = 44
    inst = hi.df_instance(n, 4 * n, seed=12, name="df44b")
    kap = hi.random_kappa(n, seed=13, sigma=0.02)
    rng = np.random.default_rng(14)
    g1 = rng.standard_normal((n, n))
    g1 = g1 + g1.T
    g2 = hi.symmetrize_eri(rng.standard_normal((n,) * 4))
    g = oracle.gradient(inst, kap, g1, g2)
    dh, de, dk = pkg.hci_rotate_backward(torch.tensor(kap).cuda(), torch.tensor(inst.h).cuda(),
                                         torch.tensor(inst.eri).cuda(), torch.tensor(g1).cuda(),
                                         torch.tensor(g2).cuda())
    assert np.abs(dh.cpu().numpy() - g["dh"]).max() < 1e-11 * np.abs(g["dh"]).max()
    assert np.abs(de.cpu().numpy() - g["deri"]).max() < 1e-13 * np.abs(g["deri"]).max()
    assert np.abs(dk.cpu().numpy() - g["dkappa"]).max() < 1e-11 * np.abs(g["dkappa"]).max()
