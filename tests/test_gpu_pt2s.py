"""GPU semistochastic second-order correction (Sec. II.B, Eq. semistoc)
against the oracle on the same seeded inputs:

* the draws are bit-identical (Philox4x64-10 and the integer inverse CDF);
* every sample's E2^S(eps2) and E2^S(eps2_det) within 1e-10 of the oracle's
  value on those draws, closed and open shell, all pairs and screened;
* E2^D equals hci_pt2 at eps2_det (to rounding order); eps2_det = eps2
  leaves exactly E2^D;
  the hash-class split does not change a sample; invalid arguments are
  refused.
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


def _compare(got, want, rel=1e-10):
    assert np.array_equal(got["draws"].cpu().numpy(), want["draws"])
    g, w = got["samples"], want["samples"]
    assert np.abs(g - w).max() <= rel * max(1e-12, np.abs(w).max()), np.abs(g - w).max()
    assert abs(got["e2_det"] - want["e2_det"]) <= 1e-11 * max(1e-12, abs(want["e2_det"]))
    assert abs(got["estimate"] - want["estimate"]) <= rel * max(1e-12, abs(want["estimate"]))


@pytest.fixture(scope="module")
def poly8_state(pkg):
    inst = hi.ppp_polyene(8)
    with solver(pkg, inst) as s:
        out = s.solve(1e-3, dav_tol=1e-10)
    return inst, out


def test_semistochastic_polyene8_matches_oracle(pkg, poly8_state):
    inst, out = poly8_state
    keys, c, e0 = out["keys"], out["c"], out["E"]
    args = (e0, 1e-6, 3e-5, 40, 20, 1708)
    with solver(pkg, inst) as s:
        got = s.pt2_semistochastic(keys, c, *args)
        e2d, _ = s.pt2(keys, c, 3e-5, e0)
    want = oracle.pt2_semistochastic(inst, host_keys(keys), c.cpu().numpy(), *args)
    _compare(got, want)
    # separate calls sum the same terms in an order set by the walk's atomics
    assert abs(got["e2_det"] - e2d) <= 1e-13 * abs(e2d)
    assert got["error"] > 0.0


@pytest.mark.parametrize("name,make,nv,eps2,eps2d,nd,ns", [
    ("tiny7_all", lambda: hi.random_tiny(7, 3, 2, 51), 150, -1.0, 1e-3, 30, 6),
    ("df12", lambda: hi.df_12o(), 800, 1e-5, 1e-3, 200, 4),
    ("polyene8_open", lambda: hi.Instance("p8o", 8, 5, 3, hi.ppp_polyene(8).h, hi.ppp_polyene(8).eri, 0.3), 300,
     0.0, 1e-4, 64, 5),
])
def test_semistochastic_random_space_matches_oracle(pkg, name, make, nv, eps2, eps2d, nd, ns):
    inst = make()
    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, nv, seed=nv + 81)
    c = hi.random_vector(len(keys), seed=nv + 82)
    c[::11] = 0.0                      # never drawn
    c /= np.linalg.norm(c)
    e0 = float(oracle.diag(inst, keys).min()) - 0.5
    args = (e0, eps2, eps2d, nd, ns, 99 + nv)
    with solver(pkg, inst) as s:
        got = s.pt2_semistochastic(dev_keys(keys), torch.tensor(c).cuda(), *args)
    want = oracle.pt2_semistochastic(inst, keys, c, *args)
    _compare(got, want)
    d = got["draws"].cpu().numpy()
    assert not np.isin(np.arange(0, len(keys), 11), d).any()


def test_semistochastic_classes_and_equal_thresholds(pkg, poly8_state):
    inst, out = poly8_state
    keys, c, e0 = out["keys"], out["c"], out["E"]
    with solver(pkg, inst) as s:
        one = s.pt2_semistochastic(keys, c, e0, 1e-7, 1e-5, 50, 4, 5)
        many = s.pt2_semistochastic(keys, c, e0, 1e-7, 1e-5, 50, 4, 5, max_pairs=300)
        same = s.pt2_semistochastic(keys, c, e0, 1e-5, 1e-5, 50, 4, 5)
        e2d, _ = s.pt2(keys, c, 1e-5, e0)
    assert np.array_equal(one["draws"].cpu().numpy(), many["draws"].cpu().numpy())
    assert np.abs(one["samples"] - many["samples"]).max() <= 1e-12 * np.abs(one["samples"]).max()
    assert same["estimate"] == same["e2_det"] and same["error"] == 0.0
    assert abs(same["e2_det"] - e2d) <= 1e-13 * abs(e2d)


def test_semistochastic_invalid_and_empty(pkg, poly8_state):
    inst, out = poly8_state
    keys, c, e0 = out["keys"], out["c"], out["E"]
    with solver(pkg, inst) as s:
        with pytest.raises(pkg.HCIError):
            s.pt2_semistochastic(keys, c, e0, 1e-6, 1e-5, 1, 4)
        with pytest.raises(pkg.HCIError):
            s.pt2_semistochastic(keys, c, e0, 1e-4, 1e-5, 10, 4)
        r = s.pt2_semistochastic(keys[:0], c[:0], e0, 1e-6, 1e-5, 10, 3)
        assert r["estimate"] == 0.0 and r["error"] == 0.0
