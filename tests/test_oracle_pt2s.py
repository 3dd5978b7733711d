"""Pins of the oracle's semistochastic second-order correction (Sec. II.B,
Eq. semistoc) against things other than itself:

* its Philox4x64-10 against numpy's independent implementation (numpy
  advances the counter before its first block);
* the integer inverse CDF against the bit rule it reduces to when the
  weights are powers of two;
* the sampled estimator's exact expectation, summed over every ordered
  draw sequence with its probability, against the deterministic E2 with
  the same screen (itself pinned against the Jordan-Wigner FCI);
* eps2_det = eps2 leaves exactly E2^D; and on a polyene HCI state the
  sample means agree with E2 within five standard errors.
"""
import itertools

import numpy as np
import pytest

import hci_inputs as hi
import oracle


def _next(ctr):
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if c[0] == 0:
        c[1] += 1
    return c


@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((1, 2, 3, 4), (5, 6)),
                                     ((2**64 - 2, 7, 0, 9), (2**64 - 1, 123)),
                                     ((17, 3, 0, 0), (20170823, 0))])
def test_philox_matches_numpy(ctr, key):
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(8)]
    c1 = _next(ctr)
    c2 = _next(c1)
    assert list(oracle.philox4x64(c1, key)) + list(oracle.philox4x64(c2, key)) == raw


def test_inverse_cdf_power_of_two_weights():
    c = np.array([0.5, 0.0, -0.25, 0.25])
    W, total = oracle.sample_weights(c)
    assert W == [2**39, 0, 2**38, 2**38] and total == 2**40
    seed = 99
    d = oracle.sample_draws(c, 50, 3, seed)
    for s in range(3):
        for k in range(50):
            r = oracle.philox4x64((k, s, 0, 0), (seed, 0))[0]
            want = 0 if r < 2**63 else (2 if r < 3 * 2**62 else 3)
            assert d[s, k] == want


def test_weights_proportional_to_abs_c():
    c = hi.random_vector(500, seed=5)
    c[::7] = 0.0
    W, total = oracle.sample_weights(c)
    W = np.array(W, dtype=np.float64)
    assert np.all((W > 0) == (c != 0))
    a = np.abs(c)
    assert np.abs(W / W.max() - a / a.max()).max() < 2.0**-38


def test_weights_above_2_22_determinants_keep_the_sum_below_2_62():
    n = (1 << 22) + 5                      # ceil(log2 n) = 23: scale 2^39
    c = np.full(n, 1e-3)
    c[0] = -0.9
    c[7] = 0.0
    W, total = oracle.sample_weights(c)
    assert total < 2**62
    W = np.array(W, dtype=np.float64)
    assert 2.0**38 <= W.max() <= 2.0**39 and W[7] == 0.0 and W[W > 0].min() >= 1.0
    a = np.abs(c)
    assert np.abs(W / W.max() - a / a.max()).max() < 2.0**-37


def _expectation(inst, keys, c, e0, nd, eps2, eps2d):
    W, total = oracle.sample_weights(c)
    p = np.array([w / total for w in W])
    acc = np.zeros(2)
    for seq in itertools.product(range(len(keys)), repeat=nd):
        prob = np.prod(p[list(seq)])
        if prob == 0.0:
            continue
        idx, cnt = np.unique(seq, return_counts=True)
        acc += prob * np.array(oracle.pt2_sampled(inst, keys, c, idx, cnt, p, nd, eps2, eps2d, e0))
    return acc


@pytest.mark.parametrize("nalpha,nbeta,nd,eps2,eps2d", [(2, 2, 3, -1.0, 2e-2), (3, 1, 2, 1e-3, 5e-2),
                                                       (2, 2, 4, 0.0, 1e-2)])
def test_estimator_expectation_is_e2(nalpha, nbeta, nd, eps2, eps2d):
    inst = hi.random_tiny(5, nalpha, nbeta, 31 + nd)
    keys = hi.random_det_keys(5, nalpha, nbeta, 4, seed=40 + nd)
    c = hi.random_vector(4, seed=41 + nd)
    c[1] = 0.0        # never drawn; contributes nothing either way
    e0 = float(oracle.diag(inst, keys).min()) - 0.3
    got = _expectation(inst, keys, c, e0, nd, eps2, eps2d)
    want = [oracle.pt2(inst, keys, c, eps2, e0)[0], oracle.pt2(inst, keys, c, eps2d, e0)[0]]
    assert want[0] != want[1]
    assert np.abs(got - want).max() < 1e-12 * max(1.0, abs(want[0])), (got, want)


def test_single_determinant_sample_is_exact():
    inst = hi.random_tiny(5, 2, 2, 3)
    keys = hi.random_det_keys(5, 2, 2, 1, seed=4)
    c = np.array([1.0])
    e0 = float(oracle.diag(inst, keys)[0])
    est = oracle.pt2_sampled(inst, keys, c, [0], [5], [1.0], 5, 0.0, 1e-2, e0)
    want = [oracle.pt2(inst, keys, c, 0.0, e0)[0], oracle.pt2(inst, keys, c, 1e-2, e0)[0]]
    assert np.abs(np.array(est) - want).max() < 1e-13 * abs(want[0])


@pytest.fixture(scope="module")
def poly8():
    inst = hi.ppp_polyene(8)
    out = oracle.hci(inst, 1e-3)
    return inst, out


def test_equal_thresholds_leave_deterministic(poly8):
    inst, out = poly8
    r = oracle.pt2_semistochastic(inst, out["keys"], out["c"], out["E"], 1e-4, 1e-4, 20, 5, 7)
    assert r["estimate"] == r["e2_det"] and r["error"] == 0.0
    assert np.array_equal(r["samples"][:, 0], r["samples"][:, 1])


def test_sample_means_agree_with_e2(poly8):
    inst, out = poly8
    eps2, eps2d = 1e-6, 3e-5
    r = oracle.pt2_semistochastic(inst, out["keys"], out["c"], out["E"], eps2, eps2d, 40, 300, 1708)
    e2 = oracle.pt2(inst, out["keys"], out["c"], eps2, out["E"])[0]
    e2d = oracle.pt2(inst, out["keys"], out["c"], eps2d, out["E"])[0]
    s = r["samples"]
    se = s.std(axis=0, ddof=1) / np.sqrt(len(s))
    assert abs(s[:, 0].mean() - e2) < 5 * se[0]
    assert abs(s[:, 1].mean() - e2d) < 5 * se[1]
    assert abs(r["estimate"] - e2) < 5 * r["error"]
    # the correlated difference is far less noisy than either estimate
    assert e2d != 0.0 and r["error"] < 0.5 * se[0]
    assert r["draws"].min() >= 0 and r["draws"].max() < len(out["keys"])
