"""hci_qtrans, one quarter transform of the integral rotation (Sec. III.A),
out[J*n + p] = sum_a in[a*n^3 + J] M[a*n + p], on the bf16 tensor cores as
exact products of balanced 8-bit digits rounded once to FP64:

* integer inputs whose products and sums are exact in FP64 come back
  bit-exact (every padded width 16/32/48/64, ragged last tiles, n = 1);
* general inputs, with row scales spread over 60 orders of magnitude, stay
  within 2^-50 n max_a|in[a][J]| max_a|M[a][p]| of the FP64 result (the
  normwise bound of the digit truncation plus FP64's own rounding);
* zero rows give zeros, subnormal entries count as zero, a lone huge entry
  does not disturb the other rows;
* n outside [1, 64] and null pointers are refused.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1708_07544_gb300 import build

    build.build()
    import paper_1708_07544_gb300 as p

    return p


def _ref(inp, M):
    n = M.shape[0]
    return np.einsum("aJ,ap->Jp", inp.reshape(n, n ** 3), M).reshape(-1)


def _run(pkg, inp, M):
    return pkg.hci_qtrans(torch.tensor(inp).cuda(), torch.tensor(M).cuda()).cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 33, 48, 49, 64])
def test_integer_inputs_bit_exact(pkg, n):
    rng = np.random.default_rng(n)
    inp = rng.integers(-1000, 1001, size=n ** 4).astype(np.float64)
    M = rng.integers(-50, 51, size=(n, n)).astype(np.float64)
    got = _run(pkg, inp, M)
    assert np.array_equal(got, _ref(inp, M))


@pytest.mark.parametrize("n", [5, 17, 44, 49])
def test_general_inputs_within_normwise_bound(pkg, n):
    rng = np.random.default_rng(100 + n)
    inp = rng.standard_normal((n, n ** 3)) * 10.0 ** rng.uniform(-30, 30, size=n ** 3)[None, :]
    M = rng.standard_normal((n, n))
    got = _run(pkg, inp.reshape(-1), M).reshape(n ** 3, n)
    want = _ref(inp.reshape(-1), M).reshape(n ** 3, n)
    bound = 2.0 ** -50 * n * np.abs(inp).max(axis=0)[:, None] * np.abs(M).max(axis=0)[None, :]
    assert np.all(np.abs(got - want) <= bound)


def test_zero_subnormal_and_isolated_rows(pkg):
    n = 20
    rng = np.random.default_rng(7)
    inp = rng.standard_normal((n, n ** 3))
    inp[:, 5] = 0.0                         # a zero row (J = 5)
    inp[:, 6] = 1e-310                      # subnormal entries count as zero
    inp[3, 7] = 1e300                       # one huge entry in row J = 7
    M = rng.standard_normal((n, n))
    got = _run(pkg, inp.reshape(-1), M).reshape(n ** 3, n)
    want = _ref(inp.reshape(-1), M).reshape(n ** 3, n)
    assert np.all(got[5] == 0.0) and np.all(got[6] == 0.0)
    assert np.abs(got[7] - want[7]).max() <= 2.0 ** -50 * n * 1e300 * np.abs(M).max()
    rest = np.ones(n ** 3, bool)
    rest[[5, 6, 7]] = False
    assert np.abs(got[rest] - want[rest]).max() <= 2.0 ** -50 * n * np.abs(inp).max() * np.abs(M).max()


def test_refusals(pkg):
    from paper_1708_07544_gb300 import _abi

    L = _abi.load()
    x = torch.zeros(16, dtype=torch.float64).cuda()
    for n in (0, 65):
        assert L.hci_qtrans(n, x.data_ptr(), x.data_ptr(), x.data_ptr(), 1, None) == _abi.HCI_ERR_INVALID
    assert L.hci_qtrans(2, None, x.data_ptr(), x.data_ptr(), 1, None) == _abi.HCI_ERR_INVALID
    assert b"hci_qtrans" in L.hci_last_error(None)
