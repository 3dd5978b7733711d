"""The allocation-free rotation entry point, called through the C ABI.

hci_rotate_noalloc serves callers that cannot allocate device memory when
they rotate the integrals (a host thread inside another framework's memory
pool, or one that must not let cudaMalloc/cudaFree synchronise the device).
It must return what hci_rotate returns, on consecutive calls that share its
static scratch array, and reject sizes beyond that array.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import hci_inputs as hi

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12     # the rotation tests' bar against the oracle


@pytest.fixture(scope="module")
def lib():
    from paper_1708_07544_gb300 import build

    build.build()
    from paper_1708_07544_gb300 import _abi

    return _abi.load()


def _call(fn, n, kap, h, eri):
    U = torch.empty_like(h)
    h2 = torch.empty_like(h)
    e2 = torch.empty_like(eri)
    st = fn(n, kap.data_ptr(), h.data_ptr(), eri.data_ptr(), U.data_ptr(), h2.data_ptr(), e2.data_ptr(),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, U, h2, e2


def test_noalloc_rotation_matches_allocating_entry_point(lib):
    cases = [(12, 101, 0.2), (32, 202, 0.05)]      # two calls in a row, the second at the size limit
    for n, seed, sigma in cases:
        inst = hi.df_instance(n, 2 * n, seed=seed, name=f"df{n}")
        kap = torch.tensor(hi.random_kappa(n, seed=seed + 1, sigma=sigma)).cuda()
        h = torch.tensor(inst.h).cuda()
        eri = torch.tensor(inst.eri).cuda()
        st_ref, U_ref, h_ref, e_ref = _call(lib.hci_rotate, n, kap, h, eri)
        assert st_ref == 0
        st, U, h2, e2 = _call(lib.hci_rotate_noalloc, n, kap, h, eri)
        assert st == 0, lib.hci_last_error(None)
        assert torch.max(torch.abs(U - U_ref)).item() < TOL
        assert torch.max(torch.abs(h2 - h_ref)).item() < TOL
        assert torch.max(torch.abs(e2 - e_ref)).item() < TOL


def test_noalloc_rotation_rejects_oversize(lib):
    n = 33
    z = torch.zeros((n, n), dtype=torch.float64).cuda()
    e = torch.zeros((n,) * 4, dtype=torch.float64).cuda()
    st, *_ = _call(lib.hci_rotate_noalloc, n, z, z, e)
    assert st == 1
    assert b"outside [1,32]" in lib.hci_last_error(None)
