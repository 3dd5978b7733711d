"""Failure paths of the C ABI, provoked on the host only (no device fault,
trap or hang is ever caused):

* allocation failure: with HCI_FAIL_ALLOC_AFTER=k the context refuses its
  (k+1)-th device allocation as if the device were out of memory.  Every
  allocating entry point is swept over k = 0, 1, 2, ... until it succeeds:
  each refusal must come back as HCI_ERR_NOMEM with a message, leave the
  context destroyable, and the first success must give the result of an
  unrestricted run;
* Davidson and the z-vector solve stopped at their iteration limit return
  HCI_ERR_NOT_CONVERGED with the last iterate (a normalised vector whose
  Rayleigh quotient lies above the converged energy); Davidson also stops,
  with the exact pair, when its correction falls inside an exhausted
  subspace;
* checkpoint and resume of the selection loop (Sec. II.A: V^{mu+1} depends
  only on V^mu and c^mu): a state saved to host memory at some mu and
  resumed in a fresh context reaches the uninterrupted solve's space and
  energy.
"""
import os

import numpy as np
import pytest

import hci_inputs as hi

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ENV = "HCI_FAIL_ALLOC_AFTER"


@pytest.fixture(scope="module")
def pkg():
    from paper_1708_07544_gb300 import build

    build.build()
    import paper_1708_07544_gb300 as p

    return p


@pytest.fixture()
def inst():
    return hi.ppp_polyene(8)


def _solver(pkg, inst):
    return pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, torch.tensor(inst.h).cuda(),
                         torch.tensor(inst.eri).cuda(), inst.e_core)


def _space(pkg, inst):
    with _solver(pkg, inst) as s:
        out = s.solve(1e-3)
    return out["keys"], out["c"], out["E"]


def _calls(pkg, inst, keys, c, E):
    """name -> function(solver) returning a comparable result."""
    return {
        "select": lambda s: s.select(1e-4, keys, c).cpu().numpy(),
        "sigma": lambda s: s.sigma(keys, c).cpu().numpy(),
        "davidson": lambda s: np.array([s.davidson(keys, None)[0]]),
        "rdm12": lambda s: torch.cat([t.flatten() for t in s.rdm12(keys, c)]).cpu().numpy(),
        "solve": lambda s: np.array([s.solve(1e-3)["E"]]),
        "pt2": lambda s: np.array(s.pt2(keys, c, 1e-5, E), dtype=np.float64),
        "pt2_rdms": lambda s: np.concatenate([np.array(s.pt2(keys, c, 1e-5, E, rdms=True)[:2], np.float64)]),
        "pt2_stochastic": lambda s: np.array([s.pt2_semistochastic(keys, c, E, 1e-6, 1e-5, 50, 3, seed=3)["estimate"]]),
        "relaxed_rdm12": lambda s: s.relaxed_rdm12(keys, c, E, 1e-5)[1].cpu().numpy(),
        "davidson_roots": lambda s: np.array(s.davidson_roots(keys, 2)[0]),
        "solve_roots": lambda s: np.array(s.solve_roots(2, 1e-3)["E"]),
        "direct_sigma": lambda s: (s.set_sigma_mode(pkg._abi.SIGMA_DIRECT), s.sigma(keys, c).cpu().numpy())[1],
    }


def test_every_allocating_entry_point_reports_nomem(pkg, inst):
    keys, c, E = _space(pkg, inst)
    calls = _calls(pkg, inst, keys, c, E)
    want = {}
    for name, fn in calls.items():
        with _solver(pkg, inst) as s:
            want[name] = fn(s)
    try:
        for name, fn in calls.items():
            refused = 0
            for k in range(0, 2000):
                os.environ[ENV] = str(k)
                try:
                    s = _solver(pkg, inst)
                except pkg.HCIError as e:
                    assert e.status == pkg._abi.HCI_ERR_NOMEM and "injected" in str(e), (name, k, str(e))
                    refused += 1
                    continue
                try:
                    got = fn(s)
                except pkg.HCIError as e:
                    assert e.status == pkg._abi.HCI_ERR_NOMEM and "injected" in str(e), (name, k, str(e))
                    refused += 1
                    continue
                finally:
                    s.close()
                np.testing.assert_allclose(got, want[name], rtol=1e-9, atol=1e-10, err_msg=name)
                break
            else:
                pytest.fail(f"{name}: no success within 2000 allocations")
            assert refused > 3, name
    finally:
        os.environ.pop(ENV, None)
    # the library works as before once the variable is gone
    with _solver(pkg, inst) as s:
        assert abs(s.solve(1e-3)["E"] - E) < 1e-10


def test_rotation_allocation_failure(pkg, inst):
    n = inst.norb
    kap = torch.tensor(hi.random_kappa(n, seed=3, sigma=0.05)).cuda()
    h = torch.tensor(inst.h).cuda()
    eri = torch.tensor(inst.eri).cuda()
    ref = pkg.hci_rotate(kap, h, eri)
    try:
        for k in range(0, 64):
            os.environ[ENV] = str(k)
            try:
                out = pkg.hci_rotate(kap, h, eri)
            except pkg.HCIError as e:
                assert e.status == pkg._abi.HCI_ERR_NOMEM and "injected" in str(e)
                continue
            assert k > 0
            assert all(torch.equal(a, b) for a, b in zip(out, ref))
            break
        else:
            pytest.fail("rotation never succeeded")
        os.environ[ENV] = "0"
        with pytest.raises(pkg.HCIError) as ei:
            pkg.hci_rotate_backward(kap, h, eri, torch.eye(n, dtype=torch.float64).cuda(),
                                    torch.zeros((n,) * 4, dtype=torch.float64).cuda())
        assert ei.value.status == pkg._abi.HCI_ERR_NOMEM
    finally:
        os.environ.pop(ENV, None)


def test_davidson_stopped_at_its_limit(pkg, inst):
    keys, c, E = _space(pkg, inst)
    with _solver(pkg, inst) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.davidson(keys, None, tol=1e-13, maxit=1)
        assert ei.value.status == pkg._abi.HCI_ERR_NOT_CONVERGED
        e1, c1, it = s.davidson(keys, None, tol=1e-13, maxit=2, allow_unconverged=True)
        assert it == 2
        assert abs(torch.linalg.norm(c1).item() - 1.0) < 1e-12
        assert e1 > E + 1e-6                    # Rayleigh quotient of a non-converged vector
        # the whole loop reports it too
        with pytest.raises(pkg.HCIError) as ej:
            s.solve(1e-3, dav_tol=1e-13, dav_maxit=1)
        assert ej.value.status == pkg._abi.HCI_ERR_NOT_CONVERGED
        # z-vector: one CG step is not enough
        rhs = torch.randn(keys.shape[0], dtype=torch.float64, device="cuda")
        with pytest.raises(pkg.HCIError) as ez:
            s.zvector(keys, c, E, rhs, tol=1e-13, maxit=1)
        assert ez.value.status == pkg._abi.HCI_ERR_NOT_CONVERGED


def test_davidson_stops_when_the_subspace_is_exhausted(pkg, inst):
    """With tol = 0 the residual test never succeeds; once the subspace
    spans the whole (small) space the next correction lies inside it and
    Davidson stops there (not at maxit) with the exact lowest eigenpair,
    reported as HCI_ERR_NOT_CONVERGED."""
    import oracle

    keys = hi.random_det_keys(inst.norb, inst.nalpha, inst.nbeta, 12, seed=77)
    want = np.linalg.eigvalsh(oracle.hamiltonian(inst, keys).toarray())[0]
    kd = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64).reshape(-1, 2)).cuda()
    with _solver(pkg, inst) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.davidson(kd, None, tol=0.0, maxit=100)
        assert ei.value.status == pkg._abi.HCI_ERR_NOT_CONVERGED
        e, c, it = s.davidson(kd, None, tol=0.0, maxit=100, allow_unconverged=True)
    assert it < 100
    assert abs(e - want) < 1e-12
    H = oracle.hamiltonian(inst, keys)
    c = c.cpu().numpy()
    assert abs(np.linalg.norm(c) - 1.0) < 1e-12
    assert np.abs(H @ c - want * c).max() < 1e-10


@pytest.mark.parametrize("stop", [1, 3])
def test_resume_from_saved_state(pkg, stop):
    inst = hi.df_12o()
    eps1 = 3e-4
    with _solver(pkg, inst) as s:
        full = s.solve(eps1)
    # the same loop stepped by hand up to mu = stop, saved to host memory
    with _solver(pkg, inst) as s:
        a0, b0 = (1 << inst.nalpha) - 1, (1 << inst.nbeta) - 1
        keys = torch.tensor([[a0, b0]], dtype=torch.int64).cuda()
        c = torch.ones(1, dtype=torch.float64).cuda()
        for _ in range(stop):
            new = s.select(eps1, keys, c)
            assert new.shape[0] > 0
            keys, c0 = s.merge(keys, c, new)
            _, c, _ = s.davidson(keys, c0)
        saved = (keys.cpu().numpy().copy(), c.cpu().numpy().copy())
    with _solver(pkg, inst) as s2:
        res = s2.solve_from(torch.from_numpy(saved[0]).cuda(), torch.from_numpy(saved[1]).cuda(), eps1)
    assert torch.equal(res["keys"].cpu(), full["keys"].cpu())
    assert abs(res["E"] - full["E"]) < 1e-9
    assert res["iters"] == full["iters"] - stop
    # resuming from the converged state selects nothing and returns its energy
    with _solver(pkg, inst) as s3:
        again = s3.solve_from(full["keys"], full["c"], eps1)
    assert again["iters"] == 0 and torch.equal(again["keys"].cpu(), full["keys"].cpu())
    assert abs(again["E"] - full["E"]) < 1e-10


def test_resume_rejects_unsorted_start(pkg, inst):
    keys, c, E = _space(pkg, inst)
    with _solver(pkg, inst) as s:
        with pytest.raises(pkg.HCIError) as ei:
            s.solve_from(keys.flip(0).contiguous(), c, 1e-3)
        assert ei.value.status == pkg._abi.HCI_ERR_INVALID
