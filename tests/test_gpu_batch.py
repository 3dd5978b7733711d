"""Batched solve of uneven active spaces against one-at-a-time solves."""
import numpy as np
import pytest

import hci_inputs as hi

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_1708_07544_gb300 import build

    build.build()
    import paper_1708_07544_gb300 as p

    return p


def _lst(insts):
    return [(i.norb, i.nalpha, i.nbeta, torch.tensor(i.h).cuda(), torch.tensor(i.eri).cuda(), i.e_core)
            for i in insts]


def test_batch_equals_individual_solves(pkg):
    insts = hi.df_batch(64)[:10] + [hi.ppp_polyene(8)]
    lst = _lst(insts)
    en4, nv4, r1, r2 = pkg.hci_solve_batch(lst, 1e-4, dav_tol=1e-10, nstreams=4, want_rdm=True)
    en1, nv1, _, _ = pkg.hci_solve_batch(lst, 1e-4, dav_tol=1e-10, nstreams=1)
    assert np.array_equal(nv4, nv1)
    assert np.abs(en4 - en1).max() < 1e-9
    for k in (0, 5, 10):
        n, na, nb, h, eri, ec = lst[k]
        with pkg.HCISolver(n, na, nb, h, eri, ec) as s:
            out = s.solve(1e-4, dav_tol=1e-10)
            g1, g2 = s.rdm12(out["keys"], out["c"])
        assert out["keys"].shape[0] == nv4[k]
        assert abs(out["E"] - en4[k]) < 1e-9
        assert torch.max(torch.abs(g1 - r1[k])).item() < 1e-8
        assert torch.max(torch.abs(g2 - r2[k])).item() < 1e-8


def test_batch_reports_a_failing_instance(pkg):
    insts = hi.df_batch(64)[:3]
    lst = _lst(insts)
    n, na, nb, h, eri, ec = lst[1]
    lst[1] = (n, n + 1, nb, h, eri, ec)       # more electrons than orbitals
    with pytest.raises(pkg.HCIError) as ei:
        pkg.hci_solve_batch(lst, 1e-4, nstreams=2)
    assert "instance 1" in str(ei.value)


def test_batch_matches_oracle(pkg):
    """Three instances of the uneven batch (norb 10, 17 and 24) solved
    concurrently: energies within 1e-9 Ha, space sizes equal and RDMs within
    1e-8 of the oracle's HCI (Sec. II.A) and RDMs (Sec. IV); the selected
    sets of the same instances (single-instance solves, which the batch
    reproduces above) equal the oracle's."""
    import oracle

    allb = hi.df_batch(64)
    insts = [allb[0], allb[7], allb[59]]
    assert [i.norb for i in insts] == [10, 17, 24]
    lst = _lst(insts)
    en, nv, r1, r2 = pkg.hci_solve_batch(lst, 1e-4, dav_tol=1e-10, nstreams=3, want_rdm=True)
    for k, inst in enumerate(insts):
        ref = oracle.hci(inst, 1e-4)
        assert nv[k] == len(ref["keys"]), (k, nv[k], len(ref["keys"]))
        assert abs(en[k] - ref["E"]) < 1e-9, (k, en[k], ref["E"])
        w1, w2 = oracle.rdm12(inst.norb, ref["keys"], ref["c"])
        assert np.abs(r1[k].cpu().numpy() - w1).max() < 1e-8
        assert np.abs(r2[k].cpu().numpy() - w2).max() < 1e-8
        n, na, nb, h, eri, ec = lst[k]
        with pkg.HCISolver(n, na, nb, h, eri, ec) as s:
            out = s.solve(1e-4, dav_tol=1e-10)
        got = out["keys"].cpu().numpy().view(np.uint64).reshape(-1, 2)
        assert np.array_equal(got, ref["keys"])
