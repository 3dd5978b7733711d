"""Full-size workloads (the sizes bench.py times), checked where the oracle
can follow: sampled rows of H c, the selection criterion on sampled
sources (a converged space yields no new determinant, Sec. II.A), the RDM
invariants and E = sum h rdm1 + 1/2 sum (pq|rs) rdm2 (Sec. IV), and the
vHCISCF gradient (Eq. vdedk2) against central finite differences at fixed V
and against the oracle's chain rule applied to the GPU RDMs, and the
perturbative correction's independence of its hash-class split.
"""
import numpy as np
import pytest

import hci_inputs as hi
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

E_TOL = 1e-9
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


def host_keys(t):
    return t.cpu().numpy().view(np.uint64).reshape(-1, 2)


def solve(pkg, inst, eps1, kap):
    h = torch.tensor(inst.h).cuda()
    eri = torch.tensor(inst.eri).cuda()
    k = torch.tensor(kap).cuda()
    _, h2, e2 = pkg.hci_rotate(k, h, eri)
    s = pkg.HCISolver(inst.norb, inst.nalpha, inst.nbeta, h2, e2, inst.e_core)
    out = s.solve(eps1, dav_tol=1e-10, cap=1 << 22)
    R, _ = oracle.rotate(inst, kap)
    return s, out, R, (h, eri, k)


def check_space(pkg, s, out, R, eps1, nrows=24, nsrc=48):
    keys_d, c_d = out["keys"], out["c"]
    keys = host_keys(keys_d)
    c = c_d.cpu().numpy()
    nV = len(keys)
    # sampled rows of H c against the oracle's row-by-row enumeration
    sig = s.sigma(keys_d, c_d).cpu().numpy()
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([np.argsort(-np.abs(c))[:4], rng.choice(nV, nrows, replace=False)]))
    ref = oracle.sigma_rows(R, keys, c, rows)
    assert np.abs(sig[rows] - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
    # eigenpair: residual and Rayleigh quotient
    e = float(c @ sig)
    assert abs(e - out["E"]) < E_TOL
    assert np.linalg.norm(sig - out["E"] * c) < 1e-8
    # convergence of the selection: sampled sources generate nothing new
    src = np.unique(np.concatenate([np.argsort(-np.abs(c))[:nsrc // 2], rng.choice(nV, nsrc // 2, replace=False)]))
    new, _, ties = oracle.select(R, keys, c, eps1, sources=src)
    tie = {tuple(x) for x in ties.tolist()}
    assert {tuple(x) for x in new.tolist()} - tie == set()
    # RDM invariants and the energy expression
    r1, r2 = s.rdm12(keys_d, c_d)
    r1, r2 = r1.cpu().numpy(), r2.cpu().numpy()
    N = R.nalpha + R.nbeta
    assert abs(np.trace(r1) - N) < RDM_TOL
    assert abs(np.einsum("pprr->", r2) - N * (N - 1)) < 1e-6
    assert np.abs(np.einsum("pqrr->pq", r2) - (N - 1) * r1).max() < 1e-7
    assert np.abs(r1 - r1.T).max() < RDM_TOL
    assert np.abs(r2 - r2.transpose(2, 3, 0, 1)).max() < RDM_TOL
    assert np.abs(r2 - r2.transpose(1, 0, 3, 2)).max() < RDM_TOL
    assert abs(oracle.energy_from_rdm(R, r1, r2) - out["E"]) < E_TOL
    return r1, r2


def test_pentacene22_full(pkg):
    inst = hi.ppp_pentacene()
    kap = np.zeros((22, 22))
    s, out, R, _ = solve(pkg, inst, 5e-5, kap)
    try:
        assert out["keys"].shape[0] > 300000
        check_space(pkg, s, out, R, 5e-5)
    finally:
        s.close()


def test_df44_bench_configuration(pkg):
    inst = hi.df_44o()
    kap = hi.random_kappa(44, seed=1709, sigma=0.01)
    s, out, R, (h, eri, k) = solve(pkg, inst, 1e-4, kap)
    try:
        assert 1e6 < out["keys"].shape[0] < 1e7
        r1, r2 = check_space(pkg, s, out, R, 1e-4, nrows=8, nsrc=16)
        # perturbative correction at eps2 = 1e-5 (Sec. II.B, Eq. pt_hci): the
        # same sum when the targets are split into many hash classes; a
        # looser eps2 keeps fewer targets and a smaller |E2|
        e2, n2 = s.pt2(out["keys"], out["c"], 1e-5, out["E"])
        e2m, n2m = s.pt2(out["keys"], out["c"], 1e-5, out["E"], max_pairs=1 << 22)
        e2l, n2l = s.pt2(out["keys"], out["c"], 3e-5, out["E"])
        assert abs(e2m - e2) < 1e-12 * abs(e2) and n2m == n2
        assert e2 < e2l < 0.0 and n2l < n2
        # its density matrices (Sec. V): tr Gamma^dc_1 = N <c|d> = 0,
        # sum_pr Gamma^dd_pprr = (N - 1) tr Gamma^dd_1, Gamma^dd_1 symmetric
        e2r, n2r, (r1dd, r2dd, r1dc, r2dc) = s.pt2(out["keys"], out["c"], 1e-5, out["E"], rdms=True)
        assert abs(e2r - e2) < 1e-12 * abs(e2) and n2r == n2
        r1dd, r2dd, r1dc = r1dd.cpu().numpy(), r2dd.cpu().numpy(), r1dc.cpu().numpy()
        N = R.nalpha + R.nbeta
        assert np.trace(r1dd) > 0.0 and abs(np.trace(r1dc)) < 1e-10
        assert abs(np.einsum("pprr->", r2dd) - (N - 1) * np.trace(r1dd)) < 1e-8 * N * N * np.trace(r1dd)
        assert np.abs(r1dd - r1dd.T).max() < 1e-12
        # semistochastic E2(1e-5) from E2^D(3e-5) (Eq. semistoc): within five
        # standard errors of the deterministic value; one sample of 200
        # draws against the oracle on the same draws
        keys_h = out["keys"].cpu().numpy().view(np.uint64).reshape(-1, 2)
        c_h = out["c"].cpu().numpy()
        r = s.pt2_semistochastic(out["keys"], out["c"], out["E"], 1e-5, 3e-5, 1000, 12, seed=11)
        assert abs(r["e2_det"] - e2l) <= 1e-12 * abs(e2l)
        assert r["error"] > 0.0 and abs(r["estimate"] - e2) < 5 * r["error"]
        one = s.pt2_semistochastic(out["keys"], out["c"], out["E"], 1e-5, 3e-5, 200, 1, seed=12)
        d = oracle.sample_draws(c_h, 200, 1, 12)
        assert np.array_equal(one["draws"].cpu().numpy(), d)
        W, tot = oracle.sample_weights(c_h)
        p = np.array(W, np.float64) / float(tot)
        idx, cnt = np.unique(d[0], return_counts=True)
        want = oracle.pt2_sampled(R, keys_h, c_h, idx, cnt, p, 200, 1e-5, 3e-5, out["E"])
        assert np.abs(one["samples"][0] - want).max() <= 1e-10 * abs(want[0])
    finally:
        s.close()
    # backward through the rotation against the oracle's chain rule on the same RDMs
    dh, de, dk = pkg.hci_rotate_backward(k, h, eri, torch.tensor(r1).cuda(), torch.tensor(r2).cuda())
    g = oracle.gradient(inst, kap, r1, r2)
    assert np.abs(dk.cpu().numpy() - g["dkappa"]).max() < 1e-8


def test_df12_gradient_full_size_fd(pkg):
    """(12e,12o) DF at eps1 = 1e-4: dE/dkappa from the RDM backward equals
    central finite differences (step 1e-5) of the energy at fixed V."""
    inst = hi.df_12o()
    kap = hi.random_kappa(12, seed=1709, sigma=0.01)
    s, out, R, (h, eri, k) = solve(pkg, inst, 1e-4, kap)
    keys_d = out["keys"]
    try:
        r1, r2 = s.rdm12(keys_d, out["c"])
    finally:
        s.close()
    _, _, dk = pkg.hci_rotate_backward(k, h, eri, r1, r2)
    dk = dk.cpu().numpy()
    g = oracle.gradient(inst, kap, r1.cpu().numpy(), r2.cpu().numpy())["dkappa"]
    assert np.abs(dk - g).max() < 1e-8
    step = 1e-5
    for p, q in [(0, 7), (3, 9), (5, 6)]:
        vals = []
        for sg in (1, -1):
            d = kap.copy()
            d[p, q] += sg * step
            d[q, p] -= sg * step
            _, h2, e2 = pkg.hci_rotate(torch.tensor(d).cuda(), h, eri)
            with pkg.HCISolver(12, 6, 6, h2, e2, 0.0) as s2:
                vals.append(s2.davidson(keys_d, out["c"], tol=1e-11)[0])
        fd = (vals[0] - vals[1]) / (2 * step)
        an = dk[p, q] - dk[q, p]
        assert abs(fd - an) < 1e-6, (p, q, fd, an)
