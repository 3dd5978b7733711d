"""Plain CPU oracle for the variational HCI solve of arXiv:1708.07544.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py may import this package.  It
shares no code with the CUDA library and never imports it.

What each function follows:

* ``select``      -- Eq. (criteria) with the HCI importance function
                     f(D_a) = max_i |H_ai c_i| (Sec. II.A), by enumerating
                     every single and double of every D_i (liborc_hci.so).
* ``hamiltonian`` -- Slater-Condon matrix elements on V (Sec. II.A; the
                     rules are pinned by the Jordan-Wigner FCI in fci_jw.py).
* ``ground_state``-- minimum of the energy functional Eq. (variational)
                     on a fixed V (a library eigensolver stands in for
                     Davidson: the result is the same lowest eigenpair).
* ``hci``         -- the variational stage V^{mu+1} = V^mu + C^mu(eps1)
                     (Sec. II.A, Fig. 1) iterated until C^mu is empty;
                     ``hci_roots`` the same for several lowest states.
* ``rdm12``       -- the variational RDMs by their definition (Sec. IV).
* ``pt2``         -- the screened Epstein-Nesbet correction E2(eps2),
                     Eq. (pt_hci) of Sec. II.B, by enumerating every single
                     and double of every D_i (terms with |H_ai c_i| > eps2
                     kept; pinned against numerators taken from the
                     Jordan-Wigner FCI matrix); ``pt2_rdm`` its density
                     matrices Gamma^dd and Gamma^dc by their definition.
* ``pt2_semistochastic`` -- Eq. (semistoc): E2^D(eps2_det) plus the mean
                     over samples of E2^S(eps2) - E2^S(eps2_det), each
                     sample the unbiased multinomial estimator of the cited
                     semistochastic HCI work (``pt2_sampled``; pinned by its
                     exact expectation over every draw sequence), the draws
                     made by ``philox4x64`` (pinned against numpy's Philox)
                     and an exact integer inverse CDF (``sample_draws``).
* ``hci_parity`` -- the variational stage restricted to states of one spin
                     parity in the S_z = 0 sector (the singlet / triplet
                     states of Sec. VI told apart by the spin-flip symmetry
                     of the spin-free Hamiltonian): the space is closed under
                     exchanging the alpha and beta strings, and the state is
                     the lowest eigenvector of H in the subspace c(beta,
                     alpha) = p c(alpha, beta) (``parity_ground_state``,
                     pinned against Jordan-Wigner spectra sorted by S).
* ``rotate`` / ``gradient`` -- vHCISCF gradient Eq. (vdedk2): the
                     derivative of the rotated integrals contracted with
                     the RDMs, chained through U = exp(kappa) (Sec. III.B).

Readings where the paper is silent (strict '>', eps1 <= 0 accepts every
single/double, aufbau start, stop at an empty C^mu, phase of c, spin-summed
RDM order) are stated in the functions below.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        L.orc_diag.argtypes = [ctypes.c_int, P, P, d, P, i64, P]
        L.orc_hamiltonian.argtypes = [ctypes.c_int, P, P, d, P, i64]
        L.orc_hamiltonian.restype = P
        L.orc_csr_nnz.argtypes = [P]
        L.orc_csr_nnz.restype = i64
        L.orc_csr_copy.argtypes = [P, P, P, P]
        L.orc_csr_free.argtypes = [P]
        L.orc_sigma_rows.argtypes = [ctypes.c_int, P, P, d, P, i64, P, P, i64, P]
        L.orc_select.argtypes = [ctypes.c_int, P, P, P, P, i64, d, ctypes.c_int, P, i64]
        L.orc_select.restype = P
        L.orc_sel_count.argtypes = [P]
        L.orc_sel_count.restype = i64
        L.orc_sel_copy.argtypes = [P, P, P]
        L.orc_sel_free.argtypes = [P]
        L.orc_rdm12.argtypes = [ctypes.c_int, P, i64, P, P, P]
        L.orc_pt2.argtypes = [ctypes.c_int, P, P, d, P, P, i64, d, d, P, P]
        L.orc_pt2_rdm.argtypes = [ctypes.c_int, P, P, d, P, P, i64, d, d, P, P, P, P]
        L.orc_pt2_sampled.argtypes = [ctypes.c_int, P, P, d, P, i64, P, P, P, i64, i64, d, d, d, P]
        L.orc_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_lib().orc_num_threads())


class Problem:
    """Minimal view of an instance: norb, nalpha, nbeta, h, eri, e_core."""

    def __init__(self, norb, nalpha, nbeta, h, eri, e_core=0.0):
        self.norb, self.nalpha, self.nbeta = int(norb), int(nalpha), int(nbeta)
        self.h = _c(h, np.float64)
        self.eri = _c(eri, np.float64)
        self.e_core = float(e_core)

    @staticmethod
    def of(inst) -> "Problem":
        if isinstance(inst, Problem):
            return inst
        return Problem(inst.norb, inst.nalpha, inst.nbeta, inst.h, inst.eri, inst.e_core)


# ----------------------------------------------------------------------------
# determinant-level primitives (C++)
# ----------------------------------------------------------------------------

def diag(inst, keys) -> np.ndarray:
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    out = np.zeros(len(keys))
    _lib().orc_diag(P.norb, _p(P.h), _p(P.eri), P.e_core, _p(keys), len(keys), _p(out))
    return out


def hamiltonian(inst, keys) -> sp.csr_matrix:
    """<D_i|H|D_j> on V (Slater-Condon), E_core on the diagonal."""
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    L = _lib()
    h = L.orc_hamiltonian(P.norb, _p(P.h), _p(P.eri), P.e_core, _p(keys), len(keys))
    try:
        nnz = L.orc_csr_nnz(h)
        rp = np.zeros(len(keys) + 1, np.int64)
        col = np.zeros(nnz, np.int64)
        val = np.zeros(nnz)
        L.orc_csr_copy(h, _p(rp), _p(col), _p(val))
    finally:
        L.orc_csr_free(h)
    return sp.csr_matrix((val, col, rp), shape=(len(keys), len(keys)))


def sigma_rows(inst, keys, c, rows) -> np.ndarray:
    """(H c)_i for the listed rows, by enumerating the excitations of D_i."""
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    rows = _c(rows, np.int64)
    out = np.zeros(len(rows))
    _lib().orc_sigma_rows(P.norb, _p(P.h), _p(P.eri), P.e_core, _p(keys), len(keys), _p(c),
                          _p(rows), len(rows), _p(out))
    return out


def pt2(inst, keys, c, eps2, e0):
    """Screened second-order Epstein-Nesbet correction (Sec. II.B,
    Eq. pt_hci): E2 = sum over D_a outside V of (sum'_i H_ai c_i)^2 /
    (e0 - H_aa), the screened sum keeping the terms with |H_ai c_i| > eps2
    (strict, as for eps1).  Returns (E2, |C(eps2)|)."""
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    e2 = ctypes.c_double(0.0)
    n_ext = ctypes.c_int64(0)
    _lib().orc_pt2(P.norb, _p(P.h), _p(P.eri), P.e_core, _p(keys), _p(c), len(keys), float(eps2), float(e0),
                   ctypes.byref(e2), ctypes.byref(n_ext))
    return e2.value, n_ext.value


def pt2_rdm(inst, keys, c, eps2, e0):
    """Density matrices of the perturbative correction (Sec. V,
    Computational Details), spin-summed like rdm12:
    Gamma^dd = sum_a d_a^2 <D_a|op|D_a> and Gamma^dc = sum over the screened
    pairs of c_i d_a <D_i|op|D_a>, d_a = (sum'_i H_ai c_i) / (e0 - H_aa),
    the pairs being those of pt2 (|H_ai c_i| > eps2).  Returns
    (rdm1_dd, rdm2_dd, rdm1_dc, rdm2_dc)."""
    P = Problem.of(inst)
    n = P.norb
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    out = [np.zeros((n, n)), np.zeros((n,) * 4), np.zeros((n, n)), np.zeros((n,) * 4)]
    _lib().orc_pt2_rdm(n, _p(P.h), _p(P.eri), P.e_core, _p(keys), _p(c), len(keys), float(eps2), float(e0),
                       *[_p(x) for x in out])
    return tuple(out)


def spin_square(norb, keys, c):
    """<S^2> of the state sum_i c_i |D_i> (the spin of the states Sec. VI
    compares): S^2 = S_- S_+ + S_z (S_z + 1), with ||S_+ c||^2 evaluated by
    applying S_+ = sum_p a+_{p alpha} a_{p beta} to every determinant (alpha
    block then beta block, ascending: the sign of a+_{p alpha} a_{p beta} is
    (-1)^(n_alpha + #beta below p + #alpha below p)).  Small spaces only."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    c = np.asarray(c, np.float64)
    if len(keys) == 0:
        return 0.0
    na = bin(int(keys[0, 0])).count("1")
    nb = bin(int(keys[0, 1])).count("1")
    out = {}
    for (ka, kb), ci in zip(keys.tolist(), c.tolist()):
        if ci == 0.0:
            continue
        for p in range(norb):
            if not (kb >> p) & 1 or (ka >> p) & 1:
                continue
            below = (1 << p) - 1
            sgn = -1.0 if (na + bin(kb & below).count("1") + bin(ka & below).count("1")) % 2 else 1.0
            t = (ka | (1 << p), kb & ~(1 << p))
            out[t] = out.get(t, 0.0) + sgn * ci
    sz = 0.5 * (na - nb)
    return float(sum(v * v for v in out.values()) + sz * (sz + 1.0) * float(c @ c))


# ----------------------------------------------------------------------------
# semistochastic second-order correction (Sec. II.B, Eq. semistoc)
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def philox4x64(ctr, key, rounds=10):
    """Philox4x64-R counter-based generator (Salmon, Moraes, Dror, Shaw,
    SC'11), from its published definition: each round multiplies words 0
    and 2 by two fixed odd constants into 128-bit products and mixes the
    halves with words 1 and 3 and the key; the key is bumped by two Weyl
    constants between rounds.  ctr: 4 words, key: 2 words (ints < 2^64)."""
    c0, c1, c2, c3 = (int(x) & _M64 for x in ctr)
    k0, k1 = (int(x) & _M64 for x in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + 0x9E3779B97F4A7C15) & _M64
            k1 = (k1 + 0xBB67AE8584CAA73B) & _M64
        p0 = 0xD2E7470EE14C6C93 * c0
        p1 = 0xCA5A826395121157 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & _M64, (p0 >> 64) ^ c3 ^ k1, p0 & _M64)
    return c0, c1, c2, c3


def sample_weights(c):
    """Integer sampling weights W_i proportional to |c_i| (reading: p_i =
    |c_i| / sum_j |c_j| to 2^-B relative): W_i = ceil(|c_i| 2^(B - E))
    with 2^(E-1) <= max|c| < 2^E, B = 40 for up to 2^22 determinants and
    62 - ceil(log2 n) above (so that the sum stays below 2^62); every
    non-zero c_i has W_i >= 1 and the weights and their prefix sums are
    exact integers in any order.  Returns (W as Python ints, total)."""
    a = np.abs(np.asarray(c, np.float64))
    if a.size == 0 or a.max() == 0.0:
        return [0] * a.size, 0
    lg = 0
    while (1 << lg) < a.size:
        lg += 1
    B = 40 if lg <= 22 else 62 - lg
    e = int(np.frexp(a.max())[1])
    W = [int(x) for x in np.ceil(np.ldexp(a, B - e))]
    return W, sum(W)


def sample_draws(c, n_draws, n_samples, seed):
    """Draw k of sample s: r = first word of philox4x64((k, s, 0, 0),
    (seed, 0)), u = floor(r * total / 2^64) in [0, total), and the drawn
    index is the first i whose inclusive prefix sum of W exceeds u, so D_i
    is drawn with probability W_i / total.  Returns an int64 array
    (n_samples, n_draws)."""
    W, total = sample_weights(c)
    cum = np.cumsum(np.array(W, dtype=np.int64))      # exact: total < 2^63
    out = np.zeros((n_samples, n_draws), np.int64)
    for s in range(n_samples):
        for k in range(n_draws):
            r = philox4x64((k, s, 0, 0), (int(seed), 0))[0]
            u = (r * total) >> 64
            out[s, k] = int(np.searchsorted(cum, np.int64(u), side="right"))
    return out


def pt2_sampled(inst, keys, c, idx, counts, p, n_draws, eps2, eps2_det, e0):
    """One sample of the stochastic correction: the distinct drawn
    determinants idx (into V), drawn counts[j] times out of n_draws with
    probability p[idx[j]].  Returns (E2^S(eps2), E2^S(eps2_det)), the
    unbiased estimates of E2 with each screen (orc_pt2_sampled)."""
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    idx = _c(idx, np.int64)
    f = _c(np.asarray(counts, np.float64) / np.asarray(p, np.float64)[idx], np.float64)
    sk = _c(keys[idx], np.uint64)
    sc = _c(c[idx], np.float64)
    out = np.zeros(2)
    _lib().orc_pt2_sampled(P.norb, _p(P.h), _p(P.eri), P.e_core, _p(keys), len(keys), _p(sk), _p(sc), _p(f),
                           len(idx), int(n_draws), float(eps2), float(eps2_det), float(e0), _p(out))
    return float(out[0]), float(out[1])


def pt2_semistochastic(inst, keys, c, e0, eps2, eps2_det, n_draws, n_samples, seed):
    """Eq. (semistoc): E2 ~ E2^D(eps2_det) + mean_s [E2^S_s(eps2) -
    E2^S_s(eps2_det)], both stochastic terms of a sample from the same
    draws; the error is the standard error of that mean.  Returns a dict
    with estimate, error, e2_det, samples (n_samples x 2) and draws."""
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    e2d, _ = pt2(inst, keys, c, eps2_det, e0)
    W, total = sample_weights(c)
    p = np.array([w / total for w in W]) if total else np.zeros(len(W))
    draws = sample_draws(c, n_draws, n_samples, seed)
    samples = np.zeros((n_samples, 2))
    for s in range(n_samples):
        idx, cnt = np.unique(draws[s], return_counts=True)
        samples[s] = pt2_sampled(inst, keys, c, idx, cnt, p, n_draws, eps2, eps2_det, e0)
    diff = samples[:, 0] - samples[:, 1]
    err = float(np.std(diff, ddof=1) / np.sqrt(n_samples)) if n_samples > 1 else 0.0
    return {"estimate": e2d + float(diff.mean()), "error": err, "e2_det": e2d, "samples": samples,
            "draws": draws}


def select(inst, keys, c, eps1, band=1e-12, sources=None):
    """One selection step, Eq. (criteria) with f_HCI (Sec. II.A).

    Returns (new_keys, f_new, tie_keys): new_keys are the determinants not
    in V with max_i |H_ai c_i| > eps1 (strict inequality, as the criterion is stated),
    sorted by (alpha, beta); eps1 <= 0 accepts every single and double
    excitation (reading: the symmetry-zero elements left by the MO
    transform would otherwise make the set depend on rounding).
    tie_keys lists determinants with |f - eps1| <= band*eps1, whose
    membership may legitimately differ under a different summation order.
    `sources` restricts the D_i that generate (sampled verification).
    """
    P = Problem.of(inst)
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    L = _lib()
    allx = 1 if eps1 <= 0 else 0
    floor = eps1 * (1.0 - band) if eps1 > 0 else 0.0
    if sources is not None:
        src = _c(sources, np.int64)
        hs = L.orc_select(P.norb, _p(P.h), _p(P.eri), _p(keys), _p(c), len(keys), floor, allx,
                          _p(src), len(src))
    else:
        hs = L.orc_select(P.norb, _p(P.h), _p(P.eri), _p(keys), _p(c), len(keys), floor, allx,
                          None, 0)
    try:
        m = L.orc_sel_count(hs)
        k = np.zeros((m, 2), np.uint64)
        f = np.zeros(m)
        L.orc_sel_copy(hs, _p(k), _p(f))
    finally:
        L.orc_sel_free(hs)
    if eps1 <= 0:
        return k, f, np.zeros((0, 2), np.uint64)
    sel = f > eps1
    tie = np.abs(f - eps1) <= band * eps1
    return k[sel], f[sel], k[tie]


def rdm12(norb, keys, c):
    """rdm1[p,q] = sum_s <a+_ps a_qs>, rdm2[p,q,r,s] = sum_st <a+_ps a+_rt a_st a_qs>
    (spin-summed, the order in which E = sum h rdm1 + 1/2 sum (pq|rs) rdm2)."""
    keys = _c(keys, np.uint64).reshape(-1, 2)
    c = _c(c, np.float64)
    r1 = np.zeros((norb, norb))
    r2 = np.zeros((norb,) * 4)
    _lib().orc_rdm12(norb, _p(keys), len(keys), _p(c), _p(r1), _p(r2))
    return r1, r2


# ----------------------------------------------------------------------------
# eigenproblem, HCI loop
# ----------------------------------------------------------------------------

def fix_phase(c: np.ndarray) -> np.ndarray:
    """Reading: the largest-|c| component (lowest index on ties) is positive."""
    if len(c) == 0:
        return c
    a = np.abs(c)
    i = int(np.argmax(a))      # argmax returns the first maximum
    return -c if c[i] < 0 else c


def ground_state(inst, keys, v0=None, H=None):
    """Lowest eigenpair of H restricted to V (Eq. variational on a fixed V)."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    if H is None:
        H = hamiltonian(inst, keys)
    nV = len(keys)
    if nV <= 2500:
        w, v = np.linalg.eigh(H.toarray())
        e, c = float(w[0]), v[:, 0]
    else:
        if v0 is not None and np.linalg.norm(v0) > 0:
            v0 = np.asarray(v0, dtype=np.float64)
            v0 = v0 + 1e-3 * np.random.default_rng(0).standard_normal(nV) / np.sqrt(nV)
        w, v = spla.eigsh(H, k=1, which="SA", v0=v0, tol=0, ncv=min(nV, 40))
        e, c = float(w[0]), v[:, 0]
        r = H @ c - e * c
        if np.linalg.norm(r) > 1e-9:
            w, v = spla.eigsh(H, k=1, which="SA", v0=c, tol=0, ncv=min(nV, 80), maxiter=20000)
            e, c = float(w[0]), v[:, 0]
    c = c / np.linalg.norm(c)
    return e, fix_phase(c)


def lowest_states(inst, keys, nroots):
    """The nroots lowest eigenpairs of H restricted to V (ascending; each
    vector with the phase of fix_phase)."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    H = hamiltonian(inst, keys)
    if len(keys) <= 2500:
        w, v = np.linalg.eigh(H.toarray())
    else:
        w, v = spla.eigsh(H, k=nroots, which="SA", tol=0, ncv=min(len(keys), max(40, 4 * nroots)))
        order = np.argsort(w)
        w, v = w[order], v[:, order]
    return w[:nroots].astype(float), np.stack([fix_phase(v[:, r] / np.linalg.norm(v[:, r])) for r in range(nroots)])


def hci_roots(inst, eps1, nroots, max_iter=30):
    """Variational HCI for the nroots lowest states: a determinant enters when
    max_r |H_ai c_i^(r)| > eps1 for some D_i, i.e. the selection of the
    single-state loop with c_i replaced by max_r |c_i^(r)|; V^0 = {aufbau}
    (one state), then after each merge the nroots lowest states, or all of
    them while V holds fewer determinants (reading: the paper is silent;
    the space must reach nroots determinants by the end)."""
    P = Problem.of(inst)
    keys = aufbau(P.nalpha, P.nbeta)
    ceff = np.array([1.0])
    es, cs = None, None
    for mu in range(max_iter):
        new, _, _ = select(P, keys, ceff, eps1)
        if len(new) == 0:
            break
        keys, _ = merge(keys, np.zeros(len(keys)), new)
        es, cs = lowest_states(P, keys, min(nroots, len(keys)))
        ceff = np.abs(cs).max(axis=0)
    if len(keys) < nroots:
        raise ValueError("space smaller than the number of roots")
    return {"keys": keys, "c": cs, "E": es}


def merge(keys, c, new_keys):
    """Sorted union V + C (Sec. II.A) with c padded by zeros (warm start)."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    new_keys = np.asarray(new_keys, np.uint64).reshape(-1, 2)
    allk = np.concatenate([keys, new_keys])
    allc = np.concatenate([np.asarray(c, np.float64), np.zeros(len(new_keys))])
    order = np.lexsort((allk[:, 1], allk[:, 0]))
    return allk[order], allc[order]


def aufbau(nalpha, nbeta):
    """Reading: the first V is the aufbau determinant in the given orbital order."""
    return np.array([[(1 << nalpha) - 1, (1 << nbeta) - 1]], dtype=np.uint64)


def hci(inst, eps1, max_iter=30, verbose=False):
    """Variational HCI (Sec. II.A): V^0 = {aufbau}, c^0 = [1]; repeat
    select C^mu(eps1), V^{mu+1} = V^mu + C^mu, lowest eigenpair on V^{mu+1};
    stop when C^mu is empty (reading: the paper leaves the convergence
    test open) or after max_iter iterations."""
    P = Problem.of(inst)
    keys = aufbau(P.nalpha, P.nbeta)
    c = np.array([1.0])
    e = float(diag(P, keys)[0])
    history = []
    for mu in range(max_iter):
        new, _, ties = select(P, keys, c, eps1)
        history.append({"mu": mu, "nV": len(keys), "n_new": len(new), "E": e, "n_ties": len(ties)})
        if verbose:
            print(history[-1])
        if len(new) == 0:
            break
        keys, c = merge(keys, c, new)
        e, c = ground_state(P, keys, v0=c)
    return {"keys": keys, "c": c, "E": e, "history": history}


# ----------------------------------------------------------------------------
# spin parity in the S_z = 0 sector (spin-flip symmetry)
# ----------------------------------------------------------------------------
# The spin flip F exchanges a+_{p alpha} and a+_{p beta}.  With m = n_alpha =
# n_beta, F |alpha, beta> = (-1)^(m m) |beta, alpha> = (-1)^m |beta, alpha>
# (the m beta creators move past the m alpha ones), F commutes with the
# spin-free H, and an eigenstate of total spin S has F = (-1)^(m + S).  So
# the states of spin parity p = (-1)^S are the vectors with
# c(beta, alpha) = p c(alpha, beta): even S (singlets, quintets) p = +1, odd S
# (triplets) p = -1; a determinant with alpha = beta belongs to p = +1 only.

def flip_keys(keys):
    """(alpha, beta) -> (beta, alpha) for every determinant."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    return np.ascontiguousarray(keys[:, ::-1])


def close_under_flip(keys):
    """The sorted union of a key set and its spin-flipped partners."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    allk = np.unique(np.concatenate([keys, flip_keys(keys)]), axis=0)
    return allk[np.lexsort((allk[:, 1], allk[:, 0]))]


def flip_partner(keys):
    """index of the spin-flipped partner of every determinant of a
    flip-closed V (ValueError when one is missing)."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    n = len(keys)
    allk = np.concatenate([keys, flip_keys(keys)])
    uniq, inv = np.unique(allk, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    if len(uniq) != n:
        raise ValueError("space not closed under the spin flip")
    pos = np.empty(n, np.int64)
    pos[inv[:n]] = np.arange(n)
    return pos[inv[n:]]


def parity_basis(keys, parity):
    """Orthonormal basis (sparse nV x nb) of {c : c(b, a) = parity c(a, b)}
    on a flip-closed V: (e_D + parity e_Dbar) / sqrt(2) per pair D != Dbar,
    e_D for alpha = beta when parity = +1."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    part = flip_partner(keys)
    idx = np.arange(len(keys))
    selfp = idx[part == idx] if parity > 0 else idx[:0]
    lo = idx[part > idx]
    nb_self, nb_pair = len(selfp), len(lo)
    r = 1.0 / np.sqrt(2.0)
    rows = np.concatenate([selfp, lo, part[lo]])
    cols = np.concatenate([np.arange(nb_self), nb_self + np.arange(nb_pair), nb_self + np.arange(nb_pair)])
    vals = np.concatenate([np.ones(nb_self), np.full(nb_pair, r), np.full(nb_pair, parity * r)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(keys), nb_self + nb_pair))


def parity_ground_state(inst, keys, parity):
    """Lowest eigenpair of H on a flip-closed V restricted to spin parity
    `parity` (Eq. variational in that symmetry sector); c in the determinant
    basis with the phase of fix_phase."""
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    B = parity_basis(keys, parity)
    if B.shape[1] == 0:
        raise ValueError("no state of this spin parity in V")
    H = hamiltonian(inst, keys)
    Hs = (B.T @ H @ B).tocsr()
    if Hs.shape[0] <= 2500:
        w, v = np.linalg.eigh(Hs.toarray())
        e, y = float(w[0]), v[:, 0]
    else:
        w, v = spla.eigsh(Hs, k=1, which="SA", tol=0, ncv=min(Hs.shape[0], 40))
        e, y = float(w[0]), v[:, 0]
    c = B @ y
    return e, fix_phase(c / np.linalg.norm(c))


def hci_parity(inst, eps1, parity, max_iter=30):
    """Variational HCI for the lowest state of spin parity `parity` in the
    S_z = 0 sector (Sec. II.A with the sector of Sec. VI's singlet and
    triplet states).  Reading: V^0 = {aufbau}, c^0 = [1] (the first
    selection is made from the aufbau determinant whatever its parity);
    each selection C^mu(eps1) of Eq. (criteria) is completed by the spin-flip
    partners of its determinants, V^{mu+1} = V^mu + C^mu + F C^mu, and the
    state on V^{mu+1} is the lowest eigenvector of spin parity `parity`;
    stop when C^mu is empty."""
    P = Problem.of(inst)
    if P.nalpha != P.nbeta:
        raise ValueError("spin parity needs n_alpha = n_beta")
    keys = aufbau(P.nalpha, P.nbeta)
    c = np.array([1.0])
    e = None
    for mu in range(max_iter):
        new, _, _ = select(P, keys, c, eps1)
        if len(new) == 0:
            break
        new = close_under_flip(new)
        keys, _ = merge(keys, np.zeros(len(keys)), new)
        e, c = parity_ground_state(P, keys, parity)
    if e is None:
        e, c = parity_ground_state(P, keys, parity)
    return {"keys": keys, "c": c, "E": e}


# ----------------------------------------------------------------------------
# orbital rotation and vHCISCF gradient
# ----------------------------------------------------------------------------

def expm(kappa):
    return scipy.linalg.expm(np.asarray(kappa, dtype=np.float64))


def rotate(inst, kappa):
    """h' = U^T h U, (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd), U = exp(kappa)."""
    P = Problem.of(inst)
    U = expm(kappa)
    h2 = U.T @ P.h @ U
    e2 = np.einsum("abcd,ap,bq,cr,ds->pqrs", P.eri, U, U, U, U, optimize=True)
    return Problem(P.norb, P.nalpha, P.nbeta, h2, e2, P.e_core), U


def energy_from_rdm(inst, rdm1, rdm2):
    P = Problem.of(inst)
    return float(np.sum(P.h * rdm1) + 0.5 * np.sum(P.eri * rdm2) + P.e_core)


def gradient(inst, kappa, rdm1, rdm2):
    """Gradient of E(h', eri') with dE/dh' = rdm1, dE/d(pq|rs)' = rdm2/2
    (Hellmann-Feynman at fixed V, c: dE/dc = 0, Eq. vdedk2), chained
    through the rotation (all four index positions, no symmetry assumed)
    and through U = exp(kappa) by the adjoint Frechet derivative of expm.
    Returns dict(dh, deri, dU, dkappa) with dkappa the derivative with
    respect to every entry of the full kappa matrix."""
    P = Problem.of(inst)
    U = expm(kappa)
    D = 0.5 * np.asarray(rdm2)
    g1 = np.asarray(rdm1)
    dh = U @ g1 @ U.T
    deri = np.einsum("pqrs,ap,bq,cr,ds->abcd", D, U, U, U, U, optimize=True)
    gU = P.h @ U @ g1.T + P.h.T @ U @ g1
    E = P.eri
    gU = gU + np.einsum("xbcd,bq,cr,ds,yqrs->xy", E, U, U, U, D, optimize=True)
    gU = gU + np.einsum("axcd,ap,cr,ds,pyrs->xy", E, U, U, U, D, optimize=True)
    gU = gU + np.einsum("abxd,ap,bq,ds,pqys->xy", E, U, U, U, D, optimize=True)
    gU = gU + np.einsum("abcx,ap,bq,cr,pqry->xy", E, U, U, U, D, optimize=True)
    dk = scipy.linalg.expm_frechet(np.asarray(kappa, dtype=np.float64).T, gU, compute_expm=False)
    return {"dh": dh, "deri": deri, "dU": gU, "dkappa": dk}


def energy_fixed_space(inst, kappa, keys, v0=None):
    """E at fixed V after rotating the integrals by exp(kappa) (for central
    finite differences of the vHCISCF gradient)."""
    R, _ = rotate(inst, kappa)
    e, c = ground_state(R, keys, v0=v0)
    return e, c
