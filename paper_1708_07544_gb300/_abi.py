"""ctypes binding of libhci.so: one Python function per C entry point, same
names, argument marshalling only (torch tensors -> device pointers).

Keys are int64 torch tensors of shape (nV, 2) holding the (alpha, beta)
uint64 bit patterns; coefficient vectors and integrals are float64.
Every computation runs in the CUDA library; there is no CPU fallback, and
loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhci.so")

HCI_OK = 0
HCI_ERR_INVALID = 1
HCI_ERR_CAPACITY = 2
HCI_ERR_NOT_CONVERGED = 3
HCI_ERR_CUDA = 4
HCI_ERR_NOMEM = 5
_NAMES = {0: "OK", 1: "INVALID", 2: "CAPACITY", 3: "NOT_CONVERGED", 4: "CUDA", 5: "NOMEM"}

EXPORTS = ["hci_create", "hci_destroy", "hci_last_error", "hci_build_lists", "hci_select", "hci_merge",
           "hci_sigma", "hci_davidson", "hci_rdm12", "hci_solve", "hci_rotate", "hci_rotate_backward",
           "hci_stats", "hci_profile", "hci_timers", "hci_launch_count", "hci_rotate_noalloc",
           "hci_solve_batch", "hci_pt2", "hci_zvector", "hci_relaxed_rdm12", "hci_davidson_roots",
           "hci_solve_roots", "hci_pt2_stochastic", "hci_set_sigma_mode", "hci_spin_square", "hci_solve_from", "hci_set_spin_parity",
           "hci_qtrans"]
PHASES = ["lists", "walk", "dedup", "merge", "graph", "sigma", "davidson", "rdm", "singles", "graph_space",
          "graph_rows", "graph_merge", "rdm_diag", "hdiag"]
STATS = ["graph_nnz", "last_candidates", "sigma_calls", "sigma_rows", "sigma_nnz", "select_calls",
         "select_sources", "candidates", "graph_builds", "walk_entries", "singles_exact", "rows_refilled",
         "sigma_direct", "graph_half"]
SIGMA_AUTO, SIGMA_STORED, SIGMA_DIRECT, SIGMA_HALF = 0, 1, 2, 3


class HCIError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"HCI_ERR_{_NAMES.get(status, status)}: {msg}")
        self.status = status


_LIB = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libhci.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libhci.so not built at {p}; run __graft_entry__.build()")
    L = ctypes.CDLL(p)
    V = ctypes.c_void_p
    I = ctypes.c_int
    I64 = ctypes.c_int64
    D = ctypes.c_double
    P = ctypes.POINTER
    L.hci_create.argtypes = [P(V), I, I, I, V, V, D, V]
    L.hci_destroy.argtypes = [V]
    L.hci_last_error.argtypes = [V]
    L.hci_last_error.restype = ctypes.c_char_p
    L.hci_build_lists.argtypes = [V]
    L.hci_select.argtypes = [V, D, V, V, I64, V, I64, P(I64)]
    L.hci_merge.argtypes = [V, V, V, I64, V, I64, V, V]
    L.hci_sigma.argtypes = [V, V, I64, V, V, I]
    L.hci_davidson.argtypes = [V, V, I64, V, P(D), D, I, P(I)]
    L.hci_rdm12.argtypes = [V, V, I64, V, V, V]
    L.hci_pt2.argtypes = [V, D, V, V, I64, D, I64, P(D), P(I64), V, V, V, V, V]
    L.hci_set_sigma_mode.argtypes = [V, I, I64]
    L.hci_set_spin_parity.argtypes = [V, I]
    L.hci_spin_square.argtypes = [V, V, P(D)]
    L.hci_pt2_stochastic.argtypes = [V, V, V, I64, D, D, D, I64, I, ctypes.c_uint64, I64, V, V, V]
    L.hci_zvector.argtypes = [V, V, I64, V, D, V, V, D, I, P(I)]
    L.hci_davidson_roots.argtypes = [V, V, I64, I, V, V, D, I, P(I)]
    L.hci_solve_roots.argtypes = [V, I, D, I, D, I, V, V, I64, P(I64), V, P(I)]
    L.hci_relaxed_rdm12.argtypes = [V, D, V, V, I64, D, I64, D, I, P(D), V, V]
    L.hci_solve.argtypes = [V, D, I, D, I, V, V, I64, P(I64), P(D), P(I)]
    L.hci_solve_from.argtypes = [V, V, V, I64, D, I, D, I, V, V, I64, P(I64), P(D), P(I)]
    L.hci_rotate.argtypes = [I, V, V, V, V, V, V, V]
    L.hci_rotate_backward.argtypes = [I, V, V, V, V, V, V, V, V, V]
    L.hci_rotate_noalloc.argtypes = [I, V, V, V, V, V, V, V]
    L.hci_qtrans.argtypes = [I, V, V, V, I, V]
    L.hci_solve_batch.argtypes = [I, V, V, V, V, V, V, D, I, D, I, I, V, V, V, V, V]
    L.hci_stats.argtypes = [V, V, I]
    L.hci_profile.argtypes = [V, I]
    L.hci_timers.argtypes = [V, V, V, I]
    L.hci_launch_count.argtypes = []
    for name in EXPORTS:
        getattr(L, name).restype = I
    L.hci_last_error.restype = ctypes.c_char_p
    L.hci_launch_count.restype = I64
    if path is None:
        _LIB = L
    return L


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(status: int, ctx=None):
    if status != HCI_OK:
        msg = load().hci_last_error(ctx)
        raise HCIError(status, (msg or b"").decode())


def hci_create(norb, nalpha, nbeta, h, eri, e_core=0.0, stream=None):
    """Returns an opaque context handle (int)."""
    L = load()
    out = ctypes.c_void_p()
    h = h.to(torch.float64).contiguous()
    eri = eri.to(torch.float64).contiguous()
    st = L.hci_create(ctypes.byref(out), int(norb), int(nalpha), int(nbeta), _ptr(h), _ptr(eri), float(e_core),
                      _stream_ptr(stream))
    _check(st, None)
    return out.value


def hci_destroy(ctx):
    _check(load().hci_destroy(ctx), None)


def hci_last_error(ctx=None) -> str:
    return (load().hci_last_error(ctx) or b"").decode()


def hci_build_lists(ctx):
    _check(load().hci_build_lists(ctx), ctx)


def hci_select(ctx, eps1, keys, c, cap=None):
    """New determinants (sorted, unique, not in V) as an (n_new, 2) int64 tensor."""
    L = load()
    nV = keys.shape[0]
    n = ctypes.c_int64(0)
    if cap is None:
        cap = max(1024, 4 * nV)
    out = torch.empty((cap, 2), dtype=torch.int64, device=keys.device)
    st = L.hci_select(ctx, float(eps1), _ptr(keys), _ptr(c), nV, _ptr(out), cap, ctypes.byref(n))
    if st == HCI_ERR_CAPACITY:
        cap = int(n.value)
        out = torch.empty((max(cap, 1), 2), dtype=torch.int64, device=keys.device)
        st = L.hci_select(ctx, float(eps1), _ptr(keys), _ptr(c), nV, _ptr(out), cap, ctypes.byref(n))
    _check(st, ctx)
    return out[: int(n.value)]


def hci_merge(ctx, keys, c, new_keys):
    L = load()
    nV, nn = keys.shape[0], new_keys.shape[0]
    ok = torch.empty((nV + nn, 2), dtype=torch.int64, device=keys.device)
    oc = torch.empty(nV + nn, dtype=torch.float64, device=keys.device) if c is not None else None
    _check(L.hci_merge(ctx, _ptr(keys), _ptr(c), nV, _ptr(new_keys) if nn else None, nn, _ptr(ok), _ptr(oc)), ctx)
    return ok, oc


def hci_sigma(ctx, keys, c):
    """H c for c of shape (nV,) or (nvec, nV)."""
    L = load()
    nV = keys.shape[0]
    nvec = 1 if c.dim() == 1 else c.shape[0]
    out = torch.empty_like(c)
    _check(L.hci_sigma(ctx, _ptr(keys), nV, _ptr(c), _ptr(out), nvec), ctx)
    return out


def hci_davidson(ctx, keys, c0=None, tol=1e-10, maxit=400, allow_unconverged=False):
    """(E, c, iterations); c0 is copied (zero/None => start at the lowest diagonal)."""
    L = load()
    nV = keys.shape[0]
    c = torch.zeros(nV, dtype=torch.float64, device=keys.device) if c0 is None else c0.clone().contiguous()
    e = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    st = L.hci_davidson(ctx, _ptr(keys), nV, _ptr(c), ctypes.byref(e), float(tol), int(maxit), ctypes.byref(it))
    if not (allow_unconverged and st == HCI_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return e.value, c, it.value


def hci_pt2(ctx, keys, c, eps2, e0, max_pairs=0, norb=None, grad=False):
    """Screened second-order Epstein-Nesbet correction; returns (E2, |C(eps2)|),
    and with norb given also (rdm1_dd, rdm2_dd, rdm1_dc, rdm2_dc), and with
    grad also dE2/dc (appended last)."""
    L = load()
    e2 = ctypes.c_double(0.0)
    n_ext = ctypes.c_int64(0)
    rd = [None] * 4
    if norb is not None:
        shapes = [(norb, norb), (norb,) * 4, (norb, norb), (norb,) * 4]
        rd = [torch.empty(sh, dtype=torch.float64, device=keys.device) for sh in shapes]
    g = torch.empty(keys.shape[0], dtype=torch.float64, device=keys.device) if grad else None
    _check(L.hci_pt2(ctx, float(eps2), _ptr(keys), _ptr(c), keys.shape[0], float(e0), int(max_pairs),
                     ctypes.byref(e2), ctypes.byref(n_ext), *[_ptr(x) if x is not None else None for x in rd],
                     _ptr(g) if g is not None else None), ctx)
    out = (e2.value, n_ext.value)
    if norb is not None:
        out = out + (tuple(rd),)
    if grad:
        out = out + (g,)
    return out


def hci_set_spin_parity(ctx, parity):
    _check(load().hci_set_spin_parity(ctx, int(parity)), ctx)


def hci_spin_square(ctx, rdm2):
    """<S^2> from the spin-summed 2-RDM of hci_rdm12."""
    s2 = ctypes.c_double(0.0)
    _check(load().hci_spin_square(ctx, _ptr(rdm2.contiguous()), ctypes.byref(s2)), ctx)
    return s2.value


def hci_set_sigma_mode(ctx, mode, graph_budget=0):
    """Stored connections (SIGMA_STORED), searched again per traversal
    (SIGMA_DIRECT), or stored while they fit graph_budget bytes (SIGMA_AUTO)."""
    _check(load().hci_set_sigma_mode(ctx, int(mode), int(graph_budget)), ctx)


def hci_pt2_stochastic(ctx, keys, c, e0, eps2, eps2_det, n_draws, n_samples, seed=0, max_pairs=0):
    """Semistochastic E2 (Eq. semistoc): dict with estimate, error, e2_det,
    samples [n_samples, 2] (E2^S(eps2), E2^S(eps2_det)) and draws
    [n_samples, n_draws] (device int32 indices into V)."""
    L = load()
    res = (ctypes.c_double * 3)()
    smp = np.zeros((int(n_samples), 2))
    draws = torch.empty((int(n_samples), int(n_draws)), dtype=torch.int32, device=keys.device)
    _check(L.hci_pt2_stochastic(ctx, _ptr(keys), _ptr(c), keys.shape[0], float(e0), float(eps2), float(eps2_det),
                                int(n_draws), int(n_samples), int(seed), int(max_pairs), res,
                                smp.ctypes.data_as(ctypes.c_void_p), _ptr(draws)), ctx)
    return {"estimate": res[0], "error": res[1], "e2_det": res[2], "samples": smp, "draws": draws}


def hci_davidson_roots(ctx, keys, nroots, c0=None, tol=1e-10, maxit=400):
    """(energies [nroots], c [nroots, nV], total iterations)."""
    L = load()
    nV = keys.shape[0]
    c = torch.zeros((nroots, nV), dtype=torch.float64, device=keys.device) if c0 is None else c0.clone().contiguous()
    e = (ctypes.c_double * nroots)()
    it = ctypes.c_int(0)
    _check(L.hci_davidson_roots(ctx, _ptr(keys), nV, int(nroots), _ptr(c), e, float(tol), int(maxit),
                                ctypes.byref(it)), ctx)
    return np.array(e[:]), c, it.value


def hci_solve_roots(ctx, nroots, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 22, device=None):
    """Multi-state variational HCI: (keys [nV, 2] int64, c [nroots, nV], energies, selections)."""
    L = load()
    dev = device if device is not None else torch.device("cuda")
    keys = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    c = torch.empty((nroots, cap), dtype=torch.float64, device=dev)
    nv = ctypes.c_int64(0)
    e = (ctypes.c_double * nroots)()
    it = ctypes.c_int(0)
    _check(L.hci_solve_roots(ctx, int(nroots), float(eps1), int(max_iter), float(dav_tol), int(dav_maxit),
                             _ptr(keys), _ptr(c), cap, ctypes.byref(nv), e, ctypes.byref(it)), ctx)
    n = nv.value
    cflat = c.reshape(-1)[: nroots * n].reshape(nroots, n).clone()
    return keys[:n].clone(), cflat, np.array(e[:]), it.value


def hci_zvector(ctx, keys, c, e0, rhs, tol=1e-10, maxit=500):
    """z with (H - e0) z = P rhs, z orthogonal to c; returns (z, iterations)."""
    L = load()
    z = torch.empty_like(c)
    it = ctypes.c_int(0)
    _check(L.hci_zvector(ctx, _ptr(keys), keys.shape[0], _ptr(c), float(e0), _ptr(rhs), _ptr(z), float(tol),
                         int(maxit), ctypes.byref(it)), ctx)
    return z, it.value


def hci_relaxed_rdm12(ctx, keys, c, e0, eps2, norb, max_pairs=0, zv_tol=1e-10, zv_maxit=500):
    """Relaxed density matrices of E_var + E2; returns (E2, rdm1, rdm2)."""
    L = load()
    e2 = ctypes.c_double(0.0)
    r1 = torch.empty((norb, norb), dtype=torch.float64, device=keys.device)
    r2 = torch.empty((norb,) * 4, dtype=torch.float64, device=keys.device)
    _check(L.hci_relaxed_rdm12(ctx, float(eps2), _ptr(keys), _ptr(c), keys.shape[0], float(e0), int(max_pairs),
                               float(zv_tol), int(zv_maxit), ctypes.byref(e2), _ptr(r1), _ptr(r2)), ctx)
    return e2.value, r1, r2


def hci_rdm12(ctx, keys, c, norb):
    L = load()
    r1 = torch.empty((norb, norb), dtype=torch.float64, device=keys.device)
    r2 = torch.empty((norb,) * 4, dtype=torch.float64, device=keys.device)
    _check(L.hci_rdm12(ctx, _ptr(keys), keys.shape[0], _ptr(c), _ptr(r1), _ptr(r2)), ctx)
    return r1, r2


def hci_solve(ctx, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 24, device="cuda"):
    """Whole variational stage; returns (keys, c, E, iterations)."""
    L = load()
    nv = ctypes.c_int64(0)
    e = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    keys = torch.empty((cap, 2), dtype=torch.int64, device=device)
    c = torch.empty(cap, dtype=torch.float64, device=device)
    st = L.hci_solve(ctx, float(eps1), int(max_iter), float(dav_tol), int(dav_maxit), _ptr(keys), _ptr(c), cap,
                     ctypes.byref(nv), ctypes.byref(e), ctypes.byref(it))
    if st == HCI_ERR_CAPACITY:
        cap = int(nv.value)
        keys = torch.empty((cap, 2), dtype=torch.int64, device=device)
        c = torch.empty(cap, dtype=torch.float64, device=device)
        st = L.hci_solve(ctx, float(eps1), int(max_iter), float(dav_tol), int(dav_maxit), _ptr(keys), _ptr(c), cap,
                         ctypes.byref(nv), ctypes.byref(e), ctypes.byref(it))
    _check(st, ctx)
    n = int(nv.value)
    return keys[:n], c[:n], e.value, it.value


def hci_solve_from(ctx, keys0, c0, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 24):
    """Variational stage resumed from (keys0, c0); returns (keys, c, E, iterations)."""
    L = load()
    keys0 = keys0.contiguous()
    c0 = c0.to(torch.float64).contiguous()
    nv = ctypes.c_int64(0)
    e = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    cap = max(cap, keys0.shape[0])
    dev = keys0.device

    def run(cap):
        keys = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        c = torch.empty(cap, dtype=torch.float64, device=dev)
        st = L.hci_solve_from(ctx, _ptr(keys0), _ptr(c0), keys0.shape[0], float(eps1), int(max_iter),
                              float(dav_tol), int(dav_maxit), _ptr(keys), _ptr(c), cap, ctypes.byref(nv),
                              ctypes.byref(e), ctypes.byref(it))
        return st, keys, c

    st, keys, c = run(cap)
    if st == HCI_ERR_CAPACITY:
        st, keys, c = run(int(nv.value))
    _check(st, ctx)
    n = int(nv.value)
    return keys[:n], c[:n], e.value, it.value


def hci_rotate(kappa, h, eri, stream=None):
    """(U, h', eri') with U = exp(kappa)."""
    L = load()
    n = h.shape[0]
    U = torch.empty_like(h)
    h2 = torch.empty_like(h)
    e2 = torch.empty_like(eri)
    _check(L.hci_rotate(n, _ptr(kappa.contiguous()), _ptr(h.contiguous()), _ptr(eri.contiguous()), _ptr(U),
                        _ptr(h2), _ptr(e2), _stream_ptr(stream)), None)
    return U, h2, e2


def hci_qtrans(inp, M, out=None, check=True, stream=None):
    """One quarter transform out[J*n + p] = sum_a inp[a*n^3 + J] M[a*n + p]."""
    L = load()
    n = M.shape[0]
    if out is None:
        out = torch.empty_like(inp)
    _check(L.hci_qtrans(n, _ptr(inp.contiguous()), _ptr(M.contiguous()), _ptr(out), 1 if check else 0,
                        _stream_ptr(stream)), None)
    return out


def hci_rotate_backward(kappa, h, eri, rdm1, rdm2, want_dh=True, want_deri=True, want_dkappa=True, stream=None):
    L = load()
    n = h.shape[0]
    dh = torch.empty_like(h) if want_dh else None
    de = torch.empty_like(eri) if want_deri else None
    dk = torch.empty_like(h) if want_dkappa else None
    _check(L.hci_rotate_backward(n, _ptr(kappa.contiguous()), _ptr(h.contiguous()), _ptr(eri.contiguous()),
                                 _ptr(rdm1.contiguous()), _ptr(rdm2.contiguous()), _ptr(dh), _ptr(de), _ptr(dk),
                                 _stream_ptr(stream)), None)
    return dh, de, dk


def hci_stats(ctx):
    """Work counters of the context as a dict (names in STATS)."""
    import numpy as np

    out = np.zeros(len(STATS), dtype=np.int64)
    _check(load().hci_stats(ctx, out.ctypes.data, len(STATS)), ctx)
    return {k: int(out[i]) for i, k in enumerate(STATS)}


def hci_profile(ctx, enable=True):
    _check(load().hci_profile(ctx, 1 if enable else 0), ctx)


def hci_timers(ctx):
    """Read and reset the per-phase device times: {phase: (ms, count)}."""
    import numpy as np

    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().hci_timers(ctx, ms.ctypes.data, cnt.ctypes.data, len(PHASES)), ctx)
    return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}


def hci_launch_count():
    return int(load().hci_launch_count())


def hci_solve_batch(instances, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, nstreams=8, want_rdm=False,
                    device="cuda"):
    """Solve many active spaces concurrently.  instances: list of
    (norb, nalpha, nbeta, h, eri, e_core) with h, eri CUDA float64 tensors.
    Returns (energies, nV, rdm1 list or None, rdm2 list or None)."""
    import numpy as np

    L = load()
    cnt = len(instances)
    norb = np.array([int(x[0]) for x in instances], dtype=np.int32)
    na = np.array([int(x[1]) for x in instances], dtype=np.int32)
    nb = np.array([int(x[2]) for x in instances], dtype=np.int32)
    hs = [x[3].to(torch.float64).contiguous() for x in instances]
    es = [x[4].to(torch.float64).contiguous() for x in instances]
    hp = np.array([_ptr(t) for t in hs], dtype=np.uint64)
    ep = np.array([_ptr(t) for t in es], dtype=np.uint64)
    ec = np.array([float(x[5]) for x in instances], dtype=np.float64)
    en = np.zeros(cnt)
    nv = np.zeros(cnt, dtype=np.int64)
    stat = np.zeros(cnt, dtype=np.int32)
    r1 = r2 = None
    r1p = r2p = None
    if want_rdm:
        r1 = [torch.empty((int(n), int(n)), dtype=torch.float64, device=device) for n in norb]
        r2 = [torch.empty((int(n),) * 4, dtype=torch.float64, device=device) for n in norb]
        r1p = np.array([t.data_ptr() for t in r1], dtype=np.uint64)
        r2p = np.array([t.data_ptr() for t in r2], dtype=np.uint64)
    torch.cuda.synchronize()
    st = L.hci_solve_batch(cnt, norb.ctypes.data, na.ctypes.data, nb.ctypes.data, hp.ctypes.data, ep.ctypes.data,
                           ec.ctypes.data, float(eps1), int(max_iter), float(dav_tol), int(dav_maxit), int(nstreams),
                           en.ctypes.data, nv.ctypes.data, r1p.ctypes.data if want_rdm else None,
                           r2p.ctypes.data if want_rdm else None, stat.ctypes.data)
    _check(st, None)
    return en, nv, r1, r2
