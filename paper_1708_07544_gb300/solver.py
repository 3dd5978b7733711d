"""Convenience wrappers over the C ABI: a solver object per active space and
the autograd Function of the vHCISCF energy (Sec. III.B, Eq. vdedk2)."""
from __future__ import annotations

import torch

from . import _abi


class HCISolver:
    """One context of libhci.so bound to (h, eri) on the current CUDA stream."""

    def __init__(self, norb, nalpha, nbeta, h, eri, e_core=0.0, stream=None):
        self.norb, self.nalpha, self.nbeta = int(norb), int(nalpha), int(nbeta)
        self.e_core = float(e_core)
        self.ctx = _abi.hci_create(norb, nalpha, nbeta, h, eri, e_core, stream)

    def close(self):
        if getattr(self, "ctx", None):
            _abi.hci_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def build_lists(self):
        _abi.hci_build_lists(self.ctx)

    def select(self, eps1, keys, c, cap=None):
        return _abi.hci_select(self.ctx, eps1, keys, c, cap)

    def merge(self, keys, c, new_keys):
        return _abi.hci_merge(self.ctx, keys, c, new_keys)

    def sigma(self, keys, c):
        return _abi.hci_sigma(self.ctx, keys, c)

    def davidson(self, keys, c0=None, tol=1e-10, maxit=400, allow_unconverged=False):
        return _abi.hci_davidson(self.ctx, keys, c0, tol, maxit, allow_unconverged)

    def rdm12(self, keys, c):
        return _abi.hci_rdm12(self.ctx, keys, c, self.norb)

    def pt2(self, keys, c, eps2, e0, max_pairs=0, rdms=False):
        """Screened Epstein-Nesbet correction E2(eps2) of the state (keys, c)
        with variational energy e0; returns (E2, |C(eps2)|), and with rdms
        also (rdm1_dd, rdm2_dd, rdm1_dc, rdm2_dc)."""
        return _abi.hci_pt2(self.ctx, keys, c, eps2, e0, max_pairs, self.norb if rdms else None)

    def spin_square(self, rdm2):
        """<S^2> of the state whose spin-summed 2-RDM is rdm2 (hci_rdm12)."""
        return _abi.hci_spin_square(self.ctx, rdm2)

    def set_spin_parity(self, parity):
        """+1: even total spin, -1: odd, 0: any (S_z = 0 only; hci_set_spin_parity)."""
        _abi.hci_set_spin_parity(self.ctx, parity)

    def set_sigma_mode(self, mode, graph_budget=0):
        """_abi.SIGMA_AUTO / SIGMA_STORED / SIGMA_DIRECT (see hci_set_sigma_mode)."""
        _abi.hci_set_sigma_mode(self.ctx, mode, graph_budget)

    def pt2_semistochastic(self, keys, c, e0, eps2, eps2_det, n_draws, n_samples, seed=0, max_pairs=0):
        """E2(eps2) ~ E2^D(eps2_det) + mean of E2^S(eps2) - E2^S(eps2_det)
        over n_samples samples of n_draws determinants (Eq. semistoc)."""
        return _abi.hci_pt2_stochastic(self.ctx, keys, c, e0, eps2, eps2_det, n_draws, n_samples, seed, max_pairs)

    def davidson_roots(self, keys, nroots, c0=None, tol=1e-10, maxit=400):
        return _abi.hci_davidson_roots(self.ctx, keys, nroots, c0, tol, maxit)

    def solve_roots(self, nroots, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 22):
        keys, c, e, it = _abi.hci_solve_roots(self.ctx, nroots, eps1, max_iter, dav_tol, dav_maxit, cap)
        return {"keys": keys, "c": c, "E": e, "iters": it}

    def zvector(self, keys, c, e0, rhs, tol=1e-10, maxit=500):
        return _abi.hci_zvector(self.ctx, keys, c, e0, rhs, tol, maxit)

    def relaxed_rdm12(self, keys, c, e0, eps2, max_pairs=0, zv_tol=1e-10, zv_maxit=500):
        """(E2, rdm1, rdm2): the density of E_var + E2 (Sec. III.A, Eq. lambda)."""
        return _abi.hci_relaxed_rdm12(self.ctx, keys, c, e0, eps2, self.norb, max_pairs, zv_tol, zv_maxit)

    def solve(self, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 24):
        keys, c, e, it = _abi.hci_solve(self.ctx, eps1, max_iter, dav_tol, dav_maxit, cap)
        return {"keys": keys, "c": c, "E": e, "iters": it}

    def solve_from(self, keys, c, eps1, max_iter=30, dav_tol=1e-10, dav_maxit=400, cap=1 << 24):
        """The selection loop resumed from a saved state (keys, c)."""
        keys, c, e, it = _abi.hci_solve_from(self.ctx, keys, c, eps1, max_iter, dav_tol, dav_maxit, cap)
        return {"keys": keys, "c": c, "E": e, "iters": it}

    def stats(self):
        return _abi.hci_stats(self.ctx)

    def profile(self, enable=True):
        _abi.hci_profile(self.ctx, enable)

    def timers(self):
        return _abi.hci_timers(self.ctx)


class HCIEnergy(torch.autograd.Function):
    """E(h, eri, kappa) = variational HCI energy of the rotated integrals.

    forward: U = exp(kappa), h' = U^T h U, eri' = U^4 eri, variational HCI
    on (h', eri') -> E; the selected space V and the solver context (its
    integrals and connection graph, not the CI vector) are kept for the
    backward.
    backward: c is recomputed by a cold-started Davidson on the saved V
    (the CI vector is not stored), the RDMs give dE/dh' = rdm1 and
    dE/deri' = rdm2/2 (dE/dc = 0 at the variational minimum), and the
    rotation's adjoint returns dE/dh, dE/deri and dE/dkappa for every entry
    of the full kappa matrix.
    """

    @staticmethod
    def forward(ctx, h, eri, kappa, nalpha, nbeta, e_core, eps1, max_iter=30, dav_tol=1e-10):
        n = h.shape[0]
        _, h2, e2 = _abi.hci_rotate(kappa, h, eri)
        s = HCISolver(n, nalpha, nbeta, h2, e2, e_core)
        try:
            out = s.solve(eps1, max_iter, dav_tol)
        except Exception:
            s.close()
            raise
        ctx.save_for_backward(h, eri, kappa, out["keys"])
        ctx.solver = s
        ctx.cfg = (n, nalpha, nbeta, e_core, dav_tol)
        ctx.nV = out["keys"].shape[0]
        return torch.tensor(out["E"], dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, gE):
        h, eri, kappa, keys = ctx.saved_tensors
        n, na, nb, e_core, tol = ctx.cfg
        s = ctx.solver
        ctx.solver = None
        if s is None:
            # a second backward through the same graph: a fresh context
            _, h2, e2 = _abi.hci_rotate(kappa, h, eri)
            s = HCISolver(n, na, nb, h2, e2, e_core)
        try:
            _, c, _ = s.davidson(keys, None, tol)          # zero start: cold, c recomputed
            r1, r2 = s.rdm12(keys, c)
        finally:
            s.close()
        dh, de, dk = _abi.hci_rotate_backward(kappa, h, eri, r1, r2)
        g = gE.to(torch.float64)
        return g * dh, g * de, g * dk, None, None, None, None, None, None
