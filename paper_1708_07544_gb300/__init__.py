"""GB300-native heat-bath CI active-space solver (arXiv:1708.07544).

The compute path is libhci.so (hand-written sm_103a CUDA behind a C ABI,
declared in include/hci.h).  This package only marshals torch tensors into
it: `_abi` mirrors the C entry points one to one, `HCISolver` wraps a
context, and `HCIEnergy` is the torch.autograd.Function whose backward maps
the variational energy's adjoint to dE/dh = rdm1, dE/d(pq|rs) = rdm2/2 and,
through U = exp(kappa), to the orbital gradient dE/dkappa (Eq. vdedk2).
"""
from __future__ import annotations

from ._abi import (HCIError, hci_build_lists, hci_create, hci_davidson, hci_destroy, hci_last_error,  # noqa: F401
                   hci_launch_count, hci_merge, hci_profile, hci_qtrans, hci_rdm12, hci_rotate, hci_rotate_backward,
                   hci_select, hci_sigma, hci_solve, hci_solve_batch, hci_stats, hci_timers, load)
from .solver import HCIEnergy, HCISolver  # noqa: F401

__all__ = ["HCIError", "HCISolver", "HCIEnergy", "load", "hci_create", "hci_destroy", "hci_last_error",
           "hci_build_lists", "hci_select", "hci_merge", "hci_sigma", "hci_davidson", "hci_rdm12", "hci_solve",
           "hci_rotate", "hci_rotate_backward", "hci_stats", "hci_profile", "hci_timers", "hci_launch_count",
           "hci_solve_batch", "hci_qtrans"]
