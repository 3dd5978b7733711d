"""The C-ABI library loads and exports every entry point declared in
include/hci.h (no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hci.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hci_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_07544_gb300 import build

    path = build.build()
    import paper_1708_07544_gb300 as pkg

    return pkg.load(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hci_select" in names and "hci_rdm12" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1708_07544_gb300 import _abi

    assert sorted(_abi.EXPORTS) == _declared()


def test_create_rejects_bad_sizes_without_gpu(lib):
    import ctypes

    out = ctypes.c_void_p()
    # validation happens before any device call
    assert lib.hci_create(ctypes.byref(out), 65, 1, 1, None, None, 0.0, None) == 1
    assert b"norb" in lib.hci_last_error(None)
    assert lib.hci_create(ctypes.byref(out), 8, 9, 1, None, None, 0.0, None) == 1


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_1708_07544_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "hci_oracle" not in src and "orc_" not in src, f


def _enum_values():
    txt = open(os.path.join(ROOT, "include", "hci.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(HCI_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}


def test_binding_constants_match_header():
    from paper_1708_07544_gb300 import _abi

    ev = _enum_values()
    assert ev["HCI_ST_COUNT"] == len(_abi.STATS)
    for i, name in enumerate(_abi.STATS):
        assert ev["HCI_ST_" + name.upper()] == i, name
    assert (ev["HCI_SIGMA_AUTO"], ev["HCI_SIGMA_STORED"], ev["HCI_SIGMA_DIRECT"], ev["HCI_SIGMA_HALF"]) == \
        (_abi.SIGMA_AUTO, _abi.SIGMA_STORED, _abi.SIGMA_DIRECT, _abi.SIGMA_HALF)
    assert ev["HCI_PH_COUNT"] == len(_abi.PHASES)
    for i, name in enumerate(_abi.PHASES):
        assert ev["HCI_PH_" + name.upper()] == i, name
    for name in ["INVALID", "CAPACITY", "NOT_CONVERGED", "CUDA", "NOMEM"]:
        assert ev["HCI_ERR_" + name] == getattr(_abi, "HCI_ERR_" + name), name


def test_create_reports_injected_allocation_failure_without_gpu(lib, monkeypatch):
    """HCI_FAIL_ALLOC_AFTER=0 refuses the context's first device allocation
    on the host, before any device call: hci_create returns HCI_ERR_NOMEM
    with a message that names the injection (no GPU needed)."""
    import ctypes

    monkeypatch.setenv("HCI_FAIL_ALLOC_AFTER", "0")
    out = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)          # never dereferenced: the refusal comes first
    assert lib.hci_create(ctypes.byref(out), 8, 4, 4, dummy, dummy, 0.0, None) == 5
    assert b"injected" in lib.hci_last_error(None)
    assert out.value is None
