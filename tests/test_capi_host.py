"""The C-ABI library loads and exports every symbol include/*.h declares, and
its host-side argument checks work without a GPU (no device work is issued)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_6720_gb300 import build
    build.build()
    from paper_1307_6720_gb300 import mhs
    return mhs


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^MHS_API\s+[\w\s\*]+?\b(mhs_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["mhs_create", "mhs_set_lower_bz", "mhs_solve", "mhs_fields", "mhs_get_phi", "mhs_destroy",
                     "mhs_set_stream", "mhs_status_string", "mhs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.mhs_status_string(0) == "MHS_OK"
    assert lib.mhs_status_string(lib.MHS_ERR_NOT_ELLIPTIC) == "MHS_ERR_NOT_ELLIPTIC"
    assert lib.mhs_version().startswith("mhs-gb300")


@pytest.mark.parametrize("n", [(4, 5, 5), (5, 6, 5), (3, 5, 5), (5, 5, 0)])
def test_create_rejects_bad_sizes(lib, n):
    with pytest.raises(lib.MhsError) as e:
        lib.mhs_create(*n, 1.0, 1.0, 1.0, 0.0)
    assert e.value.status == lib.MHS_ERR_INVALID_ARG


def test_create_rejects_bad_lengths(lib):
    with pytest.raises(lib.MhsError) as e:
        lib.mhs_create(9, 9, 9, 1.0, -1.0, 1.0, 0.0)
    assert e.value.status == lib.MHS_ERR_INVALID_ARG


def test_create_rejects_non_elliptic_xi(lib):
    """xi >= 1 on an interior plane makes eq. (scalar_pot) non-elliptic (Sect. 2.1)."""
    xi = lib.xi_params(lib.MHS_XI_EXP, 1.05, 0.1)
    with pytest.raises(lib.MhsError) as e:
        lib.mhs_create(9, 9, 9, 1.0, 1.0, 1.0, 0.5, xi)
    assert e.value.status == lib.MHS_ERR_NOT_ELLIPTIC
    assert "elliptic" in lib.mhs_last_error()


def test_create_rejects_indefinite_alpha(lib):
    with pytest.raises(lib.MhsError) as e:
        lib.mhs_create(9, 9, 9, 1.0, 1.0, 1.0, 10.0)
    assert e.value.status == lib.MHS_ERR_NOT_ELLIPTIC


def test_create_rejects_bad_atmosphere(lib):
    with pytest.raises(lib.MhsError) as e:
        lib.mhs_create(9, 9, 9, 1.0, 1.0, 1.0, 0.0, None, lib.atmos_params(mu0=0.0))
    assert e.value.status == lib.MHS_ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.LIB.mhs_solve(None, 1e-10, 0, None) == lib.MHS_ERR_INVALID_ARG
    assert lib.LIB.mhs_set_lower_bz(None, None) == lib.MHS_ERR_INVALID_ARG
    lib.mhs_destroy(None)
