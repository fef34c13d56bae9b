"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol the header declares, validates arguments before touching CUDA, and
its float64 host filter-bank builder matches the oracle's construction."""

import ctypes

import numpy as np
import pytest

from oracle import bank as Bk
from paper_2006_04591_gb300 import _build, shearlet as S


@pytest.fixture(scope="module")
def L():
    _build.build()
    return S.lib()


def test_exports_every_header_symbol(L):
    names = S.header_symbols()
    assert len(names) >= 14
    raw = ctypes.CDLL(S.library_path())
    missing = [n for n in names if not hasattr(raw, n)]
    assert missing == []


def test_checked_library_exports_the_same_symbols(L):
    """libshearlet_checked.so (the -DSHL_CHECKED build) carries the same C ABI
    and says that it is the checked build; the main library says it is not."""
    import ctypes
    from paper_2006_04591_gb300 import _build
    from paper_2006_04591_gb300 import shearlet as S
    raw = ctypes.CDLL(_build.LIB_CHECKED)
    for n in S.header_symbols():
        assert hasattr(raw, n), n
    raw.shl_checked_build.restype = ctypes.c_int
    assert raw.shl_checked_build() == 1
    assert S.shl_checked_build() == 0


def test_version_and_status_strings(L):
    assert L.shl_abi_version() == 1
    assert L.shl_status_str(0) == b"ok"
    assert L.shl_status_str(4) == b"unsupported"


def test_unsupported_sizes_rejected(L):
    h = ctypes.c_void_p()
    for r, c in [(4097, 16), (16, 0), (0, 5), (16, 5000), (-3, 8)]:
        st = L.shl_bank_create(r, c, 2, None, 0, -1, ctypes.byref(h))
        assert st == 4 and not h.value
    st = L.shl_bank_create(16, 16, 2, None, 0, -1, None)
    assert st == 1
    # the GPU builder covers the power-of-two sizes only; it rejects others
    # before touching a device
    st = L.shl_bank_create_gpu(15, 16, 2, None, 0, 0, ctypes.byref(h))
    assert st == 4 and not h.value


def test_bank_path_selection(L):
    for (r, c, general) in [(16, 16, 0), (2048, 16, 0), (15, 16, 1), (8, 16, 1), (4096, 16, 1),
                            (1, 1, 1), (17, 4093, 1)]:
        G = np.ones((1, r, c))
        h = S.shl_bank_create_from_spectra(G, device=-1)
        assert S.shl_bank_path(h) == general
        S.shl_bank_destroy(h)
    h = S.shl_bank_create_general(np.ones((1, 16, 16)), device=-1)
    assert S.shl_bank_path(h) == 1
    S.shl_bank_destroy(h)


def test_complex_bank_hermitian_check_and_info():
    rng = np.random.default_rng(3)
    g = rng.standard_normal((3, 9, 7))                     # real, non-symmetric filters
    G = np.fft.fft2(g, axes=(-2, -1))                      # Hermitian spectra
    h = S.shl_bank_create_general(G, idx=np.arange(9).reshape(3, 3), device=-1)
    info = S.shl_bank_copy_info(h)
    np.testing.assert_array_equal(info["spectra"], G.real)
    np.testing.assert_array_equal(S.shl_bank_copy_spectra_imag(h), G.imag)
    np.testing.assert_allclose(info["dual_w"], np.sum(np.abs(G) ** 2, axis=0), rtol=1e-14)
    np.testing.assert_allclose(info["rms"], np.sqrt(np.sum(np.abs(G) ** 2, axis=(1, 2)) / 63),
                               rtol=1e-14)
    np.testing.assert_array_equal(info["idx"], np.arange(9).reshape(3, 3))
    S.shl_bank_destroy(h)
    bad = G.copy()
    bad[1, 2, 3] += 0.5j                                   # breaks G(-k) = conj G(k)
    with pytest.raises(S.ShearletError) as e:
        S.shl_bank_create_general(bad, device=-1)
    assert e.value.status == 1 and "Hermitian" in str(e.value)
    # a real bank given to the complex entry point must still be even
    with pytest.raises(S.ShearletError):
        S.shl_bank_create_general(g, device=-1)


def test_non_even_spectrum_rejected():
    rng = np.random.default_rng(0)
    G = rng.standard_normal((2, 16, 16))
    with pytest.raises(S.ShearletError) as e:
        S.shl_bank_create_from_spectra(G, device=-1)
    assert e.value.status == 1


def test_zero_dual_weight_rejected():
    G = np.zeros((1, 16, 16))
    G[0, 0, 0] = 1.0
    with pytest.raises(S.ShearletError) as e:
        S.shl_bank_create_from_spectra(G, device=-1)
    assert e.value.status == 1


def test_host_only_bank_rejects_transform_calls(L):
    h = S.shl_bank_create(16, 16, 1, device=-1)
    n = ctypes.c_size_t()
    assert L.shl_workspace_size(h, 0, 2, ctypes.byref(n)) == 0 and n.value > 0
    fake = ctypes.c_void_p(1 << 20)
    st = L.shl_decompose(h, fake, 1, fake, 0, 0, fake, n.value, None)
    assert st == 1 and b"host-only" in L.shl_last_error_detail()
    assert L.shl_workspace_size(None, 0, 1, ctypes.byref(n)) == 1
    S.shl_bank_destroy(h)


@pytest.mark.parametrize("rows,cols,J,levels,full", [
    (32, 32, 2, None, False), (64, 64, 3, None, False), (32, 64, 2, None, False),
    (64, 32, 2, [1, 2], True), (32, 32, 1, [0], False),
    # general sizes: float64 Bluestein line DFTs in the host builder
    (45, 60, 2, None, False), (33, 33, 1, None, True), (100, 72, 2, None, False),
    (127, 128, 2, None, False), (7, 5, 1, None, False), (35, 27, 2, [1, 2], True),
])
def test_host_bank_builder_matches_oracle(rows, cols, J, levels, full):
    h = S.shl_bank_create(rows, cols, J, levels, full, device=-1)
    info = S.shl_bank_copy_info(h)
    S.shl_bank_destroy(h)
    ref = Bk.shearlet_bank(rows, cols, J, levels, full)
    assert info["spectra"].shape == ref["spectra"].shape
    np.testing.assert_array_equal(info["idx"], ref["idx"])
    np.testing.assert_allclose(info["spectra"], ref["spectra"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(info["rms"], ref["rms"], rtol=1e-12)
    np.testing.assert_allclose(info["dual_w"], ref["dual_w"], rtol=1e-12)


def test_bad_levels_rejected():
    with pytest.raises(S.ShearletError):
        S.shl_bank_create(32, 32, 2, [1, 7], device=-1)
