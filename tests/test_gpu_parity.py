"""GPU parity: the CUDA transform against the FP64 oracle, element by element.

Inputs are seeded (``synth``); the filter banks are built by the oracle and
handed to the library with ``shl_bank_create_from_spectra``, so no oracle
input comes from the CUDA path.  Error measure: max |gpu - oracle| / max
|oracle| per image (float32 path <= 1e-5, bfloat16-stored coefficients
<= 1e-2).  Thresholded reconstructions compare |c| with the same float32
threshold on both sides, so the keep/zero decisions are identical.
"""

import numpy as np
import pytest

from oracle import apps as OA
from oracle import bank as Bk
from oracle import transform as OT
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 1e-2


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_BANKS = {}


def _bank(rows, cols, J):
    key = (rows, cols, J)
    if key not in _BANKS:
        from paper_2006_04591_gb300.shearlet import Bank
        ref = Bk.shearlet_bank(rows, cols, J)
        _BANKS[key] = (ref, Bank.from_spectra(ref["spectra"], ref["idx"], device=0))
    return _BANKS[key]


def _images(B, rows, cols, seed):
    return np.stack([synth.cartoon(rows, cols, seed + b) +
                     synth.gaussian_noise((rows, cols), 0.05, 900 + seed + b)
                     for b in range(B)]).astype(np.float32)


CASES = [(16, 16, 1, 1), (16, 32, 2, 3), (64, 16, 2, 2), (32, 32, 2, 2),
         (128, 128, 3, 2), (256, 256, 3, 8), (64, 2048, 2, 1), (2048, 32, 2, 1)]


@pytest.mark.parametrize("rows,cols,J,B", CASES)
def test_decompose_f32(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    x = _images(B, rows, cols, 10)
    c = bank.decompose(torch.from_numpy(x).cuda()).cpu().numpy()
    want, imag = OT.decompose_batch(x, ref["psi_hat"])
    assert imag < 1e-9 * np.abs(want).max()
    for b in range(B):
        assert _rel(c[b], want[b]) <= TOL32, b


@pytest.mark.parametrize("rows,cols,J,B", CASES[:6])
def test_decompose_bf16(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    x = _images(B, rows, cols, 20)
    c = bank.decompose(torch.from_numpy(x).cuda(), dtype=torch.bfloat16)
    c = c.float().cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    for b in range(B):
        assert _rel(c[b], want[b]) <= TOL16, b


@pytest.mark.parametrize("rows,cols,J,B", CASES)
def test_reconstruct_and_adjoint_f32(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    K = ref["spectra"].shape[0]
    rng = np.random.default_rng(rows * 7 + cols)
    c = rng.standard_normal((B, K, rows, cols)).astype(np.float32)
    ct = torch.from_numpy(c).cuda()
    rec = bank.reconstruct(ct).cpu().numpy()
    adj = bank.adjoint(ct).cpu().numpy()
    want_r, _ = OT.reconstruct_batch(c, ref["psi_hat"])
    want_a, _ = OT.reconstruct_batch(c, ref["psi_hat"], adjoint_only=True)
    for b in range(B):
        assert _rel(rec[b], want_r[b]) <= TOL32, b
        assert _rel(adj[b], want_a[b]) <= TOL32, b


@pytest.mark.parametrize("rows,cols,J,B", CASES[:6])
def test_reconstruct_bf16_input(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    K = ref["spectra"].shape[0]
    rng = np.random.default_rng(5)
    c16 = torch.from_numpy(rng.standard_normal((B, K, rows, cols)).astype(np.float32)).bfloat16()
    rec = bank.reconstruct(c16.cuda()).cpu().numpy()
    want, _ = OT.reconstruct_batch(c16.float().numpy(), ref["psi_hat"])
    for b in range(B):
        assert _rel(rec[b], want[b]) <= TOL32, b


@pytest.mark.parametrize("rows,cols,J,B", [(32, 32, 2, 2), (256, 256, 3, 3), (32, 64, 2, 2)])
def test_dual_weighted_decompose(rows, cols, J, B):
    ref, bank = _bank(rows, cols, J)
    x = _images(B, rows, cols, 30)
    c = bank.decompose(torch.from_numpy(x).cuda(), dual=True).cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"], dual=True)
    for b in range(B):
        assert _rel(c[b], want[b]) <= TOL32, b


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_thresholded_reconstruct(dtype):
    rows = cols = 64
    ref, bank = _bank(rows, cols, 2)
    K = ref["spectra"].shape[0]
    B = 3
    rng = np.random.default_rng(11)
    c = torch.from_numpy(rng.standard_normal((B, K, rows, cols)).astype(np.float32))
    if dtype == "bf16":
        c = c.bfloat16()
    th = torch.from_numpy(rng.uniform(0, 1.5, size=(B, K)).astype(np.float32))
    th[0, 0] = 0.0
    cf = c.float().numpy()
    thn = th.numpy()
    kept = np.where(np.abs(cf) >= thn[:, :, None, None], cf, 0.0)   # same f32 compare
    want, _ = OT.reconstruct_batch(kept, ref["psi_hat"])
    got = bank.reconstruct(c.cuda(), thresh=th.cuda()).cpu().numpy()
    for b in range(B):
        assert _rel(got[b], want[b]) <= TOL32


def test_threshold_tie_is_kept():
    ref, bank = _bank(16, 16, 1)
    K = ref["spectra"].shape[0]
    c = np.zeros((1, K, 16, 16), np.float32)
    c[0, 1, 3, 4] = 0.5
    c[0, 2, 5, 6] = -0.5
    c[0, 3, 7, 8] = 0.49999997
    th = np.full((1, K), 0.5, np.float32)
    got = bank.reconstruct(torch.from_numpy(c).cuda(), thresh=torch.from_numpy(th).cuda())
    kept = c.copy()
    kept[0, 3, 7, 8] = 0.0
    want, _ = OT.reconstruct_batch(kept, ref["psi_hat"])
    assert _rel(got.cpu().numpy()[0], want[0]) <= TOL32


def test_masked_decompose():
    rows = cols = 64
    ref, bank = _bank(rows, cols, 2)
    B = 2
    fm = _images(B, rows, cols, 40)
    fe = _images(B, rows, cols, 50)
    m = np.stack([synth.bernoulli_mask(rows, cols, 0.5, 60 + b) for b in range(B)])
    u = (m * (fm - fe) + fe).astype(np.float32)
    got = bank.decompose_masked(torch.from_numpy(fm).cuda(),
                                torch.from_numpy(m.astype(np.uint8)).cuda(),
                                torch.from_numpy(fe).cuda()).cpu().numpy()
    want, _ = OT.decompose_batch(u, ref["psi_hat"])
    for b in range(B):
        assert _rel(got[b], want[b]) <= TOL32


def test_subband_absmax():
    ref, bank = _bank(32, 32, 2)
    rng = np.random.default_rng(3)
    c = rng.standard_normal((2, 17, 32, 32)).astype(np.float32)
    got = bank.subband_absmax(torch.from_numpy(c).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, np.abs(c).max(axis=(2, 3)))
    got = bank.subband_absmax(torch.from_numpy(c).cuda(), by_rms=True).cpu().numpy()
    np.testing.assert_allclose(got, np.abs(c).max(axis=(2, 3)) / ref["rms"][None], rtol=1e-6)


def test_empty_batch_is_noop():
    ref, bank = _bank(32, 32, 2)
    x = torch.empty((0, 32, 32), device="cuda")
    c = bank.decompose(x)
    assert c.shape == (0, 17, 32, 32)
    r = bank.reconstruct(c)
    assert r.shape == (0, 32, 32)


def test_perfect_reconstruction_property():
    ref, bank = _bank(256, 256, 3)
    x = torch.from_numpy(_images(4, 256, 256, 70)).cuda()
    r = bank.reconstruct(bank.decompose(x))
    assert (r - x).abs().max().item() <= TOL32 * x.abs().max().item()


def test_library_bank_matches_oracle_on_device():
    from paper_2006_04591_gb300.shearlet import Bank
    b = Bank.create(64, 64, 3, device=0)
    ref = Bk.shearlet_bank(64, 64, 3)
    np.testing.assert_allclose(b.info()["spectra"], ref["spectra"], atol=1e-12)
    x = _images(2, 64, 64, 80)
    c = b.decompose(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    for i in range(2):
        assert _rel(c[i], want[i]) <= TOL32


# --------------------------------------------- full size (bench launch config)
def test_full_size_512_k49_sampled():
    """512 x 512, K = 49, B = 16 in one call; sampled subbands vs the oracle."""
    ref, bank = _bank(512, 512, 4)
    B = 16
    x = np.stack([synth.cartoon(512, 512, 100 + b) for b in range(B)]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    c = bank.decompose(xt)
    rng = np.random.default_rng(0)
    for _ in range(6):
        b, i = int(rng.integers(B)), int(rng.integers(49))
        want = OT.decompose(x[b], ref["psi_hat"][i:i + 1]).real[0]
        assert _rel(c[b, i].cpu().numpy(), want) <= TOL32, (b, i)
    r = bank.reconstruct(c)
    for b in (0, B - 1):
        want = OT.reconstruct(c[b].cpu().numpy().astype(np.float64), ref["psi_hat"]).real
        assert _rel(r[b].cpu().numpy(), want) <= TOL32
    assert (r - xt).abs().max().item() <= TOL32 * xt.abs().max().item()


# ------------------------------------------------------------ rows of 512
@pytest.mark.parametrize("rows,J,B", [(16, 1, 3), (256, 3, 2), (1024, 2, 1), (512, 2, 5)])
def test_rows_of_512_decompose_f32_bf16_dual(rows, J, B):
    """Rows of 512 (the benchmark's row length) with other column lengths and
    batches of odd subband counts, in float32, bfloat16 and dual-weighted
    form."""
    ref, bank = _bank(rows, 512, J)
    x = _images(B, rows, 512, 90)
    xt = torch.from_numpy(x).cuda()
    c32 = bank.decompose(xt).cpu().numpy()
    c16 = bank.decompose(xt, dtype=torch.bfloat16).float().cpu().numpy()
    cd = bank.decompose(xt, dual=True).cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    want_d, _ = OT.decompose_batch(x, ref["psi_hat"], dual=True)
    for b in range(B):
        assert _rel(c32[b], want[b]) <= TOL32, b
        assert _rel(c16[b], want[b]) <= TOL16, b
        assert _rel(cd[b], want_d[b]) <= TOL32, b


def test_chunking_does_not_change_results():
    """One staging chunk (the default of the staged kernels, which run the
    512 x 256 planes) and many small chunks (the fixed scratch of
    shl_decompose_noalloc: three chunks here) run the same arithmetic: equal
    bits."""
    from paper_2006_04591_gb300 import shearlet as S
    ref, bank = _bank(512, 256, 3)
    x = torch.from_numpy(_images(4, 512, 256, 95)).cuda()
    a = bank.decompose(x)
    b = torch.empty_like(a)
    S.shl_decompose_noalloc(bank.handle, x, 4, b, S.SHL_F32, 0)
    assert torch.equal(a, b)


# ------------------------------------------- images in mapped pinned memory
def test_pinned_host_images_give_the_same_bits():
    """Images in pinned host memory are read / written by the first / last
    kernel over the CPU-GPU link: the same bits as with device images."""
    ref, bank = _bank(256, 256, 3)
    x = _images(3, 256, 256, 97)
    xd = torch.from_numpy(x).cuda()
    xh = torch.from_numpy(x).pin_memory()
    c_dev = bank.decompose(xd)
    c_host = bank.decompose(xh)
    torch.cuda.synchronize()
    assert torch.equal(c_dev, c_host)
    yh = torch.empty((3, 256, 256), dtype=torch.float32).pin_memory()
    bank.reconstruct(c_dev, out=yh)
    torch.cuda.synchronize()
    assert torch.equal(bank.reconstruct(c_dev).cpu(), yh)
    th = torch.full((3, bank.K), 0.05)
    sh = torch.empty((3, 256, 256), dtype=torch.float32).pin_memory()
    bank.shrink(xh, th, out=sh)
    torch.cuda.synchronize()
    assert torch.equal(bank.shrink(xd, th).cpu(), sh)


def test_unmapped_host_memory_is_rejected():
    from paper_2006_04591_gb300 import shearlet as S
    ref, bank = _bank(32, 32, 2)
    x = torch.zeros((1, 32, 32))                       # pageable, not registered
    c = torch.empty((1, bank.K, 32, 32), device="cuda")
    ws = bank.workspace(S.SHL_OP_DECOMPOSE, 1)
    with pytest.raises(S.ShearletError):
        S.shl_decompose(bank.handle, x, 1, c, S.SHL_F32, 0, ws)


# ----------------------------------------------------- sizes and degenerate banks
def test_max_size_2048():
    """2048 x 2048 (the largest size the library takes), 2 scales: sampled
    subbands against the oracle, perfect reconstruction, adjoint identity."""
    ref, bank = _bank(2048, 2048, 2)
    x = _images(1, 2048, 2048, 123)
    xt = torch.from_numpy(x).cuda()
    c = bank.decompose(xt)
    c16 = bank.decompose(xt, dtype=torch.bfloat16)     # bfloat16 staging at 2048-long rows
    for i in (0, 5, 16):
        want = OT.decompose(x[0], ref["psi_hat"][i:i + 1]).real[0]
        assert _rel(c[0, i].cpu().numpy(), want) <= TOL32, i
        assert _rel(c16[0, i].float().cpu().numpy(), want) <= TOL16, i
    del c16
    r = bank.reconstruct(c)
    assert (r - xt).abs().max().item() <= TOL32 * xt.abs().max().item()
    w = torch.randn(c.shape, generator=torch.Generator().manual_seed(3)).cuda()
    a = bank.adjoint(w)
    lhs = (c.double() * w.double()).sum().item()
    rhs = (xt.double() * a.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_identity_bank_is_identity():
    """One filter G = 1 (W = 1): decomposition and reconstruction return the image."""
    from paper_2006_04591_gb300.shearlet import Bank
    bank = Bank.from_spectra(np.ones((1, 64, 128)), device=0)
    x = torch.from_numpy(_images(2, 64, 128, 7)).cuda()
    c = bank.decompose(x)
    assert c.shape == (2, 1, 64, 128)
    assert (c[:, 0] - x).abs().max().item() <= 1e-6 * x.abs().max().item()
    assert (bank.reconstruct(c) - x).abs().max().item() <= 1e-6 * x.abs().max().item()
    assert (bank.adjoint(c) - x).abs().max().item() <= 1e-6 * x.abs().max().item()


def test_single_scale_bank():
    """J = 1 (one scale, shear level 1): parity and perfect reconstruction."""
    ref, bank = _bank(128, 64, 1)
    x = _images(2, 128, 64, 11)
    c = bank.decompose(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    for b in range(2):
        assert _rel(c[b], want[b]) <= TOL32
    r = bank.reconstruct(torch.from_numpy(c).cuda()).cpu().numpy()
    assert np.abs(r - x).max() <= TOL32 * np.abs(x).max()
