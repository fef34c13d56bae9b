"""Filter-bank construction on the GPU (shl_bank_create_gpu) against the host
float64 builder and against the oracle's bank: the same construction in
float64, so the spectra agree to float64 rounding; and a transform with the
GPU-built bank matches the oracle."""

import numpy as np
import pytest

from oracle import bank as Bk
from oracle import transform as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rows,cols,J,levels,full", [
    (64, 64, 2, None, 0), (128, 256, 3, None, 0), (256, 128, 3, None, 1),
    (512, 512, 4, None, 0), (64, 128, 3, [0, 1, 3], 0), (2048, 32, 2, None, 0)])
def test_gpu_bank_equals_host_bank(rows, cols, J, levels, full):
    from paper_2006_04591_gb300 import shearlet as S
    host = S.shl_bank_copy_info(S.shl_bank_create(rows, cols, J, levels, full, device=-1))
    gpu = S.Bank.create(rows, cols, J, levels, bool(full), device=0, on_gpu=True).info()
    np.testing.assert_array_equal(gpu["idx"], host["idx"])
    scale = np.abs(host["spectra"]).max()
    assert np.abs(gpu["spectra"] - host["spectra"]).max() <= 1e-12 * scale
    assert np.abs(gpu["dual_w"] - host["dual_w"]).max() <= 1e-12 * np.abs(host["dual_w"]).max()
    np.testing.assert_allclose(gpu["rms"], host["rms"], rtol=1e-12)


def test_gpu_bank_matches_oracle_and_transforms():
    from paper_2006_04591_gb300 import shearlet as S
    from paper_2006_04591_gb300 import synth
    ref = Bk.shearlet_bank(128, 128, 3)
    bank = S.Bank.create(128, 128, 3, device=0, on_gpu=True)
    info = bank.info()
    assert np.abs(info["spectra"] - ref["spectra"]).max() <= 1e-10
    x = np.stack([synth.cartoon(128, 128, 40 + b) for b in range(2)]).astype(np.float32)
    c = bank.decompose(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    for b in range(2):
        assert np.abs(c[b] - want[b]).max() <= 1e-5 * np.abs(want[b]).max()
    r = bank.reconstruct(torch.from_numpy(c).cuda()).cpu().numpy()
    assert np.abs(r - x).max() <= 1e-5 * np.abs(x).max()


def test_gpu_bank_rejects_bad_arguments():
    from paper_2006_04591_gb300 import shearlet as S
    with pytest.raises(S.ShearletError):
        S.shl_bank_create_gpu(100, 128, 3, device=0)
    with pytest.raises(S.ShearletError):
        S.shl_bank_create_gpu(128, 128, 3, device=-1)
    with pytest.raises(S.ShearletError):
        S.shl_bank_create_gpu(128, 128, 2, [0, 5], device=0)
