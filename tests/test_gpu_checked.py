"""The bounds-checked build (libshearlet_checked.so, -DSHL_CHECKED) on small
planes: every guarded global access of the transform kernels compares its
index with its buffer's extent and records a miss in a device word instead of
accessing.  Each case runs in a child process that loads the checked library
(SHL_LIBRARY=checked), checks decomposition (float32, bfloat16, dual-weighted,
masked input), reconstruction (plain, thresholded), adjoint, the fused
threshold step and the subband maxima against the FP64 oracle, and requires
the guard word to stay 0."""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:            # the child process runs this file as a script
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 1e-2


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _case(rows, cols, J, B):
    from oracle import bank as Bk
    from oracle import transform as OT
    from paper_2006_04591_gb300 import synth
    from paper_2006_04591_gb300 import shearlet as S
    assert S.shl_checked_build() == 1
    ref = Bk.shearlet_bank(rows, cols, J)
    bank = S.Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    K = ref["spectra"].shape[0]
    x = np.stack([synth.cartoon(rows, cols, 40 + b) for b in range(B)]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    c = bank.decompose(xt)
    assert _rel(c.cpu().numpy(), want) <= TOL32
    assert _rel(bank.decompose(xt, dtype=torch.bfloat16).float().cpu().numpy(), want) <= TOL16
    want_d, _ = OT.decompose_batch(x, ref["psi_hat"], dual=True)
    assert _rel(bank.decompose(xt, dual=True).cpu().numpy(), want_d) <= TOL32
    cc = c.cpu().numpy().astype(np.float64)
    want_r, _ = OT.reconstruct_batch(cc, ref["psi_hat"])
    want_a, _ = OT.reconstruct_batch(cc, ref["psi_hat"], adjoint_only=True)
    assert _rel(bank.reconstruct(c).cpu().numpy(), want_r) <= TOL32
    assert _rel(bank.adjoint(c).cpu().numpy(), want_a) <= TOL32
    th = np.full((B, K), 0.05, np.float32)
    kept = np.where(np.abs(c.cpu().numpy()) >= th[:, :, None, None], c.cpu().numpy(), 0.0)
    want_t, _ = OT.reconstruct_batch(kept, ref["psi_hat"])
    tht = torch.from_numpy(th).cuda()
    assert _rel(bank.reconstruct(c, thresh=tht).cpu().numpy(), want_t) <= TOL32
    assert _rel(bank.shrink(xt, tht).cpu().numpy(), want_t) <= TOL32
    m = np.stack([synth.bernoulli_mask(rows, cols, 0.5, 60 + b) for b in range(B)])
    fe = np.zeros_like(x)
    got_m = bank.decompose_masked(xt, torch.from_numpy(m.astype(np.uint8)).cuda(),
                                  torch.from_numpy(fe).cuda()).cpu().numpy()
    want_m, _ = OT.decompose_batch((m * x).astype(np.float32), ref["psi_hat"])
    assert _rel(got_m, want_m) <= TOL32
    amax = bank.subband_absmax(c).cpu().numpy()
    np.testing.assert_array_equal(amax, np.abs(c.cpu().numpy()).max(axis=(2, 3)))
    assert S.shl_check_status(0) == 0


def _child(*args):
    env = dict(os.environ, SHL_LIBRARY="checked")
    cmd = [sys.executable, os.path.abspath(__file__)] + [str(a) for a in args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout


@pytest.mark.parametrize("rows,cols,J,B", [(16, 16, 1, 2), (16, 16, 2, 3), (32, 64, 2, 2),
                                          (64, 16, 1, 3), (16, 512, 2, 1)])
def test_checked_build_small_planes(rows, cols, J, B):
    _child(rows, cols, J, B)


if __name__ == "__main__":
    from paper_2006_04591_gb300 import _build
    _build.build()
    _case(*[int(a) for a in sys.argv[1:5]])
    print("checked ok")
