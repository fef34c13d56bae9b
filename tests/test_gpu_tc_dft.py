"""GPU parity of the tensor-core column pass of the bfloat16-output
decomposition (tcgen05 DFT stages, switched on with SHL_TC_DFT=1, read once
per process) against the FP64 oracle.

Each test runs its checks in a child process with the switch set and asserts,
from the library's launch profile, which column pass ran.  Planes with 512
rows use the tensor-core pass (512-point columns as a 32 x 16 Cooley-Tukey
split, both stages bfloat16 GEMMs with float32 accumulation); other planes,
and planes with fewer than 8 column frequencies, keep the CUDA-core pass.
Error measure max |gpu - oracle| / max |oracle| per image, <= 1e-2 as for
every bfloat16-stored decomposition; the child also prints the error of the
CUDA-core pass on the same input for comparison.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:            # the child process runs this file as a script
    sys.path.insert(0, ROOT)

from oracle import bank as Bk
from oracle import transform as OT
from paper_2006_04591_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL16 = 1e-2
_BANKS = {}


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _bank(rows, cols, J):
    key = (rows, cols, J)
    if key not in _BANKS:
        from paper_2006_04591_gb300.shearlet import Bank
        ref = Bk.shearlet_bank(rows, cols, J)
        _BANKS[key] = (ref, Bank.from_spectra(ref["spectra"], ref["idx"], device=0))
    return _BANKS[key]


def _images(B, rows, cols, seed):
    return np.stack([synth.cartoon(rows, cols, seed + b) +
                     synth.gaussian_noise((rows, cols), 0.05, 700 + seed + b)
                     for b in range(B)]).astype(np.float32)


def _profile():
    from paper_2006_04591_gb300 import shearlet as S
    return S.shl_profile_read()


def _case_decompose(rows, cols, J, B, expect_tc):
    """bfloat16 decomposition, plain and dual-weighted, against the oracle."""
    ref, bank = _bank(rows, cols, J)
    x = _images(B, rows, cols, 20 + J)
    xt = torch.from_numpy(x).cuda()
    _profile()
    c16 = bank.decompose(xt, dtype=torch.bfloat16).float().cpu().numpy()
    cd16 = bank.decompose(xt, dtype=torch.bfloat16, dual=True).float().cpu().numpy()
    torch.cuda.synchronize()
    prof = _profile()
    assert ("dec_lines_tc" in prof) == expect_tc, sorted(prof)
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    want_d, _ = OT.decompose_batch(x, ref["psi_hat"], dual=True)
    c32 = bank.decompose(xt).cpu().numpy()          # float32 storage, CUDA-core pass
    for b in range(B):
        e16, ed = _rel(c16[b], want[b]), _rel(cd16[b], want_d[b])
        print("image %d: tensor-core %.2e (dual %.2e), float32 pass rounded %.2e"
              % (b, e16, ed, _rel(c32[b].astype(np.float32), want[b])))
        assert e16 <= TOL16, (b, e16)
        assert ed <= TOL16, (b, ed)


def _case_masked():
    """The masked decomposition M (f_m - f) + f of the inpainting step."""
    rows, cols = 512, 64
    ref, bank = _bank(rows, cols, 2)
    B = 2
    fm = _images(B, rows, cols, 40)
    fe = _images(B, rows, cols, 50)
    m = np.stack([synth.bernoulli_mask(rows, cols, 0.5, 60 + b) for b in range(B)])
    u = (m * (fm - fe) + fe).astype(np.float32)
    _profile()
    got = bank.decompose_masked(torch.from_numpy(fm).cuda(),
                                torch.from_numpy(m.astype(np.uint8)).cuda(),
                                torch.from_numpy(fe).cuda(),
                                dtype=torch.bfloat16).float().cpu().numpy()
    torch.cuda.synchronize()
    assert "dec_lines_tc" in _profile()
    want, _ = OT.decompose_batch(u, ref["psi_hat"])
    for b in range(B):
        assert _rel(got[b], want[b]) <= TOL16, b


def _case_chunks():
    """Lines are transformed independently of the tile they share: the
    library's fixed scratch (several staging chunks) gives the same bits as
    one chunk, and a second call repeats them."""
    from paper_2006_04591_gb300 import shearlet as S
    ref, bank = _bank(512, 256, 3)
    x = torch.from_numpy(_images(4, 512, 256, 95)).cuda()
    a = bank.decompose(x, dtype=torch.bfloat16)
    b = torch.empty_like(a)
    S.shl_decompose_noalloc(bank.handle, x, 4, b, S.SHL_BF16, 0)
    assert torch.equal(a, b)
    assert torch.equal(a, bank.decompose(x, dtype=torch.bfloat16))
    torch.cuda.synchronize()
    assert "dec_lines_tc" in _profile()


def _child(name, *args):
    env = dict(os.environ, SHL_TC_DFT="1")
    cmd = [sys.executable, os.path.abspath(__file__), name] + [str(a) for a in args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "tc ok" in r.stdout
    print(r.stdout)


# rows, cols, J, batch, tensor-core pass expected (512 rows and >= 8 column frequencies)
CASES = [(512, 512, 4, 3, 1), (512, 512, 2, 1, 1), (512, 256, 3, 2, 1), (512, 32, 1, 2, 1),
         (512, 1024, 2, 1, 1), (512, 16, 1, 3, 1), (256, 512, 2, 1, 0)]


@pytest.mark.parametrize("rows,cols,J,B,tc", CASES)
def test_tc_decompose_bf16_and_dual(rows, cols, J, B, tc):
    _child("decompose", rows, cols, J, B, tc)


def test_tc_masked_decompose():
    _child("masked")


def test_tc_chunks_and_repeat_give_the_same_bits():
    _child("chunks")


if __name__ == "__main__":
    from paper_2006_04591_gb300 import _build
    from paper_2006_04591_gb300 import shearlet as S
    _build.build()
    S.shl_profile_enable(1)
    name, rest = sys.argv[1], sys.argv[2:]
    args = [int(a) for a in rest]
    if name == "decompose":
        args[-1] = bool(args[-1])
    globals()["_case_" + name](*args)
    torch.cuda.synchronize()
    S.shl_sync()                    # raises if a bounded MMA wait ran out
    print("tc ok")
