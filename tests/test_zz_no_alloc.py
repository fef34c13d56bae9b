"""shl_decompose_noalloc: the decomposition for callers that cannot allocate.

Callers such as plug-ins whose host framework owns all device memory, or
latency-critical loops that must not call cudaMalloc, use this entry point;
it takes its scratch from an array compiled into the library instead of a
caller-provided workspace.  Its results must equal those of shl_decompose
(same kernels, same arithmetic), call after call: the shared scratch keeps the
previous call's contents, which must not leak into the next result.

This file is collected last so that a run stopping at the first failure has
run every other test before it; it sets up everything it needs itself, so it
also passes alone in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _rel(a, b):
    a = a.double()
    b = b.double()
    return ((a - b).abs().max() / b.abs().max().clamp_min(1e-300)).item()


def test_noalloc_matches_workspace_entry_on_consecutive_calls():
    from paper_2006_04591_gb300 import _build, synth
    from paper_2006_04591_gb300 import shearlet as S
    _build.build()
    bank = S.Bank.create(256, 256, 3, device=0)
    B = 4
    xs = [torch.from_numpy(np.stack([synth.cartoon(256, 256, 300 + 10 * k + b)
                                     for b in range(B)]).astype(np.float32)).cuda()
          for k in range(2)]
    for flags, dtype, code in [(0, torch.float32, S.SHL_F32),
                               (S.SHL_DUAL_WEIGHTED, torch.bfloat16, S.SHL_BF16)]:
        for x in xs:                       # two calls in a row, different inputs
            want = bank.decompose(x, dtype=dtype, dual=bool(flags))
            got = torch.full_like(want, float("nan"))
            S.shl_decompose_noalloc(bank.handle, x, B, got, code, flags)
            torch.cuda.synchronize()
            assert torch.isfinite(got.float()).all()
            tol = TOL32 if dtype == torch.float32 else 1e-2
            assert _rel(got.float(), want.float()) <= tol


def test_noalloc_rejects_batches_beyond_its_scratch():
    """The first batch beyond the documented limit is refused.  The buffers are
    sized for that batch, so a regression in the bound check gives a wrong
    result and a failed assertion here, never an access out of bounds."""
    from paper_2006_04591_gb300 import _build
    from paper_2006_04591_gb300 import shearlet as S
    _build.build()
    N = 512
    bank = S.Bank.create(N, N, 2, device=0)
    ok = S.noalloc_max_batch(N, N)
    assert ok == 30                       # the header's example: batch <= 30 at 512 x 512
    bad = ok + 1
    x = torch.zeros((bad, N, N), device="cuda")
    c = torch.zeros((bad, bank.K, N, N), device="cuda")
    with pytest.raises(S.ShearletError) as e:
        S.shl_decompose_noalloc(bank.handle, x, bad, c, S.SHL_F32, 0)
    assert e.value.status == 1 and "batch too large" in str(e.value)
    # the wrapper refuses buffers smaller than the batch before any launch
    with pytest.raises(ValueError):
        S.shl_decompose_noalloc(bank.handle, x[:1], 2, c, S.SHL_F32, 0)


def test_noalloc_general_size_matches_workspace_entry():
    """A bank on the general kernels (non-power-of-two size) through the same
    fixed scratch: two calls in a row equal shl_decompose bit for bit."""
    from oracle import bank as Bk
    from paper_2006_04591_gb300 import _build, synth
    from paper_2006_04591_gb300 import shearlet as S
    _build.build()
    N, M = 45, 60
    ref = Bk.shearlet_bank(N, M, 2)
    bank = S.Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    assert bank.general
    B = 3
    for k in range(2):
        x = torch.from_numpy(np.stack([synth.cartoon(N, M, 700 + 10 * k + b)
                                       for b in range(B)]).astype(np.float32)).cuda()
        want = bank.decompose(x)
        got = torch.full_like(want, float("nan"))
        S.shl_decompose_noalloc(bank.handle, x, B, got, S.SHL_F32, 0)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
