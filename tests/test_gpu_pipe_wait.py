"""The pipelined decomposition (opt-in, SHL_PIPE=1) against the oracle and,
bit for bit with float32 coefficients, against the two-launch path; and its waits are bounded: with every ROW wait made
unsatisfiable (SHL_PIPE_STALL_TEST=1, a count that no item reaches), the
launch ends by itself, shl_sync reports SHL_ETIMEOUT, and the same process
then decomposes correctly.  Runs in a child process so that the variable
stays out of the other tests."""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, time, numpy as np, torch
    from oracle import bank as Bk
    from oracle import transform as OT
    from paper_2006_04591_gb300 import shearlet as S
    ref = Bk.shearlet_bank(512, 512, 2)
    bank = S.Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 512, 512)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    L = S.lib()
    os.environ["SHL_PIPE_STALL_TEST"] = "1"
    t0 = time.time()
    bank.decompose(xt)
    st = L.shl_sync(None)
    dt = time.time() - t0
    os.environ["SHL_PIPE_STALL_TEST"] = "0"
    assert st == S.SHL_ETIMEOUT, st
    assert dt < 30, dt
    c = bank.decompose(xt).cpu().numpy()
    assert L.shl_sync(None) == 0
    want, _ = OT.decompose_batch(x, ref["psi_hat"])
    err = np.abs(c - want).max() / np.abs(want).max()
    assert err <= 1e-5, err
    print("stall ok %.2f s" % dt)
""")


def test_pipe_wait_runs_out_and_reports():
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    env["SHL_PIPE"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "stall ok" in r.stdout


PARITY = textwrap.dedent("""
    import numpy as np, torch
    from oracle import bank as Bk
    from oracle import transform as OT
    from paper_2006_04591_gb300 import shearlet as S
    from paper_2006_04591_gb300 import synth
    for (rows, cols, J, B) in [(512, 512, 2, 5), (512, 1024, 2, 1), (512, 512, 4, 2)]:
        ref = Bk.shearlet_bank(rows, cols, J)
        bank = S.Bank.from_spectra(ref["spectra"], ref["idx"], device=0)
        x = np.stack([synth.cartoon(rows, cols, 40 + b) for b in range(B)]).astype(np.float32)
        xt = torch.from_numpy(x).cuda()
        for dt, dual, tol in [(torch.float32, False, 1e-5), (torch.bfloat16, False, 1e-2),
                              (torch.float32, True, 1e-5)]:
            c = bank.decompose(xt, dtype=dt, dual=dual)
            assert S.lib().shl_sync(None) == 0
            # the two-launch path with a small staging area: the same
            # arithmetic for float32 coefficients (bfloat16 coefficients: it
            # stages the half spectra in bfloat16, the pipelined path in
            # float32, so both are held to the oracle below instead)
            c2 = torch.empty_like(c)
            S.shl_decompose_noalloc(bank.handle, xt, B, c2, S._dtype_code(dt),
                                    S.SHL_DUAL_WEIGHTED if dual else 0)
            if dt == torch.float32:
                assert torch.equal(c, c2), (rows, cols, J, B, dt, dual)
            else:
                w16, _ = OT.decompose_batch(x, ref["psi_hat"], dual=dual)
                g16 = c2.float().cpu().numpy()
                for b in range(B):
                    e16 = np.abs(g16[b] - w16[b]).max() / np.abs(w16[b]).max()
                    assert e16 <= tol, (rows, cols, J, b, dt, dual, e16)
            want, _ = OT.decompose_batch(x, ref["psi_hat"], dual=dual)
            got = c.float().cpu().numpy()
            for b in range(B):
                err = np.abs(got[b] - want[b]).max() / np.abs(want[b]).max()
                assert err <= tol, (rows, cols, J, b, dt, dual, err)
    print("pipe parity ok")
""")


def test_pipe_parity_and_bit_equality():
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    env["SHL_PIPE"] = "1"
    r = subprocess.run([sys.executable, "-c", PARITY], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "pipe parity ok" in r.stdout
