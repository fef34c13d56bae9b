"""Checkpoint / resume of the learned parts and the on-disk filter-bank
cache (host-only banks and CPU modules: no GPU needed)."""

import os

import numpy as np
import pytest
import torch

from paper_2006_04591_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def test_bank_cache_round_trip(tmp_path):
    from paper_2006_04591_gb300.shearlet import Bank
    d = str(tmp_path)
    for rows, cols, J, general in ((32, 64, 2, False), (45, 60, 2, True)):
        a = Bank.cached(d, rows, cols, J, device=-1)
        key = Bank.cache_key(rows, cols, J)
        path = os.path.join(d, "bank_%s.npz" % key)
        assert os.path.exists(path) and a.general == general
        mtime = os.path.getmtime(path)
        b = Bank.cached(d, rows, cols, J, device=-1)          # served from the file
        assert os.path.getmtime(path) == mtime and b.general == general
        ia, ib = a.info(), b.info()
        np.testing.assert_array_equal(ia["spectra"], ib["spectra"])
        np.testing.assert_array_equal(ia["idx"], ib["idx"])
        np.testing.assert_array_equal(ia["dual_w"], ib["dual_w"])
        with pytest.raises(ValueError):
            Bank.load(path, device=-1, key="not-this-one")
    assert Bank.cache_key(32, 64, 2) != Bank.cache_key(32, 64, 2, full=True)
    assert Bank.cache_key(32, 64, 2) != Bank.cache_key(32, 64, 2, [1, 2])


def test_bank_cache_key_tracks_builder_and_cleans_up(tmp_path, monkeypatch):
    """A changed builder version changes the key (no stale spectra), and a
    save that fails leaves no temporary file in the cache directory."""
    from paper_2006_04591_gb300 import shearlet as S
    k1 = S.Bank.cache_key(32, 64, 2)
    monkeypatch.setattr(S, "bank_builder_version", lambda: 10**6)
    assert S.Bank.cache_key(32, 64, 2) != k1

    def boom(self, path, key=""):
        open(path, "wb").write(b"partial")
        raise OSError("disk full")
    monkeypatch.setattr(S.Bank, "save", boom)
    with pytest.raises(OSError):
        S.Bank.cached(str(tmp_path), 32, 64, 2, device=-1)
    assert os.listdir(str(tmp_path)) == []


def test_complex_bank_save_load(tmp_path):
    from paper_2006_04591_gb300.shearlet import Bank
    g = np.random.default_rng(0).standard_normal((3, 9, 7))
    G = np.fft.fft2(g, axes=(-2, -1))
    a = Bank.from_complex_spectra(G, device=-1)
    p = str(tmp_path / "c.npz")
    a.save(p)
    b = Bank.load(p, device=-1)
    assert b.general
    np.testing.assert_array_equal(b.info()["spectra_imag"], G.imag)


def test_checkpoint_round_trip(tmp_path):
    from paper_2006_04591_gb300 import nn
    net = nn.CoeffNet(5, ch=8, seed=1, device="cpu", tc=False)
    opt = nn.Adam(net.parameters(), lr=3e-4, betas=(0.9, 0.99))
    for k, (m, v) in enumerate(zip(opt.m, opt.v)):
        m.fill_(0.1 * k)
        v.fill_(0.01 * k)
    opt.step_count = 17
    p = str(tmp_path / "ck.pt")
    nn.save_checkpoint(p, net, opt, step=17, meta={"domain": "test"})
    net2 = nn.CoeffNet(5, ch=8, seed=2, device="cpu", tc=False)
    opt2 = nn.Adam(net2.parameters())
    step, meta = nn.load_checkpoint(p, net2, opt2)
    assert step == 17 and meta == {"domain": "test"}
    for (k, a), (_, b) in zip(net.state_dict().items(), net2.state_dict().items()):
        assert torch.equal(a, b), k
    assert opt2.step_count == 17 and opt2.lr == 3e-4 and opt2.b2 == 0.99
    assert all(torch.equal(a, b) for a, b in zip(opt.m + opt.v, opt2.m + opt2.v))
    with pytest.raises(ValueError):
        nn.load_checkpoint(p, nn.CoeffNet(6, ch=8, device="cpu", tc=False))
    st = torch.load(p, weights_only=False)
    st["version"] = 99
    torch.save(st, p)
    with pytest.raises(ValueError):
        nn.load_checkpoint(p, net2)


def test_lpd_resume_checks_the_run_and_keeps_the_schedule(tmp_path):
    """A learned primal-dual checkpoint is resumed only by a run of the same
    domain, size, angle and scale counts; the cosine schedule is the one the
    checkpoint records (held at its end when a run asks for more steps)."""
    from paper_2006_04591_gb300 import lpd, nn
    net = nn.CoeffNet(3, ch=4, seed=0, device="cpu", tc=False)
    p = str(tmp_path / "lpd.pt")
    meta = {"domain": "shearlet", "size": 128, "angles": 30, "scales": 2, "steps": 400, "lr": 1e-3}
    nn.save_checkpoint(p, net, step=200, meta=meta)
    assert lpd.resume_meta(p, "shearlet", 128, 30, 2)["steps"] == 400
    for bad in (("image", 128, 30, 2), ("shearlet", 64, 30, 2), ("shearlet", 128, 60, 2),
                ("shearlet", 128, 30, 3)):
        with pytest.raises(ValueError):
            lpd.resume_meta(p, *bad)
    assert lpd.cosine_lr(1e-3, 0, 400) == pytest.approx(1e-3)
    assert lpd.cosine_lr(1e-3, 200, 400) == pytest.approx(0.5e-3)
    assert lpd.cosine_lr(1e-3, 400, 400) == pytest.approx(0.0, abs=1e-12)
    assert lpd.cosine_lr(1e-3, 900, 400) == pytest.approx(0.0, abs=1e-12)
