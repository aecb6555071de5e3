"""A8: the differentiable TOD chi^2 on the GPU (autograd Function with the
hand-written adjoint) against the FP64 oracle's value and gradients, and a
central finite difference through the GPU forward."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_03509_gb300 as tg
    cfg = synth.scaled(synth.CONFIGS["chi2"], nscan=3, len_lo=16384, len_hi=16384, flag_frac=0.02)
    band = synth.make_band(cfg)
    ing = tg.ingest(band)
    off = ing["offsets"]
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"],
                   ing["psi_streams"], cluster_size=2)
    dev = torch.device("cuda:0")
    N = int(off[-1])
    pix = torch.empty(N, dtype=torch.int32, device=dev)
    psi = torch.empty(N, dtype=torch.int16, device=dev)
    plan.decode(pix, psi)
    m32 = band.map_tqu.T.astype(np.float32)                    # (npix, 3), FP32 values
    return dict(tg=tg, torch=torch, cfg=cfg, band=band, ing=ing, plan=plan, dev=dev, pix=pix, psi=psi,
                m32=m32, d=torch.from_numpy(ing["tod"]).to(dev),
                flags=torch.from_numpy(ing["flag_words"].view(np.int32)).to(dev))


def _oracle(S, map_tqu_3n, gains, psd):
    band, ing = S["band"], S["ing"]
    off = ing["offsets"]
    nq = len(off) - 1
    pix = np.concatenate([band.pix[q][:off[q + 1] - off[q]] for q in range(nq)])
    psi = np.concatenate([band.psi[q][:off[q + 1] - off[q]] for q in range(nq)])
    mask = (~ing["flags"]).astype(np.float64)
    return oracle.chi2_band(map_tqu_3n, pix, psi, ing["tod"].astype(np.float64), gains, mask, psd, off,
                            S["cfg"].ndet, S["cfg"].fsamp)


def test_chi2_value_and_gradients_match_oracle(setup):
    S = setup
    torch = S["torch"]
    from paper_2201_03509_gb300.chi2 import tod_chi2
    gains = S["band"].gain.copy()
    psd = S["band"].psd.copy()
    tm = torch.from_numpy(S["m32"].astype(np.float64)).to(S["dev"]).requires_grad_(True)
    tgain = torch.from_numpy(gains).to(S["dev"]).requires_grad_(True)
    tpsd = torch.from_numpy(psd).to(S["dev"]).requires_grad_(True)
    L = tod_chi2(tm, tgain, tpsd, S["plan"], S["d"], S["flags"], S["pix"], S["psi"])
    L.backward()
    S["plan"].status()
    ref = _oracle(S, S["m32"].T.astype(np.float64), gains, psd)
    assert float(L) == pytest.approx(ref["L"], rel=1e-6)
    gm = tm.grad.cpu().numpy().T
    assert np.abs(gm - ref["dm"]).max() <= 1e-4 * np.abs(ref["dm"]).max()
    gg = tgain.grad.cpu().numpy()
    assert np.abs(gg - ref["dg"]).max() <= 1e-4 * np.abs(ref["dg"]).max()
    gp = tpsd.grad.cpu().numpy()
    for j in range(3):
        assert np.abs(gp[:, j] - ref["dpsd"][:, j]).max() <= 1e-4 * np.abs(ref["dpsd"][:, j]).max()


def test_chi2_gain_gradient_matches_gpu_finite_difference(setup):
    """Central difference of the GPU forward itself.  The chi-squared is
    quadratic in each gain, so the central difference is exact for any step;
    a step of the gain's own size keeps the difference far above the FP32
    rounding of the transforms (FP64 sums of FP32 values)."""
    S = setup
    torch = S["torch"]
    from paper_2201_03509_gb300.chi2 import tod_chi2
    gains = torch.from_numpy(S["band"].gain.copy()).to(S["dev"])
    psd = torch.from_numpy(S["band"].psd.copy()).to(S["dev"])
    tm = torch.from_numpy(S["m32"].astype(np.float64)).to(S["dev"])
    g = gains.clone().requires_grad_(True)
    L = tod_chi2(tm, g, psd, S["plan"], S["d"], S["flags"], S["pix"], S["psi"])
    L.backward()
    q = 1
    h = 1.0
    gp, gmn = gains.clone(), gains.clone()
    gp[q] += h
    gmn[q] -= h
    num = (float(tod_chi2(tm, gp, psd, S["plan"], S["d"], S["flags"], S["pix"], S["psi"]))
           - float(tod_chi2(tm, gmn, psd, S["plan"], S["d"], S["flags"], S["pix"], S["psi"]))) / (2 * h)
    assert float(g.grad[q]) == pytest.approx(num, rel=1e-4)
