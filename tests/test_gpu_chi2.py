"""A8: the differentiable TOD chi^2 on the GPU (autograd Function with the
hand-written adjoint) against the FP64 oracle's value and gradients, in the
FP32 and FP64 variants, on a small flagged band and on the full autograd
workload (4 detectors x 200 scans x 65536 samples, Nside 256); and central
finite differences of the GPU's own FP64 chi^2 in the map, a gain and every
noise parameter against its analytic gradient (1e-4 relative)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup(cfg):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_03509_gb300 as tg
    band = synth.make_band(cfg)
    ing = tg.ingest(band)
    off = ing["offsets"]
    plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, off, ing["pix_streams"], ing["psi_streams"])
    dev = torch.device("cuda:0")
    m32 = band.map_tqu.T.astype(np.float32)                    # (npix, 3), FP32 values
    # noise parameters away from the simulation's, so that no gradient sits at a stationary point
    psd = band.psd.copy()
    psd[:, 0] *= 1.1
    psd[:, 1] *= 1.2
    psd[:, 2] += 0.1
    return dict(tg=tg, torch=torch, cfg=cfg, band=band, ing=ing, plan=plan, dev=dev, m32=m32, psd=psd,
                d=torch.from_numpy(ing["tod"]).to(dev),
                flags=torch.from_numpy(ing["flag_words"].view(np.int32)).to(dev))


@pytest.fixture(scope="module")
def small():
    return _setup(synth.scaled(synth.CONFIGS["chi2"], nscan=3, len_lo=16384, len_hi=16384, flag_frac=0.02))


@pytest.fixture(scope="module")
def full():
    return _setup(synth.CONFIGS["chi2"])


def _oracle(S):
    band, ing = S["band"], S["ing"]
    off = ing["offsets"]
    nq = len(off) - 1
    pix = np.concatenate([band.pix[q][:off[q + 1] - off[q]] for q in range(nq)])
    psi = np.concatenate([band.psi[q][:off[q + 1] - off[q]] for q in range(nq)])
    mask = (~ing["flags"]).astype(np.float64)
    return oracle.chi2_band(S["m32"].T.astype(np.float64), pix, psi, ing["tod"].astype(np.float64),
                            band.gain.copy(), mask, S["psd"], off, S["cfg"].ndet, S["cfg"].fsamp)


def _gpu(S, precision, m=None, g=None, psd=None, grad=True):
    torch = S["torch"]
    from paper_2201_03509_gb300.chi2 import tod_chi2
    tm = torch.from_numpy(S["m32"].astype(np.float64) if m is None else m).to(S["dev"]).requires_grad_(grad)
    tg_ = torch.from_numpy(S["band"].gain.copy() if g is None else g).to(S["dev"]).requires_grad_(grad)
    tp = torch.from_numpy(S["psd"] if psd is None else psd).to(S["dev"]).requires_grad_(grad)
    L = tod_chi2(tm, tg_, tp, S["plan"], S["d"], S["flags"], precision)
    if grad:
        L.backward()
    S["plan"].status()
    if not grad:
        return float(L)
    return float(L), tm.grad.cpu().numpy().T, tg_.grad.cpu().numpy(), tp.grad.cpu().numpy()


def _check_against_oracle(S, precision, tol_L, tol_g):
    ref = _oracle(S)
    L, gm, gg, gp = _gpu(S, precision)
    assert L == pytest.approx(ref["L"], rel=tol_L)
    assert np.abs(gm - ref["dm"]).max() <= tol_g * np.abs(ref["dm"]).max()
    assert np.abs(gg - ref["dg"]).max() <= tol_g * np.abs(ref["dg"]).max()
    for j in range(3):
        assert np.abs(gp[:, j] - ref["dpsd"][:, j]).max() <= tol_g * np.abs(ref["dpsd"][:, j]).max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_chi2_small_band_matches_oracle(small, prec):
    p = small["tg"].Plan.PREC_F64 if prec == "f64" else small["tg"].Plan.PREC_F32
    _check_against_oracle(small, p, 1e-6 if prec == "f32" else 1e-11, 1e-4 if prec == "f32" else 1e-9)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_chi2_autograd_workload_matches_oracle(full, prec):
    p = full["tg"].Plan.PREC_F64 if prec == "f64" else full["tg"].Plan.PREC_F32
    _check_against_oracle(full, p, 1e-6 if prec == "f32" else 1e-11, 1e-4 if prec == "f32" else 1e-9)


def test_chi2_f64_gradients_match_gpu_finite_differences(full):
    """Central differences of the GPU's FP64 chi^2.  It is quadratic in the
    map and in each gain, so there the difference is exact for any step (the
    steps keep it far above the rounding of L); in the noise parameters the
    relative step 1e-5 leaves a truncation error near 1e-10."""
    S = full
    F64 = S["tg"].Plan.PREC_F64
    L0, gm, gg, gp = _gpu(S, F64)
    m0 = S["m32"].astype(np.float64)
    rng = np.random.default_rng(4)
    # the map: T, Q, U of a few well-observed pixels
    off = S["ing"]["offsets"]
    kept = [S["band"].pix[q][:int(off[q + 1] - off[q])] for q in range(8)]
    hits = np.bincount(np.concatenate(kept), minlength=S["band"].npix)
    for p in rng.choice(np.nonzero(hits > 0)[0], 3, replace=False):
        for c in range(3):
            h = 1e-4
            mp, mm = m0.copy(), m0.copy()
            mp[p, c] += h
            mm[p, c] -= h
            num = (_gpu(S, F64, m=mp, grad=False) - _gpu(S, F64, m=mm, grad=False)) / (2 * h)
            assert gm[c, p] == pytest.approx(num, rel=1e-4), (p, c)
    # a gain
    g0 = S["band"].gain.copy()
    q = 17
    gpl, gmi = g0.copy(), g0.copy()
    gpl[q] += 1e-3
    gmi[q] -= 1e-3
    num = (_gpu(S, F64, g=gpl, grad=False) - _gpu(S, F64, g=gmi, grad=False)) / 2e-3
    assert gg[q] == pytest.approx(num, rel=1e-4)
    # every noise parameter of one detector
    det = 2
    for j in range(3):
        h = 1e-5 * abs(S["psd"][det, j])
        pp, pm = S["psd"].copy(), S["psd"].copy()
        pp[det, j] += h
        pm[det, j] -= h
        num = (_gpu(S, F64, psd=pp, grad=False) - _gpu(S, F64, psd=pm, grad=False)) / (2 * h)
        assert gp[det, j] == pytest.approx(num, rel=1e-4), j


def test_chi2_f32_gain_gradient_matches_gpu_finite_difference(small):
    """The FP32 variant's own central difference in a gain: chi^2 is
    quadratic in each gain, so a step of the gain's size is exact and keeps
    the difference far above the FP32 rounding of the transforms."""
    S = small
    F32 = S["tg"].Plan.PREC_F32
    _, _, gg, _ = _gpu(S, F32)
    g0 = S["band"].gain.copy()
    q = 1
    gpl, gmi = g0.copy(), g0.copy()
    gpl[q] += 1.0
    gmi[q] -= 1.0
    num = (_gpu(S, F32, g=gpl, grad=False) - _gpu(S, F32, g=gmi, grad=False)) / 2.0
    assert gg[q] == pytest.approx(num, rel=1e-4)
