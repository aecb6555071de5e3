"""Pins of the oracle's noise-PSD step (row A10): the log-likelihood of the
correlated-noise spectrum against a closed form and against the truth of
simulated spectra, the Philox proposal numbers against their distributions,
and the Metropolis chain against the posterior integrated on a grid."""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle

FS = 32.5


def _pc(n, s0, fk, al):
    """Pc_k = s0^2 (f_k / fk)^al for k = 1..n-1, f_k = k FS / (2n) (written
    here from the model, not taken from the oracle)."""
    k = np.arange(1, n, dtype=np.float64)
    return s0 ** 2 * (k * FS / (2.0 * n) / fk) ** al


def test_loglike_closed_form_unit_spectrum():
    # xhat_k = sqrt(Pc_k): every term is 1 + ln Pc_k, and
    # sum_k ln Pc_k = N ln s0^2 + al (ln (n-1)! + N ln(FS / (2 n fk)))
    for n, s0, fk, al in ((64, 1e-3, 0.05, -1.5), (1001, 2e-3, 0.2, -2.7), (4096, 0.8e-3, 0.01, -0.6)):
        xh = np.zeros(n)
        xh[1:] = np.sqrt(_pc(n, s0, fk, al))
        xh[0] = 123.0                               # the offset mode does not enter
        N = n - 1
        want = -0.5 * (N + N * math.log(s0 ** 2) + al * (special.gammaln(n) + N * math.log(FS / (2.0 * n * fk))))
        got = oracle.psd_loglike([xh], [n], FS, s0, fk, al)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-9)


def _simulate(truth, lengths, seed):
    s0, fk, al = truth
    rng = np.random.default_rng(seed)
    out = []
    for n in lengths:
        xh = np.zeros(n)
        xh[1:] = np.sqrt(_pc(n, s0, fk, al)) * rng.standard_normal(n - 1)
        out.append(xh)
    return out


def test_loglike_peaks_at_the_truth():
    truth = (1e-3, 0.08, -1.6)
    lengths = [30000, 41000, 52000, 37000]
    sp = _simulate(truth, lengths, 7)
    lnfks = np.log(truth[1]) + np.linspace(-0.5, 0.5, 41)
    als = truth[2] + np.linspace(-0.3, 0.3, 61)
    grid = np.array([[oracle.psd_loglike(sp, lengths, FS, truth[0], math.exp(a), b) for b in als] for a in lnfks])
    i, j = np.unravel_index(np.argmax(grid), grid.shape)
    assert abs(lnfks[i] - math.log(truth[1])) <= 0.1
    assert abs(als[j] - truth[2]) <= 0.03


def test_proposal_numbers_have_their_distributions():
    z1, z2, u = np.array([oracle.psd_proposal(5, 2, det, step, 9)
                          for det in range(3) for step in range(700)]).T
    assert stats.kstest(z1, "norm").pvalue > 1e-3
    assert stats.kstest(z2, "norm").pvalue > 1e-3
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 0.1
    # distinct counters give distinct numbers
    assert oracle.psd_proposal(5, 2, 0, 0, 9) != oracle.psd_proposal(5, 2, 0, 1, 9)
    assert oracle.psd_proposal(5, 2, 0, 0, 9) != oracle.psd_proposal(5, 2, 1, 0, 9)


def test_metropolis_matches_the_grid_posterior():
    truth = (1e-3, 0.1, -1.2)
    lengths = [1500]
    sp = _simulate(truth, lengths, 3)
    # posterior on a grid (flat prior in the box, which the mass sits well inside)
    lnfks = np.linspace(math.log(0.1) - 1.5, math.log(0.1) + 1.5, 121)
    als = np.linspace(-2.2, -0.3, 121)
    lg = np.array([[oracle.psd_loglike(sp, lengths, FS, truth[0], math.exp(a), b) for b in als] for a in lnfks])
    w = np.exp(lg - lg.max())
    w /= w.sum()
    mean_lnfk, mean_al = float((w.sum(1) * lnfks).sum()), float((w.sum(0) * als).sum())
    sd_al = math.sqrt(float((w.sum(0) * (als - mean_al) ** 2).sum()))
    sd_lnfk = math.sqrt(float((w.sum(1) * (lnfks - mean_lnfk) ** 2).sum()))
    # the chain, one Metropolis step per call (the state carries over)
    psd = np.array([truth], dtype=np.float64)
    chain = []
    for it in range(6000):
        psd, _ = oracle.sample_noise_psd([sp], [lengths], FS, psd, 11, 0, it, 1, 0.8 * sd_lnfk, 0.8 * sd_al)
        if it >= 500:
            chain.append((math.log(psd[0, 1]), psd[0, 2]))
    c = np.array(chain)
    assert abs(c[:, 0].mean() - mean_lnfk) < 0.25 * sd_lnfk
    assert abs(c[:, 1].mean() - mean_al) < 0.25 * sd_al
    assert c[:, 1].std() == pytest.approx(sd_al, rel=0.25)
    assert c[:, 0].std() == pytest.approx(sd_lnfk, rel=0.25)


def test_proposals_outside_the_box_are_rejected():
    truth = (1e-3, 0.1, -0.3)                       # alpha 0.05 inside the upper edge
    lengths = [800]
    sp = _simulate(truth, lengths, 4)
    psd, acc = oracle.sample_noise_psd([sp], [lengths], FS, [truth], 1, 0, 0, 200, 1e3, 1e3)
    assert acc[0] == 0                              # every huge step leaves the box
    np.testing.assert_allclose(psd[0], truth, rtol=1e-14)
    psd, acc = oracle.sample_noise_psd([sp], [lengths], FS, [truth], 1, 0, 0, 300, 0.05, 0.2)
    assert acc[0] > 0
    assert oracle.psd_in_box(math.log(psd[0, 1]), psd[0, 2])
