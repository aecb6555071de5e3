"""The multi-band Gibbs sweep: the TOD steps of several bands (each its own
plan, e.g. the 30, 44 and 70 GHz bands) run concurrently on their own
streams, iteration after iteration (paper Sect. 5: the TOD steps of the
frequency bands are independent given the sky model, so they run side by
side).  Each band carries its map from one iteration to the next (the
map the step solves is the next step's input) and, with the noise-PSD step
(row A10), its noise parameters: the n_corr draw writes its spectra and
`psd_steps` Metropolis steps update the band's (f_knee, alpha) before the
next iteration.  Gains are drawn afresh every iteration from their
conditional.  Only marshals and sequences C-ABI calls."""
from __future__ import annotations

import numpy as np

from . import MODE_DRAW, Plan, Rng
from .step import GibbsTODStep


class BandChain:
    """One band's Gibbs chain: its plan, step buffers and stream.  `map_tqu`
    (float64 [3, npix]) starts the chain."""

    def __init__(self, plan: Plan, psd: np.ndarray, flag_words: np.ndarray, tod: np.ndarray,
                 map_tqu: np.ndarray, band_id: int, cg_tol: float = 1e-6, psd_steps: int = 0,
                 psd_step_sizes=(2e-4, 2e-4)):
        import torch
        self.plan, self.band_id = plan, int(band_id)
        self.step = GibbsTODStep(plan, psd, flag_words, cg_tol=cg_tol)
        # the bands already share the GPU: no next-step decode under the draw
        self.step.lookahead = False
        self.step.set_tod(tod)
        m4 = np.zeros((plan.npix, 4), np.float32)
        m4[:, :3] = np.asarray(map_tqu, np.float64).T
        self.step.map32.copy_(torch.from_numpy(m4))
        self.psd_steps = int(psd_steps)
        self.psd_step_sizes = tuple(float(x) for x in psd_step_sizes)
        dev = self.step.d.device
        self.stream = torch.cuda.Stream(device=dev)
        if self.psd_steps:
            self.spec = torch.empty(plan.N, dtype=torch.float32, device=dev)
            self.psd_next = torch.empty_like(self.step.psd)
            self.accepted = torch.zeros(plan.ndet, dtype=torch.int32, device=dev)

    @property
    def nsamples(self) -> int:
        return int(self.plan.N)

    def enqueue(self, seed: int, it: int, mode: int = MODE_DRAW):
        """Queue iteration `it` of this band on its stream."""
        import torch
        st, p = self.step, self.plan
        rng = Rng(seed, self.band_id, it)
        with torch.cuda.stream(self.stream):
            if self.psd_steps:
                p.set_ncorr_spectrum(self.spec)
            # the map solved by the previous iteration is this one's input:
            # the projection reads it before the solve overwrites it
            st.run(st.map32, rng, mode, self.stream)
            if self.psd_steps:
                p.set_ncorr_spectrum(None)
                p.sample_noise_psd(self.spec, st.psd, rng, self.psd_steps, self.psd_step_sizes[0],
                                   self.psd_step_sizes[1], self.psd_next, self.accepted, stream=self.stream)
                st.psd.copy_(self.psd_next)


class MultiBandSweep:
    """Runs the bands' chains side by side, one stream per band."""

    def __init__(self, chains: list):
        self.chains = list(chains)

    @property
    def nsamples(self) -> int:
        return sum(c.nsamples for c in self.chains)

    def run(self, n_iter: int, seed: int, it0: int = 0, mode: int = MODE_DRAW, on_iteration=None,
            concurrent: bool = True) -> dict:
        """Queue n_iter iterations of every band (iterations it0 ..
        it0 + n_iter - 1) and wait for them.  The caller's stream waits for
        every band.  With concurrent=False each band's iteration waits for the
        previous band's (the bands take turns on the GPU; same results).
        Returns the elapsed time and, per band, the time from the start to
        the end of its last iteration (CUDA events).  on_iteration(k) is
        called after iteration k is queued (e.g. to copy results out)."""
        import torch
        cur = torch.cuda.current_stream()
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(cur)
        for c in self.chains:
            c.stream.wait_event(t0)
        for k in range(n_iter):
            for i, c in enumerate(self.chains):
                if not concurrent and (i or k):
                    prev = torch.cuda.Event()
                    prev.record(self.chains[i - 1].stream)
                    c.stream.wait_event(prev)
                c.enqueue(seed, it0 + k, mode)
            if on_iteration is not None:
                on_iteration(k)
        ends = []
        for c in self.chains:
            e = torch.cuda.Event(enable_timing=True)
            e.record(c.stream)
            cur.wait_event(e)
            ends.append(e)
        t1 = torch.cuda.Event(enable_timing=True)
        t1.record(cur)
        torch.cuda.synchronize()
        return {"ms": t0.elapsed_time(t1), "band_ms": [t0.elapsed_time(e) for e in ends],
                "samples_per_iteration": self.nsamples}
