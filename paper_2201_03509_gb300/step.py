"""One Gibbs TOD step on the GPU (paper Listing `code:gibbs`, step 1):
decode -> project -> sample gain -> sample n_corr -> bin -> solve, as a
sequence of the C-ABI calls on one stream.  Holds the device buffers.

With ``data_streams`` the detector data and flags stay compressed on the
device too (Sect. 4.1; the plan must have them attached) and every step
decodes them along with the pointing.  With ``gain_prior`` each step draws
every detector's scan gains jointly under the smooth prior across scans
(tod_sample_gain_smooth) in place of the independent per-scan draws.  With
``shard`` (a shard.ShardedMaps) the plan holds one process's scan range and
the binning + solve become the reduction over processes (Sect. 2.3-2.4)."""
from __future__ import annotations

import numpy as np

from . import MODE_DRAW, Plan, Rng


class GibbsTODStep:
    def __init__(self, plan: Plan, psd: np.ndarray, flag_words: np.ndarray | None, rcond_min: float = 1e-6,
                 cg_tol: float = 1e-6, cg_maxiter: int = 500, data_streams: bool = False,
                 gain_prior: np.ndarray | None = None, shard=None):
        import torch
        dev = torch.device("cuda", plan.device)
        N, nq, npix = plan.N, plan.nq, plan.npix
        self.plan = plan
        self.rcond_min, self.cg_tol, self.cg_maxiter = rcond_min, cg_tol, cg_maxiter
        f32, f64, i32 = torch.float32, torch.float64, torch.int32
        self.psd = torch.from_numpy(np.ascontiguousarray(psd, np.float64)).to(dev)
        self.data_streams = data_streams
        # optional smooth prior across scans: float64[ndet, 2] (sigma_g, alpha_g)
        self.gain_prior = (None if gain_prior is None else
                           torch.from_numpy(np.ascontiguousarray(gain_prior, np.float64).reshape(plan.ndet, 2)).to(dev))
        self.gain_iters = torch.zeros(plan.ndet, dtype=torch.int32, device=dev)
        if data_streams:
            self.flags = torch.zeros((N + 31) // 32, dtype=i32, device=dev)   # decoded every step
        else:
            self.flags = torch.from_numpy(np.ascontiguousarray(flag_words, np.uint32).view(np.int32)).to(dev)
        self.d = torch.empty(N, dtype=f32, device=dev)
        self.pix = torch.empty(N, dtype=i32, device=dev)
        self.psi = torch.empty(N, dtype=torch.int16, device=dev)
        self.s = torch.empty(N, dtype=f32, device=dev)
        self.ncorr = torch.empty(N, dtype=f32, device=dev)
        self.gain = torch.zeros(nq, dtype=f64, device=dev)
        self.mu = torch.zeros(nq, dtype=f64, device=dev)
        self.sigma = torch.zeros(nq, dtype=f64, device=dev)
        self.cg_iters = torch.zeros(nq, dtype=i32, device=dev)
        self.A = torch.zeros((npix, 6), dtype=f64, device=dev)
        self.b = torch.zeros((npix, 3), dtype=f64, device=dev)
        self.hits = torch.zeros(npix, dtype=i32, device=dev)
        self.map = torch.zeros((3, npix), dtype=f64, device=dev)
        self.map32 = torch.zeros((npix, 4), dtype=f32, device=dev)
        self.rcond = torch.zeros(npix, dtype=f64, device=dev)
        self.valid = torch.zeros(npix, dtype=torch.uint8, device=dev)
        # each step decodes the next step's pointing under its n_corr draw
        # (a spare pix/psi pair); the last step's lookahead is extra work
        self.lookahead = True
        self.shard = shard
        self._pointing_ready = False
        self._pix_next = self._psi_next = None
        self._d_next = self._flags_next = None

    def set_tod(self, d, stream=None):
        """Copy this band's detector data (host numpy float32 or a tensor)."""
        import torch
        if isinstance(d, np.ndarray):
            d = torch.from_numpy(np.ascontiguousarray(d, np.float32))
        self.d.copy_(d, non_blocking=True)

    def prefetch_tod(self, d_host, stream=None):
        """Start copying the next step's detector data (a pinned host float32
        tensor of N samples) into a second device buffer on a copy stream, so
        that the copy overlaps the step that is running.  The next run()
        on `stream` waits for the copy and then uses that buffer; the copy
        itself waits until the last step that read that buffer is done."""
        import torch
        if self.data_streams:
            raise ValueError("the detector data are decoded on the device: nothing to prefetch")
        if getattr(self, "_copy_stream", None) is None:
            self._copy_stream = torch.cuda.Stream(device=self.d.device)
            self._d_spare = torch.empty_like(self.d)
            self._spare_free = None
        cs = self._copy_stream
        if self._spare_free is None:      # never read by a step: after what is already queued
            self._spare_free = torch.cuda.Event()
            self._spare_free.record(self._stream(stream))
        cs.wait_event(self._spare_free)
        with torch.cuda.stream(cs):
            self._d_spare.copy_(d_host, non_blocking=True)
        self._copied = torch.cuda.Event()
        self._copied.record(cs)

    def _streams(self):
        """(high-priority stream for the step, side stream for the n_corr
        preparation, low-priority stream for the next step's decode)."""
        import torch
        if getattr(self, "_hp", None) is None:
            lo_pri, hi_pri = torch.cuda.Stream.priority_range()
            dev = self.d.device
            self._hp = torch.cuda.Stream(device=dev, priority=hi_pri)
            self._side = torch.cuda.Stream(device=dev, priority=hi_pri)
            self._lo = torch.cuda.Stream(device=dev, priority=lo_pri)
        return self._hp, self._side, self._lo

    def _stream(self, stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream(self.d.device)

    def _take_prefetched(self, stream):
        import torch
        if getattr(self, "_copied", None) is None:
            return
        st = self._stream(stream)
        st.wait_event(self._copied)
        self._copied = None
        # the buffer that becomes spare was last read by the step that
        # recorded _d_done (or by none since it was last swapped in)
        done = getattr(self, "_d_done", None)
        if done is None:
            done = torch.cuda.Event()
            done.record(st)
        self.d, self._d_spare = self._d_spare, self.d
        self._spare_free = done
        self._d_done = None

    def _mark_d_done(self, stream):
        import torch
        if getattr(self, "_copy_stream", None) is None:
            return
        self._d_done = torch.cuda.Event()
        self._d_done.record(self._stream(stream))     # self.d is read by nothing queued after this

    def run(self, map32_in, rng: Rng, mode: int = MODE_DRAW, stream=None, gain_event=None):
        """Enqueue one step; the new map lands in self.map / self.map32.
        Uses the detector data of a pending prefetch_tod() if there is one.
        gain_event, if given, is recorded once the gains are drawn."""
        import torch
        self._take_prefetched(stream)
        p = self.plan
        st = self._stream(stream)
        hp, side, lo = self._streams()
        # the step's own work runs on a high-priority stream ordered after
        # the caller's; the caller's stream waits for all of it at the end
        hp.wait_stream(st)
        # the n_corr gap preconditioner depends on the PSD alone: it is built
        # on a side stream while decode, projection and the gain draw run
        # (after everything already queued, so the previous step's draw has
        # finished with the old tables)
        side.wait_stream(st)
        p.ncorr_prepare(self.psd, side)
        prepared = torch.cuda.Event()
        prepared.record(side)
        if self._pointing_ready:
            # decoded by the previous step, under its n_corr draw
            self.pix, self._pix_next = self._pix_next, self.pix
            self.psi, self._psi_next = self._psi_next, self.psi
            if self.data_streams:
                self.d, self._d_next = self._d_next, self.d
                self.flags, self._flags_next = self._flags_next, self.flags
            self._pointing_ready = False
        else:
            p.decode(self.pix, self.psi, hp)
            if self.data_streams:
                p.decode_data(self.d, self.flags, hp)
        p.project(map32_in, self.pix, self.psi, None, self.s, hp)
        p.sample_gain(self.d, self.s, self.flags, self.psd, rng, mode, self.gain, self.mu, self.sigma, hp)
        if self.gain_prior is not None:
            # every detector's scans drawn jointly from their conditionals and the prior
            p.sample_gain_smooth(self.mu, self.sigma, self.gain_prior, rng, mode, self.gain, self.gain_iters,
                                 stream=hp)
        if gain_event is not None:
            gain_event.record(hp)
        hp.wait_event(prepared)
        lookahead = self.lookahead
        if lookahead:
            gained = torch.cuda.Event()
            gained.record(hp)
        p.sample_ncorr_prepared(self.d, self.s, self.gain, self.flags, self.psd, rng, mode, self.ncorr,
                                self.cg_iters, self.cg_tol, self.cg_maxiter, hp)
        if lookahead:
            # the next step's pointing (the compressed streams do not change),
            # decoded at low priority: its CTAs fill the SMs between the
            # n_corr pass kernels' CTAs and in the draw's serial tails
            if self._pix_next is None:
                self._pix_next = torch.empty_like(self.pix)
                self._psi_next = torch.empty_like(self.psi)
            if self.data_streams and self._d_next is None:
                self._d_next = torch.empty_like(self.d)
                self._flags_next = torch.empty_like(self.flags)
            lo.wait_event(gained)
            p.decode(self._pix_next, self._psi_next, lo)
            if self.data_streams:
                p.decode_data(self._d_next, self._flags_next, lo)
            self._pointing_ready = True
        if self.shard is None:
            p.bin(self.psi, self.d, self.ncorr, self.gain, self.flags, self.psd, self.A, self.b, self.hits, hp)
            p.solve_maps(self.A, self.b, self.hits, self.rcond_min, self.map, self.map32, self.rcond,
                         self.valid, hp)
        else:
            # this process's partials, reduced over processes by pixel range, solved and gathered
            with torch.cuda.stream(hp):
                m, m32, va = self.shard.reduce_and_solve(self.psi, self.d, self.ncorr, self.gain, self.flags,
                                                         self.psd, self.rcond_min)
                self.map.copy_(m)
                self.map32.copy_(m32)
                self.valid.copy_(va)
        st.wait_stream(hp)
        if lookahead:
            st.wait_stream(lo)
        self._mark_d_done(stream)

    # decode x2, project, gain (scalars, three passes, draw), n_corr (flag
    # index 4, coarse correction, right-hand side 3, CG start and its list,
    # 8 launched CG iterations x (3 passes, update, list), cooperative tail,
    # list, correction 3, finish), bin + reduce, solve; plus the
    # preconditioner preparation (Plan.toeplitz_prep_launches)
    LAUNCHES_PER_STEP = 2 + 1 + 5 + (4 + 1 + 3 + 2 + 8 * 5 + 1 + 1 + 3 + 1) + 2 + 1
    DATA_LAUNCHES = 2       # with data_streams: decode of the TOD and of the flags

    @property
    def launches_per_step(self) -> int:
        return (self.LAUNCHES_PER_STEP + self.plan.toeplitz_prep_launches
                + (self.DATA_LAUNCHES if self.data_streams else 0)
                + (1 if self.gain_prior is not None else 0))

    def capture(self, map32_in, seed: int, band: int = 0, mode: int = MODE_DRAW):
        """Capture the step into CUDA graphs.  The Gibbs iteration is read by
        the kernels from a device word, so replay(it) draws fresh numbers.

        With lookahead, two graphs are captured that take their pointing
        from the two pix/psi pairs in turn and do not decode it; replay()
        alternates between them, launches the graph on the high-priority
        stream and, once the graph has drawn the gains (an event recorded
        inside it), decodes the other pair (the next replay's pointing) with
        eager launches on the low-priority stream beside the n_corr draw.
        (A graph's kernels run at the priority of the stream it is launched
        into, so a decode captured inside the graph would compete with the
        draw at equal priority.)  Without lookahead one graph decodes
        in-step."""
        import torch
        self.iter_dev = torch.zeros(1, dtype=torch.int64, device=self.d.device)
        self._rng_graph = Rng(seed, band, 0, self.iter_dev.data_ptr())
        self._map_graph = map32_in
        side = torch.cuda.Stream(device=self.d.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(map32_in, self._rng_graph, mode)          # untimed first run off the capture
        torch.cuda.current_stream().wait_stream(side)
        lookahead = self.lookahead
        self.graphs = []
        self._graph_pairs = []
        if lookahead:
            p = self.plan
            if self._pix_next is None:
                self._pix_next = torch.empty_like(self.pix)
                self._psi_next = torch.empty_like(self.psi)
            if self.data_streams and self._d_next is None:
                self._d_next = torch.empty_like(self.d)
                self._flags_next = torch.empty_like(self.flags)
            # both pairs decoded before the first replay
            cur = torch.cuda.current_stream()
            p.decode(self.pix, self.psi, cur)
            p.decode(self._pix_next, self._psi_next, cur)
            if self.data_streams:
                p.decode_data(self.d, self.flags, cur)
                p.decode_data(self._d_next, self._flags_next, cur)
            self.lookahead = False
        self._graph_gained = []
        try:
            for _ in range(2 if lookahead else 1):
                ev = None
                if lookahead:
                    self._pointing_ready = True                 # run() swaps the pairs and does not decode
                    try:
                        ev = torch.cuda.Event(external=True)    # a record node the host can wait on
                    except TypeError:
                        ev = None
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self.run(map32_in, self._rng_graph, mode, gain_event=ev)
                self.graphs.append(g)
                self._graph_gained.append(ev)
                # the pair this graph does not read: the other graph's, decoded beside this one
                self._graph_pairs.append((self._pix_next, self._psi_next, self._d_next, self._flags_next))
        finally:
            self.lookahead = lookahead
            self._pointing_ready = False
        self._next_graph = 0
        self.graph = self.graphs[0]
        return self.graph

    def replay(self, it: int):
        """Run the captured step at Gibbs iteration ``it`` (current stream)."""
        import torch
        self.iter_dev.fill_(int(it))
        i = self._next_graph
        g = self.graphs[i]
        self._next_graph = (i + 1) % len(self.graphs)
        if len(self.graphs) == 1:
            g.replay()
            return
        cur = torch.cuda.current_stream(self.d.device)
        hp, _, lo = self._streams()
        hp.wait_stream(cur)
        # the pair the other graph reads: free once everything queued so far
        # is done; decoded after this replay's gain draw (else from its start)
        pix, psi, d, fl = self._graph_pairs[i]
        gained = self._graph_gained[i]
        if gained is None:
            gained = torch.cuda.Event()
            gained.record(hp)
        with torch.cuda.stream(hp):
            g.replay()
        lo.wait_event(gained)
        self.plan.decode(pix, psi, lo)
        if self.data_streams:
            self.plan.decode_data(d, fl, lo)
        cur.wait_stream(hp)
        cur.wait_stream(lo)
