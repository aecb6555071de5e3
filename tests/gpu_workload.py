"""Shared set-up for the GPU tests: a synthetic band ingested by the library,
its plan, and device copies of the per-step inputs.  Inputs come from synth
and the oracle only; nothing here feeds GPU output to the oracle."""
import numpy as np

import oracle
import paper_2201_03509_gb300 as tg
import synth


class Workload:
    def __init__(self, cfg, tile_pairs=0, with_noise=True, max_radix=0):
        import torch
        self.cfg = cfg
        self.band = synth.make_band(cfg, with_noise=with_noise)
        self.ing = tg.ingest(self.band)
        self.off = self.ing["offsets"]
        self.nq = len(self.off) - 1
        self.N = int(self.off[-1])
        self.plan = tg.Plan(cfg.nside, cfg.ndet, cfg.nscan, cfg.fsamp, self.off,
                            self.ing["pix_streams"], self.ing["psi_streams"], tile_pairs=tile_pairs,
                            max_radix=max_radix)
        dev = torch.device("cuda:0")
        self.dev = dev
        self.pix_ref = np.concatenate([self.band.pix[q][:self.off[q + 1] - self.off[q]]
                                       for q in range(self.nq)]).astype(np.int64)
        self.psi_ref = np.concatenate([self.band.psi[q][:self.off[q + 1] - self.off[q]]
                                       for q in range(self.nq)]).astype(np.int64)
        self.flags = self.ing["flags"]
        self.mask = (~self.flags).astype(np.float64)
        self.d32 = self.ing["tod"]
        self.t_d = torch.from_numpy(self.d32).to(dev)
        self.t_flags = torch.from_numpy(self.ing["flag_words"].view(np.int32)).to(dev)
        self.t_psd = torch.from_numpy(self.band.psd.copy()).to(dev)
        m4 = np.zeros((self.band.npix, 4), np.float32)
        m4[:, :3] = self.band.map_tqu.T
        self.t_map = torch.from_numpy(m4).to(dev)
        # FP64 projection at unit gain (oracle), its FP32 copy is the GPU input
        self.s64 = oracle.project(self.band.map_tqu, self.pix_ref, self.psi_ref)
        self.s32 = self.s64.astype(np.float32)
        self.t_s = torch.from_numpy(self.s32).to(dev)

    def sl(self, q):
        return slice(int(self.off[q]), int(self.off[q + 1]))

    def det(self, q):
        return q % self.cfg.ndet
