"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2202_08612_gb300 import binding, synth


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    if scale == 0.0:
        return float(np.abs(got).max()) if np.size(got) else 0.0
    return float(np.abs(np.asarray(got) - ref).max() / scale)


class Case:
    """A seeded synthetic system with states, multipliers and dipoles."""

    def __init__(self, NO, NV, no, nv, NJ, seed=synth.DEFAULT_SEED, nstates=2, core=False):
        self.sys = synth.make_system(NO, NV, no, nv, NJ, seed=seed, core=core)
        self.st = synth.make_states(self.sys, nstates, seed=seed + 1,
                                    cvs_states=tuple(range(nstates)) if core else ())
        self.lam1, self.lam2 = synth.make_multipliers(self.sys, seed=seed + 2)
        self.mu = synth.make_dipole(self.sys, seed=seed + 3)
        self.D00_in = synth.reference_density(self.sys)
        self.dims = (NO, NV, no, nv, NJ)
        self.core = core

    # -- oracle ---------------------------------------------------------------
    def oracle_ctx(self):
        return O.make_ctx(self.sys)

    # -- library --------------------------------------------------------------
    def context(self, precision=binding.MLCC3_FP64, device=True):
        import torch
        ctx = binding.Context(*self.dims, precision=precision,
                              core_mask=self.sys.core_mask if self.core else None)
        conv = self.to_dev if device else np.ascontiguousarray
        s = self.sys
        ctx.build_integrals(conv(s.chol), conv(s.t1), conv(s.eps), conv(s.t2c), conv(s.t2x))
        torch.cuda.synchronize()
        return ctx

    @staticmethod
    def to_dev(x):
        import torch
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()

    @staticmethod
    def empty_dev(shape):
        import torch
        return torch.zeros(shape, dtype=torch.float64, device="cuda")

    @staticmethod
    def host(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else x
