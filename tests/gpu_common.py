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

    def __init__(self, NO, NV, no, nv, NJ, seed=synth.DEFAULT_SEED, nstates=2, core=False,
                 t2_norm=None, singles_weight=0.95):
        self.sys = synth.make_system(NO, NV, no, nv, NJ, seed=seed, core=core, t2_norm=t2_norm)
        self.st = synth.make_states(self.sys, nstates, seed=seed + 1,
                                    cvs_states=tuple(range(nstates)) if core else (),
                                    singles_weight=singles_weight)
        self.lam1, self.lam2 = synth.make_multipliers(self.sys, seed=seed + 2)
        self.mu = synth.make_dipole(self.sys, seed=seed + 3)
        self.D00_in = synth.reference_density(self.sys)
        self.dims = (NO, NV, no, nv, NJ)
        self.core = core

    # -- oracle ---------------------------------------------------------------
    def oracle_ctx(self):
        return O.make_ctx(self.sys)

    # -- library --------------------------------------------------------------
    def context(self, precision=binding.MLCC3_FP64, device=True, params=None):
        import torch
        ctx = binding.Context(*self.dims, precision=precision,
                              core_mask=self.sys.core_mask if self.core else None)
        for k, v in (params or {}).items():
            ctx.set_param(k, v)
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


def oracle_all(c):
    """Oracle Omega, rho, sigma (state 0) and the three densities of a Case."""
    o, st = c.oracle_ctx(), c.st
    w = float(st.omega[0])
    ref = {}
    ref["o1"], r2 = O.triples_omega(o)
    ref["o2"] = O.from_full(o, r2)
    r1, r2 = O.jacobian_right(o, w, st.R1[0], O.to_full(o, st.R2[0]))
    ref["rho1"], ref["rho2"] = r1, O.from_full(o, r2)
    s1, s2 = O.jacobian_left(o, w, st.L1[0], O.to_full(o, st.L2[0]))
    ref["sig1"], ref["sig2"] = s1, O.from_full(o, s2)
    ref["D00"], ref["Dm0"], ref["D0m"] = O.transition_densities(
        o, w, c.lam1, O.to_full(o, c.lam2), st.R1[0], O.to_full(o, st.R2[0]), st.L1[0],
        O.to_full(o, st.L2[0]), c.D00_in)
    return ref


def run_all(c, g):
    """The same quantities from library context g (state 0 of the Case)."""
    st = c.st
    NO, NV = c.sys.dims.n_occ, c.sys.dims.n_vir
    nmo = NO + NV
    out = {}
    o1, o2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    g.triples_omega(o1, o2)
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    sig1, sig2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
    D = [c.empty_dev((nmo, nmo)) for _ in range(3)]
    g.transition_density(float(st.omega[0]), c.to_dev(c.lam1), c.to_dev(c.lam2),
                         c.to_dev(st.R1[0]), c.to_dev(st.R2[0]), c.to_dev(st.L1[0]),
                         c.to_dev(st.L2[0]), c.to_dev(c.D00_in), *D)
    out["o1"], out["o2"] = c.host(o1), c.host(o2)
    out["rho1"], out["rho2"] = c.host(rho1)[0], c.host(rho2)[0]
    out["sig1"], out["sig2"] = c.host(sig1)[0], c.host(sig2)[0]
    out["D00"], out["Dm0"], out["D0m"] = map(c.host, D)
    return out


def full_densities(c, D0m_T, Dm0_T, v=0):
    """CCSD-level leading-order transition densities plus the triples parts
    (D^{0-m}_{AI} += R^A_I, D^{m-0}_{IA} += L^A_I), as the oscillator strength
    takes them."""
    NO = c.sys.dims.n_occ
    D0m, Dm0 = np.array(D0m_T, copy=True), np.array(Dm0_T, copy=True)
    D0m[NO:, :NO] += c.st.R1[v]
    Dm0[:NO, NO:] += c.st.L1[v].T
    return D0m, Dm0


def oracle_f(c, ref):
    """The oracle's oscillator strength of state 0 from oracle_all's densities."""
    o = c.oracle_ctx()
    D0m, Dm0 = full_densities(c, ref["D0m"], ref["Dm0"])
    return O.oscillator_strength(o, float(c.st.omega[0]), D0m, Dm0, c.mu)


def library_f(c, g, got):
    """The library's oscillator strength of state 0 from run_all's densities."""
    D0m, Dm0 = full_densities(c, got["D0m"], got["Dm0"])
    return g.oscillator_strength(float(c.st.omega[0]), c.to_dev(D0m), c.to_dev(Dm0),
                                 c.to_dev(c.mu))
