"""Parity at the benchmark's full size (N_O=20, N_V=200, n_o=12, n_v=60, N_J=600,
the configuration and precision bench.py times) and at N_O=40, N_V=500, n_o=20,
n_v=120, N_J=1500 (swept in chunks by the default memory budget), where the
oracle can still compute single triples blocks but not the full sums:

* sampled n_v^3 blocks tau^{abc}_{ijk} against the oracle's tau3_block;
* properties that hold at any size: the adjoint identity <L, A R> = <A^T L, R>,
  finite differences of Omega in t2 against rho(omega = 0) (FP64 path), and the
  split path's bound against the FP64 path on every output, f and the
  excitation-energy Rayleigh quotient."""
import numpy as np
import pytest

import oracle as O
from gpu_common import rel_err
from paper_2202_08612_gb300 import binding, synth

pytestmark = pytest.mark.gpu

C2 = (20, 200, 12, 60, 600)
C3 = (40, 500, 20, 120, 1500)
SAMPLES = [(1, 0, 0), (5, 3, 1), (11, 11, 0), (11, 10, 9), (7, 7, 7)]  # i >= j >= k; (7,7,7) is not stored


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class Full:
    """A full-size seeded system on the device (the bench's seeds)."""

    def __init__(self, dims, seed=2022, t2_norm=None):
        torch = _torch()
        self.dims = dims
        self.s = synth.make_system(*dims, seed=seed, t2_norm=t2_norm)
        self.st = synth.make_states(self.s, 1, seed=seed + 1)
        self.lam1, self.lam2 = synth.make_multipliers(self.s, seed=seed + 2)
        self.mu = synth.make_dipole(self.s, seed=seed + 3)
        self.D00_in = synth.reference_density(self.s)
        self.d = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        self.z = lambda sh: torch.zeros(sh, dtype=torch.float64, device="cuda")

    def context(self, precision):
        g = binding.Context(*self.dims, precision=precision)
        s, d = self.s, self.d
        g.build_integrals(d(s.chol), d(s.t1), d(s.eps), d(s.t2c), d(s.t2x))
        return g

    def outputs(self, g):
        s, st, d, z = self.s, self.st, self.d, self.z
        NO, NV = s.dims.n_occ, s.dims.n_vir
        nmo = NO + NV
        o = {}
        o1, o2 = z((NV, NO)), z(s.t2c.shape)
        g.triples_omega(o1, o2)
        r1, r2, s1, s2 = z(st.R1.shape), z(st.R2.shape), z(st.R1.shape), z(st.R2.shape)
        g.jacobian_right(st.omega, d(st.R1), d(st.R2), r1, r2)
        g.jacobian_left(st.omega, d(st.L1), d(st.L2), s1, s2)
        w = float(st.omega[0])
        D = [z((nmo, nmo)) for _ in range(3)]
        g.transition_density(w, d(self.lam1), d(self.lam2), d(st.R1[0]), d(st.R2[0]),
                             d(st.L1[0]), d(st.L2[0]), d(self.D00_in), *D)
        D0m, Dm0 = D[2].clone(), D[1].clone()
        D0m[NO:, :NO] += d(st.R1[0])
        Dm0[:NO, NO:] += d(st.L1[0].T)
        o["f"] = g.oscillator_strength(w, D0m, Dm0, d(self.mu))
        o["rq"] = g.rayleigh_quotient(w, d(st.R1[0]), d(st.R2[0]), d(st.L1[0]), d(st.L2[0]), 0.0)
        for k, v in (("o1", o1), ("o2", o2), ("rho1", r1), ("rho2", r2), ("sig1", s1),
                     ("sig2", s2), ("D00", D[0]), ("Dm0", D[1]), ("D0m", D[2])):
            o[k] = v.cpu().numpy()
        return o

    def adjoint_gap(self, o):
        st, dm = self.st, self.s.dims
        a = synth.sd_dot(dm, st.L1[0], st.L2[0], o["rho1"][0], o["rho2"][0])
        b = synth.sd_dot(dm, o["sig1"][0], o["sig2"][0], st.R1[0], st.R2[0])
        return abs(a - b) / abs(a)


def _sampled_tau(full, g, tol):
    """tau blocks of the context's (first) chunk against the oracle's blocks."""
    oc = O.make_ctx(full.s)
    no = full.s.dims.n_act_occ
    nv3 = full.s.dims.n_act_vir ** 3
    o1 = full.z((full.s.dims.n_vir, full.s.dims.n_occ))
    o2 = full.z(full.s.t2c.shape)
    g.triples_omega(o1, o2)  # leaves the tau of the (only) chunk in the "tau" buffer
    order = [(i, j, k) for i in range(no) for j in range(i + 1) for k in range(j + 1)
             if not (i == j == k)]
    nb = g.nbatches()
    assert nb == len(order)
    # with one chunk the buffer holds every unique batch in this order
    tau = g.debug_fetch("tau", nb * nv3).reshape(nb, -1)
    checked = 0
    for (i, j, k) in SAMPLES:
        if i >= no or (i == j == k):
            continue
        ref = O.tau3_block(oc, i, j, k).reshape(-1)
        assert rel_err(tau[order.index((i, j, k))], ref) < tol, (i, j, k)
        checked += 1
    assert checked >= 3


@pytest.fixture(scope="module")
def c2():
    _torch()
    f = Full(C2)
    f.split = f.outputs(f.context(binding.MLCC3_SPLIT_BF16X3))
    f.fp64 = f.outputs(f.context(binding.MLCC3_FP64))
    return f


def test_c2_sampled_tau_blocks_split(c2):
    g = c2.context(binding.MLCC3_SPLIT_BF16X3)  # one chunk at this size
    _sampled_tau(c2, g, 1e-4)
    g.close()


def test_c2_adjoint_identity(c2):
    assert c2.adjoint_gap(c2.fp64) < 1e-12
    assert c2.adjoint_gap(c2.split) < 1e-5


def test_c2_split_against_fp64_path(c2):
    for k in ("o1", "o2", "rho1", "rho2", "sig1", "sig2", "D00", "Dm0", "D0m"):
        assert rel_err(c2.split[k], c2.fp64[k]) < 5e-5, k
    assert abs(c2.split["f"] - c2.fp64["f"]) < 5e-5 * abs(c2.fp64["f"])
    assert abs(c2.split["rq"] - c2.fp64["rq"]) < 1e-5  # Hartree


def test_c2_molecule_scaled_f_and_excitation_energy():
    """The accuracy target of the split path at the benchmark size, on the
    molecule-scaled variant of the recipe (doubles norm 0.3, f of physical
    size): |f_split - f_FP64| < 1e-6 and the excitation-energy Rayleigh
    quotients within 1e-5 Hartree, both against the FP64 GPU path."""
    f = Full(C2, t2_norm=0.3)
    g = f.context(binding.MLCC3_SPLIT_BF16X3)
    split = f.outputs(g)
    g.close()
    g = f.context(binding.MLCC3_FP64)
    fp64 = f.outputs(g)
    g.close()
    assert 1e-4 < abs(fp64["f"]) < 10.0
    assert abs(split["f"] - fp64["f"]) < 1e-6, (split["f"], fp64["f"])
    assert abs(split["rq"] - fp64["rq"]) < 1e-5
    for k in ("o1", "o2", "rho1", "rho2", "sig1", "sig2", "D00", "Dm0", "D0m"):
        assert rel_err(split[k], fp64[k]) < 5e-5, k


def test_c2_finite_differences_in_t2_fp64(c2):
    """Omega(t2 + h Rbar) - Omega(t2 - h Rbar) over 2h = rho(omega = 0, R1 = 0, R2)
    (the Jacobian is the derivative of the residual, Sec. 2)."""
    s, d, z = c2.s, c2.d, c2.z
    oc = O.make_ctx(s)
    R2 = c2.st.R2[0]
    dt = O.from_full(oc, O.delta(O.to_full(oc, R2)))
    h = 1e-5
    outs = []
    for sign in (1, -1):
        g = binding.Context(*C2, precision=binding.MLCC3_FP64)
        g.build_integrals(d(s.chol), d(s.t1), d(s.eps), d(s.t2c + sign * h * dt), d(s.t2x))
        o1, o2 = z((s.dims.n_vir, s.dims.n_occ)), z(s.t2c.shape)
        g.triples_omega(o1, o2)
        outs.append((o1.cpu().numpy(), o2.cpu().numpy()))
        g.close()
    g = c2.context(binding.MLCC3_FP64)
    r1, r2 = z(c2.st.R1.shape), z(c2.st.R2.shape)
    g.jacobian_right([0.0], d(np.zeros_like(c2.st.R1)), d(c2.st.R2), r1, r2)
    assert rel_err((outs[0][1] - outs[1][1]) / (2 * h), r2.cpu().numpy()[0]) < 1e-6
    assert rel_err((outs[0][0] - outs[1][0]) / (2 * h), r1.cpu().numpy()[0]) < 1e-6


def test_c3_chunked_split_sampled_tau_and_adjoint():
    _torch()
    f = Full(C3)
    g = f.context(binding.MLCC3_SPLIT_BF16X3)
    # one chunk for the tau check (the buffer then holds every batch), then the
    # whole path swept in chunks of 400 batches for the adjoint identity
    g.set_param("chunk_blocks", 1 << 20)
    _sampled_tau(f, g, 1e-4)
    g.set_param("chunk_blocks", 400)
    o = f.outputs(g)
    assert f.adjoint_gap(o) < 1e-5
    g.close()
