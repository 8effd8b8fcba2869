"""The Davidson driver's host logic on CPU (subspace growth, restarts, the
self-consistent omega cycles), with the triples right transformation supplied
by the oracle through an object that has the library context's call signature.
The GPU tests repeat this through the library itself."""
import numpy as np
import pytest

import oracle as O
import sdbasis
from paper_2202_08612_gb300 import synth

torch = pytest.importorskip("torch")
from paper_2202_08612_gb300.davidson import Davidson  # noqa: E402


class OracleRight:
    """jacobian_right(omega[n_vec], R1, R2, rho1, rho2) on CPU tensors (R2 and
    rho2 in the active-pair block layout), computed by the oracle."""

    def __init__(self, o):
        self.o = o
        self.calls = 0

    def jacobian_right(self, omega, R1, R2, rho1, rho2):
        self.calls += 1
        for n in range(R1.shape[0]):
            r1, r2 = O.jacobian_right(self.o, float(omega[n]), R1[n].numpy(),
                                      O.to_full(self.o, R2[n].numpy()))
            rho1[n] = torch.from_numpy(r1)
            rho2[n] = torch.from_numpy(O.from_full(self.o, r2))


def test_davidson_host_logic_reaches_the_explicit_eigenpair():
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    w, R1, R2, L1, L2, sd = sdbasis.fixed_point_eigenpair(s, o)
    ctx = OracleRight(o)
    dv = Davidson(ctx, s.eps, (3, 4, 2, 2), torch.device("cpu"))
    res = dv.solve(tol=1e-10)
    assert abs(res.omega - w) < 1e-9, (res.omega, w)
    assert res.residual < 1e-9
    ref = np.concatenate([R1.ravel(), R2.ravel()])
    got = np.concatenate([res.R1.numpy().ravel(), res.R2.numpy().ravel()])
    ref, got = ref / np.linalg.norm(ref), got / np.linalg.norm(got)
    assert min(np.abs(got - ref).max(), np.abs(got + ref).max()) < 1e-6
    assert res.iterations == ctx.calls


def test_davidson_restarts_keep_the_root():
    """A subspace cap of 3 forces restarts from the Ritz vector; the root is
    the same as without them."""
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    a = Davidson(OracleRight(o), s.eps, (3, 4, 2, 2), torch.device("cpu")).solve(tol=1e-10)
    b = Davidson(OracleRight(o), s.eps, (3, 4, 2, 2), torch.device("cpu")).solve(
        tol=1e-10, max_subspace=3)
    assert abs(a.omega - b.omega) < 1e-9, (a.omega, b.omega)
