"""The autograd adjoint's host logic on CPU: with the oracle's right and left
transformations behind the library context's call signature, the backward of
JacobianRight (the left transformation with the block weights) satisfies
<g, A R> = <grad, R> for block-symmetric R and an arbitrary incoming gradient
g.  The GPU tests repeat this through the library."""
import numpy as np
import pytest

import oracle as O
from paper_2202_08612_gb300 import synth

torch = pytest.importorskip("torch")
from paper_2202_08612_gb300 import autograd  # noqa: E402


class OracleContext:
    def __init__(self, o, NJ):
        self.o = o
        self.dims = (o.NO, o.NV, o.no, o.nv, NJ)

    def _apply(self, f, omega, X1, X2, out1, out2):
        for n in range(X1.shape[0]) if X1.dim() == 3 else [None]:
            x1 = (X1[n] if n is not None else X1).numpy()
            x2 = (X2[n] if n is not None else X2).numpy()
            r1, r2 = f(self.o, float(omega[0 if n is None else n]), x1, O.to_full(self.o, x2))
            if n is None:
                out1.copy_(torch.from_numpy(r1))
                out2.copy_(torch.from_numpy(O.from_full(self.o, r2)))
            else:
                out1[n] = torch.from_numpy(r1)
                out2[n] = torch.from_numpy(O.from_full(self.o, r2))

    def jacobian_right(self, omega, R1, R2, rho1, rho2):
        self._apply(O.jacobian_right, omega, R1, R2, rho1, rho2)

    def jacobian_left(self, omega, L1, L2, s1, s2):
        self._apply(O.jacobian_left, omega, L1, L2, s1, s2)


@pytest.mark.parametrize("core", [False, True])
def test_backward_is_the_weighted_left_transformation(core):
    s = synth.make_system(5, 9, 3, 4, 12, seed=21, core=core)
    o = O.make_ctx(s)
    st = synth.make_states(s, 1, seed=22, cvs_states=(0,) if core else ())
    ctx = OracleContext(o, 12)
    w = float(st.omega[0])
    R1 = torch.from_numpy(st.R1[0].copy()).requires_grad_(True)
    R2 = torch.from_numpy(st.R2[0].copy()).requires_grad_(True)
    rho1, rho2 = autograd.jacobian_right(ctx, w, R1, R2)
    rng = np.random.default_rng(3)
    g1 = torch.from_numpy(rng.normal(size=tuple(rho1.shape)))
    g2 = torch.from_numpy(rng.normal(size=tuple(rho2.shape)))   # not block-symmetric
    val = (g1 * rho1).sum() + (g2 * rho2).sum()                  # Euclidean <g, A R>
    gR1, gR2 = torch.autograd.grad(val, (R1, R2))
    lhs = val.item()
    rhs = ((gR1 * R1).sum() + (gR2 * R2).sum()).item()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30), (lhs, rhs)
    # a missing weight or symmetrisation in the backward breaks it: the plain
    # left transformation of g is not the gradient
    s1, s2 = torch.zeros_like(g1), torch.zeros_like(g2)
    ctx.jacobian_left([w], g1, autograd.symmetrize_block(g2, 3, 4), s1, s2)
    plain = ((s1 * R1).sum() + (s2 * R2).sum()).item()
    assert abs(plain - lhs) > 1e-8 * abs(lhs)
