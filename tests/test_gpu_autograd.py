"""The autograd adjoint (forward: right transformation, backward: the hand-written
left transformation) and the paper-level identities on the CUDA path itself:
the dot-product test <L, A R> = <A^T L, R>, and finite differences of the
triples residual in t2 (step 1e-5) against rho(omega = 0, R1 = 0, R2 = dt2)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import autograd, binding, synth

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", [binding.MLCC3_FP64, binding.MLCC3_SPLIT_BF16X3])
def test_autograd_backward_is_left_transformation(precision):
    torch = _torch()
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=2)
    g = c.context(precision=precision)
    st = c.st
    w = float(st.omega[0])
    R1 = c.to_dev(st.R1[0]).requires_grad_(True)
    R2 = c.to_dev(st.R2[0]).requires_grad_(True)
    rho1, rho2 = autograd.jacobian_right(g, w, R1, R2)
    # the dot product with the left vector L of the other state
    L1, L2 = c.to_dev(st.L1[1]), c.to_dev(st.L2[1])
    d = c.sys.dims
    W = autograd.block_weights(d.n_act_occ, d.n_act_vir, d.n_occ, d.n_vir, "cuda")
    val = (L1 * rho1).sum() + (W * L2 * rho2).sum()         # <L, A R>_w
    gR1, gR2 = torch.autograd.grad(val, (R1, R2))
    lhs = val.item()
    rhs = ((gR1 * R1).sum() + (gR2 * R2).sum()).item()       # <grad, R> (Euclidean)
    tol = 1e-10 if precision == binding.MLCC3_FP64 else 1e-4
    assert abs(lhs - rhs) <= tol * abs(lhs)
    # grad = w * sigma(L) (the left transformation itself)
    s1, s2 = c.empty_dev(st.R1.shape[1:]), c.empty_dev(st.R2.shape[1:])
    g.jacobian_left([w], L1, L2, s1, s2)
    assert rel_err(c.host(gR1), c.host(s1)) < 1e-12
    assert rel_err(c.host(gR2), c.host(W * s2)) < 1e-12


def test_dot_product_identity_on_gpu():
    torch = _torch()
    c = Case(NO=9, NV=70, no=6, nv=20, NJ=90, nstates=2)
    g = c.context()
    st = c.st
    w = [float(st.omega[0])] * 2
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    sig1, sig2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right(w, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    g.jacobian_left(w, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
    d = c.sys.dims
    for m in range(2):
        for n in range(2):
            a = synth.sd_dot(d, st.L1[m], st.L2[m], c.host(rho1)[n], c.host(rho2)[n])
            b = synth.sd_dot(d, c.host(sig1)[m], c.host(sig2)[m], st.R1[n], st.R2[n])
            assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def test_finite_differences_in_t2():
    """Omega^(T)(t2 + h Rbar) - Omega^(T)(t2 - h Rbar) over 2h = rho(omega=0) with R1 = 0
    (the Jacobian is the derivative of the residual, Sec. 2), step 1e-5, FP64 path."""
    torch = _torch()
    c = Case(NO=6, NV=24, no=4, nv=8, NJ=72, nstates=1)
    s, st = c.sys, c.st
    oc = O.make_ctx(s)
    R2 = st.R2[0]
    dt = O.from_full(oc, O.delta(O.to_full(oc, R2)))   # Rbar in block form
    # t2x is not read by the residual; keep it consistent anyway
    h = 1e-5
    outs = []
    for sign in (1, -1):
        ctx = binding.Context(*c.dims)
        dev = c.to_dev
        ctx.build_integrals(dev(s.chol), dev(s.t1), dev(s.eps), dev(s.t2c + sign * h * dt), dev(s.t2x))
        o1, o2 = c.empty_dev((s.dims.n_vir, s.dims.n_occ)), c.empty_dev(s.t2c.shape)
        ctx.triples_omega(o1, o2)
        outs.append((c.host(o1), c.host(o2)))
        ctx.close()
    fd1 = (outs[0][0] - outs[1][0]) / (2 * h)
    fd2 = (outs[0][1] - outs[1][1]) / (2 * h)
    g = c.context()
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right([0.0], c.to_dev(np.zeros_like(st.R1)), c.to_dev(st.R2), rho1, rho2)
    assert rel_err(fd2, c.host(rho2)[0]) < 1e-7
    assert rel_err(fd1, c.host(rho1)[0]) < 1e-7
