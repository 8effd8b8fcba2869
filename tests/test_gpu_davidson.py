"""The Davidson solver of the omega-nonlinear eigenproblem J(omega) R = omega R
(orbital-energy model of the singles-doubles block plus the library's triples
right transformation): on a tiny system it must reach the eigenpair that the
explicit-matrix fixed-point iteration finds (J built column by column from the
oracle), and on a larger one the split-precision path must give the FP64 path's
excitation energy within 1e-5 Hartree."""
import numpy as np
import pytest

import oracle as O
import sdbasis
from gpu_common import Case
from paper_2202_08612_gb300 import binding, synth
from paper_2202_08612_gb300.davidson import Davidson

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-9), (binding.MLCC3_SPLIT_BF16X3, 1e-5)])
def test_davidson_reaches_the_explicit_eigenpair(precision, tol):
    torch = _torch()
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    w, R1, R2, L1, L2, sd = sdbasis.fixed_point_eigenpair(s, o)
    c = Case(3, 4, 2, 2, 10, seed=5, nstates=1)
    g = c.context(precision=precision)
    dv = Davidson(g, s.eps, (3, 4, 2, 2), torch.device("cuda"))
    res = dv.solve(tol=1e-10 if precision == binding.MLCC3_FP64 else 1e-7)
    assert abs(res.omega - w) < tol, (res.omega, w)
    # the eigenvector, up to normalisation and sign
    x1, x2 = res.R1.cpu().numpy(), res.R2.cpu().numpy()
    ref = np.concatenate([R1.ravel(), R2.ravel()])
    got = np.concatenate([x1.ravel(), x2.ravel()])
    ref, got = ref / np.linalg.norm(ref), got / np.linalg.norm(got)
    assert min(np.abs(got - ref).max(), np.abs(got + ref).max()) < 1e3 * tol
    g.close()


def test_davidson_split_excitation_energy_within_1e5_hartree():
    torch = _torch()
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    om = []
    for precision in (binding.MLCC3_FP64, binding.MLCC3_SPLIT_BF16X3):
        g = c.context(precision=precision)
        dv = Davidson(g, c.sys.eps, c.dims[:4], torch.device("cuda"))
        res = dv.solve(tol=1e-8)
        assert res.residual < 1e-6, res.residual
        om.append(res.omega)
        g.close()
    assert abs(om[0] - om[1]) < 1e-5, om


def test_davidson_with_a_caller_block_equal_to_the_model():
    """A caller-supplied singles-doubles product (here the same diagonal model,
    passed as a function) gives the same root as the built-in model."""
    torch = _torch()
    c = Case(NO=6, NV=24, no=4, nv=8, NJ=72, nstates=1)
    g = c.context()
    dv0 = Davidson(g, c.sys.eps, c.dims[:4], torch.device("cuda"))
    r0 = dv0.solve(tol=1e-9)
    dv1 = Davidson(g, c.sys.eps, c.dims[:4], torch.device("cuda"),
                   sd_apply=lambda v: (dv0.D1 * v[0], dv0.D2 * v[1]))
    r1 = dv1.solve(tol=1e-9)
    assert abs(r0.omega - r1.omega) < 1e-10, (r0.omega, r1.omega)
    g.close()


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-9), (binding.MLCC3_SPLIT_BF16X3, 1e-5)])
def test_block_davidson_reaches_the_explicit_roots(precision, tol):
    """Three roots at once, the expansions of every root transformed at every
    root's frequency in one sweep replay: the self-consistent roots of the
    explicit-matrix iteration."""
    torch = _torch()
    from paper_2202_08612_gb300.davidson import BlockDavidson
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    ref = sdbasis.fixed_point_roots(s, o, 3)
    c = Case(3, 4, 2, 2, 10, seed=5, nstates=1)
    g = c.context(precision=precision)
    bd = BlockDavidson([(g, s.eps, (3, 4, 2, 2))], torch.device("cuda"), 3)
    res = bd.solve(tol=1e-10 if precision == binding.MLCC3_FP64 else 1e-7)[0]
    assert np.all(res.residual < 1e-6), res.residual
    assert np.abs(np.sort(res.omega) - np.sort(ref)).max() < tol, (res.omega, ref)
    assert res.sweeps > 1
    bd.close()
    g.close()


def test_block_davidson_two_systems_in_one_sweep():
    """Two uneven systems solved together (one graph replay per expansion for
    both): each gets the roots that the single-root solver finds for it."""
    torch = _torch()
    from paper_2202_08612_gb300.davidson import BlockDavidson
    cs = [Case(NO=6, NV=24, no=4, nv=8, NJ=72, nstates=1), Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)]
    gs = [c.context() for c in cs]
    bd = BlockDavidson([(g, c.sys.eps, c.dims[:4]) for g, c in zip(gs, cs)], torch.device("cuda"), 2)
    res = bd.solve(tol=1e-9)
    for r, g, c in zip(res, gs, cs):
        assert np.all(r.residual < 1e-7), r.residual
        single = Davidson(g, c.sys.eps, c.dims[:4], torch.device("cuda")).solve(tol=1e-9)
        assert np.abs(r.omega - single.omega).min() < 1e-8, (r.omega, single.omega)
    bd.close()
    for g in gs:
        g.close()
