"""The large workloads' device-side input generator (bench.device_system) on
CPU: the same recipe as the host generator (symmetric Cholesky vectors,
MP2-like doubles from the bare (ai|DL) integrals over the orbital-energy
denominators, the exchange block, pair-symmetric trial vectors), checked
against the formulas recomputed here in numpy."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("core", [False, True])
def test_device_system_recipe(core):
    NO, NV, no, nv, NJ, nvec = 6, 10, 3, 4, 8, 2
    x, omega = bench.device_system(NO, NV, no, nv, NJ, nvec, 7, torch.device("cpu"), core)
    x = {k: v.numpy() for k, v in x.items()}
    chol, eps = x["chol"], x["eps"]
    assert np.array_equal(chol, chol.transpose(0, 2, 1))
    assert (eps[0] == -10.0) == core
    assert np.all(eps[1 if core else 0:NO] < -0.29) and np.all(eps[NO:] > 0.09)
    Lvo = chol[:, NO:, :NO]
    eo, ev = eps[:NO], eps[NO:]
    den = (eo[:no, None, None, None] + eo[None, None, :, None]
           - ev[None, :nv, None, None] - ev[None, None, None, :])
    t2c = np.einsum('Jai,JDL->iaLD', Lvo[:, :nv, :no], Lvo) / den
    t2x = np.einsum('JaL,JDi->iaLD', Lvo[:, :nv, :], Lvo[:, :, :no]) / den
    assert np.allclose(x["t2c"], t2c, rtol=1e-12, atol=0)
    assert np.allclose(x["t2x"], t2x, rtol=1e-12, atol=0)
    assert np.array_equal(x["lam2"], x["t2c"])
    for k in ("R2", "L2"):
        aa = x[k][:, :, :, :no, :nv]
        assert np.allclose(aa, aa.transpose(0, 3, 4, 1, 2), rtol=0, atol=1e-15)
    for n in range(nvec):
        assert abs(np.sum(x["R1"][n] ** 2) - 0.95) < 1e-12
        assert abs(np.sum(x["R2"][n] ** 2) - 0.05) < 1e-12
    assert np.all((omega >= 0.3) & (omega <= 0.6)) and omega.shape == (nvec,)
    mu = x["mu"]
    assert np.array_equal(mu, mu.transpose(0, 2, 1))
