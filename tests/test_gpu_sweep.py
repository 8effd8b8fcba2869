"""Batched sweep: the right transformations of several uneven systems and all
of their trial vectors in one captured CUDA graph, replayed with new
frequencies, against the oracle and against the contexts' own eager calls."""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu

SYSTEMS = [  # (N_O, N_V, n_o, n_v, N_J), trial vectors
    ((6, 24, 4, 8, 72), 2),
    ((7, 30, 5, 13, 40), 3),
    ((10, 40, 6, 10, 60), 2),
]


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def cases():
    _cuda()
    out = []
    for q, (dims, nvec) in enumerate(SYSTEMS):
        c = Case(*dims, nstates=nvec, seed=100 + q)
        c.octx = c.oracle_ctx()
        out.append(c)
    return out


def oracle_rho(c, omega):
    o, st = c.octx, c.st
    r1, r2 = [], []
    for v in range(len(omega)):
        a, b = O.jacobian_right(o, float(omega[v]), st.R1[v], O.to_full(o, st.R2[v]))
        r1.append(a)
        r2.append(O.from_full(o, b))
    return np.array(r1), np.array(r2)


def run_sweep(cases, precision, tune):
    ctxs = [c.context(precision=precision) for c in cases]
    sw = binding.Sweep(ctxs, tune=tune)
    outs = []
    for q, c in enumerate(cases):
        R1, R2 = c.to_dev(c.st.R1), c.to_dev(c.st.R2)
        rho1, rho2 = c.empty_dev(c.st.R1.shape), c.empty_dev(c.st.R2.shape)
        sw.set_system(q, R1, R2, rho1, rho2)
        outs.append((rho1, rho2))
    return ctxs, sw, outs


def check(cases, outs, omegas, tol):
    for c, (rho1, rho2), w in zip(cases, outs, omegas):
        r1, r2 = oracle_rho(c, w)
        assert rel_err(c.host(rho1), r1) < tol
        assert rel_err(c.host(rho2), r2) < tol


def test_sweep_fp64_matches_oracle_and_replays(cases):
    ctxs, sw, outs = run_sweep(cases, binding.MLCC3_FP64, tune=True)
    omegas = [c.st.omega for c in cases]
    sw.run(np.concatenate(omegas))
    check(cases, outs, omegas, 1e-10)
    info = sw.info()
    assert info["graph_nodes"] > 0 and len(info["systems"]) == len(cases)
    assert all(s["bstc_fill"] in (0, 2, 4, 8) for s in info["systems"])
    # replay with new frequencies (no new capture)
    nodes = info["graph_nodes"]
    omegas2 = [w + 0.05 for w in omegas]
    sw.run(np.concatenate(omegas2))
    check(cases, outs, omegas2, 1e-10)
    assert sw.info()["graph_nodes"] == nodes
    # the same results from the contexts' own eager calls, mixed with the sweep
    for c, g, (rho1, rho2), w in zip(cases, ctxs, outs, omegas2):
        e1, e2 = c.empty_dev(c.st.R1.shape), c.empty_dev(c.st.R2.shape)
        g.jacobian_right(w, c.to_dev(c.st.R1), c.to_dev(c.st.R2), e1, e2)
        assert rel_err(c.host(rho1), c.host(e1)) < 1e-12
        assert rel_err(c.host(rho2), c.host(e2)) < 1e-12
    # a new integral build forces a new capture; results stay right
    s = cases[0].sys
    d = cases[0].to_dev
    ctxs[0].build_integrals(d(s.chol), d(s.t1), d(s.eps), d(s.t2c), d(s.t2x))
    sw.run(np.concatenate(omegas))
    check(cases, outs, omegas, 1e-10)
    sw.close()


def test_sweep_split_matches_oracle(cases):
    ctxs, sw, outs = run_sweep(cases, binding.MLCC3_SPLIT_BF16X3, tune=False)
    omegas = [c.st.omega for c in cases]
    sw.run(np.concatenate(omegas))
    check(cases, outs, omegas, 1e-4)
    sw.close()


def test_sweep_split_tuned_matches_oracle(cases):
    """The autotuner on: per system the split-K fill, the triples-build tile
    grouping, the launch form and the accumulation-chain cap are timed and the
    fastest kept; the tuned graph still meets the split bar, also after a
    replay with new frequencies."""
    ctxs, sw, outs = run_sweep(cases, binding.MLCC3_SPLIT_BF16X3, tune=True)
    omegas = [c.st.omega for c in cases]
    sw.run(np.concatenate(omegas))
    check(cases, outs, omegas, 1e-4)
    info = sw.info()
    for sy in info["systems"]:
        assert sy["tc_group"] in (1, 2, 4) and sy["tc_kcap"] in (8, 16)
        assert sy["tc_persist_from"] in (304, 0, 1 << 30)
        assert set(sy["tc_ms"]) >= {"tc_persist_from", "tc_kcap"}
        assert all(ms > 0 for _, ms in sy["tc_ms"]["tc_kcap"])
    omegas2 = [w + 0.05 for w in omegas]
    sw.run(np.concatenate(omegas2))
    check(cases, outs, omegas2, 1e-4)
    sw.close()


def test_sweep_errors(cases):
    torch = _cuda()
    g = cases[0].context()
    with pytest.raises(binding.MLCC3Error):
        binding.Sweep([g, g])
    sw = binding.Sweep([g], tune=False)
    host = np.zeros(cases[0].st.R1.shape)
    with pytest.raises(binding.MLCC3Error):
        sw.set_system(0, host, host, host, host)
    c = cases[0]
    sw.set_system(0, c.to_dev(c.st.R1), c.to_dev(c.st.R2), c.empty_dev(c.st.R1.shape),
                  c.empty_dev(c.st.R2.shape))
    with pytest.raises(binding.MLCC3Error):
        sw.run(np.array([np.nan, 0.4]))
    sw.close()
    del torch
