"""Davidson solver for the omega-nonlinear excitation eigenproblem of the
(ML)CC3 Jacobian, J(omega) R = omega R (Sec. 2: the triples amplitudes depend
on the excitation energy through their denominators, so the effective
singles-doubles Jacobian does too).

J(omega) = D + A_T(omega): A_T(omega) R is the triples contribution that the
library's right transformation returns (mlcc3_jacobian_right, one batched call
per expansion of the subspace); D is the caller's singles-doubles block, by
default the orbital-energy-difference model eps_a - eps_i (singles) and
eps_a + eps_b - eps_i - eps_j (doubles) that stands in for the CCSD Jacobian on
synthetic inputs.  Vectors are device tensors in the library's layouts
(singles [N_V][N_O], doubles as the active-pair block), with the unique-element
inner product (doubly stored elements weighted 1/2).

The nonlinearity is solved self-consistently: a Davidson iteration on J(omega)
at fixed omega gives the Ritz value closest to omega; omega takes that value,
the subspace products are recomputed at the new omega, and the cycle repeats
until omega and the residual norm converge.  The small projected eigenproblem
is solved on the host (numpy); all vector work stays on the device.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class DavidsonResult:
    omega: float
    R1: object       # [N_V][N_O] device tensor
    R2: object       # active-pair doubles block, device tensor
    residual: float  # unique-element norm of J(omega) R - omega R (R normalised)
    iterations: int  # right-transformation calls
    omega_cycles: int


class Davidson:
    """One excitation at a time from the lowest diagonal element of D (or from a
    given guess).  ctx: a binding.Context whose integrals are built; eps: host
    orbital energies (occupied first); dims: (N_O, N_V, n_o, n_v).  diag: the
    singles-doubles diagonal (host arrays in the vector layouts; default the
    orbital-energy differences), the preconditioner; sd_apply: the caller's
    singles-doubles block, (v1, v2) -> (y1, y2) on device tensors (default: the
    diagonal model D v)."""

    def __init__(self, ctx, eps, dims, device, diag=None, sd_apply=None):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.sd_apply = sd_apply
        NO, NV, no, nv = dims
        self.dims = dims
        self.dev = device
        eps = np.asarray(eps, dtype=np.float64)
        eo, ev = eps[:NO], eps[NO:]
        if diag is None:
            d1 = ev[:, None] - eo[None, :]
            d2 = (ev[None, :nv, None, None] + ev[None, None, None, :]
                  - eo[:no, None, None, None] - eo[None, None, :, None])
        else:
            d1, d2 = diag
        self.D1 = torch.as_tensor(np.ascontiguousarray(d1), dtype=torch.float64, device=device)
        self.D2 = torch.as_tensor(np.ascontiguousarray(d2), dtype=torch.float64, device=device)
        w = np.ones((no, nv, NO, NV))
        w[:, :, :no, :nv] = 0.5
        for i in range(no):
            for a in range(nv):
                w[i, a, i, a] = 1.0
        self.W2 = torch.as_tensor(w, dtype=torch.float64, device=device)

    # ---- vector algebra (unique-element inner product) ----
    def dot(self, x, y):
        return float((x[0] * y[0]).sum() + (self.W2 * x[1] * y[1]).sum())

    def apply(self, omega, vecs):
        """J(omega) v for a list of vectors: one batched right transformation."""
        torch = self.torch
        R1 = torch.stack([v[0] for v in vecs]).contiguous()
        R2 = torch.stack([v[1] for v in vecs]).contiguous()
        rho1, rho2 = torch.empty_like(R1), torch.empty_like(R2)
        self.ctx.jacobian_right(np.full(len(vecs), omega), R1, R2, rho1, rho2)
        self.calls += 1
        out = []
        for k, v in enumerate(vecs):
            y = self.sd_apply(v) if self.sd_apply else (self.D1 * v[0], self.D2 * v[1])
            out.append((y[0] + rho1[k], y[1] + rho2[k]))
        return out

    def _orthonormalize(self, v, basis):
        for _ in range(2):
            for b in basis:
                c = self.dot(b, v)
                v = (v[0] - c * b[0], v[1] - c * b[1])
        n = np.sqrt(max(self.dot(v, v), 0.0))
        return None if n < 1e-10 else (v[0] / n, v[1] / n)

    def _guess(self):
        torch = self.torch
        k = int(torch.argmin(self.D1).item())
        v1 = torch.zeros_like(self.D1).view(-1)
        v1[k] = 1.0
        return (v1.view_as(self.D1), torch.zeros_like(self.D2))

    def solve(self, guess=None, omega=None, tol=1e-8, omega_tol=1e-10, max_subspace=24,
              max_cycles=30, max_iter=200):
        """Converged (omega, R) of the root that starts at `guess` (default: the
        unit vector of the lowest singles diagonal element, omega = that element)."""
        self.calls = 0
        v = guess if guess is not None else self._guess()
        v = self._orthonormalize(v, [])
        if omega is None:
            omega = self.dot(v, (self.D1 * v[0], self.D2 * v[1]))
        basis, prods = [v], None
        res, cycles = np.inf, 0
        for cycles in range(1, max_cycles + 1):
            prods = self.apply(omega, basis)          # the whole subspace at this omega
            theta, x, jx = omega, basis[0], prods[0]
            while True:
                n = len(basis)
                H = np.array([[self.dot(basis[i], prods[j]) for j in range(n)] for i in range(n)])
                ev, evec = np.linalg.eig(H)
                k = int(np.argmin(np.abs(ev - omega)))
                theta = float(ev[k].real)
                y = evec[:, k].real
                x = (sum(y[i] * basis[i][0] for i in range(n)), sum(y[i] * basis[i][1] for i in range(n)))
                jx = (sum(y[i] * prods[i][0] for i in range(n)), sum(y[i] * prods[i][1] for i in range(n)))
                nx = np.sqrt(self.dot(x, x))
                x, jx = (x[0] / nx, x[1] / nx), (jx[0] / nx, jx[1] / nx)
                r = (jx[0] - theta * x[0], jx[1] - theta * x[1])
                res = np.sqrt(self.dot(r, r))
                if res < tol or self.calls >= max_iter:
                    break
                # diagonal preconditioner (theta - D)^-1, kept away from zero
                d1 = theta - self.D1
                d2 = theta - self.D2
                d1 = self.torch.where(d1.abs() < 1e-4, self.torch.full_like(d1, 1e-4), d1)
                d2 = self.torch.where(d2.abs() < 1e-4, self.torch.full_like(d2, 1e-4), d2)
                t = self._orthonormalize((r[0] / d1, r[1] / d2), basis)
                if t is None:
                    break
                if len(basis) >= max_subspace:      # restart from the Ritz vector
                    basis, prods = [x], [jx]
                    t = self._orthonormalize(t, basis)
                    if t is None:
                        break
                basis.append(t)
                prods.append(self.apply(omega, [t])[0])
            converged = abs(theta - omega) < omega_tol and res < tol
            omega = theta
            basis = [x]
            if converged or self.calls >= max_iter:
                break
        return DavidsonResult(omega, x[0], x[1], float(res), self.calls, cycles)


@dataclass
class BlockResult:
    omega: np.ndarray      # [k] converged excitation energies
    R1: object             # [k][N_V][N_O] device tensor
    R2: object             # [k][n_o][n_v][N_O][N_V] device tensor
    residual: np.ndarray   # [k] unique-element norms of J(omega_r) R_r - omega_r R_r
    sweeps: int            # mlcc3_sweep_run calls (one graph replay each)
    omega_cycles: int


class BlockDavidson:
    """Several roots of the omega-nonlinear eigenproblem J(omega) R = omega R for
    one or more systems at once (Sec. 2), with one shared subspace per system.

    J(omega) = D + A_T(omega) as in Davidson.  Root r of a system keeps its own
    frequency omega_r and the products P_r = J(omega_r) V of the whole subspace
    V; the projected matrices H_r = V^T W P_r (W the unique-element weights) of
    all roots come from one batched device GEMM, and root r takes the r-th
    eigenvalue (by real part) of H_r.  Every expansion (the preconditioned
    residuals of the unconverged roots, orthonormalised against V) is
    transformed at every root's frequency in ONE mlcc3_sweep_run over all
    systems: the systems' k x k vector slots (expansion vector s at frequency
    omega_r) are a captured CUDA graph, replayed with new vectors copied into
    its fixed buffers.  At fixed frequencies the inner iteration runs until the
    residuals fall below tol; then omega_r takes the Ritz value and the
    subspace restarts from the Ritz vectors (macro cycles), until the
    frequencies settle.

    systems: list of (ctx, eps, dims) or (ctx, eps, dims, (d1, d2)) with dims =
    (N_O, N_V, n_o, n_v) and an optional singles-doubles diagonal."""

    def __init__(self, systems, device, nroots, tune=False):
        import torch
        from . import binding
        self.torch = torch
        self.dev = device
        self.k = int(nroots)
        self.sys = []
        for spec in systems:
            ctx, eps, dims = spec[:3]
            NO, NV, no, nv = dims
            eps = np.asarray(eps, dtype=np.float64)
            eo, ev = eps[:NO], eps[NO:]
            if len(spec) > 3 and spec[3] is not None:
                d1, d2 = spec[3]
            else:
                d1 = ev[:, None] - eo[None, :]
                d2 = (ev[None, :nv, None, None] + ev[None, None, None, :]
                      - eo[:no, None, None, None] - eo[None, None, :, None])
            n1, n2 = NV * NO, no * nv * NO * NV
            w = np.ones((no, nv, NO, NV))
            w[:, :, :no, :nv] = 0.5
            for i in range(no):
                for a in range(nv):
                    w[i, a, i, a] = 1.0
            f = lambda x: torch.as_tensor(np.ascontiguousarray(x).reshape(-1), dtype=torch.float64,
                                          device=device)
            slots = self.k * self.k
            s = {"ctx": ctx, "dims": dims, "n1": n1, "n2": n2,
                 "D": torch.cat([f(d1), f(d2)]), "w": torch.cat([f(np.ones(n1)), f(w)]),
                 "R1": torch.zeros((slots, NV, NO), dtype=torch.float64, device=device),
                 "R2": torch.zeros((slots, no, nv, NO, NV), dtype=torch.float64, device=device)}
            s["rho1"], s["rho2"] = torch.zeros_like(s["R1"]), torch.zeros_like(s["R2"])
            self.sys.append(s)
        self.sweep = binding.Sweep([s["ctx"] for s in self.sys], tune=tune)
        for q, s in enumerate(self.sys):
            self.sweep.set_system(q, s["R1"], s["R2"], s["rho1"], s["rho2"])
        self.sweeps = 0

    def close(self):
        self.sweep.close()

    # ---- vectors are flat: singles [N_V N_O] then the doubles block ----
    def _unflat(self, s, X):
        NO, NV, no, nv = s["dims"]
        return X[:, :s["n1"]].reshape(-1, NV, NO), X[:, s["n1"]:].reshape(-1, no, nv, NO, NV)

    def _orth(self, s, T, V):
        """Orthonormalise the rows of T against the rows of V and each other (two
        Gram-Schmidt passes, unique-element inner product); drops dependent rows."""
        w = s["w"]
        out = []
        for t in T:
            for _ in range(2):
                if V is not None and V.shape[0]:
                    t = t - ((V * w) @ t) @ V
                for u in out:
                    t = t - (u * w * t).sum() * u
            n = float(((t * w * t).sum()).clamp_min(0.0).sqrt())
            if n > 1e-10:
                out.append(t / n)
        return self.torch.stack(out) if out else None

    def _products(self, todo):
        """todo[q] = (T [m][n], omegas [k]): J_T(omega_r) t_s for all s, r of every
        system in one sweep; returns per system [k][m][n] (A_T parts + D t)."""
        torch = self.torch
        oms = []
        for s, (T, om) in zip(self.sys, todo):
            m = 0 if T is None else T.shape[0]
            R1, R2 = s["R1"], s["R2"]
            R1.zero_()
            R2.zero_()
            if m:
                t1, t2 = self._unflat(s, T)
                for r in range(self.k):
                    R1[r * self.k:r * self.k + m] = t1
                    R2[r * self.k:r * self.k + m] = t2
            oms.append(np.repeat(np.asarray(om, dtype=np.float64), self.k))
        self.sweep.run(np.concatenate(oms))
        self.sweeps += 1
        out = []
        for s, (T, om) in zip(self.sys, todo):
            if T is None or T.shape[0] == 0:
                out.append(None)
                continue
            m = T.shape[0]
            rho = torch.cat([s["rho1"].reshape(self.k * self.k, -1),
                             s["rho2"].reshape(self.k * self.k, -1)], 1)
            P = rho.reshape(self.k, self.k, -1)[:, :m] + (s["D"] * T)[None]
            out.append(P)
        return out

    def _guess(self, s):
        torch = self.torch
        idx = torch.argsort(s["D"][:s["n1"]])[:self.k]
        G = torch.zeros((self.k, s["n1"] + s["n2"]), dtype=torch.float64, device=self.dev)
        G[torch.arange(self.k, device=self.dev), idx] = 1.0
        return G, s["D"][idx].cpu().numpy()

    def solve(self, tol=1e-8, omega_tol=1e-10, max_subspace=24, max_cycles=30, max_sweeps=300):
        torch = self.torch
        k = self.k
        st = []
        for s in self.sys:
            G, om = self._guess(s)
            st.append({"V": self._orth(s, G, None), "om": om.copy(), "done": False,
                       "theta": om.copy(), "res": np.full(k, np.inf), "X": None})
        cycles = 0
        for cycles in range(1, max_cycles + 1):
            # products of the (restarted) subspace at the current frequencies
            for x in st:
                x["P"] = None
            pending = [(x["V"], x["om"]) for x in st]
            for x, P in zip(st, self._products(pending)):
                x["P"] = P
            inner_done = [False] * len(st)
            while not all(inner_done) and self.sweeps < max_sweeps:
                todo = []
                for q, (s, x) in enumerate(zip(self.sys, st)):
                    if inner_done[q]:
                        todo.append((None, x["om"]))
                        continue
                    V, P, w = x["V"], x["P"], s["w"]
                    H = torch.matmul((V * w)[None], P.transpose(1, 2)).cpu().numpy()  # [k][nb][nb]
                    Y = np.zeros((k, V.shape[0]))
                    for r in range(k):
                        ev, evec = np.linalg.eig(H[r])
                        o = np.argsort(ev.real)
                        x["theta"][r] = float(ev[o[r]].real)
                        Y[r] = evec[:, o[r]].real
                    Yd = torch.as_tensor(Y, dtype=torch.float64, device=self.dev)
                    X = Yd @ V
                    JX = torch.bmm(Yd[:, None, :], P).squeeze(1)
                    nx = ((X * w * X).sum(1)).sqrt()[:, None]
                    X, JX = X / nx, JX / nx
                    Rr = JX - torch.as_tensor(x["theta"], device=self.dev)[:, None] * X
                    x["res"] = ((Rr * w * Rr).sum(1)).sqrt().cpu().numpy()
                    x["X"] = X
                    open_r = [r for r in range(k) if x["res"][r] >= tol]
                    if not open_r:
                        inner_done[q] = True
                        todo.append((None, x["om"]))
                        continue
                    th = torch.as_tensor(x["theta"][open_r], device=self.dev)[:, None]
                    den = th - s["D"][None]
                    den = torch.where(den.abs() < 1e-4, torch.full_like(den, 1e-4), den)
                    T = self._orth(s, Rr[open_r] / den, V)
                    if T is None:
                        inner_done[q] = True
                        todo.append((None, x["om"]))
                        continue
                    if V.shape[0] + T.shape[0] > max_subspace:   # restart from the Ritz vectors
                        x["V"] = self._orth(s, X, None)
                        x["restart"] = True
                        todo.append((x["V"], x["om"]))
                        continue
                    x["restart"] = False
                    x["T"] = T
                    todo.append((T, x["om"]))
                prods = self._products(todo)
                for q, (x, P) in enumerate(zip(st, prods)):
                    if P is None:
                        continue
                    if x.get("restart"):
                        x["P"] = P
                    else:
                        x["V"] = torch.cat([x["V"], x["T"]])
                        x["P"] = torch.cat([x["P"], P], 1)
            conv = True
            for s, x in zip(self.sys, st):
                if np.max(np.abs(x["theta"] - x["om"])) >= omega_tol or np.max(x["res"]) >= tol:
                    conv = False
                x["om"] = x["theta"].copy()
                x["V"] = self._orth(s, x["X"], None)
            if conv or self.sweeps >= max_sweeps:
                break
        out = []
        for s, x in zip(self.sys, st):
            R1, R2 = self._unflat(s, x["X"])
            out.append(BlockResult(x["theta"].copy(), R1, R2, x["res"].copy(), self.sweeps, cycles))
        return out
