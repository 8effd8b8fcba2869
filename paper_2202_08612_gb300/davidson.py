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
