"""The unique singles / active-pair doubles space of the library's vectors as an
explicit basis (orthonormal under the unique-element inner product), and the
omega-nonlinear eigenpair of J(omega) = Delta-eps + A_T(omega) on it, built
from the oracle (CPU only)."""
import numpy as np

import oracle as O


def unique_basis(d):
    """Unique singles and active-pair doubles elements (orthonormal under the
    unique-element inner product) as (kind, index) pairs."""
    NO, NV, no, nv = d.n_occ, d.n_vir, d.n_act_occ, d.n_act_vir
    basis = [("s", (A, I)) for A in range(NV) for I in range(NO)]
    for i in range(no):
        for a in range(nv):
            for L in range(NO):
                for D in range(NV):
                    if L < no and D < nv and (L * nv + D) < (i * nv + a):
                        continue  # stored twice: keep one representative
                    basis.append(("d", (i, a, L, D)))
    return basis


def to_vec(d, basis, c):
    NO, NV, no, nv = d.n_occ, d.n_vir, d.n_act_occ, d.n_act_vir
    x1 = np.zeros((NV, NO))
    x2 = np.zeros((no, nv, NO, NV))
    for (kind, idx), v in zip(basis, c):
        if kind == "s":
            x1[idx] = v
        else:
            i, a, L, D = idx
            x2[i, a, L, D] = v
            if L < no and D < nv:
                x2[L, D, i, a] = v
    return x1, x2


def coef(d, basis, x1, x2):
    return np.array([x1[idx] if kind == "s" else x2[idx] for kind, idx in basis])




def fixed_point_eigenpair(s, o):
    """(omega*, R1, R2, L1, L2, sd_part): J(omega*) R = omega* R, L J(omega*) =
    omega* L with <L, R> = 1, J = diag(Delta-eps) + A_T(omega) (the diagonal is
    the orbital-energy model of the singles-doubles block); sd_part = <L, diag R>.
    Doubles in the active-pair block layout."""
    d = s.dims
    basis = unique_basis(d)
    eps, NO = s.eps, d.n_occ

    def diag(kind, idx):
        if kind == "s":
            A, I = idx
            return eps[NO + A] - eps[I]
        i, a, L, D = idx
        return eps[NO + a] + eps[NO + D] - eps[i] - eps[L]

    dvec = np.array([diag(k, idx) for k, idx in basis])

    def jmat(w):
        cols = []
        for nu in range(len(basis)):
            e = np.zeros(len(basis))
            e[nu] = 1.0
            r1, r2 = to_vec(d, basis, e)
            y1, y2 = O.jacobian_right(o, w, r1, O.to_full(o, r2))
            cols.append(coef(d, basis, y1, O.from_full(o, y2)))
        return np.diag(dvec) + np.array(cols).T

    w = float(np.sort(dvec)[0])
    for _ in range(30):
        ev = np.linalg.eigvals(jmat(w))
        w_new = float(ev[np.argmin(np.abs(ev - w))].real)
        if abs(w_new - w) < 1e-13:
            w = w_new
            break
        w = w_new
    J = jmat(w)
    evr, vr = np.linalg.eig(J)
    evl, vl = np.linalg.eig(J.T)
    kr, kl = np.argmin(np.abs(evr - w)), np.argmin(np.abs(evl - w))
    assert abs(evr[kr].imag) < 1e-12 and abs(evr[kr].real - w) < 1e-10
    R, L = vr[:, kr].real, vl[:, kl].real
    L = L / (L @ R)
    R1, R2 = to_vec(d, basis, R)
    L1, L2 = to_vec(d, basis, L)
    return w, R1, R2, L1, L2, float(L @ (dvec * R))


def fixed_point_roots(s, o, k):
    """The k lowest self-consistent roots of J(omega) = diag(Delta-eps) + A_T(omega)
    on the explicit unique basis: omega_r = the r-th eigenvalue (by real part)
    of J(omega_r), iterated from the r-th lowest singles diagonal element."""
    d = s.dims
    basis = unique_basis(d)
    eps, NO = s.eps, d.n_occ

    def diag(kind, idx):
        if kind == "s":
            A, I = idx
            return eps[NO + A] - eps[I]
        i, a, L, D = idx
        return eps[NO + a] + eps[NO + D] - eps[i] - eps[L]

    dvec = np.array([diag(kk, idx) for kk, idx in basis])
    cols_cache = {}

    def jmat(w):
        if w not in cols_cache:
            cols = []
            for nu in range(len(basis)):
                e = np.zeros(len(basis))
                e[nu] = 1.0
                r1, r2 = to_vec(d, basis, e)
                y1, y2 = O.jacobian_right(o, w, r1, O.to_full(o, r2))
                cols.append(coef(d, basis, y1, O.from_full(o, y2)))
            cols_cache[w] = np.diag(dvec) + np.array(cols).T
        return cols_cache[w]

    singles = np.sort(np.array([dvec[n] for n, (kk, _) in enumerate(basis) if kk == "s"]))
    out = []
    for r in range(k):
        w = float(singles[r])
        for _ in range(60):
            ev = np.sort_complex(np.linalg.eigvals(jmat(w)))
            ev = ev[np.argsort(ev.real, kind="stable")]
            w_new = float(ev[r].real)
            if abs(w_new - w) < 1e-13:
                w = w_new
                break
            w = w_new
        out.append(w)
    return np.array(out)
