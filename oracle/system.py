"""O5/O6: the Jacobi-symmetrised DDA system of Eqs. (2)-(3).

Eq. (2): A_ii = I, A_ij = -beta_i G_ij beta_j (i != j); Eq. (3): solve
A x = beta E_inc, then P = beta x.  Vectors use the (3, N) "component, dipole"
layout; the dense matrix flattens them component-major (index mu*N + i).

E_inc(r) = e exp(i kappa a . r) with phase origin at the box centre (the paper
is silent on the origin; any choice only multiplies P by a constant phase).
"""
import numpy as np

from .green import green_tensor


def incident_field(pos, kd, prop, pol):
    """(3, N) complex incident field e exp(i kappa a.r) at dipole centres."""
    a = np.asarray(prop, dtype=np.float64)
    e = np.asarray(pol, dtype=np.complex128)
    phase = np.exp(1j * kd * (pos @ a))
    return e[:, None] * phase[None, :]


def rhs(beta, pos, kd, prop, pol):
    """Eq. (3) right-hand side b = beta E_inc, (3, N)."""
    return beta * incident_field(pos, kd, prop, pol)


def dense_matrix(pos, beta, kd):
    """Eq. (2) as a dense (3N, 3N) complex matrix (component-major ordering)."""
    n = pos.shape[0]
    delta = pos[:, None, :] - pos[None, :, :]
    g = green_tensor(delta, kd)                       # (N, N, 3, 3), G(0)=0
    a = np.empty((3 * n, 3 * n), dtype=np.complex128)
    for mu in range(3):
        for nu in range(3):
            blk = -(beta[mu][:, None] * beta[nu][None, :]) * g[:, :, mu, nu]
            if mu == nu:
                blk = blk + np.eye(n)
            a[mu * n:(mu + 1) * n, nu * n:(nu + 1) * n] = blk
    return a


def matvec_bruteforce(pos, beta, kd, x, chunk=512):
    """O6: y = x - beta (G (beta x)) by the direct O(N^2) sum, (3, N) -> (3, N)."""
    n = pos.shape[0]
    u = beta * x
    out = np.zeros((3, n), dtype=np.complex128)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        delta = pos[s:e, None, :] - pos[None, :, :]
        g = green_tensor(delta, kd)                   # (c, N, 3, 3)
        out[:, s:e] = np.einsum("ijmn,nj->mi", g, u)
    return x - beta * out


def matvec_rows(pos, beta, kd, x, rows, chunk=1 << 21):
    """O6 for selected outputs: (A x)_i = x_i - beta_i sum_j G(r_i - r_j) beta_j x_j
    (Eq. 3) for the dipoles i in `rows` only, by the direct sum over all j in
    chunks.  G u is applied as exp(i kappa rho)/rho^3 [(kappa^2 rho^2 - 1 +
    i kappa rho) u - (kappa^2 rho^2 - 3 + 3 i kappa rho) d (d.u)/rho^2] (O4), so
    no 3x3 tensors are formed and large lattices fit.  Returns (3, len(rows))."""
    n = pos.shape[0]
    u = beta * x
    out = np.zeros((3, len(rows)), dtype=np.complex128)
    for k, i in enumerate(rows):
        acc = np.zeros(3, dtype=np.complex128)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            d = pos[i][None, :] - pos[s:e]                # (c, 3)
            rho2 = np.sum(d * d, axis=1)
            zero = rho2 == 0.0
            rho2s = np.where(zero, 1.0, rho2)
            rho = np.sqrt(rho2s)
            kr = kd * rho
            pref = np.exp(1j * kr) / (rho2s * rho)
            pref[zero] = 0.0                              # G(0) = 0
            ca = (kr * kr - 1.0 + 1j * kr) * pref
            cb = (kr * kr - 3.0 + 3j * kr) / rho2s * pref
            uc = u[:, s:e]
            du = np.sum(d.T * uc, axis=0)                 # d . u_j
            acc += uc @ ca - (d.T * (cb * du)[None, :]).sum(axis=1)
        out[:, k] = x[:, i] - beta[:, i] * acc
    return out


def solve_dense(pos, beta, kd, b):
    """Exact solution of Eq. (3) by LU (numpy.linalg.solve); returns (3, N)."""
    a = dense_matrix(pos, beta, kd)
    x = np.linalg.solve(a, b.reshape(-1))
    return x.reshape(3, -1)
