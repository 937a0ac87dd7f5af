"""O9: the four Krylov solvers of Sec. 2 (CGNR, Bi-CGSTAB, Bi-CG, QMR).

Sec. 2 names the solvers and notes that Bi-CG and QMR exploit the complex
symmetry A = A^T of Eq. (2) (they use the bilinear form u^T v, no
conjugation); the stopping rule is the relative residual norm
||b - A x||_2 / ||b||_2 < eps with eps = 1e-5 by default (Sec. 2, Sec. 3.1).
The algorithms are restated from the standard literature as mathematics:

* QMR-CS: Lanczos with the bilinear form and unit-norm Lanczos vectors,
  quasi-minimal residual iterates, coupled two-term recurrences, residual kept
  by r_i = r_{i-1} - s_i with s_i built from A p_i (no extra product);
* Bi-CG-CS (COCG): conjugate gradients with u^T v in place of u^H v;
* Bi-CGSTAB: van der Vorst's method with Hermitian products, shadow r0;
* CGNR: CG on A^H A x = A^H b, with A^H y = conj(A conj(y)).

Every solver starts from x0 = 0 and returns (x, info) where info holds the
status ("ok", "not_converged", "breakdown"), iteration and product counts, the
recurrence residual history (relative) and the true relative residual at exit.
"""
import numpy as np

OK, NOT_CONVERGED, BREAKDOWN = "ok", "not_converged", "breakdown"
# The paper's solvers have no look-ahead (Sec. 2), so a vanishing bilinear
# form u^T u stops QMR-CS and Bi-CG-CS.  In floating point an exact zero shows
# up as rounding noise: |u^T u| <= BREAK ||u||^2 counts as zero.
BREAK = 1e-12


def dotu(a, b):
    """Bilinear form a^T b (no conjugation)."""
    return complex(np.sum(a * b))


def dotc(a, b):
    """Hermitian form a^H b."""
    return complex(np.sum(np.conj(a) * b))


def norm2(a):
    return float(np.sqrt(np.sum(a.real * a.real + a.imag * a.imag)))


def _finish(matvec, b, x, status, iters, nmv, hist):
    r = b - matvec(x)
    rel = norm2(r) / norm2(b)
    return x, dict(status=status, iters=iters, matvecs=nmv, hist=np.array(hist),
                   rel_res_true=rel, rel_res_recur=hist[-1])


def qmr_cs(matvec, b, tol=1e-5, maxiter=10000):
    """QMR for complex-symmetric A (Freund's QMR with the bilinear form).

    Lanczos vectors v_i are scaled to unit Euclidean norm, delta_i = v_i^T v_i
    carries the bilinear normalisation, and the iteration runs on coupled
    two-term recurrences (Freund and Nachtigal's implementation of QMR without
    look-ahead; for A = A^T the left and right Lanczos sequences coincide, so
    one product per step):
        p_i = v_i - (rho_i delta_i / eps_{i-1}) p_{i-1},   pt = A p_i,
        eps_i = p_i^T pt,  beta_i = eps_i / delta_i,  vt = pt - beta_i v_i,
        rho_{i+1} = ||vt||,  theta_i = rho_{i+1} / (g_{i-1} |beta_i|),
        g_i = 1 / sqrt(1 + theta_i^2),
        eta_i = -eta_{i-1} rho_i g_i^2 / (beta_i g_{i-1}^2),
        d_i = eta_i p_i + (theta_{i-1} g_i)^2 d_{i-1},
        s_i = eta_i pt + (theta_{i-1} g_i)^2 s_{i-1},
        x_i = x_{i-1} + d_i,  r_i = r_{i-1} - s_i.
    The iterate minimises ||rho_1 e_1 - H z|| over the Krylov space, H the
    (i+1) x i Lanczos matrix in the unit-norm basis (the quasi-minimal
    residual property).  delta_i = 0, eps_i = 0 or beta_i = 0 is a breakdown
    (no look-ahead)."""
    bn = norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    vt = b.copy()
    rho = bn
    g_prev, eta_prev, theta_prev, eps_prev = 1.0, -1.0 + 0.0j, 0.0, 1.0 + 0.0j
    p = np.zeros_like(b)
    d = np.zeros_like(b)
    s = np.zeros_like(b)
    hist = [1.0]
    nmv = 0
    status = NOT_CONVERGED
    k = 0
    for k in range(1, maxiter + 1):
        v = vt / rho
        delta = dotu(v, v)
        if abs(delta) <= BREAK * norm2(v) ** 2:
            status = BREAKDOWN
            break
        p = v if k == 1 else v - (rho * delta / eps_prev) * p
        pt = matvec(p); nmv += 1
        eps = dotu(p, pt)
        beta = eps / delta
        if eps == 0 or beta == 0:
            status = BREAKDOWN
            break
        vt = pt - beta * v
        rho_next = norm2(vt)
        theta = rho_next / (g_prev * abs(beta))
        g = 1.0 / np.sqrt(1.0 + theta * theta)
        eta = -eta_prev * rho * g * g / (beta * g_prev * g_prev)
        c = (theta_prev * g) ** 2
        d = eta * p + c * d
        s = eta * pt + c * s
        x = x + d
        r = r - s
        res = norm2(r) / bn
        hist.append(res)
        if res < tol:
            status = OK
            break
        if rho_next == 0:            # invariant subspace: the update above is exact
            status = OK if res < tol else BREAKDOWN
            break
        rho, g_prev, eta_prev, theta_prev, eps_prev = rho_next, g, eta, theta, eps
    x, info = _finish(matvec, b, x, status, k, nmv, hist)
    if info["status"] == OK and info["rel_res_true"] >= tol:
        info["status"] = NOT_CONVERGED
    return x, info


def bicg_cs(matvec, b, tol=1e-5, maxiter=10000):
    """Bi-CG for complex-symmetric A (COCG)."""
    bn = norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = dotu(r, r)
    hist = [1.0]
    nmv = 0
    status = NOT_CONVERGED
    k = 0
    for k in range(1, maxiter + 1):
        q = matvec(p); nmv += 1
        mu = dotu(p, q)
        if mu == 0 or abs(rho) <= BREAK * norm2(r) ** 2:
            status = BREAKDOWN
            hist.append(hist[-1])
            break
        alpha = rho / mu
        x = x + alpha * p
        r = r - alpha * q
        res = norm2(r) / bn
        hist.append(res)
        if res < tol:
            status = OK
            break
        rho_new = dotu(r, r)
        p = r + (rho_new / rho) * p
        rho = rho_new
    x, info = _finish(matvec, b, x, status, k, nmv, hist)
    if info["status"] == OK and info["rel_res_true"] >= tol:
        info["status"] = NOT_CONVERGED
    return x, info


def bicgstab(matvec, b, tol=1e-5, maxiter=10000):
    """Bi-CGSTAB (Hermitian inner products, shadow residual r0 = b)."""
    bn = norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    rho_prev = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = [1.0]
    nmv = 0
    status = NOT_CONVERGED
    k = 0
    for k in range(1, maxiter + 1):
        rho = dotc(rh, r)
        if rho == 0 or omega == 0:
            status = BREAKDOWN
            hist.append(hist[-1])
            break
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p); nmv += 1
        alpha = rho / dotc(rh, v)
        s = r - alpha * v
        sres = norm2(s) / bn
        if sres < tol:
            x = x + alpha * p
            hist.append(sres)
            status = OK
            break
        t = matvec(s); nmv += 1
        tt = dotc(t, t)
        omega = dotc(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_prev = rho
        res = norm2(r) / bn
        hist.append(res)
        if res < tol:
            status = OK
            break
    x, info = _finish(matvec, b, x, status, k, nmv, hist)
    if info["status"] == OK and info["rel_res_true"] >= tol:
        info["status"] = NOT_CONVERGED
    return x, info


def cgnr(matvec, b, tol=1e-5, maxiter=10000, matvec_h=None):
    """CGNR: CG on the normal equations A^H A x = A^H b.  A^H defaults to
    conj(A conj(.)), valid because A is complex symmetric (Eq. 2)."""
    if matvec_h is None:
        def matvec_h(y):
            return np.conj(matvec(np.conj(y)))
    bn = norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    z = matvec_h(r); nmv = 1
    p = z.copy()
    zz = dotc(z, z).real
    hist = [1.0]
    status = NOT_CONVERGED
    k = 0
    for k in range(1, maxiter + 1):
        w = matvec(p); nmv += 1
        ww = dotc(w, w).real
        if ww == 0:
            status = BREAKDOWN
            hist.append(hist[-1])
            break
        alpha = zz / ww
        x = x + alpha * p
        r = r - alpha * w
        res = norm2(r) / bn
        hist.append(res)
        if res < tol:
            status = OK
            break
        z = matvec_h(r); nmv += 1
        zz_new = dotc(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
    x, info = _finish(matvec, b, x, status, k, nmv, hist)
    if info["status"] == OK and info["rel_res_true"] >= tol:
        info["status"] = NOT_CONVERGED
    return x, info


SOLVERS = {"qmr_cs": qmr_cs, "bicg_cs": bicg_cs, "bicgstab": bicgstab, "cgnr": cgnr}
