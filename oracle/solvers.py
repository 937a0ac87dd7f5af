"""O9: the four Krylov solvers of Sec. 2 (CGNR, Bi-CGSTAB, Bi-CG, QMR).

Sec. 2 names the solvers and notes that Bi-CG and QMR exploit the complex
symmetry A = A^T of Eq. (2) (they use the bilinear form u^T v, no
conjugation); the stopping rule is the relative residual norm
||b - A x||_2 / ||b||_2 < eps with eps = 1e-5 by default (Sec. 2, Sec. 3.1).
The algorithms are restated from the standard literature as mathematics:

* QMR-CS: Lanczos with the bilinear form, Givens rotations on the tridiagonal
  matrix, residual kept by r_k = r_{k-1} - tau_k A p_k (no extra product);
* Bi-CG-CS (COCG): conjugate gradients with u^T v in place of u^H v;
* Bi-CGSTAB: van der Vorst's method with Hermitian products, shadow r0;
* CGNR: CG on A^H A x = A^H b, with A^H y = conj(A conj(y)).

Every solver starts from x0 = 0 and returns (x, info) where info holds the
status ("ok", "not_converged", "breakdown"), iteration and product counts, the
recurrence residual history (relative) and the true relative residual at exit.
"""
import numpy as np

OK, NOT_CONVERGED, BREAKDOWN = "ok", "not_converged", "breakdown"


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
    """QMR for complex-symmetric A (Lanczos with the bilinear form)."""
    bn = norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    beta_k = 0.0 + 0.0j                  # beta_1 multiplies v_0 = 0
    beta_next = np.sqrt(complex(dotu(b, b)))
    v_prev = np.zeros_like(b)
    v = b / beta_next
    p1 = np.zeros_like(b); p2 = np.zeros_like(b)
    ap1 = np.zeros_like(b); ap2 = np.zeros_like(b)
    c1, s1 = 1.0, 0.0j                   # G_{k-1}
    c2, s2 = 1.0, 0.0j                   # G_{k-2}
    t = beta_next
    hist = [1.0]
    nmv = 0
    status = NOT_CONVERGED
    k = 0
    for k in range(1, maxiter + 1):
        w = matvec(v); nmv += 1
        alpha = dotu(v, w)
        vt = w - alpha * v - beta_k * v_prev
        vtv = dotu(vt, vt)
        beta_next = np.sqrt(complex(vtv))
        # previous rotations applied to column (beta_k, alpha_k, beta_{k+1})
        eps = s2 * beta_k
        tmp = c2 * beta_k
        delta = c1 * tmp + s1 * alpha
        gt = -np.conj(s1) * tmp + c1 * alpha
        if gt == 0:
            c, s = 0.0, 1.0 + 0.0j
        else:
            c = abs(gt) / np.sqrt(abs(gt) ** 2 + abs(beta_next) ** 2)
            s = c * np.conj(beta_next / gt)
        gamma = c * gt + s * beta_next
        if gamma == 0:
            status = BREAKDOWN
            hist.append(hist[-1])
            break
        tau = c * t
        t = -np.conj(s) * t
        p = (v - delta * p1 - eps * p2) / gamma
        ap = (w - delta * ap1 - eps * ap2) / gamma
        x = x + tau * p
        r = r - tau * ap
        p2, p1 = p1, p
        ap2, ap1 = ap1, ap
        c2, s2, c1, s1 = c1, s1, c, s
        res = norm2(r) / bn
        hist.append(res)
        if res < tol:
            status = OK
            break
        if abs(vtv) < 1e-30 * norm2(vt) ** 2:
            status = BREAKDOWN
            break
        v_prev, v = v, vt / beta_next
        beta_k = beta_next
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
        if mu == 0 or rho == 0:
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
