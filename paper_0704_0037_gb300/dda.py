"""Thin ctypes binding of the C-ABI in include/dda.h (argument marshalling only).

Every function here has the name and meaning of the C entry point it wraps;
all arithmetic runs in libdda.so (hand-written sm_103a CUDA).  Device buffers
are torch CUDA tensors (complex128 or complex64, contiguous, [nrhs][3][N_occ]);
host arrays are numpy arrays.  Negative statuses raise DDAError carrying
dda_last_error(); the non-fatal solver outcomes (DDA_NOT_CONVERGED,
DDA_BREAKDOWN) are returned.

There is no CPU fallback: if libdda.so is missing or cannot be loaded this
module raises on first use.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdda.so")

DDA_OK, DDA_NOT_CONVERGED, DDA_BREAKDOWN = 0, 1, 2
DDA_ERR_ARG, DDA_ERR_CUDA, DDA_ERR_OOM, DDA_ERR_STATE, DDA_ERR_NONFINITE, DDA_ERR_TIMEOUT = \
    -1, -2, -3, -4, -5, -6
DDA_CM, DDA_RR, DDA_LDR, DDA_CLDR = 0, 1, 2, 3
DDA_QMR_CS, DDA_BICG_CS, DDA_BICGSTAB, DDA_CGNR = 0, 1, 2, 3
DDA_FP64, DDA_FP32_REFINED, DDA_FP64_PAIR = 0, 1, 2
DDA_ENGINE_AUTO, DDA_ENGINE_STOCKHAM = 0, 1

STATUS_NAMES = {0: "ok", 1: "not_converged", 2: "breakdown", -1: "err_arg", -2: "err_cuda",
                -3: "err_oom", -4: "err_state", -5: "err_nonfinite", -6: "err_timeout"}
POL = {"cm": DDA_CM, "rr": DDA_RR, "ldr": DDA_LDR, "cldr": DDA_CLDR}
SOLVER = {"qmr_cs": DDA_QMR_CS, "bicg_cs": DDA_BICG_CS, "bicgstab": DDA_BICGSTAB, "cgnr": DDA_CGNR}
PREC = {"fp64": DDA_FP64, "fp32_refined": DDA_FP32_REFINED}

# every entry point declared in include/dda.h
EXPORTS = ("dda_init_lattice", "dda_build_Dmatrix", "dda_set_beta", "dda_matvec",
           "dda_matvec_adjoint", "dda_solve", "dda_solve_batch", "dda_solve_many", "dda_scatter", "dda_mueller_plane",
           "dda_mueller_plane_full", "dda_asymmetry", "dda_symmetry", "dda_mueller_plane_sym",
           "dda_orientation_average",
           "dda_farfield_noalloc", "dda_trace",
           "dda_trace_read", "dda_n_occ", "dda_kd", "dda_grid", "dda_positions", "dda_last_error",
           "dda_free", "dda_release_cached_memory", "dda_set_fft_engine", "dda_set_pass_tiles",
           "dda_get_pass_tiles", "dda_set_memory_limit",
           "dda_memory_in_use", "dda_residual", "dda_checkpoint_bytes", "dda_pcnet_create",
           "dda_pcnet_free", "dda_pcnet_params", "dda_pcnet_last_error", "dda_pcnet_get_weights",
           "dda_pcnet_set_weights", "dda_pcnet_get_grads", "dda_pcnet_apply", "dda_pcnet_train_step",
           "dda_solve_pc", "dda_pcnet_pair")


class DDAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("pol", ctypes.c_int), ("prec", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("checkpoint_every", ctypes.c_int), ("inner_cap", ctypes.c_int),
                ("checkpoint_host", ctypes.c_void_p), ("checkpoint_bytes", ctypes.c_longlong),
                ("checkpoint_stop", ctypes.c_int), ("resume", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("matvecs_fp64", ctypes.c_int), ("outer", ctypes.c_int),
                ("rel_res_true", ctypes.c_double), ("rel_res_recur", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.c_int


def lib():
    """Load libdda.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_0704_0037_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "dda_init_lattice": ([ctypes.POINTER(_vp), _ip, _ip, _ip, ctypes.POINTER(ctypes.c_uint8), _ip,
                              _dp, ctypes.c_double, _ip, _vp], _ip),
        "dda_build_Dmatrix": ([_vp, _ip], _ip),
        "dda_set_fft_engine": ([_vp, _ip], _ip),
        "dda_set_pass_tiles": ([_vp, _ip, ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_get_pass_tiles": ([_vp, _ip, ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_set_memory_limit": ([ctypes.c_ulonglong], _ip),
        "dda_memory_in_use": ([ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)], _ip),
        "dda_set_beta": ([_vp, _ip, _ip, _dp, _dp], _ip),
        "dda_matvec": ([_vp, _ip, _vp, _vp, _ip], _ip),
        "dda_matvec_adjoint": ([_vp, _ip, _vp, _vp, _ip], _ip),
        "dda_solve": ([_vp, ctypes.POINTER(SolveOpts), _ip, _dp, _dp, _vp, _dp, _ip,
                       ctypes.POINTER(SolveInfo)], _ip),
        "dda_solve_batch": ([_vp, ctypes.POINTER(SolveOpts), _ip, _dp, _dp, _vp,
                             ctypes.POINTER(SolveInfo)], _ip),
        "dda_solve_many": ([_ip, ctypes.POINTER(_vp), ctypes.POINTER(SolveOpts), ctypes.POINTER(_ip),
                            ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.POINTER(_vp),
                            ctypes.POINTER(ctypes.POINTER(SolveInfo)), _ip, ctypes.POINTER(_ip)], _ip),
        "dda_scatter": ([_vp, _ip, _vp, _ip, _dp, _dp, _ip, _dp, _dp, _dp, _dp], _ip),
        "dda_residual": ([_vp, _ip, _ip, _dp, _dp, _vp, _dp], _ip),
        "dda_checkpoint_bytes": ([_vp, _ip, _ip, ctypes.POINTER(ctypes.c_longlong)], _ip),
        "dda_pcnet_create": ([ctypes.POINTER(_vp), ctypes.c_ulonglong], _ip),
        "dda_pcnet_free": ([_vp], _ip),
        "dda_pcnet_params": ([_vp, ctypes.POINTER(ctypes.c_longlong)], _ip),
        "dda_pcnet_last_error": ([_vp], ctypes.c_char_p),
        "dda_pcnet_get_weights": ([_vp, ctypes.POINTER(ctypes.c_float)], _ip),
        "dda_pcnet_set_weights": ([_vp, ctypes.POINTER(ctypes.c_float)], _ip),
        "dda_pcnet_get_grads": ([_vp, ctypes.POINTER(ctypes.c_float)], _ip),
        "dda_pcnet_apply": ([_vp, _vp, _vp, _vp], _ip),
        "dda_pcnet_train_step": ([_vp, _vp, _vp, _vp, _vp, ctypes.c_float, _dp], _ip),
        "dda_solve_pc": ([_vp, _vp, ctypes.POINTER(SolveOpts), _dp, _dp, _vp, _dp, _ip,
                          ctypes.POINTER(SolveInfo)], _ip),
        "dda_pcnet_pair": ([_vp, _ip, _dp, _dp, _vp, _vp, _vp, _vp], _ip),
        "dda_mueller_plane": ([_ip, _dp, _dp, _dp, _dp], _ip),
        "dda_mueller_plane_full": ([_ip, _dp, _dp, _dp, _dp], _ip),
        "dda_asymmetry": ([_ip, _dp, _dp, _dp, _dp, _dp], _ip),
        "dda_symmetry": ([_vp, ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_mueller_plane_sym": ([_vp, _ip, _vp, _ip, _dp, _dp, _dp], _ip),
        "dda_orientation_average": ([_vp, ctypes.POINTER(SolveOpts), _ip, _ip, _ip, _ip, _dp, _dp,
                                     _dp, ctypes.POINTER(SolveInfo)], _ip),
        "dda_farfield_noalloc": ([_vp, _vp, _ip, _vp, _vp], _ip),
        "dda_trace": ([_vp, _ip], _ip),
        "dda_release_cached_memory": ([], _ip),
        "dda_trace_read": ([_vp, _ip, ctypes.c_char_p, _dp, ctypes.POINTER(ctypes.c_longlong),
                            ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_n_occ": ([_vp, ctypes.POINTER(ctypes.c_longlong)], _ip),
        "dda_kd": ([_vp, _dp], _ip),
        "dda_grid": ([_vp, ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_positions": ([_vp, ctypes.POINTER(ctypes.c_int)], _ip),
        "dda_last_error": ([_vp], ctypes.c_char_p),
        "dda_free": ([_vp], _ip),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _dptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _check(h, rc):
    if rc < 0:
        msg = lib().dda_last_error(h).decode() if h else ""
        raise DDAError(rc, msg)
    return rc


def _stream_ptr(stream):
    """cudaStream_t of a torch stream (or of torch's current one), or a raw handle."""
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return _vp(stream.cuda_stream)
    return _vp(int(stream))


def _dev_ptr(t, dtype=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("device buffers must be contiguous CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return _vp(t.data_ptr())


def _vecs(prop, pol, nrhs):
    a = np.ascontiguousarray(np.asarray(prop, dtype=np.float64).reshape(nrhs, 3))
    e = np.asarray(pol, dtype=np.complex128).reshape(nrhs, 3)
    e2 = np.ascontiguousarray(np.stack([e.real, e.imag], axis=-1).reshape(nrhs, 6))
    return a, e2


# ---------------------------------------------------------------- entry points

def dda_init_lattice(occ, m_list, kd, volume_corrected=False, stream=None):
    """occ: uint8 (nz, ny, nx) material indices; m_list: refractive indices.
    Returns the handle (ctypes void pointer)."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    nz, ny, nx = occ.shape
    m = np.asarray(m_list, dtype=np.complex128).reshape(-1)
    m2 = np.ascontiguousarray(np.stack([m.real, m.imag], axis=-1).reshape(-1))
    h = _vp()
    rc = lib().dda_init_lattice(ctypes.byref(h), nx, ny, nz,
                                occ.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), m.size,
                                _dptr(m2), float(kd), int(bool(volume_corrected)),
                                _stream_ptr(stream))
    if rc < 0:
        raise DDAError(rc, "dda_init_lattice failed")
    return h


def dda_set_fft_engine(h, engine):
    return _check(h, lib().dda_set_fft_engine(h, int(engine)))


def dda_set_pass_tiles(h, prec, tiles=None):
    """Tile variants (y forward, z, y inverse) of one arithmetic's products:
    0 default, 1 half the lines per block, -1 autotuned (None: all -1)."""
    arr = None if tiles is None else (ctypes.c_int * 3)(*[int(t) for t in tiles])
    return _check(h, lib().dda_set_pass_tiles(h, int(prec), arr))


def dda_get_pass_tiles(h, prec):
    arr = (ctypes.c_int * 3)()
    _check(h, lib().dda_get_pass_tiles(h, int(prec), arr))
    return tuple(arr)


def dda_set_memory_limit(nbytes):
    """Cap on the device bytes held by the library's live handles (0: none)."""
    return lib().dda_set_memory_limit(int(nbytes))


def dda_memory_in_use():
    """(bytes held by live handles, bytes in the cache of freed blocks)."""
    a, b = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    rc = lib().dda_memory_in_use(ctypes.byref(a), ctypes.byref(b))
    if rc < 0:
        raise DDAError(rc, "dda_memory_in_use")
    return a.value, b.value


def dda_build_Dmatrix(h, prec=DDA_FP64):
    return _check(h, lib().dda_build_Dmatrix(h, int(prec)))


def dda_set_beta(h, pol_prescription, prop, pol):
    nrhs = int(np.asarray(prop).size // 3)
    a, e = _vecs(prop, pol, nrhs)
    return _check(h, lib().dda_set_beta(h, int(pol_prescription), nrhs, _dptr(a), _dptr(e)))


def dda_matvec(h, prec, x, y, nrhs=1):
    import torch
    dt = torch.complex64 if prec == DDA_FP32_REFINED else torch.complex128
    return _check(h, lib().dda_matvec(h, int(prec), _dev_ptr(x, dt), _dev_ptr(y, dt), int(nrhs)))


def dda_matvec_adjoint(h, prec, x, y, nrhs=1):
    import torch
    dt = torch.complex128 if prec == DDA_FP64 else torch.complex64
    return _check(h, lib().dda_matvec_adjoint(h, int(prec), _dev_ptr(x, dt), _dev_ptr(y, dt),
                                              int(nrhs)))


def _opts(opts):
    if isinstance(opts, dict):
        o = SolveOpts(solver=opts.get("solver", DDA_QMR_CS), pol=opts.get("pol", DDA_LDR),
                         prec=opts.get("prec", DDA_FP64), tol=opts.get("tol", 1e-5),
                         maxiter=opts.get("maxiter", 10000), inner_tol=opts.get("inner_tol", 1e-3),
                         checkpoint_every=opts.get("checkpoint_every", 0),
                         inner_cap=opts.get("inner_cap", 0))
        buf = opts.get("checkpoint")
        if buf is not None:
            # a writable numpy uint8 array owned by the caller
            o.checkpoint_host = buf.ctypes.data_as(ctypes.c_void_p)
            o.checkpoint_bytes = int(buf.nbytes)
        o.checkpoint_stop = int(bool(opts.get("checkpoint_stop", False)))
        o.resume = int(bool(opts.get("resume", False)))
        return o
    return opts


def dda_solve(h, opts, prop, pol, P, hist_len=0):
    """opts: SolveOpts or dict.  Returns (status, [info dicts], hist or None)."""
    import torch
    o = _opts(opts)
    nrhs = int(np.asarray(prop).size // 3)
    a, e = _vecs(prop, pol, nrhs)
    info = (SolveInfo * nrhs)()
    hist = np.full((nrhs, hist_len), -1.0) if hist_len > 0 else None
    rc = lib().dda_solve(h, ctypes.byref(o), nrhs, _dptr(a), _dptr(e),
                         _dev_ptr(P, torch.complex128), _dptr(hist), int(hist_len), info)
    _check(h, rc)
    return rc, [i.as_dict() for i in info], hist


def dda_solve_batch(h, opts, prop, pol, P):
    """All right-hand sides at once (QMR-CS).  Returns (status, [info dicts])."""
    import torch
    o = _opts(opts)
    nrhs = int(np.asarray(prop).size // 3)
    a, e = _vecs(prop, pol, nrhs)
    info = (SolveInfo * nrhs)()
    rc = lib().dda_solve_batch(h, ctypes.byref(o), nrhs, _dptr(a), _dptr(e),
                               _dev_ptr(P, torch.complex128), info)
    _check(h, rc)
    return rc, [i.as_dict() for i in info]


def dda_solve_many(handles, opts, props, pols, Ps, n_threads=8):
    """Particles in parallel host threads (each handle on its own stream).
    Returns (worst status, [status per particle], [[info dicts] per particle])."""
    import torch
    o = _opts(opts)
    n = len(handles)
    hs = (_vp * n)(*handles)
    nr = (_ip * n)()
    keep = []
    pa = (_dp * n)()
    pe = (_dp * n)()
    pp = (_vp * n)()
    infos = []
    ip = (ctypes.POINTER(SolveInfo) * n)()
    for i in range(n):
        k = int(np.asarray(props[i]).size // 3)
        a, e = _vecs(props[i], pols[i], k)
        keep += [a, e]
        nr[i] = k
        pa[i] = _dptr(a)
        pe[i] = _dptr(e)
        pp[i] = _dev_ptr(Ps[i], torch.complex128)
        inf = (SolveInfo * k)()
        infos.append(inf)
        ip[i] = ctypes.cast(inf, ctypes.POINTER(SolveInfo))
    st = (_ip * n)()
    rc = lib().dda_solve_many(n, hs, ctypes.byref(o), nr, pa, pe, pp, ip, int(n_threads), st)
    if rc < 0 and all(s == 0 for s in st):
        raise DDAError(rc, "dda_solve_many arguments")
    return rc, list(st), [[x.as_dict() for x in inf] for inf in infos]


def dda_checkpoint_bytes(h, prec, nrhs):
    """Size of the host buffer for checkpoints of a QMR-CS solve."""
    v = ctypes.c_longlong()
    _check(h, lib().dda_checkpoint_bytes(h, int(prec), int(nrhs), ctypes.byref(v)))
    return v.value


def dda_residual(h, pol_prescription, P, prop, pol):
    """||b - A x|| / ||b|| per right-hand side (x = P / beta), native FP64 product."""
    import torch
    nrhs = int(np.asarray(prop).size // 3)
    a, e = _vecs(prop, pol, nrhs)
    res = np.zeros(nrhs)
    _check(h, lib().dda_residual(h, int(pol_prescription), nrhs, _dptr(a), _dptr(e),
                                 _dev_ptr(P, torch.complex128), _dptr(res)))
    return res


def dda_scatter(h, pol_prescription, P, prop, pol, dirs=None, weights=None):
    """Returns (F (nrhs, n_dir, 3) complex, q (nrhs, 3) = Q_ext, Q_abs, Q_sca)."""
    import torch
    nrhs = int(np.asarray(prop).size // 3)
    a, e = _vecs(prop, pol, nrhs)
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3)) if dirs is not None \
        else np.zeros((0, 3))
    n_dir = d.shape[0]
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64)) if weights is not None else None
    F = np.zeros((nrhs, max(n_dir, 1), 6))
    q = np.zeros((nrhs, 3))
    rc = lib().dda_scatter(h, int(pol_prescription), _dev_ptr(P, torch.complex128), nrhs, _dptr(a),
                           _dptr(e), n_dir, _dptr(d) if n_dir else None, _dptr(w), _dptr(F),
                           _dptr(q))
    _check(h, rc)
    Fc = (F[..., 0::2] + 1j * F[..., 1::2])[:, :n_dir, :]
    return Fc, q


def _cplx_pairs(F):
    f = np.asarray(F, dtype=np.complex128).reshape(-1, 3)
    return np.ascontiguousarray(np.stack([f.real, f.imag], axis=-1).reshape(-1))


def dda_mueller_plane_full(theta_deg, F_xpol, F_ypol):
    """(n_theta, 4, 4) Mueller matrices in the xz plane."""
    th = np.ascontiguousarray(np.asarray(theta_deg, dtype=np.float64))
    out = np.zeros(th.size * 16)
    rc = lib().dda_mueller_plane_full(th.size, _dptr(th), _dptr(_cplx_pairs(F_xpol)),
                                      _dptr(_cplx_pairs(F_ypol)), _dptr(out))
    if rc < 0:
        raise DDAError(rc, "dda_mueller_plane_full")
    return out.reshape(-1, 4, 4)


def dda_asymmetry(dirs, weights, F, prop):
    """(<cos theta>, g_vec) from amplitudes at quadrature directions."""
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(prop, dtype=np.float64).reshape(3))
    g = np.zeros(4)
    rc = lib().dda_asymmetry(d.shape[0], _dptr(d), _dptr(w), _dptr(_cplx_pairs(F)), _dptr(a),
                             _dptr(g))
    if rc < 0:
        raise DDAError(rc, "dda_asymmetry")
    return float(g[0]), g[1:].copy()


DDA_SYM_ROT90_Z = 1


def dda_symmetry(h):
    f = ctypes.c_int(0)
    _check(h, lib().dda_symmetry(h, ctypes.byref(f)))
    return f.value


def dda_mueller_plane_sym(h, pol_prescription, P, theta_deg):
    """Mueller matrices (n, 4, 4) in the xz plane from the x-polarised
    solution alone (lattice invariant under the 90 degree rotation about z);
    also returns (F_x, F_y), each (n, 3) complex."""
    import torch
    th = np.ascontiguousarray(np.asarray(theta_deg, dtype=np.float64))
    M = np.zeros(th.size * 16)
    F = np.zeros(th.size * 12)
    _check(h, lib().dda_mueller_plane_sym(h, int(pol_prescription), _dev_ptr(P, torch.complex128),
                                          th.size, _dptr(th), _dptr(M), _dptr(F)))
    Fc = F[0::2] + 1j * F[1::2]
    Fc = Fc.reshape(-1, 2, 3)
    return M.reshape(-1, 4, 4), Fc[:, 0], Fc[:, 1]


def dda_orientation_average(h, opts, n_alpha, n_beta, n_gamma, theta_deg):
    """Returns (status, (<Q_ext>, <Q_abs>), M (n, 4, 4), [info dicts])."""
    o = _opts(opts)
    th = np.ascontiguousarray(np.asarray(theta_deg, dtype=np.float64))
    q = np.zeros(2)
    M = np.zeros(th.size * 16)
    infos = (SolveInfo * (2 * n_beta * n_gamma))()
    rc = _check(h, lib().dda_orientation_average(h, ctypes.byref(o), int(n_alpha), int(n_beta),
                                                 int(n_gamma), th.size, _dptr(th), _dptr(q),
                                                 _dptr(M), infos))
    return rc, (float(q[0]), float(q[1])), M.reshape(-1, 4, 4), [i.as_dict() for i in infos]


def dda_mueller_plane(theta_deg, F_xpol, F_ypol):
    th = np.ascontiguousarray(np.asarray(theta_deg, dtype=np.float64))
    fx = np.asarray(F_xpol, dtype=np.complex128).reshape(-1, 3)
    fy = np.asarray(F_ypol, dtype=np.complex128).reshape(-1, 3)
    fx2 = np.ascontiguousarray(np.stack([fx.real, fx.imag], axis=-1).reshape(-1))
    fy2 = np.ascontiguousarray(np.stack([fy.real, fy.imag], axis=-1).reshape(-1))
    out = np.zeros(th.size)
    rc = lib().dda_mueller_plane(th.size, _dptr(th), _dptr(fx2), _dptr(fy2), _dptr(out))
    if rc < 0:
        raise DDAError(rc, "dda_mueller_plane")
    return out


def dda_farfield_noalloc(h, P, dirs, F):
    """F(n) for one polarization vector without any device allocation by the
    library.  P: CUDA complex128 [3][N_occ] (or [1][3][N_occ]); dirs: CUDA
    float64 [n_dir][3]; F: CUDA complex128 [n_dir][3] (written)."""
    import torch
    n_dir = int(dirs.shape[0])
    return _check(h, lib().dda_farfield_noalloc(h, _dev_ptr(P, torch.complex128), n_dir,
                                                _dev_ptr(dirs, torch.float64),
                                                _dev_ptr(F, torch.complex128)))


def dda_release_cached_memory():
    """Return the device memory the library keeps for reuse to the driver."""
    return lib().dda_release_cached_memory()


def dda_trace(h, enable=True):
    return _check(h, lib().dda_trace(h, int(bool(enable))))


def dda_trace_read(h, max_n=32):
    """Returns {kernel name: (total ms, launches)}."""
    names = ctypes.create_string_buffer(32 * max_n)
    ms = np.zeros(max_n)
    cnt = np.zeros(max_n, dtype=np.int64)
    n = ctypes.c_int()
    _check(h, lib().dda_trace_read(h, max_n, names, _dptr(ms),
                                   cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                   ctypes.byref(n)))
    out = {}
    for k in range(min(n.value, max_n)):
        nm = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[k]), int(cnt[k]))
    return out


def dda_n_occ(h):
    n = ctypes.c_longlong()
    _check(h, lib().dda_n_occ(h, ctypes.byref(n)))
    return n.value


def dda_kd(h):
    v = ctypes.c_double()
    _check(h, lib().dda_kd(h, ctypes.byref(v)))
    return v.value


def dda_grid(h):
    g = (ctypes.c_int * 3)()
    _check(h, lib().dda_grid(h, g))
    return tuple(g)


def dda_positions(h):
    n = dda_n_occ(h)
    ijk = np.zeros((n, 3), dtype=np.int32)
    _check(h, lib().dda_positions(h, ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return ijk


def dda_last_error(h):
    return lib().dda_last_error(h).decode()


def dda_free(h):
    return lib().dda_free(h)


# ---------------------------------------------------------------- learned preconditioner
# (layer, cin, cout, kernel) of the network, in the order of its parameters
PCNET_LAYERS = ((7, 16, 3), (16, 32, 3), (32, 160, 3), (160, 160, 3), (192, 32, 3), (48, 16, 3),
                (16, 6, 1))


class PcNet:
    """The learned right preconditioner (dda_pcnet_*): owns one network."""

    def __init__(self, seed=0):
        self.p = _vp()
        rc = lib().dda_pcnet_create(ctypes.byref(self.p), ctypes.c_ulonglong(seed))
        if rc < 0:
            raise DDAError(rc, "dda_pcnet_create failed")
        n = ctypes.c_longlong()
        lib().dda_pcnet_params(self.p, ctypes.byref(n))
        self.nparam = n.value

    def _check(self, rc):
        if rc < 0:
            raise DDAError(rc, lib().dda_pcnet_last_error(self.p).decode())
        return rc

    def weights(self):
        w = np.zeros(self.nparam, dtype=np.float32)
        self._check(lib().dda_pcnet_get_weights(self.p, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        if w.size != self.nparam:
            raise ValueError("wrong parameter count")
        self._check(lib().dda_pcnet_set_weights(self.p, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def grads(self):
        g = np.zeros(self.nparam, dtype=np.float32)
        self._check(lib().dda_pcnet_get_grads(self.p, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return g

    def apply(self, h, v, z):
        """z = N(v): CUDA complex128 [3][N_occ] tensors on the handle's lattice."""
        import torch
        return self._check(lib().dda_pcnet_apply(self.p, h, _dev_ptr(v, torch.complex128),
                                                 _dev_ptr(z, torch.complex128)))

    def train_step(self, h, r, e, z, lr):
        """One Adam step on (r, e); z receives N(r); returns the loss."""
        import torch
        loss = ctypes.c_double()
        self._check(lib().dda_pcnet_train_step(self.p, h, _dev_ptr(r, torch.complex128),
                                               _dev_ptr(e, torch.complex128),
                                               _dev_ptr(z, torch.complex128), ctypes.c_float(lr),
                                               ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.p is not None and self.p.value:
            lib().dda_pcnet_free(self.p)
        self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dda_pcnet_pair(h, pol_prescription, prop, pol, P_star, P_k, r, e):
    """Training pair: e = (P* - P_k) / beta, r = A e (device complex128 [3][N_occ])."""
    import torch
    a, ev = _vecs(prop, pol, 1)
    return _check(h, lib().dda_pcnet_pair(h, int(pol_prescription), _dptr(a), _dptr(ev),
                                          _dev_ptr(P_star, torch.complex128),
                                          _dev_ptr(P_k, torch.complex128),
                                          _dev_ptr(r, torch.complex128), _dev_ptr(e, torch.complex128)))


def dda_solve_pc(h, net, opts, prop, pol, P, hist_len=0):
    """Flexible Bi-CGSTAB with the network as right preconditioner (net None:
    plain Bi-CGSTAB).  Returns (status, info dict, hist or None)."""
    import torch
    o = _opts(opts)
    a, e = _vecs(prop, pol, 1)
    info = (SolveInfo * 1)()
    hist = np.full(hist_len, -1.0) if hist_len > 0 else None
    rc = lib().dda_solve_pc(h, net.p if net is not None else None, ctypes.byref(o), _dptr(a), _dptr(e),
                            _dev_ptr(P, torch.complex128), _dptr(hist), int(hist_len), info)
    _check(h, rc)
    return rc, info[0].as_dict(), hist


class Particle:
    """Owns one handle; frees it on close / garbage collection."""

    def __init__(self, occ, m_list, kd, volume_corrected=False, stream=None, engine=None):
        self.h = dda_init_lattice(occ, m_list, kd, volume_corrected, stream)
        if engine is not None:
            dda_set_fft_engine(self.h, engine)
            self.grid = dda_grid(self.h)
        self.n_occ = dda_n_occ(self.h)
        self.kd = dda_kd(self.h)
        self.grid = dda_grid(self.h)

    def close(self):
        if self.h is not None:
            dda_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
