"""Python binding of libvie (include/vie.h): the FFT-accelerated PWL current-based VIE on GB300.

Argument marshalling only: every function here forwards to the C ABI entry point
of the same name; all arithmetic runs in the library's CUDA kernels.  Arrays may
be torch tensors (CUDA or CPU) or NumPy arrays (host); complex arrays use
complex128 (FP64 entry points) or complex64 (FP32 matvec) with the layout
[nrhs][12][nz][ny][nx].  The library is built in place by `build()`; importing
works without it, but every call raises if libvie.so is missing - there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvie.so")

VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_EDEVICE, VIE_ETIMEOUT, VIE_NOT_CONVERGED = 0, -1, -2, -3, -4, 1
VIE_FP64, VIE_FP32, VIE_BF16X3 = 0, 1, 2
VIE_OP_A, VIE_OP_PA, VIE_OP_NSCAT, VIE_OP_K = 0, 1, 2, 3
VIE_SOLVE_FP64, VIE_SOLVE_FP32_REFINE, VIE_SOLVE_BF16X3_REFINE = 0, 1, 2
VIE_INJECT_NONE, VIE_INJECT_OOM = 0, 1
VIE_SETUP_PWC = 1
VIE_TUCKER_APPLY = 1

EXPORTS = (
    "vie_setup", "vie_setup_green_external", "vie_destroy", "vie_matvec", "vie_rhs_planewave", "vie_rhs_dipoles", "vie_solve",
    "vie_fields", "vie_green_toeplitz", "vie_green_toeplitz_k", "vie_rhs_dipoles_h", "vie_hfields", "vie_info", "vie_strerror", "vie_last_error",
    "vie_stats_reset", "vie_stats_read", "vie_matvec_noalloc", "vie_fault_inject", "vie_tuning",
    "vie_set_permeability", "vie_jm_matvec", "vie_jm_rhs", "vie_jm_solve", "vie_jm_fields", "vie_green_tucker",
    "vie_server_create", "vie_server_destroy", "vie_submit", "vie_poll", "vie_server_stats",
)


class vie_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class vie_solve_info(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int), ("fp64_matvecs", ctypes.c_int),
                ("fp32_matvecs", ctypes.c_int), ("refinements", ctypes.c_int), ("resid", ctypes.c_double),
                ("true_resid", ctypes.c_double), ("err_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vie_request(ctypes.Structure):
    _fields_ = [("grid", vie_grid), ("freq_hz", ctypes.c_double), ("eps_real", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("dip_pos", ctypes.c_void_p),
                ("dip_mom", ctypes.c_void_p), ("tol", ctypes.c_double), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("mode", ctypes.c_int), ("x_out", ctypes.c_void_p),
                ("p_abs_out", ctypes.c_void_p), ("P_abs_out", ctypes.c_void_p)]


class vie_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nrhs", ctypes.c_int), ("iterations", ctypes.c_int),
                ("green_cached", ctypes.c_int), ("queued_s", ctypes.c_double), ("run_s", ctypes.c_double),
                ("resid", ctypes.c_double), ("start_s", ctypes.c_double), ("end_s", ctypes.c_double),
                ("dev_start_s", ctypes.c_double), ("dev_end_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VieError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        lib = _lib()
        detail = lib.vie_last_error().decode()
        super().__init__(f"{where}: {lib.vie_strerror(code).decode()} ({code}) {detail}")


_LIB = None


def build(verbose=False):
    """Compile libvie.so for sm_103a in place (nvcc) and return its path."""
    from . import _builder as _b

    return _b.build(verbose=verbose)


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; call paper_1902_02196_gb300.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.vie_setup.argtypes = [ctypes.POINTER(vie_grid), D, P, P, I, ctypes.POINTER(P)]
    lib.vie_setup_green_external.argtypes = [ctypes.POINTER(vie_grid), D, P, P, P, ctypes.POINTER(P)]
    lib.vie_destroy.argtypes = [P]
    lib.vie_destroy.restype = None
    lib.vie_matvec.argtypes = [P, I, P, P, I, I, P]
    lib.vie_matvec_noalloc.argtypes = [P, I, P, P, I, I, P]
    lib.vie_rhs_planewave.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D), P, P, P]
    lib.vie_rhs_dipoles.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D), P, P, P]
    lib.vie_solve.argtypes = [P, I, P, P, D, I, I, I, I, ctypes.POINTER(vie_solve_info), P]
    lib.vie_fields.argtypes = [P, I, P, P, P, P, ctypes.POINTER(D), P]
    lib.vie_green_toeplitz.argtypes = [P, P]
    lib.vie_green_toeplitz_k.argtypes = [P, P]
    lib.vie_rhs_dipoles_h.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D), P, P]
    lib.vie_hfields.argtypes = [P, I, P, P, P, P, ctypes.POINTER(D), P]
    lib.vie_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(S)]
    lib.vie_set_permeability.argtypes = [P, P, P]
    lib.vie_green_tucker.argtypes = [P, D, I, P, P, ctypes.POINTER(S)]
    lib.vie_jm_matvec.argtypes = [P, I, P, P, I, I, P]
    lib.vie_jm_rhs.argtypes = [P, I, P, P, P, P]
    lib.vie_jm_solve.argtypes = [P, I, P, P, D, I, I, I, I, ctypes.POINTER(vie_solve_info), P]
    lib.vie_jm_fields.argtypes = [P, I, P, P, P, P, P, P, ctypes.POINTER(D), P]
    lib.vie_strerror.argtypes = [I]
    lib.vie_strerror.restype = ctypes.c_char_p
    lib.vie_stats_reset.argtypes = [I]
    lib.vie_stats_read.argtypes = [I, P, P, P, P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)]
    lib.vie_fault_inject.argtypes = [I, I]
    lib.vie_tuning.argtypes = [P, S]
    lib.vie_last_error.argtypes = []
    lib.vie_last_error.restype = ctypes.c_char_p
    lib.vie_server_create.argtypes = [S, I, ctypes.POINTER(P)]
    lib.vie_server_destroy.argtypes = [P]
    lib.vie_server_destroy.restype = None
    lib.vie_submit.argtypes = [P, ctypes.POINTER(vie_request), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.vie_poll.argtypes = [P, ctypes.c_ulonglong, I, ctypes.POINTER(vie_result)]
    lib.vie_server_stats.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(S), ctypes.POINTER(I)]
    _LIB = lib
    return lib


def _ptr(a):
    """Raw data pointer of a torch tensor or NumPy array (must be contiguous); None -> NULL."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _stream(s):
    """cudaStream_t of a torch stream (its legacy default stream maps to cudaStreamLegacy), or None."""
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or 1
    return int(s)


def _nrhs(a, h):
    """Right-hand sides in a vector batch of handle h (h.nc components per voxel: 12 PWL, 3 PWC)."""
    n = 1
    for d in a.shape:
        n *= int(d)
    if n % (h.nc * h.nv):
        raise ValueError(f"array size is not a multiple of {h.nc} * N_V")
    return n // (h.nc * h.nv)


def _check(rc, where):
    if rc < 0:
        raise VieError(rc, where)
    return rc


class Handle:
    """Owns a vie_handle (one grid, frequency and material map)."""

    def __init__(self, ptr, grid, freq, nc=12):
        self.ptr = ptr
        self.grid = grid
        self.freq = freq
        self.nv = grid[0] * grid[1] * grid[2]
        self.nc = nc  # unknowns per voxel: 12 (PWL) or 3 (PWC)

    def close(self):
        if self.ptr:
            vie_destroy(self)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vie_setup(grid, freq_hz, eps_real, sigma, flags=0):
    """grid = (nx, ny, nz, dx, dy, dz); eps_real, sigma: float64 (nz, ny, nx) maps (host or device).
    flags = VIE_SETUP_PWC: the piecewise-constant system, vectors [nrhs][3][nz][ny][nx]."""
    lib = _lib()
    g = vie_grid(*[int(v) for v in grid[:3]], *[float(v) for v in grid[3:]])
    out = ctypes.c_void_p()
    _check(lib.vie_setup(ctypes.byref(g), float(freq_hz), _ptr(eps_real), _ptr(sigma), int(flags), ctypes.byref(out)),
           "vie_setup")
    return Handle(out.value, (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), freq_hz, 3 if flags & VIE_SETUP_PWC else 12)


def vie_setup_green_external(grid, freq_hz, eps_real, sigma, toeplitz):
    """vie_setup with the caller's Galerkin entries of N: toeplitz is complex128
    [144][2nz-1][2ny-1][2nx-1] (entry alpha * 12 + beta, offset d at index d + N - 1), host or device."""
    lib = _lib()
    g = vie_grid(*[int(v) for v in grid[:3]], *[float(v) for v in grid[3:]])
    shape = (2 * g.nz - 1, 2 * g.ny - 1, 2 * g.nx - 1)
    n = 1
    for d in toeplitz.shape:
        n *= int(d)
    if n != 144 * shape[0] * shape[1] * shape[2]:
        raise ValueError("toeplitz must hold 144 x (2nz-1) x (2ny-1) x (2nx-1) complex values")
    out = ctypes.c_void_p()
    _check(lib.vie_setup_green_external(ctypes.byref(g), float(freq_hz), _ptr(eps_real), _ptr(sigma), _ptr(toeplitz),
                                        ctypes.byref(out)), "vie_setup_green_external")
    return Handle(out.value, (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), freq_hz)


def vie_destroy(h):
    _lib().vie_destroy(h.ptr)


def vie_matvec(h, x, y, precision=VIE_FP64, op=VIE_OP_A, stream=None):
    return _check(_lib().vie_matvec(h.ptr, _nrhs(x, h), _ptr(x), _ptr(y), int(precision), int(op), _stream(stream)),
                  "vie_matvec")


def vie_matvec_noalloc(h, x, y, precision=VIE_FP64, op=VIE_OP_A, stream=None):
    """vie_matvec for callers that cannot allocate GPU memory: device tensors only, scratch in a fixed
    64 MiB static device array; oversized calls raise VieError (VIE_EINVAL)."""
    return _check(_lib().vie_matvec_noalloc(h.ptr, _nrhs(x, h), _ptr(x), _ptr(y), int(precision), int(op),
                                            _stream(stream)), "vie_matvec_noalloc")


def vie_rhs_planewave(h, pol, direction, e_inc=None, b=None, stream=None):
    D3 = ctypes.c_double * 3
    return _check(_lib().vie_rhs_planewave(h.ptr, D3(*pol), D3(*direction), _ptr(e_inc), _ptr(b), _stream(stream)),
                  "vie_rhs_planewave")


def vie_rhs_dipoles(h, pos, mom, e_inc=None, b=None, stream=None):
    import numpy as np

    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1, 3)
    Dp = ctypes.POINTER(ctypes.c_double)
    return _check(_lib().vie_rhs_dipoles(h.ptr, pos.shape[0], pos.ctypes.data_as(Dp), mom.ctypes.data_as(Dp),
                                         _ptr(e_inc), _ptr(b), _stream(stream)), "vie_rhs_dipoles")


def vie_solve(h, b, x, tol=1e-6, restart=50, maxit=200, mode=VIE_SOLVE_FP32_REFINE, guess=False, true_resid=False,
              keep_point=True, graph=True, stream=None):
    """Returns (rc, [info dict per right-hand side]); rc is VIE_OK or VIE_NOT_CONVERGED.
    keep_point=False: the handle keeps no residual point for vie_fields (flags bit 2).
    graph=False: direct launches instead of a CUDA graph per restart cycle (flags bit 3)."""
    n = _nrhs(b, h)
    info = (vie_solve_info * n)()
    flags = (1 if guess else 0) | (2 if true_resid else 0) | (0 if keep_point else 4) | (0 if graph else 8)
    rc = _check(_lib().vie_solve(h.ptr, n, _ptr(b), _ptr(x), float(tol), int(restart), int(maxit), int(mode),
                                 flags, info, _stream(stream)), "vie_solve")
    return rc, [i.as_dict() for i in info]


def vie_fields(h, x, e_inc, e_coeff=None, p_abs=None, stream=None):
    """Returns the absorbed power P_abs (W) per right-hand side as a list."""
    n = _nrhs(x, h)
    P = (ctypes.c_double * n)()
    _check(_lib().vie_fields(h.ptr, n, _ptr(x), _ptr(e_inc), _ptr(e_coeff), _ptr(p_abs), P, _stream(stream)),
           "vie_fields")
    return list(P)


def vie_rhs_dipoles_h(h, pos, mom, h_inc, stream=None):
    """Tested incident magnetic fields of the dipoles into h_inc [R][12][nz][ny][nx] complex128."""
    import numpy as np

    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1, 3)
    Dp = ctypes.POINTER(ctypes.c_double)
    return _check(_lib().vie_rhs_dipoles_h(h.ptr, pos.shape[0], pos.ctypes.data_as(Dp), mom.ctypes.data_as(Dp),
                                           _ptr(h_inc), _stream(stream)), "vie_rhs_dipoles_h")


def vie_hfields(h, x, h_inc, h_coeff=None, b1_plus=None, stream=None):
    """Magnetic field coefficients, b1+ and the magnetic energy; returns W_m (J) per right-hand side."""
    n = _nrhs(x, h)
    W = (ctypes.c_double * n)()
    _check(_lib().vie_hfields(h.ptr, n, _ptr(x), _ptr(h_inc), _ptr(h_coeff), _ptr(b1_plus), W, _stream(stream)),
           "vie_hfields")
    return list(W)


def _nrhs_jm(a, h):
    """Right-hand sides in a JM-VIE vector batch [R][2][12][nz][ny][nx]."""
    n = 1
    for d in a.shape:
        n *= int(d)
    if n % (24 * h.nv):
        raise ValueError("array size is not a multiple of 24 * N_V")
    return n // (24 * h.nv)


def vie_set_permeability(h, mu_real, mu_imag):
    """Relative permeability mu_r = mu_real - i mu_imag per voxel, float64 [nz][ny][nx]."""
    return _check(_lib().vie_set_permeability(h.ptr, _ptr(mu_real), _ptr(mu_imag)), "vie_set_permeability")


def vie_jm_matvec(h, x, y, op=VIE_OP_A, precision=VIE_FP64, stream=None):
    """y = A x or P^-1 A x of the full JM-VIE system, x, y [R][2][12][nz][ny][nx] complex128
    (VIE_FP64) or complex64 (VIE_FP32)."""
    return _check(_lib().vie_jm_matvec(h.ptr, _nrhs_jm(x, h), _ptr(x), _ptr(y), int(precision), int(op),
                                       _stream(stream)), "vie_jm_matvec")


def vie_jm_rhs(h, e_inc, h_inc, b, stream=None):
    """b = (c_e chi_e e_inc, i k0 chi_m h_inc) into b [R][2][12][nz][ny][nx]."""
    return _check(_lib().vie_jm_rhs(h.ptr, _nrhs(e_inc, h), _ptr(e_inc), _ptr(h_inc), _ptr(b), _stream(stream)),
                  "vie_jm_rhs")


def vie_jm_solve(h, b, x, tol=1e-6, restart=50, maxit=200, mode=VIE_SOLVE_FP64, guess=False, true_resid=False,
                 graph=True, stream=None):
    """GMRES on the JM system (FP64, or FP32 inner solves with FP64 refinement); returns
    (rc, [info dict per right-hand side]).  graph=False: direct launches (flags bit 3)."""
    n = _nrhs_jm(b, h)
    info = (vie_solve_info * n)()
    flags = (1 if guess else 0) | (2 if true_resid else 0) | (0 if graph else 8)
    rc = _check(_lib().vie_jm_solve(h.ptr, n, _ptr(b), _ptr(x), float(tol), int(restart), int(maxit), int(mode),
                                    flags, info, _stream(stream)), "vie_jm_solve")
    return rc, [i.as_dict() for i in info]


def vie_jm_fields(h, x, e_inc, h_inc, e_coeff=None, h_coeff=None, p_abs=None, stream=None):
    """Field coefficients and absorbed power of a JM solution; returns P_abs (W) per right-hand side."""
    n = _nrhs_jm(x, h)
    P = (ctypes.c_double * n)()
    _check(_lib().vie_jm_fields(h.ptr, n, _ptr(x), _ptr(e_inc), _ptr(h_inc), _ptr(e_coeff), _ptr(h_coeff),
                                _ptr(p_abs), P, _stream(stream)), "vie_jm_fields")
    return list(P)


def vie_green_toeplitz(h, out):
    return _check(_lib().vie_green_toeplitz(h.ptr, _ptr(out)), "vie_green_toeplitz")


def vie_green_tucker(h, tol, apply=False):
    """Tucker compression of the handle's 60 Toeplitz tensors; returns (ranks [60][3] as (rx, ry, rz),
    relative errors [60], compressed bytes).  apply=True: the Green spectra are rebuilt from the
    compressed tensors (VIE_TUCKER_APPLY)."""
    import numpy as np

    ranks = np.zeros((60, 3), dtype=np.int32)
    err = np.zeros(60)
    nb = ctypes.c_size_t()
    _check(_lib().vie_green_tucker(h.ptr, float(tol), VIE_TUCKER_APPLY if apply else 0, ranks.ctypes.data,
                                   err.ctypes.data, ctypes.byref(nb)), "vie_green_tucker")
    return ranks, err, nb.value


def vie_green_toeplitz_k(h, out):
    """The 30 Toeplitz tensors of the K operator, [30][nz][ny][nx] complex128 (host or device)."""
    return _check(_lib().vie_green_toeplitz_k(h.ptr, _ptr(out)), "vie_green_toeplitz_k")


def vie_info(h):
    L = (ctypes.c_int * 3)()
    nb = ctypes.c_size_t()
    _check(_lib().vie_info(h.ptr, L, ctypes.byref(nb)), "vie_info")
    return tuple(L), nb.value


def vie_fault_inject(kind, count=1):
    """Host-side fault injection (VIE_INJECT_OOM: the next `count` workspace growths fail)."""
    return _check(_lib().vie_fault_inject(int(kind), int(count)), "vie_fault_inject")


def vie_tuning():
    """Lines of the autotuner's measurements and choices (one per grid shape seen)."""
    lib = _lib()
    n = lib.vie_tuning(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    lib.vie_tuning(ctypes.addressof(buf), n + 1)
    return buf.value.decode().splitlines()


def vie_strerror(code):
    return _lib().vie_strerror(int(code)).decode()


def vie_stats_reset(timing=False):
    return _check(_lib().vie_stats_reset(1 if timing else 0), "vie_stats_reset")


def vie_stats_read(max_entries=256):
    """Returns (total_launches, {kernel name: (launches, device ms, algorithmic bytes)})."""
    names = ctypes.create_string_buffer(48 * max_entries)
    launches = (ctypes.c_longlong * max_entries)()
    ms = (ctypes.c_double * max_entries)()
    nbytes = (ctypes.c_double * max_entries)()
    n = ctypes.c_int()
    tot = ctypes.c_longlong()
    _check(_lib().vie_stats_read(max_entries, ctypes.addressof(names), ctypes.addressof(launches),
                                 ctypes.addressof(ms), ctypes.addressof(nbytes), ctypes.byref(n), ctypes.byref(tot)),
           "vie_stats_read")
    out = {}
    for i in range(n.value):
        nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (launches[i], ms[i], nbytes[i])
    return tot.value, out


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------
class Server:
    """The request loop of vie_server_create (arguments marshalled; the loop itself is native)."""

    def __init__(self, hbm_budget_bytes=0, max_concurrent=4):
        p = ctypes.c_void_p()
        _check(_lib().vie_server_create(int(hbm_budget_bytes), int(max_concurrent), ctypes.byref(p)),
               "vie_server_create")
        self._p = p
        self._keep = {}

    def close(self):
        if self._p:
            _lib().vie_server_destroy(self._p)
            self._p = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, grid, freq_hz, eps_real, sigma, pos, mom, tol=1e-6, restart=50, maxit=30,
               mode=VIE_SOLVE_FP32_REFINE, x_out=None, p_abs_out=None, P_abs_out=None):
        """Queue one solve; host NumPy inputs (float64), optional host outputs.  Returns the ticket."""
        import numpy as np

        eps = np.ascontiguousarray(eps_real, dtype=np.float64)
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1, 3)
        for o in (x_out, p_abs_out, P_abs_out):
            if o is not None and not (isinstance(o, np.ndarray) and o.flags["C_CONTIGUOUS"]):
                raise ValueError("outputs must be C-contiguous NumPy arrays")
        r = vie_request()
        r.grid = vie_grid(*grid)
        r.freq_hz = float(freq_hz)
        r.eps_real, r.sigma = eps.ctypes.data, sig.ctypes.data
        r.nrhs = pos.shape[0]
        r.dip_pos, r.dip_mom = pos.ctypes.data, mom.ctypes.data
        r.tol, r.restart, r.maxit, r.mode = float(tol), int(restart), int(maxit), int(mode)
        r.x_out = _ptr(x_out)
        r.p_abs_out = _ptr(p_abs_out)
        r.P_abs_out = _ptr(P_abs_out)
        t = ctypes.c_ulonglong()
        _check(_lib().vie_submit(self._p, ctypes.byref(r), ctypes.byref(t)), "vie_submit")
        self._keep[t.value] = (x_out, p_abs_out, P_abs_out)  # outputs stay alive until polled
        return t.value

    def poll(self, ticket, timeout_us=0):
        """Result dict when the request is done, None when it is still queued or running."""
        res = vie_result()
        rc = _lib().vie_poll(self._p, ctypes.c_ulonglong(ticket), int(timeout_us), ctypes.byref(res))
        if rc == VIE_ETIMEOUT:
            return None
        _check(rc, "vie_poll")
        self._keep.pop(ticket, None)
        return res.as_dict()

    def stats(self):
        q, r, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        _check(_lib().vie_server_stats(self._p, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c)),
               "vie_server_stats")
        return dict(queued=q.value, running=r.value, bytes_in_use=b.value, cache_entries=c.value)
