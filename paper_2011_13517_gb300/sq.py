"""Thin Python binding of libsq (include/sq.h): argument marshalling only.

Every entry point has the name of the C function it calls.  Device buffers are torch CUDA tensors
(passed as raw pointers with the current torch stream); host scalars come back as Python floats.
If libsq.so is missing this module raises at import of the library -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsq.so")

SQ_FP64 = 0
SQ_FP32 = 1
SQ_WANT_FORCE = 1
SQ_GAUSS = 2
SQ_KB_FMA = 4
SQ_GRAD_ANALYTIC = 0
SQ_GRAD_FD = 1

STATUS = {0: "SQ_OK", 1: "SQ_ERR_ARG", 2: "SQ_ERR_CUBE_EXCEEDS_BOX", 3: "SQ_ERR_NO_BRACKET",
          4: "SQ_ERR_NOT_FINITE", 5: "SQ_ERR_CUDA", 6: "SQ_ERR_TIMEOUT", 7: "SQ_ERR_OOM",
          8: "SQ_ERR_STATE", 9: "SQ_ERR_UNSUPPORTED"}

EXPORTS = ["sq_build_hamiltonian", "sq_density", "sq_fermi_level", "sq_fermi_weights", "sq_gauss_rule",
           "sq_fermi_resolve",
           "sq_moments_range", "sq_moments_cols", "sq_observables", "sq_energy", "sq_nonlocal_force",
           "sq_get_spectral_bounds", "sq_get_moments", "sq_copy_moments", "sq_get_cube", "sq_get_timing",
           "sq_kernel_launches", "sq_fma_throughput", "sq_mma_throughput", "sq_moments_noalloc", "sq_batch_create", "sq_batch_density",
           "sq_batch_info", "sq_batch_destroy", "sq_density_vjp", "sq_kernel_name", "sq_destroy",
           "sq_status_string", "sq_last_error", "sq_lda_pw92", "sq_pseudocharge", "sq_poisson_periodic",
           "sq_effective_potential", "sq_mixer_create", "sq_mixer_step", "sq_mixer_destroy", "sq_self_energy",
           "sq_free_energy", "sq_local_force"]


class SQError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class sq_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3), ("fd_order", ctypes.c_int)]


class sq_atoms(ctypes.Structure):
    _fields_ = [("natom", ctypes.c_int), ("R", ctypes.POINTER(ctypes.c_double)), ("lmax", ctypes.c_int),
                ("sigma", ctypes.c_double), ("rc", ctypes.c_double),
                ("energy", ctypes.POINTER(ctypes.c_double))]


_lib = None


def lib():
    """Load libsq.so (never builds implicitly; call paper_2011_13517_gb300.build.build() first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsq.so not built ({LIB_PATH}); run paper_2011_13517_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        L.sq_build_hamiltonian.argtypes = [ctypes.POINTER(sq_grid), vp, ctypes.POINTER(sq_atoms), ctypes.c_double,
                                           ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, ctypes.POINTER(vp)]
        L.sq_density.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 vp, dp, vp]
        d = ctypes.c_double
        L.sq_fermi_level.argtypes = [dp, ctypes.c_int, d, d, d, d, d, d, dp]
        L.sq_fermi_weights.argtypes = [d, ctypes.c_int, d, d, d, dp, dp, dp]
        L.sq_gauss_rule.argtypes = [dp, dp, ctypes.c_int, d, d, dp, dp]
        L.sq_fermi_resolve.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, dp, vp]
        L.sq_moments_range.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                       ctypes.c_longlong, dp, dp, vp]
        L.sq_observables.argtypes = [vp, d, d, d, dp, dp, vp, vp]
        L.sq_moments_cols.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_longlong, vp, vp]
        L.sq_fma_throughput.argtypes = [ctypes.c_int, dp, dp, vp]
        L.sq_mma_throughput.argtypes = [ctypes.c_int, dp, dp, vp]
        L.sq_energy.argtypes = [vp, dp, dp, dp, vp]
        L.sq_nonlocal_force.argtypes = [vp, vp, vp]
        L.sq_get_spectral_bounds.argtypes = [vp, dp, dp]
        L.sq_get_moments.argtypes = [vp, ip, ip, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.sq_copy_moments.argtypes = [vp, vp, vp, vp]
        L.sq_get_cube.argtypes = [vp, ip]
        L.sq_get_timing.argtypes = [vp, dp, dp, dp]
        L.sq_kernel_launches.argtypes = []
        L.sq_moments_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.sq_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.sq_batch_density.argtypes = [vp, ctypes.POINTER(vp), dp, vp]
        L.sq_batch_info.argtypes = [vp, ip, ip, ip, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.sq_batch_destroy.argtypes = [vp]
        L.sq_density_vjp.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp, vp]
        L.sq_kernel_name.argtypes = [vp]
        L.sq_kernel_name.restype = ctypes.c_char_p
        L.sq_batch_destroy.restype = None
        L.sq_destroy.argtypes = [vp]
        L.sq_destroy.restype = None
        L.sq_mixer_destroy.restype = None
        L.sq_mixer_destroy.argtypes = [vp]
        L.sq_status_string.argtypes = [ctypes.c_int]
        L.sq_status_string.restype = ctypes.c_char_p
        L.sq_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("sq_destroy", "sq_status_string", "sq_last_error", "sq_kernel_launches", "sq_batch_destroy",
                            "sq_kernel_name", "sq_mixer_destroy"):
                getattr(L, name).restype = ctypes.c_int
        L.sq_kernel_launches.restype = ctypes.c_longlong
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise SQError(status, lib().sq_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype=torch.float64, numel=None):
    """Raw pointer of a contiguous CUDA tensor of the given dtype holding at least `numel` elements.
    The library writes through these pointers without knowing the tensor's size, so a short buffer
    is rejected here, before any launch."""
    if numel is not None and t.numel() < numel:
        raise ValueError(f"buffer holds {t.numel()} elements, the call writes {numel}")
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Owns an sq_handle; remembers the sizes its outputs need (grid points, atoms, projectors)."""

    def __init__(self, ptr, N_d=None, natom=None, nproj=None):
        self.ptr = ctypes.c_void_p(ptr)
        self.N_d = N_d
        self.natom = natom
        self.nproj = nproj
        self.K = None
        self.range = None

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            lib().sq_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)


def sq_build_hamiltonian(n, L, fd_order, d_veff, R, lmax, sigma, rc, energy, R_cut,
                         lambda_min=math.nan, lambda_max=math.nan, stream=None, flags=SQ_GRAD_ANALYTIC) -> Handle:
    """sq_build_hamiltonian: grid (n, L, fd_order), device V_eff [N_d] float64, atoms R [natom, 3]
    with projector parameters, truncation half-width R_cut, optional spectral bounds, and the
    projector gradient of the force (flags: SQ_GRAD_ANALYTIC or SQ_GRAD_FD)."""
    g = sq_grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.L[a] = float(L[a])
    g.fd_order = int(fd_order)
    Rh = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 3))
    en = np.ascontiguousarray(np.asarray(energy, dtype=np.float64).reshape(-1))
    at = sq_atoms()
    at.natom = int(Rh.shape[0])
    at.R = Rh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    at.lmax = int(lmax)
    at.sigma = float(sigma)
    at.rc = float(rc)
    at.energy = en.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    N_d = int(g.n[0]) * int(g.n[1]) * int(g.n[2])
    out = ctypes.c_void_p()
    _check(lib().sq_build_hamiltonian(ctypes.byref(g), _dev_ptr(d_veff, numel=N_d), ctypes.byref(at), float(R_cut),
                                      int(flags), float(lambda_min), float(lambda_max), _stream(stream),
                                      ctypes.byref(out)))
    return Handle(out.value, N_d=N_d, natom=at.natom, nproj=1 if int(lmax) == 0 else 4)


def sq_density(h: Handle, K, kT, N_e, precision, flags, d_rho, stream=None) -> float:
    lam = ctypes.c_double()
    _check(lib().sq_density(h.ptr, int(K), float(kT), float(N_e), int(precision), int(flags),
                            _dev_ptr(d_rho, numel=h.N_d), ctypes.byref(lam), _stream(stream)))
    h.K, h.range = int(K), (0, h.N_d)
    return lam.value


def sq_fermi_resolve(h: Handle, kT, N_e, d_rho=None, stream=None) -> float:
    """Re-solve the Fermi level of the last whole-grid sq_density for another kT / N_e (device)."""
    lam = ctypes.c_double()
    _check(lib().sq_fermi_resolve(h.ptr, float(kT), float(N_e),
                                  _dev_ptr(d_rho, numel=h.N_d) if d_rho is not None else ctypes.c_void_p(None),
                                  ctypes.byref(lam), _stream(stream)))
    return lam.value


def _host_f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size < n:
        raise ValueError(f"array holds {a.size} values, {n} are needed")
    return a


def sq_fermi_level(msum, K, omega, tau, lambda_min, lambda_max, kT, N_e) -> float:
    """Pure host Fermi level from moment sums M_k (Eq. Ne); no handle, no GPU."""
    m = _host_f64(msum, int(K) + 1)
    lam = ctypes.c_double()
    _check(lib().sq_fermi_level(m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(K), float(omega), float(tau),
                                float(lambda_min), float(lambda_max), float(kT), float(N_e), ctypes.byref(lam)))
    return lam.value


def sq_fermi_weights(lambda_f, K, omega, tau, kT):
    """Host Chebyshev weights (c, d, e) [K+1] of g, lam g and s(g) at lambda_f."""
    out = [np.zeros(int(K) + 1) for _ in range(3)]
    ptr = [o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for o in out]
    _check(lib().sq_fermi_weights(float(lambda_f), int(K), float(omega), float(tau), float(kT), *ptr))
    return tuple(out)


def sq_gauss_rule(a, b, omega=0.0, tau=1.0):
    """Host Gauss rule (nodes, weights) [K] of one grid point from its Lanczos coefficients a, b [K]."""
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    b = _host_f64(b, a.size)
    nodes, weights = np.zeros(a.size), np.zeros(a.size)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().sq_gauss_rule(a.ctypes.data_as(dp), b.ctypes.data_as(dp), int(a.size), float(omega), float(tau),
                               nodes.ctypes.data_as(dp), weights.ctypes.data_as(dp)))
    return nodes, weights


def sq_moments_range(h: Handle, K, precision, flags, q_begin, q_end, stream=None):
    """Recursion over columns [q_begin, q_end): returns (partial M_k [K+1], partial force moments
    [K+1, natom, nproj, 3] or None)."""
    K = int(K)
    msum = np.zeros(K + 1)
    want_force = bool(int(flags) & SQ_WANT_FORCE) and h.natom
    A = np.zeros((K + 1, h.natom, h.nproj, 3)) if want_force else None
    _check(lib().sq_moments_range(h.ptr, K, int(precision), int(flags), int(q_begin), int(q_end),
                                  msum.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if A is not None else None,
                                  _stream(stream)))
    h.K, h.range = K, (int(q_begin), int(q_end))
    return msum, A


def sq_moments_cols(h: Handle, K, precision, d_cols, d_mu_out, stream=None):
    """Moments [K+1, ncols] of the listed grid points (d_cols: CUDA int64 tensor) into d_mu_out."""
    n = int(d_cols.numel())
    dt = torch.float64 if precision == SQ_FP64 else torch.float32
    _check(lib().sq_moments_cols(h.ptr, int(K), int(precision), _dev_ptr(d_cols, torch.int64, numel=n), n,
                                 _dev_ptr(d_mu_out, dt, numel=(int(K) + 1) * n), _stream(stream)))


def sq_observables(h: Handle, lambda_f, kT, N_e, msum, A=None, d_rho=None, stream=None):
    """After sq_moments_range: total sums in, density of the range's columns out (d_rho [q_end - q_begin])."""
    if h.K is None or h.range is None:
        raise ValueError("sq_observables needs sq_moments_range first")
    m = _host_f64(msum, h.K + 1)
    Ah = _host_f64(A, (h.K + 1) * h.natom * h.nproj * 3) if A is not None else None
    n = h.range[1] - h.range[0]
    _check(lib().sq_observables(h.ptr, float(lambda_f), float(kT), float(N_e),
                                m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                Ah.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if Ah is not None else None,
                                _dev_ptr(d_rho, numel=n) if d_rho is not None else ctypes.c_void_p(None),
                                _stream(stream)))


def sq_mma_throughput(kind, stream=None):
    """Measured warp-level MMA throughput (TFLOP/s, ms): kind 0 TF32 m16n8k8, 1 BF16 m16n8k16."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().sq_mma_throughput(int(kind), ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return t.value, ms.value


def sq_fma_throughput(precision, stream=None):
    """Measured FMA ceiling (TFLOP/s, ms of the timed probe launch) of the current GPU."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().sq_fma_throughput(int(precision), ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return t.value, ms.value


def _grid(n, box):
    return (ctypes.c_int * 3)(*[int(v) for v in n]), (ctypes.c_double * 3)(*[float(v) for v in box])


def sq_lda_pw92(d_rho, d_exc, d_vxc, stream=None):
    """sq_lda_pw92: eps_xc and V_xc of the LDA (Slater + Perdew-Wang) at every point of d_rho."""
    n = d_rho.numel()
    _check(lib().sq_lda_pw92(ctypes.c_longlong(n), _dev_ptr(d_rho), _dev_ptr(d_exc, numel=n), _dev_ptr(d_vxc, numel=n),
                             _stream(stream)))


def sq_pseudocharge(n, box, R, Z, sigma_b, d_b, stream=None):
    """sq_pseudocharge: Gaussian pseudocharges of the nuclei on the grid (R [natom, 3] bohr, Z [natom])."""
    gn, gb = _grid(n, box)
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 3))
    Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1))
    if R.shape[0] != Z.size:
        raise ValueError("R and Z disagree on the atom count")
    N = int(np.prod([int(v) for v in n]))
    _check(lib().sq_pseudocharge(gn, gb, ctypes.c_int(Z.size), R.ctypes.data_as(ctypes.c_void_p),
                                 Z.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(sigma_b), _dev_ptr(d_b, numel=N),
                                 _stream(stream)))


def sq_poisson_periodic(n, box, fd_order, d_f, d_phi, tol=1e-11, max_iter=5000, stream=None):
    """sq_poisson_periodic: phi of -(1/4 pi) L_h phi = f - mean f; returns (iterations, relative residual)."""
    gn, gb = _grid(n, box)
    N = int(np.prod([int(v) for v in n]))
    it, res = ctypes.c_int(), ctypes.c_double()
    _check(lib().sq_poisson_periodic(gn, gb, ctypes.c_int(fd_order), _dev_ptr(d_f, numel=N), ctypes.c_double(tol),
                                     ctypes.c_int(max_iter), _dev_ptr(d_phi, numel=N), ctypes.byref(it),
                                     ctypes.byref(res), _stream(stream)))
    return it.value, res.value


def sq_effective_potential(n, box, fd_order, d_rho, d_b, d_phi, d_exc, d_vxc, d_veff, tol=1e-11, max_iter=5000,
                           stream=None):
    """sq_effective_potential: phi(rho + b), eps_xc, V_xc and V_eff = V_xc + phi; returns (iterations, residual)."""
    gn, gb = _grid(n, box)
    N = int(np.prod([int(v) for v in n]))
    it, res = ctypes.c_int(), ctypes.c_double()
    _check(lib().sq_effective_potential(gn, gb, ctypes.c_int(fd_order), _dev_ptr(d_rho, numel=N),
                                        _dev_ptr(d_b, numel=N), ctypes.c_double(tol), ctypes.c_int(max_iter),
                                        _dev_ptr(d_phi, numel=N), _dev_ptr(d_exc, numel=N), _dev_ptr(d_vxc, numel=N),
                                        _dev_ptr(d_veff, numel=N), ctypes.byref(it), ctypes.byref(res),
                                        _stream(stream)))
    return it.value, res.value


class Mixer:
    """Owns an sq_mixer (Anderson mixing of V_eff over SCF iterations)."""

    def __init__(self, ptr, n):
        self.ptr = ctypes.c_void_p(ptr)
        self.n = n

    def close(self):
        if self.ptr:
            lib().sq_mixer_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sq_mixer_create(n, history=5, beta=0.3):
    out = ctypes.c_void_p()
    _check(lib().sq_mixer_create(ctypes.c_longlong(int(n)), ctypes.c_int(history), ctypes.c_double(beta),
                                 ctypes.byref(out)))
    return Mixer(out.value, int(n))


def sq_mixer_step(m: Mixer, d_vin, d_vout, d_vnext, stream=None):
    """One Anderson step: writes V_next, returns |V_out - V_in| / |V_out|."""
    err = ctypes.c_double()
    _check(lib().sq_mixer_step(m.ptr, _dev_ptr(d_vin, numel=m.n), _dev_ptr(d_vout, numel=m.n),
                               _dev_ptr(d_vnext, numel=m.n), ctypes.byref(err), _stream(stream)))
    return err.value


def sq_mixer_destroy(m: Mixer):
    m.close()


def _atoms(R, Z):
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 3))
    Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1))
    if R.shape[0] != Z.size:
        raise ValueError("R and Z disagree on the atom count")
    return R, Z


def sq_self_energy(n, box, R, Z, sigma_b, stream=None):
    """sq_self_energy: E_self^h of the Gaussian pseudocharges."""
    gn, gb = _grid(n, box)
    R, Z = _atoms(R, Z)
    e = ctypes.c_double()
    _check(lib().sq_self_energy(gn, gb, ctypes.c_int(Z.size), R.ctypes.data_as(ctypes.c_void_p),
                                Z.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(sigma_b), ctypes.byref(e),
                                _stream(stream)))
    return e.value


def sq_free_energy(n, box, d_rho, d_b, d_phi, d_exc, d_vxc, F_band, E_self, stream=None):
    """sq_free_energy: the discrete free energy F^h."""
    gn, gb = _grid(n, box)
    N = int(np.prod([int(v) for v in n]))
    F = ctypes.c_double()
    _check(lib().sq_free_energy(gn, gb, *[_dev_ptr(t, numel=N) for t in (d_rho, d_b, d_phi, d_exc, d_vxc)],
                                ctypes.c_double(F_band), ctypes.c_double(E_self), ctypes.byref(F), _stream(stream)))
    return F.value


def sq_local_force(n, box, fd_order, R, Z, sigma_b, d_phi, stream=None):
    """sq_local_force: [natom, 3] local pseudopotential forces."""
    gn, gb = _grid(n, box)
    R, Z = _atoms(R, Z)
    N = int(np.prod([int(v) for v in n]))
    f = np.zeros((Z.size, 3))
    _check(lib().sq_local_force(gn, gb, ctypes.c_int(fd_order), ctypes.c_int(Z.size),
                                R.ctypes.data_as(ctypes.c_void_p), Z.ctypes.data_as(ctypes.c_void_p),
                                ctypes.c_double(sigma_b), _dev_ptr(d_phi, numel=N),
                                f.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return f


def sq_energy(h: Handle, stream=None):
    U, S, F = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sq_energy(h.ptr, ctypes.byref(U), ctypes.byref(S), ctypes.byref(F), _stream(stream)))
    return U.value, S.value, F.value


def sq_nonlocal_force(h: Handle, d_force, stream=None):
    _check(lib().sq_nonlocal_force(h.ptr, _dev_ptr(d_force, numel=3 * h.natom), _stream(stream)))


def sq_get_spectral_bounds(h: Handle):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().sq_get_spectral_bounds(h.ptr, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def sq_get_cube(h: Handle):
    m = (ctypes.c_int * 3)()
    _check(lib().sq_get_cube(h.ptr, m))
    return tuple(m)


def sq_get_timing(h: Handle):
    """(recursion_ms, moment_sum_ms, fermi_ms) of the last sq_density, from CUDA events."""
    r, m, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sq_get_timing(h.ptr, ctypes.byref(r), ctypes.byref(m), ctypes.byref(f)))
    return r.value, m.value, f.value


def sq_density_vjp(h: Handle, d_rho_bar, U_bar, checkpoint_k, d_veff_bar, stream=None):
    """sq_density_vjp: d_veff_bar = dL/dV_eff for L = sum rho_bar rho + U_bar U (see include/sq.h)."""
    _check(lib().sq_density_vjp(h.ptr, _dev_ptr(d_rho_bar, numel=h.N_d), float(U_bar), int(checkpoint_k),
                                _dev_ptr(d_veff_bar, numel=h.N_d), _stream(stream)))


def sq_kernel_name(h: Handle) -> str:
    return lib().sq_kernel_name(h.ptr).decode()


def sq_kernel_launches() -> int:
    return int(lib().sq_kernel_launches())


def sq_moments_noalloc(h: Handle, K, precision, d_mu, stream=None):
    """sq_moments_noalloc: moments [K+1, N_d] into the caller's tensor (float64 for SQ_FP64, float32
    for SQ_FP32) with no device allocation by the library; see include/sq.h for the shared fixed
    scratch array and its rules."""
    dt = torch.float64 if precision == SQ_FP64 else torch.float32
    _check(lib().sq_moments_noalloc(h.ptr, int(K), int(precision), _dev_ptr(d_mu, dt, numel=(int(K) + 1) * h.N_d),
                                    _stream(stream)))


class Batch:
    """Owns an sq_batch (the cell handles stay owned by the caller and must outlive it)."""

    def __init__(self, ptr, handles):
        self.ptr = ctypes.c_void_p(ptr)
        self.handles = handles

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            lib().sq_batch_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)


def sq_batch_create(handles, K, kT, N_e, precision, flags) -> Batch:
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    Ks = (ctypes.c_int * n)(*[int(x) for x in K])
    kTs = np.ascontiguousarray(kT, dtype=np.float64)
    Nes = np.ascontiguousarray(N_e, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().sq_batch_create(arr, n, Ks, kTs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 Nes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(precision), int(flags),
                                 ctypes.byref(out)))
    return Batch(out.value, list(handles))


def sq_batch_density(b: Batch, d_rhos, stream=None):
    n = len(b.handles)
    ptrs = (ctypes.c_void_p * n)(*[_dev_ptr(r, numel=h.N_d).value for r, h in zip(d_rhos, b.handles)])
    lam = np.zeros(n)
    _check(lib().sq_batch_density(b.ptr, ptrs, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
    return lam


def sq_batch_destroy(b: Batch):
    b.close()


def sq_destroy(h: Handle):
    h.close()


def sq_batch_info(b: Batch):
    cfg, chunk, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms, nodes = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().sq_batch_info(b.ptr, ctypes.byref(cfg), ctypes.byref(chunk), ctypes.byref(grid), ctypes.byref(ms),
                               ctypes.byref(nodes)))
    return dict(config=cfg.value, chunk=chunk.value, grid=grid.value, tuned_ms=ms.value, graph_nodes=nodes.value)


def sq_copy_moments(h: Handle, N_d, stream=None):
    """Copies of the moments mu [K+1, N_d] (recursion precision) and sums M [K+1] (float64)."""
    K, prec = ctypes.c_int(), ctypes.c_int()
    mu_p, ms_p = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().sq_get_moments(h.ptr, ctypes.byref(K), ctypes.byref(prec), ctypes.byref(mu_p), ctypes.byref(ms_p)))
    dt = torch.float64 if prec.value == SQ_FP64 else torch.float32
    mu = torch.empty((K.value + 1, int(N_d)), dtype=dt, device="cuda")
    ms = torch.empty(K.value + 1, dtype=torch.float64, device="cuda")
    _check(lib().sq_copy_moments(h.ptr, ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(ms.data_ptr()),
                                 _stream(stream)))
    return mu, ms


# ---------------------------------------------------------------------------------------------
# convenience for a generated cell (marshalling only)

def build_for_cell(cell, bounds=None, stream=None, d_veff=None, flags=SQ_GRAD_ANALYTIC):
    if d_veff is None:
        d_veff = torch.from_numpy(np.ascontiguousarray(cell.veff.reshape(-1))).to("cuda")
    lo, hi = (math.nan, math.nan) if bounds is None else bounds
    return sq_build_hamiltonian(cell.n, cell.box, cell.fd_order, d_veff, cell.R, cell.lmax, cell.proj_sigma,
                                cell.proj_rc, cell.proj_energy, cell.R_cut, lo, hi, stream=stream, flags=flags)


def solve_cell(cell, precision=SQ_FP64, force=True, bounds=None, K=None, kT=None, N_e=None, stream=None,
               grad=SQ_GRAD_ANALYTIC, extra_flags=0):
    """Build + density (+ energy, force) for one cell; returns numpy results.  extra_flags is or-ed into
    sq_density's flags (SQ_KB_FMA)."""
    h = build_for_cell(cell, bounds=bounds, stream=stream, flags=grad)
    try:
        rho = torch.empty(cell.N_d, dtype=torch.float64, device="cuda")
        lam_f = sq_density(h, cell.K if K is None else K, cell.kT if kT is None else kT,
                           cell.N_e if N_e is None else N_e, precision, (SQ_WANT_FORCE if force else 0) | extra_flags, rho,
                           stream=stream)
        U, S, F = sq_energy(h, stream=stream)
        out = dict(lam_f=lam_f, U=U, S=S, F=F, bounds=sq_get_spectral_bounds(h))
        if force:
            f = torch.empty((cell.natom, 3), dtype=torch.float64, device="cuda")
            sq_nonlocal_force(h, f, stream=stream)
            out["force"] = f.cpu().numpy()
        mu, ms = sq_copy_moments(h, cell.N_d, stream=stream)
        torch.cuda.synchronize()
        out["rho"] = rho.cpu().numpy()
        out["mu"] = mu.double().cpu().numpy()
        out["Msum"] = ms.cpu().numpy()
        return out
    finally:
        h.close()
