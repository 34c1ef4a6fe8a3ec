"""Python binding of libcl.so (the C ABI declared in include/cl.h).

Argument marshalling only: every step of the lattice evolution runs in the
library's CUDA kernels.  Arrays may be numpy arrays (host) or torch CUDA
tensors (device, passed by pointer); both must be C-contiguous with N^3
elements of the lattice's element type (float64 for CL_PREC_FP64, float32
otherwise).  The library must be built (``build_ext.build()``); importing this
module without it raises, there is no fallback.
"""
import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcl.so")

CL_OK, CL_EINVAL, CL_ENOMEM, CL_ECUDA, CL_ENAN, CL_ECONSTRAINT, CL_ETIMEOUT, CL_ESTATE, CL_EUNSUPPORTED = range(9)
CL_PREC_FP64, CL_PREC_FP32_KAHAN, CL_PREC_FP32 = 0, 1, 2
CL_INT_VV2, CL_INT_YOSHIDA4, CL_INT_RK3_3, CL_INT_RK4_5, CL_INT_YOSHIDA6, CL_INT_YOSHIDA8, CL_INT_YOSHIDA10, CL_INT_RK3_4 = \
    range(8)
CL_GAUGE_NONE, CL_GAUGE_U1_AXION = 0, 1
CL_GSPEC_E, CL_GSPEC_B, CL_GSPEC_APLUS, CL_GSPEC_AMINUS = 0, 1, 2, 3
CL_POT_LPHI4, CL_POT_M2, CL_POT_M2_G2, CL_POT_LPHI4_G2, CL_POT_POLY = 0, 1, 2, 3, 4
CL_FIELD_PHI0, CL_FIELD_PHI1, CL_FIELD_PI0, CL_FIELD_PI1 = 0, 1, 2, 3
CL_FIELD_THETA1, CL_FIELD_THETA2, CL_FIELD_THETA3, CL_FIELD_E1, CL_FIELD_E2, CL_FIELD_E3 = 4, 5, 6, 7, 8, 9
CL_FIELD_GW_V11, CL_FIELD_GW_V12, CL_FIELD_GW_V13, CL_FIELD_GW_V22, CL_FIELD_GW_V23 = 10, 11, 12, 13, 14
CL_FIELD_GW_P11, CL_FIELD_GW_P12, CL_FIELD_GW_P13, CL_FIELD_GW_P22, CL_FIELD_GW_P23 = 15, 16, 17, 18, 19
CL_OPT_GRAPH, CL_OPT_TILE_BY, CL_OPT_TILE_DZ, CL_OPT_STAGES, CL_OPT_PASS_VARIANT = 0, 1, 2, 3, 4

# Every exported entry point of include/cl.h.
EXPORTS = ["cl_init_lattice", "cl_free", "cl_set_potential", "cl_set_state", "cl_get_state", "cl_set_scalars",
           "cl_get_scalars", "cl_init_vacuum", "cl_step", "cl_sync", "cl_energies", "cl_spectrum",
           "cl_set_gauge_coupling", "cl_set_hubble_limit", "cl_set_option", "cl_get_option", "cl_last_launch_count", "cl_strerror", "cl_last_error",
           "cl_fused_pass_noalloc", "cl_surrogate_create", "cl_surrogate_free", "cl_surrogate_set_weights",
           "cl_surrogate_get_weights", "cl_surrogate_forward", "cl_surrogate_backward", "cl_surrogate_get_grads",
           "cl_surrogate_last_launch_count", "cl_surrogate_loss", "cl_surrogate_adamw", "cl_surrogate_channel_stats",
           "cl_lattice_pack", "cl_lattice_unpack", "cl_surrogate_jump", "cl_surrogate_size", "cl_autotune", "cl_gauge_spectrum", "cl_set_nonminimal", "cl_enable_gw", "cl_gw_spectrum",
           "cl_set_adaptive"]
CL_ACT_RELU, CL_ACT_GELU = 1, 2
CL_SG_BF16, CL_SG_FP32 = 0, 1


class cl_lattice_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("nfields", C.c_int32), ("precision", C.c_int32), ("integrator", C.c_int32),
                ("gauge", C.c_int32), ("expansion", C.c_int32), ("members", C.c_int32), ("dims", C.c_int32),
                ("member_N", C.POINTER(C.c_int32)), ("member_L", C.POINTER(C.c_double)),
                ("L", C.c_double), ("alpha", C.c_double), ("kappa", C.c_double), ("dt", C.c_double),
                ("a0", C.c_double), ("stream", C.c_void_p)]


class cl_vacuum_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("kcut", C.c_double), ("amp2", C.c_double),
                ("fbar", C.c_double * 2), ("dfbar", C.c_double * 2)]


class cl_energy(C.Structure):
    _fields_ = [("t", C.c_double), ("a", C.c_double), ("adot", C.c_double), ("K", C.c_double * 2),
                ("G", C.c_double * 2), ("V", C.c_double), ("KE", C.c_double), ("GB", C.c_double),
                ("rho", C.c_double), ("p", C.c_double), ("hubble_violation", C.c_double),
                ("gauss_violation", C.c_double), ("step", C.c_int64), ("ricci", C.c_double),
                ("gauss_rms_step", C.c_double), ("gauss_rms_max", C.c_double), ("dt", C.c_double),
                ("rk_error", C.c_double)]

    def as_dict(self):
        return {"t": self.t, "a": self.a, "adot": self.adot, "K0": self.K[0], "K1": self.K[1], "G0": self.G[0],
                "G1": self.G[1], "V": self.V, "KE": self.KE, "GB": self.GB, "rho": self.rho, "p": self.p,
                "hubble_violation": self.hubble_violation, "gauss_violation": self.gauss_violation,
                "step": self.step, "ricci": self.ricci, "gauss_rms_step": self.gauss_rms_step,
                "gauss_rms_max": self.gauss_rms_max, "dt": self.dt, "rk_error": self.rk_error}


class cl_pass_noalloc_desc(C.Structure):
    """One fused pass on caller-owned device arrays (see cl_fused_pass_noalloc in cl.h)."""
    _fields_ = [("N", C.c_int32), ("nfields", C.c_int32), ("precision", C.c_int32), ("expansion", C.c_int32),
                ("L", C.c_double), ("alpha", C.c_double), ("kappa", C.c_double),
                ("m2", C.c_double * 2), ("lam", C.c_double * 2), ("g2", C.c_double),
                ("drift", C.c_double), ("energy_kick", C.c_double), ("kick", C.c_double),
                ("phi_in", C.c_void_p * 2), ("pi_in", C.c_void_p * 2), ("c_in", C.c_void_p * 2),
                ("phi_out", C.c_void_p * 2), ("pi_out", C.c_void_p * 2), ("c_out", C.c_void_p * 2),
                ("scalars", C.c_void_p), ("energies", C.c_void_p), ("stream", C.c_void_p), ("status", C.c_void_p)]


class cl_surrogate_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("in_channels", C.c_int32), ("out_channels", C.c_int32), ("hidden", C.c_int32),
                ("layers", C.c_int32), ("activation", C.c_int32), ("precision", C.c_int32), ("reserved", C.c_int32),
                ("stream", C.c_void_p)]


class CLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (_strerror(status), status, msg))
        self.status = status


_lib = None


def lib():
    """Load libcl.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libcl.so is not built (run paper_2607_24978_gb300.build_ext.build())")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        L.cl_init_lattice.argtypes = [P(C.c_void_p), P(cl_lattice_params)]
        L.cl_free.argtypes = [C.c_void_p]
        L.cl_free.restype = None
        L.cl_set_potential.argtypes = [C.c_void_p, C.c_int32, P(C.c_double), C.c_int32]
        L.cl_set_state.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]
        L.cl_get_state.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]
        L.cl_set_scalars.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double]
        L.cl_get_scalars.argtypes = [C.c_void_p, C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double)]
        L.cl_init_vacuum.argtypes = [C.c_void_p, C.c_int32, P(cl_vacuum_params)]
        L.cl_step.argtypes = [C.c_void_p, C.c_int32]
        L.cl_sync.argtypes = [C.c_void_p]
        L.cl_energies.argtypes = [C.c_void_p, P(cl_energy), C.c_int32]
        L.cl_gauge_spectrum.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_int32, P(C.c_double), P(C.c_double),
                                        P(C.c_double), C.c_int32, P(C.c_int32)]
        L.cl_spectrum.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_int32, P(C.c_double),
                                  P(C.c_double), P(C.c_double), C.c_int32, P(C.c_int32)]
        L.cl_set_gauge_coupling.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.cl_set_hubble_limit.argtypes = [C.c_void_p, C.c_double]
        L.cl_set_nonminimal.argtypes = [C.c_void_p, C.c_double]
        L.cl_set_adaptive.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        L.cl_enable_gw.argtypes = [C.c_void_p]
        L.cl_gw_spectrum.argtypes = [C.c_void_p, C.c_double, C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double),
                                     C.c_int32, P(C.c_int32)]
        L.cl_set_option.argtypes = [C.c_void_p, C.c_int32, C.c_int64]
        L.cl_get_option.argtypes = [C.c_void_p, C.c_int32, P(C.c_int64)]
        L.cl_last_launch_count.argtypes = [C.c_void_p]
        L.cl_last_launch_count.restype = C.c_int64
        L.cl_strerror.argtypes = [C.c_int]
        L.cl_strerror.restype = C.c_char_p
        L.cl_last_error.argtypes = [C.c_void_p]
        L.cl_last_error.restype = C.c_char_p
        L.cl_fused_pass_noalloc.argtypes = [P(cl_pass_noalloc_desc)]
        fp = P(C.c_float)
        L.cl_surrogate_create.argtypes = [P(C.c_void_p), P(cl_surrogate_params)]
        L.cl_surrogate_free.argtypes = [C.c_void_p]
        L.cl_surrogate_free.restype = None
        L.cl_surrogate_set_weights.argtypes = [C.c_void_p, C.c_int32, fp, fp]
        L.cl_surrogate_get_weights.argtypes = [C.c_void_p, C.c_int32, fp, fp]
        L.cl_surrogate_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        L.cl_surrogate_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        L.cl_surrogate_get_grads.argtypes = [C.c_void_p, C.c_int32, fp, fp]
        L.cl_surrogate_last_launch_count.argtypes = [C.c_void_p]
        L.cl_surrogate_last_launch_count.restype = C.c_int64
        L.cl_surrogate_loss.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, P(C.c_double)]
        L.cl_surrogate_adamw.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_int64]
        L.cl_surrogate_channel_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, fp, fp]
        L.cl_lattice_pack.argtypes = [C.c_void_p, fp, fp, C.c_void_p]
        L.cl_lattice_unpack.argtypes = [C.c_void_p, fp, fp, C.c_void_p]
        L.cl_surrogate_jump.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, fp, fp, C.c_double, P(C.c_int32)]
        L.cl_surrogate_size.argtypes = [C.c_void_p]
        L.cl_autotune.argtypes = [C.c_void_p, C.c_char_p, P(C.c_double)]
        for name in EXPORTS:
            if name not in ("cl_free", "cl_last_launch_count", "cl_strerror", "cl_last_error", "cl_surrogate_free",
                            "cl_surrogate_last_launch_count"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _strerror(s):
    try:
        return lib().cl_strerror(int(s)).decode()
    except ImportError:
        return "status"


def _check(h, s):
    if s != CL_OK:
        msg = lib().cl_last_error(h).decode() if h else ""
        raise CLError(s, msg)


def _buffer(arr, dtype, n):
    """(pointer, on_device, keepalive) for a numpy array or torch CUDA tensor of n elements."""
    if hasattr(arr, "data_ptr"):  # torch tensor
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        if arr.dtype != want or not arr.is_contiguous() or arr.numel() != n:
            raise ValueError("tensor must be contiguous %s with %d elements" % (want, n))
        return C.c_void_p(arr.data_ptr()), int(arr.is_cuda), arr
    a = np.ascontiguousarray(arr, dtype=dtype)
    if a.size != n:
        raise ValueError("array must have %d elements" % n)
    return a.ctypes.data_as(C.c_void_p), 0, a


class Lattice:
    """Owns one cl_lattice handle.  Methods mirror the C calls."""

    def __init__(self, N, L, nfields=1, precision=CL_PREC_FP64, integrator=CL_INT_VV2, gauge=CL_GAUGE_NONE,
                 expansion=True, alpha=1.0, kappa=0.1, dt=0.01, a0=1.0, stream=None, member_N=None, member_L=None,
                 dims=3):
        """A single N^3 lattice (dims 2 / 1: the reduced lattice of N^2 / N sites), or
        (member_N = list of sizes) a batched ensemble whose member m has member_N[m]^3 sites
        and box side member_L[m] (default L)."""
        p = cl_lattice_params()
        p.N, p.nfields, p.precision, p.integrator = int(N), int(nfields), int(precision), int(integrator)
        p.gauge, p.expansion, p.members, p.dims = int(gauge), int(bool(expansion)), 0, int(dims)
        p.L, p.alpha, p.kappa, p.dt, p.a0 = float(L), float(alpha), float(kappa), float(dt), float(a0)
        p.stream = C.c_void_p(int(stream)) if stream else None
        keep = []
        if member_N is not None:
            mn = (C.c_int32 * len(member_N))(*[int(x) for x in member_N])
            keep.append(mn)
            p.members = len(member_N)
            p.member_N = C.cast(mn, C.POINTER(C.c_int32))
            if member_L is not None:
                ml = (C.c_double * len(member_L))(*[float(x) for x in member_L])
                keep.append(ml)
                p.member_L = C.cast(ml, C.POINTER(C.c_double))
        h = C.c_void_p()
        s = lib().cl_init_lattice(C.byref(h), C.byref(p))
        if s != CL_OK:
            raise CLError(s, "cl_init_lattice")
        self.h = h
        self.nfields, self.precision = int(nfields), int(precision)
        self.member_N = [int(x) for x in member_N] if member_N is not None else [int(N)]
        self.members = len(self.member_N)
        self.N = int(N) if member_N is None else max(self.member_N)
        self.dtype = np.float64 if precision == CL_PREC_FP64 else np.float32
        self.dims = int(dims) if dims in (1, 2) else 3
        self.n = self._sites(0)

    def close(self):
        if getattr(self, "h", None):
            lib().cl_free(self.h)
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

    def cl_set_potential(self, kind, params):
        arr = (C.c_double * len(params))(*[float(x) for x in params])
        _check(self.h, lib().cl_set_potential(self.h, int(kind), arr, len(params)))

    def _shape(self, member):
        # lattice shape of a member (z, y, x); an out-of-range member is left for the library to reject
        n = self.member_N[member if 0 <= member < self.members else 0]
        d = self.dims if self.dims in (1, 2) else 3
        return (n if d >= 3 else 1, n if d >= 2 else 1, n)

    def _sites(self, member):
        z, y, x = self._shape(member)
        return z * y * x

    def cl_set_state(self, field, data, member=0):
        ptr, dev, keep = _buffer(data, self.dtype, self._sites(member))
        _check(self.h, lib().cl_set_state(self.h, int(member), int(field), ptr, dev))

    def cl_get_state(self, field, out=None, member=0):
        """Return the field at the latest integer time (numpy), or fill `out` (tensor or array)."""
        if out is None:
            out = np.empty(self._shape(member), dtype=self.dtype)
        ptr, dev, keep = _buffer(out, self.dtype, self._sites(member))
        _check(self.h, lib().cl_get_state(self.h, int(member), int(field), ptr, dev))
        return out

    def cl_set_scalars(self, a, adot=math.nan, t=0.0, member=0):
        _check(self.h, lib().cl_set_scalars(self.h, int(member), float(a), float(adot), float(t)))

    def cl_get_scalars(self, member=0):
        a, b, t = C.c_double(), C.c_double(), C.c_double()
        _check(self.h, lib().cl_get_scalars(self.h, int(member), C.byref(a), C.byref(b), C.byref(t)))
        return a.value, b.value, t.value

    def cl_init_vacuum(self, seed, kcut, amp2, fbar, dfbar=(0.0, 0.0), member=-1):
        v = cl_vacuum_params()
        v.seed, v.kcut, v.amp2 = int(seed), float(kcut), float(amp2)
        for i in range(2):
            v.fbar[i] = float(fbar[i]) if i < len(fbar) else 0.0
            v.dfbar[i] = float(dfbar[i]) if i < len(dfbar) else 0.0
        _check(self.h, lib().cl_init_vacuum(self.h, int(member), C.byref(v)))

    def cl_step(self, nsteps=1):
        _check(self.h, lib().cl_step(self.h, int(nsteps)))

    def cl_sync(self):
        _check(self.h, lib().cl_sync(self.h))

    def cl_energies(self, count=None):
        """Energies of member 0 (a dict), or of members 0..count-1 (a list of dicts)."""
        n = 1 if count is None else int(count)
        e = (cl_energy * n)()
        _check(self.h, lib().cl_energies(self.h, e, n))
        return e[0].as_dict() if count is None else [x.as_dict() for x in e]

    def cl_spectrum(self, field, dn=1.0, type_=1, member=0):
        nb = C.c_int32()
        lib().cl_spectrum(self.h, int(member), int(field), float(dn), int(type_), None, None, None, 0, C.byref(nb))
        n = nb.value
        k, d, c = np.zeros(n), np.zeros(n), np.zeros(n)
        dp = C.POINTER(C.c_double)
        _check(self.h, lib().cl_spectrum(self.h, int(member), int(field), float(dn), int(type_),
                                         k.ctypes.data_as(dp), d.ctypes.data_as(dp), c.ctypes.data_as(dp), n,
                                         C.byref(nb)))
        return k, d, c

    def cl_gauge_spectrum(self, which, dn=1.0, type_=1):
        """Spectra of the U(1) sector: which = CL_GSPEC_E, _B, _APLUS or _AMINUS."""
        nb = C.c_int32()
        lib().cl_gauge_spectrum(self.h, int(which), float(dn), int(type_), None, None, None, 0, C.byref(nb))
        n = nb.value
        k, d, c = np.zeros(n), np.zeros(n), np.zeros(n)
        dp = C.POINTER(C.c_double)
        _check(self.h, lib().cl_gauge_spectrum(self.h, int(which), float(dn), int(type_), k.ctypes.data_as(dp),
                                               d.ctypes.data_as(dp), c.ctypes.data_as(dp), n, C.byref(nb)))
        return k, d, c

    def cl_lattice_pack(self, mu, sg, x):
        """Packed, normalised (phi, pi, a) of this lattice into the CUDA tensor x (N^3 x 3)."""
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sg = np.ascontiguousarray(sg, dtype=np.float32)
        xp, xdev, xk = _buffer(x, np.float32, self.n * 3)
        _check(self.h, lib().cl_lattice_pack(self.h, _fptr(mu), _fptr(sg), xp))

    def cl_lattice_unpack(self, mu, sg, y):
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sg = np.ascontiguousarray(sg, dtype=np.float32)
        yp, ydev, yk = _buffer(y, np.float32, self.n * 2)
        _check(self.h, lib().cl_lattice_unpack(self.h, _fptr(mu), _fptr(sg), yp))

    def cl_set_gauge_coupling(self, alphaL, ws2):
        _check(self.h, lib().cl_set_gauge_coupling(self.h, float(alphaL), float(ws2)))

    def cl_set_nonminimal(self, xi):
        _check(self.h, lib().cl_set_nonminimal(self.h, float(xi)))

    def cl_set_adaptive(self, tol, h_min=0.0, h_max=1e300):
        _check(self.h, lib().cl_set_adaptive(self.h, float(tol), float(h_min), float(h_max)))

    def cl_enable_gw(self):
        _check(self.h, lib().cl_enable_gw(self.h))

    def cl_gw_spectrum(self, dn=1.0, type_=1):
        nb = C.c_int32()
        lib().cl_gw_spectrum(self.h, float(dn), int(type_), None, None, None, 0, C.byref(nb))
        n = nb.value
        k, d, c = np.zeros(n), np.zeros(n), np.zeros(n)
        dp = C.POINTER(C.c_double)
        _check(self.h, lib().cl_gw_spectrum(self.h, float(dn), int(type_), k.ctypes.data_as(dp), d.ctypes.data_as(dp),
                                            c.ctypes.data_as(dp), n, C.byref(nb)))
        return k, d, c

    def cl_set_hubble_limit(self, limit):
        _check(self.h, lib().cl_set_hubble_limit(self.h, float(limit)))

    def cl_set_option(self, option, value):
        _check(self.h, lib().cl_set_option(self.h, int(option), int(value)))

    def cl_get_option(self, option):
        v = C.c_int64()
        _check(self.h, lib().cl_get_option(self.h, int(option), C.byref(v)))
        return v.value

    def cl_last_launch_count(self):
        return int(lib().cl_last_launch_count(self.h))

    def cl_autotune(self, cache_path=None):
        """Pick the fastest tiling from timed trial passes (state unchanged); returns
        (stages, tile_by, tile_dz, microseconds per pass, pass variant)."""
        best = (C.c_double * 5)()
        _check(self.h, lib().cl_autotune(self.h, cache_path.encode() if cache_path else None, best))
        return int(best[0]), int(best[1]), int(best[2]), float(best[3]), int(best[4])


def cl_fused_pass_noalloc(desc):
    """Queue one fused pass on caller-owned device arrays; allocates nothing.  `desc` is a
    cl_pass_noalloc_desc whose pointers are device addresses (e.g. tensor.data_ptr())."""
    s = lib().cl_fused_pass_noalloc(C.byref(desc))
    if s != CL_OK:
        raise CLError(s, "cl_fused_pass_noalloc")


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Surrogate:
    """Owns one cl_surrogate handle (see cl_surrogate_* in cl.h).  Host arrays are float32
    numpy arrays; x has shape (N, N, N, in_channels), weights (27, cout, cin)."""

    def __init__(self, N, in_channels=3, out_channels=2, hidden=48, layers=6, activation=CL_ACT_RELU,
                 precision=CL_SG_BF16, stream=None):
        p = cl_surrogate_params()
        p.N, p.in_channels, p.out_channels, p.hidden = int(N), int(in_channels), int(out_channels), int(hidden)
        p.layers, p.activation, p.precision, p.reserved = int(layers), int(activation), int(precision), 0
        p.stream = C.c_void_p(int(stream)) if stream else None
        h = C.c_void_p()
        st = lib().cl_surrogate_create(C.byref(h), C.byref(p))
        if st != CL_OK:
            raise CLError(st, "cl_surrogate_create")
        self.h = h
        self.N, self.cin, self.cout, self.hidden, self.layers = int(N), int(in_channels), int(out_channels), int(
            hidden), int(layers)
        self.shapes = [((hidden if l else in_channels), (out_channels if l == layers - 1 else hidden))
                       for l in range(layers)]

    def close(self):
        if getattr(self, "h", None):
            lib().cl_surrogate_free(self.h)
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

    def _chk(self, st, what):
        if st != CL_OK:
            raise CLError(st, what)

    def set_weights(self, layer, W, b):
        W = np.ascontiguousarray(W, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        ci, co = self.shapes[layer]
        if W.size != 27 * co * ci or b.size != co:
            raise ValueError("layer %d takes W (27, %d, %d) and b (%d,)" % (layer, co, ci, co))
        self._chk(lib().cl_surrogate_set_weights(self.h, int(layer), _fptr(W), _fptr(b)), "set_weights")

    def get_weights(self, layer):
        ci, co = self.shapes[layer]
        W = np.empty((27, co, ci), np.float32)
        b = np.empty(co, np.float32)
        self._chk(lib().cl_surrogate_get_weights(self.h, int(layer), _fptr(W), _fptr(b)), "get_weights")
        return W, b

    def forward(self, x, out=None):
        """x: (N, N, N, in_channels) float32 numpy array or CUDA tensor; returns y."""
        n = self.N ** 3
        xp, xdev, xk = _buffer(x, np.float32, n * self.cin)
        if out is None:
            out = np.empty((self.N, self.N, self.N, self.cout), np.float32) if not xdev else None
        yp, ydev, yk = _buffer(out, np.float32, n * self.cout)
        self._chk(lib().cl_surrogate_forward(self.h, xp, yp, xdev), "forward")
        return out

    def backward(self, g, want_dx=False):
        n = self.N ** 3
        gp, gdev, gk = _buffer(g, np.float32, n * self.cout)
        dx = np.empty((self.N, self.N, self.N, self.cin), np.float32) if want_dx else None
        self._chk(lib().cl_surrogate_backward(self.h, gp, dx.ctypes.data_as(C.c_void_p) if want_dx else None, gdev),
                  "backward")
        return dx

    def grads(self, layer):
        ci, co = self.shapes[layer]
        dW = np.empty((27, co, ci), np.float32)
        db = np.empty(co, np.float32)
        self._chk(lib().cl_surrogate_get_grads(self.h, int(layer), _fptr(dW), _fptr(db)), "get_grads")
        return dW, db

    def last_launch_count(self):
        return int(lib().cl_surrogate_last_launch_count(self.h))

    def loss(self, target, stride=None, scale=None):
        """Loss of the last forward against target (device tensor or host array with `stride`
        values per site); keeps dL/dy for backward(None)."""
        stride = self.cout if stride is None else int(stride)
        tp, tdev, tk = _buffer(target, np.float32, self.N ** 3 * stride)
        sc = None if scale is None else np.ascontiguousarray(scale, dtype=np.float32)
        out = C.c_double()
        self._chk(lib().cl_surrogate_loss(self.h, tp, stride, None if sc is None else sc.ctypes.data_as(C.c_void_p),
                                          tdev, C.byref(out)), "loss")
        return out.value

    def backward_from_loss(self):
        self._chk(lib().cl_surrogate_backward(self.h, None, None, 1), "backward")

    def adamw(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
        self._chk(lib().cl_surrogate_adamw(self.h, float(lr), float(beta1), float(beta2), float(eps),
                                           float(weight_decay), int(t)), "adamw")

    def channel_stats(self, x, n, channels):
        xp, xdev, xk = _buffer(x, np.float32, int(n) * int(channels))
        mean = np.zeros(3, np.float32)
        std = np.zeros(3, np.float32)
        self._chk(lib().cl_surrogate_channel_stats(self.h, xp, int(n), int(channels), _fptr(mean), _fptr(std)),
                  "channel_stats")
        return mean[:channels], std[:channels]

    def jump(self, lattice, steps, mu, sg, hubble_limit=1e-3):
        """One learned jump of `steps` lattice steps with the leapfrog as fallback; True if accepted."""
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sg = np.ascontiguousarray(sg, dtype=np.float32)
        acc = C.c_int32()
        _check(lattice.h, lib().cl_surrogate_jump(self.h, lattice.h, int(steps), _fptr(mu), _fptr(sg),
                                                  float(hubble_limit), C.byref(acc)))
        return bool(acc.value)
