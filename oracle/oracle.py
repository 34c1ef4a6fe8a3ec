"""ctypes wrapper of the FP64 CPU oracle -- test infrastructure only.

Arrays are numpy float64 in C order with shape (N, N, N) indexed [z, y, x]
(x fastest), matching the oracle's site index n = (z*N + y)*N + x.  The
functions only marshal arguments; every step of the arithmetic is in the C
files of this folder.
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build_oracle

VV2, YOSHIDA4, RK3_3, RK4_5, YOSHIDA6, YOSHIDA8, YOSHIDA10, RK3_4 = 0, 1, 2, 3, 4, 5, 6, 7
E_NAMES = ["K0", "K1", "G0", "G1", "V", "KEM", "GEM", "rho", "p", "hubble_violation", "a", "b"]


class Model(C.Structure):
    _fields_ = [("N", C.c_int32), ("nf", C.c_int32), ("expansion", C.c_int32), ("gauge", C.c_int32),
                ("L", C.c_double), ("alpha", C.c_double), ("kappa", C.c_double),
                ("m2", C.c_double * 2), ("lam", C.c_double * 2), ("g2", C.c_double),
                ("alphaL", C.c_double), ("ws2", C.c_double), ("nmc", C.c_int32), ("xi", C.c_double),
                ("dims", C.c_int32)]


_lib = None
_libs = {}


def use_threads(on):
    """Select the loop-parallel build (liboracle_omp.so, all host cores) for the calls that
    follow, or the serial one.  Only the CPU-baseline timing turns it on."""
    global _lib
    _lib = _load(bool(on))


def threads():
    """Threads the selected build runs its loops on."""
    return int(lib().orc_threads())


def lib():
    global _lib
    if _lib is None:
        _lib = _load(False)
    return _lib


def _load(omp):
    if omp not in _libs:
        path = build_oracle.build(omp=omp)
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        mp = C.POINTER(Model)
        L.orc_V.restype = C.c_double
        L.orc_V.argtypes = [mp, C.c_double, C.c_double]
        L.orc_dV.restype = C.c_double
        L.orc_dV.argtypes = [mp, C.c_int, C.c_double, C.c_double]
        L.orc_laplacian.argtypes = [C.c_int, C.c_double, dp, dp]
        L.orc_grad2_sum.restype = C.c_double
        L.orc_grad2_sum.argtypes = [C.c_int, dp]
        L.orc_kick_force.argtypes = [mp, C.c_int, dp, C.c_double, dp]
        L.orc_energies.argtypes = [mp, dp, dp, C.c_void_p, C.c_void_p, dp, dp]
        L.orc_addot.restype = C.c_double
        L.orc_addot.argtypes = [mp, C.c_double, C.c_double, C.c_double]
        L.orc_step.argtypes = [mp, C.c_int, C.c_double, C.c_int, dp, dp, C.c_void_p, C.c_void_p, dp]
        L.orc_u1_gauss.argtypes = [mp, dp, dp, dp, C.c_double, dp]
        L.orc_u1_rhs.argtypes = [mp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_u1_leapfrog.argtypes = [mp, C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_dft3.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_vacuum.argtypes = [mp, C.c_uint64, C.c_uint32, C.c_double, C.c_double, dp, dp, C.c_double,
                                 dp, dp, dp]
        L.orc_spectrum.restype = C.c_int
        L.orc_spectrum.argtypes = [C.c_int, C.c_double, dp, C.c_double, C.c_int, dp, dp, dp, C.c_int]
        L.orc_gw_force.argtypes = [mp, dp, dp, C.c_double, dp]
        L.orc_step_gw.argtypes = [mp, C.c_int, C.c_double, C.c_int, dp, dp, dp, dp, dp]
        L.orc_gw_spectrum.restype = C.c_int
        L.orc_gw_spectrum.argtypes = [mp, dp, dp, C.c_double, C.c_int, dp, dp, dp, C.c_int]
        L.orc_nmc_ricci.restype = C.c_double
        L.orc_nmc_ricci.argtypes = [mp, dp, dp, dp]
        L.orc_gauge_spectrum.restype = C.c_int
        L.orc_gauge_spectrum.argtypes = [mp, dp, dp, C.c_int, C.c_double, C.c_int, dp, dp, dp, C.c_int]
        L.orc_conv3d_fwd.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_void_p, dp]
        L.orc_conv3d_bwd_data.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
        L.orc_conv3d_bwd_weight.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_void_p]
        L.orc_act.restype = C.c_double
        L.orc_act.argtypes = [C.c_int, C.c_double]
        L.orc_act_grad.restype = C.c_double
        L.orc_act_grad.argtypes = [C.c_int, C.c_double]
        L.orc_act_array.argtypes = [C.c_int, C.c_int64, dp, dp]
        L.orc_act_bwd_array.argtypes = [C.c_int, C.c_int64, dp, dp, dp]
        L.orc_step_adaptive.argtypes = [mp, C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double, C.c_int,
                                         dp, dp, dp, dp, dp]
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = []
        _libs[omp] = L
    return _libs[omp]


def make_model(N, L, nf=1, alpha=1.0, kappa=0.0, expansion=False, m2=(0.0, 0.0), lam=(0.0, 0.0),
               g2=0.0, gauge=0, alphaL=0.0, ws2=0.0, xi=None, dims=3):
    """xi: non-minimal coupling of field 0 (None: minimally coupled).  dims: 3, or 2 / 1 for
    the reduced (2+1) / (1+1)-dimensional lattice of N^2 / N sites."""
    m = Model()
    m.dims = int(dims)
    m.nmc, m.xi = (0, 0.0) if xi is None else (1, float(xi))
    m.N, m.nf, m.expansion, m.gauge = int(N), int(nf), int(bool(expansion)), int(gauge)
    m.L, m.alpha, m.kappa = float(L), float(alpha), float(kappa)
    m.m2[0], m.m2[1] = float(m2[0]), float(m2[1])
    m.lam[0], m.lam[1] = float(lam[0]), float(lam[1])
    m.g2, m.alphaL, m.ws2 = float(g2), float(alphaL), float(ws2)
    return m


@dataclasses.dataclass
class State:
    phi: np.ndarray            # (nf, N, N, N)
    pi: np.ndarray             # (nf, N, N, N)
    abt: np.ndarray            # (3,) = a, a', t
    links: np.ndarray = None   # (3, N, N, N) theta_i = dx A_i
    efield: np.ndarray = None  # (3, N, N, N)

    def copy(self):
        return State(self.phi.copy(), self.pi.copy(), self.abt.copy(),
                     None if self.links is None else self.links.copy(),
                     None if self.efield is None else self.efield.copy())


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def extents(model):
    """(nz, ny, nx) of the model's lattice: 1 along the directions a reduced lattice lacks."""
    d = model.dims if model.dims in (1, 2) else 3
    N = model.N
    return (N if d >= 3 else 1, N if d >= 2 else 1, N)


def new_state(model, a=1.0, b=0.0, t=0.0):
    nf = model.nf
    shape = (nf,) + extents(model)
    st = State(np.zeros(shape), np.zeros(shape), np.array([a, b, t], dtype=np.float64))
    if model.gauge == 1:
        N = model.N
        st.links = np.zeros((3, N, N, N))
        st.efield = np.zeros((3, N, N, N))
    return st


def step(model, st, scheme, h, nsteps=1):
    """Advance `st` in place by nsteps steps of size h."""
    st.phi, st.pi, st.abt = _c(st.phi), _c(st.pi), _c(st.abt)
    if st.links is not None:
        st.links, st.efield = _c(st.links), _c(st.efield)
    lib().orc_step(C.byref(model), int(scheme), float(h), int(nsteps), st.phi, st.pi,
                   _ptr(st.links), _ptr(st.efield), st.abt)
    return st


def u1_leapfrog(model, st, h, nsteps=1, iters=3):
    """Leapfrog steps of a U(1) + axion state with `iters` fixed-point evaluations of the
    implicit momentum kick (step(..., VV2, ...) takes 3)."""
    st.phi, st.pi, st.abt = _c(st.phi), _c(st.pi), _c(st.abt)
    st.links, st.efield = _c(st.links), _c(st.efield)
    lib().orc_u1_leapfrog(C.byref(model), float(h), int(nsteps), int(iters), st.phi, st.pi, st.links, st.efield,
                          st.abt)
    return st


def step_adaptive(model, st, h, tol, nsteps, hmin=0.0, hmax=1e300):
    """Adaptive RK3-4 steps (always accepted; the next h from the embedded error estimate).
    Returns (h_next, h_used[nsteps], eps[nsteps])."""
    st.phi, st.pi, st.abt = _c(st.phi), _c(st.pi), _c(st.abt)
    hh = C.c_double(float(h))
    hu, ep = np.zeros(nsteps), np.zeros(nsteps)
    lib().orc_step_adaptive(C.byref(model), C.byref(hh), float(tol), float(hmin), float(hmax), int(nsteps),
                            st.phi, st.pi, st.abt, hu, ep)
    return hh.value, hu, ep


def energies(model, st):
    out = np.zeros(len(E_NAMES))
    lib().orc_energies(C.byref(model), _c(st.phi), _c(st.pi),
                       _ptr(None if st.links is None else _c(st.links)),
                       _ptr(None if st.efield is None else _c(st.efield)), _c(st.abt), out)
    return dict(zip(E_NAMES, out))


def gw_force(model, phi, gv, a):
    out = np.zeros_like(_c(gv))
    lib().orc_gw_force(C.byref(model), _c(phi), _c(gv), float(a), out)
    return out


def step_gw(model, st, gv, gp, scheme, h, nsteps=1):
    """Leapfrog steps of the scalars (st) and the five GW auxiliaries gv, gp (5, N, N, N), in place."""
    st.phi, st.pi, st.abt = _c(st.phi), _c(st.pi), _c(st.abt)
    assert gv.flags.c_contiguous and gp.flags.c_contiguous and gv.dtype == np.float64 and gp.dtype == np.float64
    lib().orc_step_gw(C.byref(model), int(scheme), float(h), int(nsteps), st.phi, st.pi, gv, gp, st.abt)
    return st


def gw_spectrum(model, gp, abt, dn=1.0, type_=1):
    N = model.N
    cap = int(np.floor(np.sqrt(3.0) * (N // 2) / dn + 0.5)) + 2
    k, d, c = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    nb = lib().orc_gw_spectrum(C.byref(model), _c(gp), _c(abt), float(dn), int(type_), k, d, c, cap)
    return k[:nb], d[:nb], c[:nb]


def nmc_ricci(model, st):
    return lib().orc_nmc_ricci(C.byref(model), _c(st.phi), _c(st.pi), _c(st.abt))


def addot(model, a, rho, p):
    return lib().orc_addot(C.byref(model), float(a), float(rho), float(p))


def potential(model, f0, f1=0.0):
    return lib().orc_V(C.byref(model), float(f0), float(f1))


def laplacian(N, dx, f):
    out = np.zeros((N, N, N))
    lib().orc_laplacian(int(N), float(dx), _c(f), out)
    return out


def grad2_sum(N, f):
    return lib().orc_grad2_sum(int(N), _c(f))


def kick_force(model, phi, f, a):
    N = model.N
    out = np.zeros((N, N, N))
    lib().orc_kick_force(C.byref(model), int(f), _c(phi), float(a), out)
    return out


def u1_gauss(model, st):
    N = model.N
    out = np.zeros((N, N, N))
    lib().orc_u1_gauss(C.byref(model), _c(st.phi), _c(st.links), _c(st.efield), float(st.abt[0]), out)
    return out


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def dft3(f_re, f_im=None, sign=-1):
    N = f_re.shape[0]
    re = _c(f_re).copy()
    im = np.zeros_like(re) if f_im is None else _c(f_im).copy()
    lib().orc_dft3(int(N), int(sign), re, im)
    return re + 1j * im


def vacuum(model, seed, kcut, amp2, fbar, dfbar, a0=1.0, member=0):
    st = new_state(model, a=a0)
    fb = np.zeros(2)
    dfb = np.zeros(2)
    fb[:len(fbar)] = fbar
    dfb[:len(dfbar)] = dfbar
    lib().orc_vacuum(C.byref(model), int(seed), int(member), float(kcut), float(amp2), fb, dfb, float(a0),
                     st.phi, st.pi, st.abt)
    return st


def spectrum(N, L, f, dn=1.0, type_=1):
    cap = int(np.floor(np.sqrt(3.0) * (N // 2) / dn + 0.5)) + 2
    k = np.zeros(cap)
    d = np.zeros(cap)
    c = np.zeros(cap)
    nb = lib().orc_spectrum(int(N), float(L), _c(f), float(dn), int(type_), k, d, c, cap)
    return k[:nb], d[:nb], c[:nb]


def gauge_spectrum(model, st, which, dn=1.0, type_=1):
    """which: 0 electric, 1 magnetic, 2 / 3 the + / - chirality of the gauge potential."""
    N = model.N
    cap = int(np.floor(np.sqrt(3.0) * (N // 2) / dn + 0.5)) + 2
    k = np.zeros(cap)
    d = np.zeros(cap)
    c = np.zeros(cap)
    nb = lib().orc_gauge_spectrum(C.byref(model), _c(st.links), _c(st.efield), int(which), float(dn), int(type_),
                                  k, d, c, cap)
    return k[:nb], d[:nb], c[:nb]


def u1_rhs(model, st):
    """Right-hand side (dphi, dpi, dtheta, dE) of the axion-U(1) system at st (a, a' fixed)."""
    N = model.N
    out = [np.zeros((1, N, N, N)), np.zeros((1, N, N, N)), np.zeros((3, N, N, N)), np.zeros((3, N, N, N))]
    lib().orc_u1_rhs(C.byref(model), _c(st.phi), _c(st.pi), _c(st.links), _c(st.efield), _c(st.abt), *out)
    return out


# ------------------------------------------------------------------ convolutional surrogate
# Activations are arrays of shape (N, N, N, C) (site-major, channels last); weights
# W[27, cout, cin] with tap t = (tz*3 + ty)*3 + tx at offset (tx-1, ty-1, tz-1), bias b[cout].
RELU, GELU = 0, 1


def conv3d_fwd(x, W, b=None):
    N, cin = x.shape[0], x.shape[3]
    cout = W.shape[1]
    y = np.zeros((N, N, N, cout))
    bb = None if b is None else _c(b)
    lib().orc_conv3d_fwd(N, cin, cout, _c(x), _c(W), _ptr(bb), y)
    return y


def conv3d_bwd_data(dy, W):
    N, cout = dy.shape[0], dy.shape[3]
    cin = W.shape[2]
    dx = np.zeros((N, N, N, cin))
    lib().orc_conv3d_bwd_data(N, cin, cout, _c(dy), _c(W), dx)
    return dx


def conv3d_bwd_weight(x, dy):
    N, cin, cout = x.shape[0], x.shape[3], dy.shape[3]
    dW = np.zeros((27, cout, cin))
    db = np.zeros(cout)
    lib().orc_conv3d_bwd_weight(N, cin, cout, _c(x), _c(dy), dW, db.ctypes.data_as(C.c_void_p))
    return dW, db


def activation(act, u):
    u = _c(u)
    h = np.empty_like(u)
    lib().orc_act_array(int(act), u.size, u, h)
    return h


def activation_bwd(act, u, dh):
    u, dh = _c(u), _c(dh)
    du = np.empty_like(u)
    lib().orc_act_bwd_array(int(act), u.size, u, dh, du)
    return du


def surrogate_forward(x, layers, act=RELU):
    """Network of periodic 3x3x3 convolutions: h_0 = x, h_{l+1} = act(conv_l(h_l)) for all but
    the last layer, out = x[..., :cout_last] + conv_last(h_last) (the residual jump).
    layers: list of (W, b).  Returns (out, cache) with cache = (inputs h_l, pre-activations u_l)."""
    h, us, hs = _c(x), [], []
    for i, (W, b) in enumerate(layers):
        hs.append(h)
        u = conv3d_fwd(h, W, b)
        us.append(u)
        h = activation(act, u) if i + 1 < len(layers) else u
    cout = layers[-1][0].shape[1]
    out = x[..., :cout] + h
    return out, (hs, us)


def surrogate_backward(cache, layers, g, act=RELU):
    """Gradients of sum(out * g): returns (dx, [(dW_l, db_l)])."""
    hs, us = cache
    grads = [None] * len(layers)
    du = _c(g)
    for i in range(len(layers) - 1, -1, -1):
        W = layers[i][0]
        grads[i] = conv3d_bwd_weight(hs[i], du)
        dh = conv3d_bwd_data(du, W)
        du = activation_bwd(act, us[i - 1], dh) if i > 0 else dh
    dx = du.copy()
    dx[..., :g.shape[3]] += g
    return dx, grads
