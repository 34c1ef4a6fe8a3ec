"""The allocation-free fused pass (cl_fused_pass_noalloc) against cl_step.

cl_fused_pass_noalloc serves callers that cannot allocate device memory when they
step a lattice (an application's fixed memory arena, hosts that forbid allocation
after start-up): it runs the fused-pass kernel on their own arrays and keeps its
scratch in a fixed static device array.  Here it runs velocity Verlet in staggered
form on caller-owned tensors -- an opening half kick, then two step passes in a row,
each followed by a synchronisation of the momenta into separate buffers -- and both
steps must agree with cl_step on a library-owned lattice from the same state, within
the tolerances of the other GPU tests (1e-10 FP64, 1e-4 FP32 + Kahan).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_noalloc_pass_matches_cl_step(prec, tol):
    import torch

    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    N, nf, box, dt = 32, 2, 10.0, 0.01
    alpha, kappa, a0, b0 = 1.0, 0.3, 1.0, 0.2
    pot = [0.5, 1.0, 0.2, 0.0, 3.0]  # m2_0, lam_0, m2_1, lam_1, g2
    phi, pi = inputs.scalar_state(N, nf, seed=21, fbar=(1.0, 0.1), amp=0.05, pamp=0.05)
    np_t = np.float64 if prec == 0 else np.float32
    t_t = torch.float64 if prec == 0 else torch.float32

    # reference: the library-owned lattice, two cl_step calls
    ref = []
    with cl.Lattice(N, box, nf, prec, cl.CL_INT_VV2, expansion=True, alpha=alpha, kappa=kappa, dt=dt) as g:
        g.cl_set_potential(cl.CL_POT_POLY, pot)
        for f in range(nf):
            g.cl_set_state(cl.CL_FIELD_PHI0 + f, phi[f].astype(np_t))
            g.cl_set_state(cl.CL_FIELD_PI0 + f, pi[f].astype(np_t))
        g.cl_set_scalars(a0, b0, 0.0)
        for _ in range(2):
            g.cl_step(1)
            ref.append((np.stack([g.cl_get_state(cl.CL_FIELD_PHI0 + f) for f in range(nf)]),
                        np.stack([g.cl_get_state(cl.CL_FIELD_PI0 + f) for f in range(nf)]),
                        g.cl_get_scalars()))

    # caller-owned device buffers
    dev = "cuda"
    buf = lambda: [torch.zeros(N ** 3, dtype=t_t, device=dev) for _ in range(nf)]
    A_phi, A_pi, A_c = buf(), buf(), buf()     # state (ping)
    B_phi, B_pi, B_c = buf(), buf(), buf()     # state (pong)
    S_phi, S_pi, S_c = buf(), buf(), buf()     # synchronised copy for comparison
    for f in range(nf):
        A_phi[f].copy_(torch.from_numpy(phi[f].astype(np_t).ravel()))
        A_pi[f].copy_(torch.from_numpy(pi[f].astype(np_t).ravel()))
    scal = torch.tensor([a0, b0, 0.0], dtype=torch.float64, device=dev)
    energies = torch.zeros(14, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def run(src, dst, coef, scalars):
        d = cl.cl_pass_noalloc_desc()
        d.N, d.nfields, d.precision, d.expansion = N, nf, prec, 1
        d.L, d.alpha, d.kappa = box, alpha, kappa
        d.m2[0], d.lam[0], d.m2[1], d.lam[1], d.g2 = pot
        d.drift, d.energy_kick, d.kick = coef
        for f in range(nf):
            d.phi_in[f], d.pi_in[f], d.c_in[f] = (src[0][f].data_ptr(), src[1][f].data_ptr(),
                                                  src[2][f].data_ptr())
            d.phi_out[f], d.pi_out[f], d.c_out[f] = (dst[0][f].data_ptr(), dst[1][f].data_ptr(),
                                                     dst[2][f].data_ptr())
        d.scalars = scalars.data_ptr()
        d.energies = energies.data_ptr()
        d.stream = stream
        cl.cl_fused_pass_noalloc(d)

    A, B, Sy = (A_phi, A_pi, A_c), (B_phi, B_pi, B_c), (S_phi, S_pi, S_c)
    h = dt
    run(A, B, (0.0, 0.0, 0.5 * h), scal)  # open the leapfrog
    cur, nxt = B, A
    for step in range(2):                   # two step passes in a row
        run(cur, nxt, (h, 0.5 * h, h), scal)
        cur, nxt = nxt, cur
        sync_scal = scal.clone()
        run(cur, Sy, (0.0, -0.5 * h, -0.5 * h), sync_scal)
        torch.cuda.synchronize()
        got_phi = np.stack([S_phi[f].cpu().numpy().reshape(N, N, N) for f in range(nf)])
        got_pi = np.stack([S_pi[f].cpu().numpy().reshape(N, N, N) for f in range(nf)])
        rphi, rpi, (ra, rb, rt) = ref[step]
        assert rel_l2(got_phi, rphi) < tol
        assert rel_l2(got_pi, rpi) < tol
        a, b, t = sync_scal.cpu().tolist()
        assert a == pytest.approx(ra, rel=tol)
        assert b == pytest.approx(rb, rel=tol)
        assert t == pytest.approx(rt, rel=1e-12)
        e = energies.cpu().numpy()
        assert e[1] == pytest.approx(ra, rel=tol) and np.isfinite(e[10])


def test_noalloc_rejects_bad_descriptors():
    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    d = cl.cl_pass_noalloc_desc()
    d.N, d.nfields, d.precision, d.L = 1, 1, 0, 1.0  # N too small
    with pytest.raises(cl.CLError) as ei:
        cl.cl_fused_pass_noalloc(d)
    assert ei.value.status == cl.CL_EINVAL
