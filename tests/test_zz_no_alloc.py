"""The allocation-free fused pass (cl_fused_pass_noalloc) against cl_step.

cl_fused_pass_noalloc serves callers that cannot allocate device memory when they
step a lattice (an application's fixed memory arena, hosts that forbid allocation
after start-up): it runs the fused-pass kernel on their own arrays and keeps its
scratch in a fixed static device array.  Here it runs velocity Verlet in staggered
form on caller-owned tensors -- an opening half kick, then two step passes in a row,
each followed by a synchronisation of the momenta into separate buffers -- and both
steps must agree with cl_step on a library-owned lattice from the same state, within
the tolerances of the other GPU tests (1e-10 FP64, 1e-4 FP32).  The device's free
memory must not change across the step passes.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# (precision, fields, N, tolerance): FP64 and FP32 + Kahan with two fields; plain FP32 with one
# field on an odd N (one element per thread) and on N = 390, whose 390 x 25 blocks of one row
# and 16 planes exceed the scratch's 8192 blocks, so that every block marches more planes.
CASES = [(0, 2, 32, 1e-10), (1, 2, 32, 1e-4), (2, 1, 33, 1e-4), (2, 1, 390, 1e-4)]


@pytest.mark.parametrize("prec,nf,N,tol", CASES)
def test_noalloc_pass_matches_cl_step(prec, nf, N, tol):
    import torch

    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    box, dt = 10.0 * N / 32, 0.01
    alpha, kappa, a0, b0 = 1.0, 0.3, 1.0, 0.2
    pot = [0.5, 1.0, 0.2, 0.0, 3.0] if nf == 2 else [0.5, 1.0, 0.0, 0.0, 0.0]  # m2_0, lam_0, m2_1, lam_1, g2
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
    torch.cuda.empty_cache()

    # caller-owned device buffers, all allocated before the first pass
    dev = "cuda"
    buf = lambda: [torch.zeros(N ** 3, dtype=t_t, device=dev) for _ in range(nf)]
    A_phi, A_pi, A_c = buf(), buf(), buf()     # state (ping)
    B_phi, B_pi, B_c = buf(), buf(), buf()     # state (pong)
    Sy = [(buf(), buf(), buf()) for _ in range(2)]  # synchronised copies for comparison
    for f in range(nf):
        A_phi[f].copy_(torch.from_numpy(phi[f].astype(np_t).ravel()))
        A_pi[f].copy_(torch.from_numpy(pi[f].astype(np_t).ravel()))
    scal = torch.tensor([a0, b0, 0.0], dtype=torch.float64, device=dev)
    sync_scal = [torch.zeros(3, dtype=torch.float64, device=dev) for _ in range(2)]
    energies = [torch.zeros(14, dtype=torch.float64, device=dev) for _ in range(2)]
    status = torch.full((3,), -1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def run(src, dst, coef, scalars, en, st):
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
        d.energies = None if en is None else en.data_ptr()
        d.status = None if st is None else st.data_ptr()
        d.stream = stream
        cl.cl_fused_pass_noalloc(d)

    A, B = (A_phi, A_pi, A_c), (B_phi, B_pi, B_c)
    h = dt
    run(A, B, (0.0, 0.0, 0.5 * h), scal, None, status[0:1])  # open the leapfrog (first call: set-up)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    cur, nxt = B, A
    for step in range(2):                   # two step passes in a row, each synchronised aside
        run(cur, nxt, (h, 0.5 * h, h), scal, None, None)
        cur, nxt = nxt, cur
        sync_scal[step].copy_(scal)
        run(cur, Sy[step], (0.0, -0.5 * h, -0.5 * h), sync_scal[step], energies[step], status[step + 1:step + 2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # the passes allocated no device memory
    assert status.cpu().tolist() == [0, 0, 0]

    for step in range(2):
        gphi = np.stack([Sy[step][0][f].cpu().numpy().reshape(N, N, N) for f in range(nf)])
        gpi = np.stack([Sy[step][1][f].cpu().numpy().reshape(N, N, N) for f in range(nf)])
        rphi, rpi, (ra, rb, rt) = ref[step]
        assert rel_l2(gphi, rphi) < tol
        assert rel_l2(gpi, rpi) < tol
        a, b, t = sync_scal[step].cpu().tolist()
        assert a == pytest.approx(ra, rel=tol)
        assert b == pytest.approx(rb, rel=tol)
        assert t == pytest.approx(rt, rel=1e-12)
        e = energies[step].cpu().numpy()
        assert e[1] == pytest.approx(ra, rel=tol) and np.isfinite(e[10]) and e[10] > 0


def test_noalloc_allocates_nothing():
    """Free device memory is unchanged across repeated passes (after the first call's set-up)."""
    import torch

    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    N, nf, prec = 64, 1, cl.CL_PREC_FP32_KAHAN
    arr = [torch.zeros(N ** 3, dtype=torch.float32, device="cuda") for _ in range(6)]
    arr[0] += 1.0
    scal = torch.tensor([1.0, 0.0, 0.0], dtype=torch.float64, device="cuda")
    d = cl.cl_pass_noalloc_desc()
    d.N, d.nfields, d.precision, d.expansion, d.L, d.alpha = N, nf, prec, 0, 20.0, 1.0
    d.m2[0], d.lam[0] = 1.0, 1.0
    d.drift, d.energy_kick, d.kick = 0.01, 0.005, 0.01
    d.phi_in[0], d.pi_in[0], d.c_in[0] = arr[0].data_ptr(), arr[1].data_ptr(), arr[2].data_ptr()
    d.phi_out[0], d.pi_out[0], d.c_out[0] = arr[3].data_ptr(), arr[4].data_ptr(), arr[5].data_ptr()
    d.scalars = scal.data_ptr()
    d.stream = torch.cuda.current_stream().cuda_stream
    cl.cl_fused_pass_noalloc(d)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        cl.cl_fused_pass_noalloc(d)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_bad_descriptors():
    import torch

    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()

    def expect_einval(d):
        with pytest.raises(cl.CLError) as ei:
            cl.cl_fused_pass_noalloc(d)
        assert ei.value.status == cl.CL_EINVAL

    d = cl.cl_pass_noalloc_desc()
    d.N, d.nfields, d.precision, d.L = 1, 1, 0, 1.0  # N too small
    expect_einval(d)

    # FP64 rows of 1535 one-element threads do not fit a 512-thread block
    d = cl.cl_pass_noalloc_desc()
    d.N, d.nfields, d.precision, d.L = 1535, 1, cl.CL_PREC_FP64, 1.0
    for k in ("phi_in", "pi_in", "phi_out", "pi_out"):
        getattr(d, k)[0] = 256
    d.scalars = 256
    expect_einval(d)

    N = 16
    dev = [torch.zeros(N ** 3, dtype=torch.float32, device="cuda") for _ in range(8)]
    scal = torch.tensor([1.0, 0.0, 0.0], dtype=torch.float64, device="cuda")

    def desc(phi_in, pi_in, phi_out, pi_out, scalars):
        d = cl.cl_pass_noalloc_desc()
        d.N, d.nfields, d.precision, d.L, d.alpha = N, 2, cl.CL_PREC_FP32, 5.0, 1.0
        d.phi_in[0], d.phi_in[1] = phi_in
        d.pi_in[0], d.pi_in[1] = pi_in
        d.phi_out[0], d.phi_out[1] = phi_out
        d.pi_out[0], d.pi_out[1] = pi_out
        d.scalars = scalars
        return d

    p = [t.data_ptr() for t in dev]
    # an output that is another field's input
    expect_einval(desc((p[0], p[1]), (p[2], p[3]), (p[4], p[5]), (p[1], p[7]), scal.data_ptr()))
    # two outputs in the same buffer
    expect_einval(desc((p[0], p[1]), (p[2], p[3]), (p[4], p[5]), (p[6], p[4]), scal.data_ptr()))
    # an output that overlaps an input partly
    expect_einval(desc((p[0], p[1]), (p[2], p[3]), (p[4], p[5]), (p[6], p[3] + 4 * 100), scal.data_ptr()))
    # host memory for the scalars
    host = np.zeros(3)
    expect_einval(desc((p[0], p[1]), (p[2], p[3]), (p[4], p[5]), (p[6], p[7]), host.ctypes.data))
    # the same descriptor with device scalars is accepted
    cl.cl_fused_pass_noalloc(desc((p[0], p[1]), (p[2], p[3]), (p[4], p[5]), (p[6], p[7]), scal.data_ptr()))
    torch.cuda.synchronize()
