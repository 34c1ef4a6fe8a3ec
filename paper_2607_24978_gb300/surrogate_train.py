"""Training and evaluation driver of the convolutional surrogate.

Orchestration only: trajectories come from the library's own leapfrog, and every
arithmetic step (packing and normalising the state, forward, loss, backward, AdamW, the
jump with its Friedmann update and its Hubble-constraint fallback, spectra) runs in
libcl.so's kernels.  The driver only decides what to call in which order.

All work (lattices, networks and the device tensors that carry states between them) is
ordered on one CUDA stream, which the caller makes torch's current stream
(`with torch.cuda.stream(st)`) and passes to every handle, so that no copy or kernel of one
handle can race another's.

Workload: lambda phi^4 in program units (V = phi^4/4, alpha = 1, the coupling entering
through the vacuum amplitude), a homogeneous phi = 1 plus vacuum fluctuations, FP32 +
Kahan VV-2.  The network is local and translation invariant, so it is trained on small
lattices and applied to a larger one with the same lattice spacing.
"""
import math
import time

import numpy as np

from . import cl


def make_lattice(N, seed, dx=0.25 * math.pi, dt=0.01, amp2=1e-4, kappa=0.1, stream=None):
    """lambda phi^4 lattice with lattice spacing dx (the box grows with N)."""
    g = cl.Lattice(N, dx * N, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, expansion=True, alpha=1.0, kappa=kappa,
                   dt=dt, stream=stream)
    g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
    kcut = 16 * 2 * math.pi / (dx * 32)  # the cut of the 32^3, L = 8 pi parity workload
    g.cl_init_vacuum(int(seed), kcut, amp2, (1.0,), (0.0,))
    return g


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


def generate(torch, N, seeds, per_traj, K, warm, mu, sg, dx=0.25 * math.pi, dt=0.01):
    """Pairs (x(t), x(t + K dt)) of packed, normalised states (N^3 x 3 device tensors)."""
    pairs = []
    for sd in seeds:
        with make_lattice(N, sd, dx=dx, dt=dt, stream=_stream(torch)) as g:
            g.cl_step(warm)
            x = torch.empty(N ** 3 * 3, device="cuda")
            g.cl_lattice_pack(mu, sg, x)
            for _ in range(per_traj):
                g.cl_step(K)
                y = torch.empty(N ** 3 * 3, device="cuda")
                g.cl_lattice_pack(mu, sg, y)
                pairs.append((x, y))
                x = y
    torch.cuda.synchronize()
    return pairs


def normalisation(torch, s, N, seed, K, warm, dx=0.25 * math.pi, dt=0.01):
    """Per-channel mean and spread of the packed state, and the rms K-step change of phi and pi
    in those units (the loss scale).  `s` must still be the untrained network, whose zero last
    layer makes it the identity jump: its loss against the state K steps later is the mean
    square change."""
    one = np.ones(3, np.float32)
    zero = np.zeros(3, np.float32)
    n = N ** 3
    with make_lattice(N, seed, dx=dx, dt=dt, stream=_stream(torch)) as g:
        g.cl_step(warm)
        raw = torch.empty(n * 3, device="cuda")
        g.cl_lattice_pack(zero, one, raw)
        mean, std = s.channel_stats(raw, n, 3)
        mu = mean.astype(np.float32)
        sg = np.maximum(std, 1e-6).astype(np.float32)
        sg[2] = max(sg[2], 1.0)  # a is homogeneous: no spread to normalise by
        x0 = torch.empty(n * 3, device="cuda")
        g.cl_lattice_pack(mu, sg, x0)
        g.cl_step(K)
        x1 = torch.empty(n * 3, device="cuda")
        g.cl_lattice_pack(mu, sg, x1)
    s.forward(x0, torch.empty(n * 2, device="cuda"))
    scale = np.zeros(2, np.float32)
    for c in range(2):  # isolate one channel by giving the other a huge scale
        sc = np.full(2, 1e30, np.float32)
        sc[c] = 1.0
        scale[c] = math.sqrt(2.0 * s.loss(x1, stride=3, scale=sc))
    return mu, sg, np.maximum(scale, 1e-6)


def train(torch, N=32, hidden=48, layers=6, K=16, seeds=(1, 2, 3, 4), per_traj=24, warm=50, iters=400, lr=2e-3,
          act=cl.CL_ACT_RELU, log=None):
    """Train a surrogate on leapfrog trajectories; returns (surrogate, mu, sg, info).  Call with a
    non-default torch stream current (see the module docstring)."""
    if _stream(torch) in (0, None):
        raise ValueError("run the driver under `with torch.cuda.stream(torch.cuda.Stream())`")
    s = cl.Surrogate(N, 3, 2, hidden, layers, act, cl.CL_SG_BF16, stream=_stream(torch))
    rg = np.random.default_rng(1234)
    for l, (ci, co) in enumerate(s.shapes):  # He-scaled start; the last layer starts at zero (identity jump)
        W = rg.standard_normal((27, co, ci)) * math.sqrt(2.0 / (27 * ci)) if l < layers - 1 else np.zeros((27, co, ci))
        s.set_weights(l, W, np.zeros(co))
    mu, sg, scale = normalisation(torch, s, N, seeds[0], K, warm)
    t0 = time.perf_counter()
    pairs = generate(torch, N, seeds, per_traj, K, warm, mu, sg)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = []
    for it in range(1, iters + 1):
        x, y = pairs[int(rg.integers(len(pairs)))]
        s.forward(x, torch.empty(N ** 3 * 2, device="cuda"))
        L = s.loss(y, stride=3, scale=scale)
        s.backward_from_loss()
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / iters))  # cosine schedule
        s.adamw(lr_t, it)
        losses.append(L)
        if log and (it % 100 == 0 or it == 1):
            log("iter %d loss %.4g" % (it, L))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    info = {"train_N": N, "pairs": len(pairs), "iters": iters, "K": K, "generate_s": t_gen, "train_s": t_train,
            "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:]))}
    return s, mu, sg, info


def spectrum_error(g_ref, g_test, field=cl.CL_FIELD_PHI0):
    """Largest relative difference of the binned Type-I spectra over the populated bins."""
    _, d_ref, c = g_ref.cl_spectrum(field)
    _, d_test, _ = g_test.cl_spectrum(field)
    m = (c > 0) & (np.arange(len(c)) > 0) & (d_ref > 0)
    return float(np.max(np.abs(d_test[m] / d_ref[m] - 1.0)))


def evaluate(torch, s_train, mu, sg, N=128, K=16, jumps=8, warm=50, seed=7, hubble_limit=1e-3, hidden=48,
             layers=6, act=cl.CL_ACT_RELU):
    """Run `jumps` surrogate jumps (leapfrog fallback) against jumps * K leapfrog steps from the same
    state on an N^3 lattice; returns timings, acceptance and the spectrum error."""
    s = cl.Surrogate(N, 3, 2, hidden, layers, act, cl.CL_SG_BF16, stream=_stream(torch))
    for l in range(layers):  # the trained weights, on the larger lattice
        s.set_weights(l, *s_train.get_weights(l))
    st = _stream(torch)
    with make_lattice(N, seed, stream=st) as ref, make_lattice(N, seed, stream=st) as sur:
        ref.cl_step(warm)
        sur.cl_step(warm)
        ref.cl_sync()
        t0 = time.perf_counter()
        ref.cl_step(jumps * K)
        ref.cl_sync()
        t_ref = time.perf_counter() - t0
        t0 = time.perf_counter()
        accepted = 0
        for _ in range(jumps):
            accepted += int(s.jump(sur, K, mu, sg, hubble_limit=hubble_limit))
        sur.cl_sync()
        t_sur = time.perf_counter() - t0
        err_phi = spectrum_error(ref, sur, cl.CL_FIELD_PHI0)
        err_pi = spectrum_error(ref, sur, cl.CL_FIELD_PI0)
        e_ref, e_sur = ref.cl_energies(), sur.cl_energies()
    s.close()
    return {"eval_N": N, "jumps": jumps, "accepted": accepted, "leapfrog_ms": t_ref * 1e3, "surrogate_ms": t_sur * 1e3,
            "speedup": t_ref / t_sur, "spectrum_err_phi": err_phi, "spectrum_err_pi": err_pi,
            "rho_rel_err": abs(e_sur["rho"] / e_ref["rho"] - 1.0),
            "hubble_violation": e_sur["hubble_violation"]}
