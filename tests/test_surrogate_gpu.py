"""Surrogate kernels on the GPU against the FP64 oracle of oracle/cnn.py.

Per operation, on the GPU's own bf16 tensors (so only that operation's rounding
differs): every convolution of the forward pass (bf16 output: within half a
bf16 unit), every weight and bias gradient (FP32 accumulation: 1e-3 relative)
and every backward-data convolution with its ReLU mask.  Then training on
trajectories of the batched solver, the Chapman-Enskog reconstruction against
the oracle, and the LBM fallback.
"""
import numpy as np
import pytest

import oracle as O
from oracle import cnn as N
from paper_1402_5487_gb300 import build, inputs as I, plbm
from paper_1402_5487_gb300 import surrogate as SG

pytestmark = pytest.mark.gpu

CIN = [4, 64, 64, 64, 64, 64]
COUT = [64, 64, 64, 64, 64, 4]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    plbm.lib()


def bf16(a):
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split(p):
    out, k = [], 0
    for ci, co in zip(CIN, COUT):
        n = 9 * ci * co
        W = p[k:k + n].reshape(3, 3, ci, co).astype(np.float64)
        k += n
        b = p[k:k + co].astype(np.float64)
        k += co
        out.append((W, b))
    return out


def close_bf16(gpu, ref):
    scale = np.max(np.abs(ref))
    return np.all(np.abs(gpu - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.fixture(scope="module", params=["tcgen05", "mma_sync"])
def net_and_pass(request):
    import torch
    net = SG.Surrogate(2, H=5, W=128, seed=7)
    net.set_tensor_path(request.param == "tcgen05")
    net.tc_path = request.param == "tcgen05"
    g = torch.Generator().manual_seed(3)
    x = torch.randn((2, 5, 128, 4), generator=g).to(torch.bfloat16).cuda()
    dout = (0.01 * torch.randn((2, 5, 128, 4), generator=g)).cuda()
    torch.cuda.synchronize()
    out = net.forward(x, 2).cpu().numpy().astype(np.float64)
    A = [x.float().cpu().numpy().astype(np.float64)]
    A += [net.tensor(0, l, 2).float().cpu().numpy().astype(np.float64) for l in range(1, 6)]
    A.append(out)
    grads = net.backward(x, dout, 2)
    dZ = [net.tensor(1, l, 2).float().cpu().numpy().astype(np.float64) for l in range(1, 6)]
    p, _ = net.params()
    assert net.check() == plbm.PLBM_OK
    yield net, A, dZ, dout.cpu().numpy().astype(np.float64), split(p), split(grads)
    net.close()


def test_forward_convolutions_match_oracle(net_and_pass):
    net, A, _, _, params, _ = net_and_pass
    for l in range(6):
        W, b = params[l]
        ref = N.conv3x3(A[l], bf16(W), b)
        if l < 5:
            assert close_bf16(A[l + 1], N.relu(ref)), l
        else:
            assert rel(A[6], ref) < 1e-5


def test_weight_gradients_match_oracle(net_and_pass):
    _, A, dZ, dout, params, grads = net_and_pass
    ups = dZ + [dout]  # upstream gradient of the convolution output of layers 1..6
    for l in range(6):
        dW, db = N.conv3x3_grad_weight(A[l], ups[l])
        assert rel(grads[l][0], dW) < 1e-3, l
        assert rel(grads[l][1], db) < 1e-3, l


def test_backward_data_convolutions_match_oracle(net_and_pass):
    net, A, dZ, dout, params, _ = net_and_pass
    # the tcgen05 path takes the output layer's upstream gradient in bf16, as it
    # does every other layer's; the mma.sync path keeps it in FP32
    ups = dZ + [bf16(dout) if net.tc_path else dout]
    for l in range(5, 0, -1):  # dZ of layer l from the upstream gradient of layer l + 1
        W, _ = params[l]
        ref = N.conv3x3_grad_input(ups[l], bf16(W)) * (A[l] > 0)
        assert close_bf16(dZ[l - 1], ref), l


def test_whole_network_gradient_close_to_fp64_chain(net_and_pass):
    # End to end against an FP64 forward/backward from the same bf16 input and weights
    # with no bf16 rounding between layers.  Each bf16 activation or gradient tensor
    # adds ~2^-9 relative noise; through five layers the first layer's weight gradient
    # drifts by up to ~10 %, the output by ~1 %.
    _, A, _, dout, params, grads = net_and_pass
    pr = [(bf16(W), b) for W, b in params]
    out, acts = N.forward(pr, A[0])
    g64 = N.backward(pr, acts, dout)
    assert rel(A[6], out) < 3e-2
    for l in range(6):
        assert rel(grads[l][0], g64[l][0]) < 0.15, l


@pytest.fixture(scope="module")
def trained():
    L, snaps = 128, 5
    stack = SG.generate(range(24), L=L, snaps=snaps, chunk=24)
    pairs = SG.pairs_of(24, snaps)
    norm = SG.fit_norm(stack, pairs)
    net = SG.Surrogate(8, H=L, W=L, seed=1)
    net.set_norm(*norm)
    losses = net.train(stack, pairs, 400, batch=8, lr=2e-3, lr_end=2e-4, log_every=50)
    yield net, stack, pairs, losses
    net.close()


def test_training_learns_more_than_persistence(trained):
    net, _, _, losses = trained
    assert losses[-1][1] < 0.5 * losses[0][1], losses
    L, snaps = 128, 5
    test_stack = SG.generate(range(1000, 1006), L=L, snaps=snaps, chunk=6)
    mse_net, mse_persist = net.evaluate(test_stack, SG.pairs_of(6, snaps))
    assert mse_net < 0.5 * mse_persist, (mse_net, mse_persist)


def test_reconstruction_matches_oracle_and_fallback_matches_lbm(trained):
    net = trained[0]
    L = 128
    fields = SG.trajectory_fields(2000, L)
    mk = lambda: plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32")
    a = mk()
    a.init(*fields)
    a.step(64)
    flags = net.advance([a], K=32, tol=1.0)
    assert flags == [0]
    assert a.diagnostics()["steps"] == 96
    m = a.moments()
    ref = N.reconstruct(SG.V5, SG.OMEGA, *m)
    got = a.get_populations()
    assert rel(got, ref) < 1e-5
    # fallback: a tolerance of zero forces K ordinary steps, identical to plain stepping
    b, c = mk(), mk()
    for s in (b, c):
        s.init(*fields)
        s.step(64)
    assert net.advance([b], K=32, tol=0.0) == [1]
    c.step(32)
    assert np.array_equal(b.get_populations(), c.get_populations())
    for s in (a, b, c):
        s.close()


def test_reported_drift_matches_fields_before_and_after(trained):
    # After an accepted advance the populations carry the predicted fields
    # exactly (projection), so the drift the library reports must equal the
    # drift of the FP64 sums of the moments before and after.
    net = trained[0]
    L = 128
    sol = plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32")
    sol.init(*SG.trajectory_fields(2001, L))
    sol.step(64)

    def sums(m):
        rho, ux, uy, th = m
        return np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(),
                         (rho * (2 * th + ux * ux + uy * uy)).sum()])

    a = sums(sol.moments())
    assert net.advance([sol], K=32, tol=1.0) == [0]
    b = sums(sol.moments())
    ref = max(abs(b[0] - a[0]) / abs(a[0]), abs(b[3] - a[3]) / abs(a[3]),
              np.hypot(b[1] - a[1], b[2] - a[2]) / (0.1 * abs(a[0])))
    got = net.last_drift()[0]
    assert abs(got - ref) <= 1e-6 + 1e-3 * ref, (got, ref)
    sol.close()


def test_conservative_projection_keeps_the_global_sums(trained):
    # With the projection option the predicted fields are shifted onto the old
    # global mass, momentum and energy: an advance then passes even a tight gate
    # and the stored populations keep the sums to FP32 rounding.
    net = trained[0]
    L = 128
    sol = plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32")
    sol.init(*SG.trajectory_fields(2002, L))
    sol.step(64)

    def sums(m):
        rho, ux, uy, th = m
        return np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(),
                         (rho * (2 * th + ux * ux + uy * uy)).sum()])

    m0 = sol.moments()
    a = sums(m0)
    net.set_conserve(True)
    try:
        flags = net.advance([sol], K=32, tol=1e-5)
        reported = net.last_drift()[0]
    finally:
        net.set_conserve(False)
    assert flags == [0]
    m1 = sol.moments()
    b = sums(m1)
    drift = max(abs(b[0] - a[0]) / abs(a[0]), abs(b[3] - a[3]) / abs(a[3]),
                np.hypot(b[1] - a[1], b[2] - a[2]) / (0.1 * abs(a[0])))
    assert drift <= 2e-6 and reported <= 2e-6, (drift, reported)
    assert np.max(np.abs(m1[1] - m0[1])) > 1e-3     # the network did move the flow
    sol.close()


@pytest.mark.parametrize("K", [32, 5])
def test_batched_fallback_equals_plain_stepping(trained, K):
    # Several fallback lattices in the row-paired layout step together in one
    # persistent launch per step; the populations must equal plain stepping bit
    # for bit, for even and odd K (the current array flips when K is odd).
    net = trained[0]
    L = 128
    mk = lambda: plbm.Solver(2, SG.V5, SG.OMEGA, L, L, theta0=SG.THETA0, prec="f32")
    a = [mk() for _ in range(3)]
    b = [mk() for _ in range(3)]
    for j, (x, y) in enumerate(zip(a, b)):
        f = SG.trajectory_fields(3000 + j, L)
        x.init(*f)
        y.init(*f)
        x.step(64)
        y.step(64)
    assert net.advance(a, K=K, tol=0.0) == [1, 1, 1]
    for x, y in zip(a, b):
        y.step(K)
        assert np.array_equal(x.get_populations(), y.get_populations())
        assert x.diagnostics()["steps"] == 64 + K
        x.step(3)
        y.step(3)
        assert np.array_equal(x.get_populations(), y.get_populations())
    for s in a + b:
        s.close()


def test_mean_penalty_enters_the_training_gradient():
    # loss = MSE + lam mean_{b,c} m_bc^2, m_bc = lattice mean of (pred - target) of
    # sample b, field c: the gradient a training step forms must equal the
    # backward pass of dout = 2 (pred - target + lam m) / n.
    import ctypes
    import torch
    net = SG.Surrogate(2, H=5, W=128, seed=11)
    g = torch.Generator().manual_seed(5)
    x = torch.randn((2, 5, 128, 4), generator=g).to(torch.bfloat16).cuda()
    y = (0.3 * torch.randn((2, 5, 128, 4), generator=g) + torch.tensor([0.2, -0.1, 0.05, 0.3])).cuda()
    p0, _ = net.params()
    lam = 7.0
    for lam_k in (0.0, lam):
        net.set_params(p0)
        net.set_mean_penalty(lam_k)
        torch.cuda.synchronize()
        assert plbm.lib().plbm_sur_train_step(net.h, 2, x.data_ptr(), y.data_ptr(), ctypes.c_float(1e-3),
                                              None) == plbm.PLBM_OK
        g_step = net.params()[1].astype(np.float64)
        net.set_params(p0)
        pred = net.forward(x, 2).clone()
        d = pred - y
        m = d.mean(dim=(1, 2), keepdim=True)
        dout = (2.0 * (d + lam_k * m) / d.numel()).contiguous()
        g_ref = net.backward(x, dout, 2).astype(np.float64)
        assert rel(g_step, g_ref) <= 1e-4, lam_k
        if lam_k == 0.0:
            g_plain = g_step
    assert rel(g_step, g_plain) > 1e-3      # the penalty does change the gradient
    net.set_mean_penalty(0.0)
    net.close()


def test_weight_gradients_over_many_tiles_per_cta_match_oracle():
    # 2 x 160 x 256 pixels = 640 tiles of 128: every CTA of the weight-gradient
    # kernels sums several tiles (the accumulators carry across tiles); the
    # 64 -> 64 layers and the 4 -> 64 input layer on both tensor paths.
    import torch
    net = SG.Surrogate(2, H=160, W=256, seed=11)
    g = torch.Generator().manual_seed(5)
    x = torch.randn((2, 160, 256, 4), generator=g).to(torch.bfloat16).cuda()
    dout = (0.01 * torch.randn((2, 160, 256, 4), generator=g)).cuda()
    for tc in (True, False):
        net.set_tensor_path(tc)
        net.forward(x, 2)
        A = [net.tensor(0, l, 2).float().cpu().numpy().astype(np.float64) for l in range(1, 5)]
        grads = split(net.backward(x, dout, 2))
        dZ = [net.tensor(1, l, 2).float().cpu().numpy().astype(np.float64) for l in range(1, 6)]
        assert net.check() == plbm.PLBM_OK
        for l in range(1, 5):   # the 64 -> 64 layers: input A_l, upstream dZ_{l+1}
            dW, db = N.conv3x3_grad_weight(A[l - 1], dZ[l])
            assert rel(grads[l][0], dW) < 1e-3, (tc, l)
            assert rel(grads[l][1], db) < 1e-3, (tc, l)
        # the 4 -> 64 input layer: input x, upstream dZ_1
        dW, db = N.conv3x3_grad_weight(x.float().cpu().numpy().astype(np.float64), dZ[0])
        assert rel(grads[0][0], dW) < 1e-3, (tc, 0)
        assert rel(grads[0][1], db) < 1e-3, (tc, 0)
    net.close()


def test_a_wait_that_runs_out_is_reported_and_the_next_pass_is_correct():
    # With a wait budget of a few nanoseconds every tcgen05 kernel of the pass
    # gives up at its first wait: it stops issuing, drains the MMAs it issued,
    # frees its tensor memory and sets the flag, which plbm_sur_check reports as
    # PLBM_E_TIMEOUT once.  With the default budget the same network then gives
    # the results of an undisturbed pass (nothing was left behind).
    import torch
    net = SG.Surrogate(1, H=3, W=128, seed=5)
    g = torch.Generator().manual_seed(9)
    x = torch.randn((1, 3, 128, 4), generator=g).to(torch.bfloat16).cuda()
    dout = (0.01 * torch.randn((1, 3, 128, 4), generator=g)).cuda()
    ref_out = net.forward(x, 1).clone()
    ref_grads = net.backward(x, dout, 1).astype(np.float64)
    assert net.check() == plbm.PLBM_OK
    net.set_wait_ns(4)
    net.forward(x, 1)
    net.backward(x, dout, 1)
    assert net.check() == plbm.PLBM_E_TIMEOUT
    assert net.check() == plbm.PLBM_OK      # reported once
    net.set_wait_ns(2_000_000_000)
    out = net.forward(x, 1).clone()
    grads = net.backward(x, dout, 1).astype(np.float64)
    assert net.check() == plbm.PLBM_OK
    assert torch.equal(out, ref_out)
    assert rel(grads, ref_grads) <= 1e-6
    net.close()


def _splitmix64(z):
    """SplitMix64 output function (Steele, Lea and Flood 2014) on uint64 arrays (wrapping)."""
    z = z + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def test_input_noise_is_the_stated_counter_based_normal_draw():
    # plbm_sur_assemble_noise adds sigma x N(0, 1) to every normalised input element,
    # the normal number of element e drawn as SplitMix64(seed ^ SplitMix64(e)) and
    # Box-Muller; restated here in FP64 NumPy from the published definitions.
    import torch
    H, W, sigma, seed = 3, 128, 0.05, 1234
    net = SG.Surrogate(2, H=H, W=W, seed=1)
    net.set_norm(np.zeros(4), np.ones(4), np.zeros(4), np.ones(4))
    npix = H * W
    g = torch.Generator().manual_seed(8)
    stack = torch.rand((2, npix, 4), generator=g).cuda()
    pairs = torch.tensor([[0, 1], [1, 0]], dtype=torch.int32).cuda()
    x0 = torch.empty((2, H, W, 4), dtype=torch.bfloat16, device="cuda")
    x1, y = torch.empty_like(x0), torch.empty((2, H, W, 4), dtype=torch.float32, device="cuda")
    L = plbm.lib()
    assert L.plbm_sur_assemble(net.h, stack.data_ptr(), npix, pairs.data_ptr(), 2, x0.data_ptr(), y.data_ptr()) == 0
    assert L.plbm_sur_assemble_noise(net.h, stack.data_ptr(), npix, pairs.data_ptr(), 2, x1.data_ptr(), y.data_ptr(),
                                     sigma, seed) == 0
    net.stream.synchronize()
    e = np.arange(2 * npix * 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _splitmix64(np.uint64(seed) ^ _splitmix64(e))
    u1 = ((h >> np.uint64(40)).astype(np.float64) + 1.0) / 2.0 ** 24
    u2 = ((h >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) / 2.0 ** 24
    gauss = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    clean = stack[pairs[:, 0].long()].cpu().numpy().astype(np.float64).reshape(-1)
    ref = bf16(clean + sigma * gauss)
    got = x1.float().cpu().numpy().astype(np.float64).reshape(-1)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6)
    d = got - x0.float().cpu().numpy().astype(np.float64).reshape(-1)
    assert abs(d.mean()) < 0.1 * sigma and abs(d.std() / sigma - 1.0) < 0.1
    assert L.plbm_sur_assemble_noise(net.h, stack.data_ptr(), npix, pairs.data_ptr(), 2, x1.data_ptr(), y.data_ptr(),
                                     -1.0, seed) == plbm.PLBM_E_ARG
    net.close()


def test_one_launch_per_model_equals_one_launch_per_lattice(trained):
    # Lattices that share a model take the moments/input and the reconstruction
    # kernels of an advance in one launch each; a set that mixes models (another
    # omega, another storage precision) takes them per lattice.  The per-node code
    # is the same and the network treats every lattice on its own, so each
    # lattice must end with the same bits either way.
    net = trained[0]
    L = 128

    def mk(seed, omega=SG.OMEGA, prec="f32"):
        s = plbm.Solver(2, SG.V5, omega, L, L, theta0=SG.THETA0, prec=prec)
        s.init(*SG.trajectory_fields(seed, L))
        s.step(64)
        return s

    same = [mk(4000), mk(4001)]                                       # one model: batched launches
    mixed = [mk(4000), mk(4001), mk(4002, omega=1.6), mk(4003, prec="f16dev")]
    alone = [mk(4002, omega=1.6), mk(4003, prec="f16dev")]
    assert net.advance(same, K=32, tol=1.0) == [0, 0]
    assert net.advance(mixed, K=32, tol=1.0) == [0, 0, 0, 0]
    for s in alone:
        assert net.advance([s], K=32, tol=1.0) == [0]
    for x, y in zip(same + alone, mixed):
        assert np.array_equal(x.get_populations(), y.get_populations())
        assert x.diagnostics()["steps"] == y.diagnostics()["steps"] == 96
    for s in same + mixed + alone:
        s.close()


@pytest.mark.parametrize("tc", [True, False])
def test_gradients_are_bitwise_reproducible(tc):
    # Every reduction of the backward pass has a fixed order (per-CTA partial sums
    # over fixed tile ranges, then an ordered sum over the CTAs), so the same pass
    # on the same inputs gives the same bits; at the training shape (16 lattices
    # of 256 x 256) the weight-gradient CTAs' row ranges cross columns and lattices.
    import torch
    B = 16
    net = SG.Surrogate(B, H=256, W=256, seed=5)
    net.set_tensor_path(tc)
    g = torch.Generator().manual_seed(9)
    x = torch.randn((B, 256, 256, 4), generator=g).to(torch.bfloat16).cuda()
    dout = (0.01 * torch.randn((B, 256, 256, 4), generator=g)).cuda()
    first = net.backward(x, dout, B).copy()
    for _ in range(3):
        again = net.backward(x, dout, B)
        assert np.array_equal(again, first), np.flatnonzero(again != first)[:10]
    assert net.check() == plbm.PLBM_OK
    net.close()


def test_training_is_bitwise_reproducible():
    # The same data, seed and steps give the same weights: the minibatches are the
    # seeded draw (their indices reach the device before the steps, which run
    # ahead of the host), the noise is counter-based and every step deterministic.
    L, snaps = 128, 3
    stack = SG.generate(range(8), L=L, snaps=snaps, chunk=8)
    pairs = SG.pairs_of(8, snaps)
    norm = SG.fit_norm(stack, pairs)
    ws = []
    for _ in range(2):
        net = SG.Surrogate(4, H=L, W=L, seed=2)
        net.set_norm(*norm)
        net.train(stack, pairs, 40, batch=4, lr=1e-3, seed=3, noise=0.2)
        ws.append(net.params()[0].copy())
        net.close()
    assert np.array_equal(ws[0], ws[1])
