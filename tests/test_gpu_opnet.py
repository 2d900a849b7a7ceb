"""The learned warm start on the GPU (include/opnet.h) against the FP64 oracle.

- the layer table and parameter layout equal the oracle's;
- forward, loss and the full parameter gradient match oracle/unet.py on the same
  FP32-rounded parameters;
- one Adam step matches the oracle's Adam on the same gradient;
- a network trained on blocks the scheme itself converged gives starting blocks
  from which the scheme needs fewer steps than from random ones.

Tolerances.  With the FP32 convolutions (opnet_set_conv OPNET_CONV_FP32) the network
runs in FP32 with FP32 accumulation over at most 27 x 144 products per output and FP32
sums over at most 2048 points per weight-gradient partial (partials summed in FP64).
Forward outputs agree to a few 1e-6 of their scale; gradients, which pass through up to
22 such layers, to 1e-4 relative per layer.

The tensor-core convolutions (the default) round activations and weights to BF16 and
accumulate in FP32.  A layer is checked against the oracle's convolution of the
BF16-rounded operands (then only the FP32 accumulation differs: K 2^-23 sum |x w| per
output); a whole forward pass against the FP32 one (BF16 rounding, 2^-9 per operand,
through 11 layers).  A layer's data gradient (opnet_conv_dgrad, the same kernel on dZ with
the tap-reversed, transposed weights) is checked the same way against the oracle's
adjoint, and the whole loss gradient with tensor-core forward and data gradients against
the FP32 one.
"""
import numpy as np
import pytest

from oracle import unet
import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402

DEV = torch.device("cuda:0")
GAMMA = 0.1


def setup(N, widths, p, seed=0, conv="fp32"):
    table = unet.layer_table(*widths, p)
    theta = syn.uniform_init(seed, unet.fans(table)).astype(np.float32).astype(np.float64)
    P = syn.warm_start_problem(seed + 5, N=N, p=p)
    net = pkg.Net(N, P.lo, P.hi, p, widths)
    net.set_conv(conv)
    net.set_params(theta)
    V = torch.from_numpy(P.V).to(DEV)
    return net, theta, P, V


def target(n, p, seed):
    Q, _ = np.linalg.qr(syn.gaussian_block(seed, n, p))
    return Q.astype(np.float32).astype(np.float64)


def layer_slices(table):
    off, out = 0, []
    for _, t, ci, co in table:
        size = t * ci * co + co
        out.append(slice(off, off + size))
        off += size
    return out


def test_layer_table_and_parameter_count_match_oracle():
    with pkg.Net(48, (-8.0,) * 3, (8.0,) * 3, 64, (24, 48, 96)) as net:
        table = unet.layer_table(24, 48, 96, 64)
        assert net.layers() == [(t, ci, co) for _, t, ci, co in table]
        assert net.count == sum(t * ci * co + co for _, t, ci, co in table) == 892720


@pytest.mark.parametrize("N,widths,p", [(8, (6, 8, 10), 8), (16, (8, 16, 24), 16),
                                        (12, (5, 7, 9), 8)])
def test_forward_matches_oracle(N, widths, p):
    net, theta, P, V = setup(N, widths, p)
    Y = net.forward(V).double().cpu().numpy()
    Y_ref, _ = unet.forward(theta, P.V, N, P.lo, P.hi, widths, p)
    assert np.abs(Y - Y_ref).max() <= 5e-6 * np.abs(Y_ref).max()
    U0 = net.infer(V).cpu().numpy()  # the FP64 warm-start block is the same Y
    np.testing.assert_array_equal(U0, Y)
    net.close()


@pytest.mark.parametrize("N,widths,p", [(8, (6, 8, 10), 8), (16, (8, 16, 24), 16)])
def test_loss_and_gradient_match_oracle(N, widths, p):
    net, theta, P, V = setup(N, widths, p, seed=1)
    Us = target(P.n, p, 3)
    loss, g = net.loss_grad(V, torch.from_numpy(Us).to(DEV, torch.float32), GAMMA)
    Y_ref, cache = unet.forward(theta, P.V, N, P.lo, P.hi, widths, p)
    L_ref, dY = unet.subspace_loss(Y_ref, Us, GAMMA)
    g_ref = unet.backward(cache, dY)
    assert loss == pytest.approx(L_ref, rel=2e-5)
    table = unet.layer_table(*widths, p)
    for (name, *_), sl in zip(table, layer_slices(table)):
        err = np.linalg.norm(g[sl] - g_ref[sl]) / np.linalg.norm(g_ref[sl])
        assert err < 1e-4, (name, err)
    net.close()


def test_adam_step_matches_oracle_adam():
    N, widths, p = 8, (6, 8, 10), 8
    net, theta, P, V = setup(N, widths, p, seed=2)
    Us = torch.from_numpy(target(P.n, p, 4)).to(DEV, torch.float32)
    _, g = net.loss_grad(V, Us, GAMMA)
    lr = 1e-3
    net.train_step(V, Us, lr, GAMMA)
    th1 = net.get_params().astype(np.float64)
    ref, _, _ = unet.adam_step(theta, g.astype(np.float64), np.zeros_like(theta),
                               np.zeros_like(theta), 1, lr)
    assert np.abs(th1 - ref).max() <= 1e-6 * lr + 1e-7 * np.abs(theta).max()
    net.close()


def test_training_reduces_the_loss():
    N, widths, p = 8, (6, 8, 10), 8
    net, theta, P, V = setup(N, widths, p, seed=3)
    Us = torch.from_numpy(target(P.n, p, 5)).to(DEV, torch.float32)
    losses = [net.train_step(V, Us, 3e-3, GAMMA) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]
    net.close()


def test_rejects_bad_configurations():
    for N, p in [(10, 8), (8, 12), (0, 8), (8, 256)]:
        with pytest.raises(pkg.OpError):
            pkg.Net(N, (-1.0,) * 3, (1.0,) * 3, p, (4, 4, 4))


# ----------------------------------------------------------------------------
# What the trained network gains over random starting blocks
# ----------------------------------------------------------------------------
def converged_block(P, seed, tol=1e-4, cap=800):
    """U* from the scheme itself (FP32 context; residual tol or cap steps) as FP32 CUDA."""
    with pkg.Solver(P.shape, P.lo, P.hi, P.V, syn.gaussian_block(seed, P.n, P.p), P.p,
                    prec="fp32") as s:
        s.solve(tol, cap, raise_on_max=False)
        return s.get_U_device(torch.float32)


def energies(P, U0, nsteps, device=False):
    """E(U0) after orthonormalisation and E after each of nsteps FP32 steps."""
    V = torch.from_numpy(P.V).to(DEV) if device else P.V
    with pkg.Solver(P.shape, P.lo, P.hi, V, U0, P.p, prec="fp32", device=device) as s:
        return np.array([s.stats()["energy"]] + [s.step(1)["energy"] for _ in range(nsteps)])


def steps_within(E, E_ref, rel):
    """First step at which |E - E_ref| <= rel |E_ref| (len(E) if never)."""
    ok = np.nonzero(np.abs(E - E_ref) <= rel * abs(E_ref))[0]
    return int(ok[0]) if ok.size else len(E)


def test_trained_warm_start_beats_random_starts():
    """A lower starting energy (the basin quantity of §3) and fewer steps until the
    energy is within 1e-3 of its converged value.  (The steps to a tight tolerance
    are set by the spectral gap at the cut and are not shortened; see the bench's
    warm-start workload.)"""
    N, p, widths = 16, 8, (8, 16, 24)
    train_seeds, test_seeds = range(1000, 1024), range(5000, 5006)
    data = []
    for sd in train_seeds:
        P = syn.warm_start_problem(sd, N=N, p=p)
        data.append((torch.from_numpy(P.V).to(DEV), converged_block(P, sd)))
    net = pkg.Net(N, (-8.0,) * 3, (8.0,) * 3, p, widths)
    net.set_params(syn.uniform_init(7, unet.fans(unet.layer_table(*widths, p))))
    first = last = None
    for epoch in range(25):
        tot = 0.0
        for V, Us in data:
            tot += net.train_step(V, Us, 2e-3, GAMMA)
        first = tot if first is None else first
        last = tot
    assert last < 0.5 * first
    rows = []
    for sd in test_seeds:
        P = syn.warm_start_problem(sd, N=N, p=p)
        Ur = syn.gaussian_block(sd, P.n, p)
        with pkg.Solver(P.shape, P.lo, P.hi, P.V, Ur, p, prec="fp32") as s:
            s.solve(1e-10, 3000, pkg.OP_STOP_ERR_E, raise_on_max=False)
            E_ref = s.stats()["energy"]
        E_rand = energies(P, Ur, 150)
        E_net = energies(P, net.infer(torch.from_numpy(P.V).to(DEV)), 150, device=True)
        rows.append((E_rand[0], E_net[0], steps_within(E_rand, E_ref, 1e-3),
                     steps_within(E_net, E_ref, 1e-3)))
    rows = np.array(rows)
    assert np.all(rows[:, 1] < rows[:, 0]), rows          # every warm start has lower energy
    assert rows[:, 3].mean() < rows[:, 2].mean(), rows    # and gets within 1e-3 sooner
    net.close()


def bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("N,taps,cin,cout", [(10, 27, 4, 24), (13, 27, 16, 8), (8, 27, 6, 128),
                                             (9, 27, 144, 48), (11, 1, 48, 64), (4, 27, 96, 16)])
def test_tensor_core_conv_layer_matches_oracle(N, taps, cin, cout):
    rng = np.random.default_rng(N * 1000 + cin + cout)
    n = N ** 3
    X = rng.standard_normal((n, cin)).astype(np.float32)
    W = (rng.standard_normal((taps * cin, cout)) / np.sqrt(taps * cin)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    Z, A = pkg.binding.net_conv("bf16_tc", torch.from_numpy(X).to(DEV), N, taps,
                                torch.from_numpy(W).to(DEV), torch.from_numpy(b).to(DEV))
    Z, A = Z.double().cpu().numpy(), A.double().cpu().numpy()
    Xr, Wr = bf16(X), bf16(W)
    if taps == 27:
        ref = unet.conv3(Xr, N, Wr.reshape(27, cin, cout), b.astype(np.float64))
        mag = unet.conv3(np.abs(Xr), N, np.abs(Wr).reshape(27, cin, cout), np.abs(b))
    else:
        ref = Xr @ Wr + b
        mag = np.abs(Xr) @ np.abs(Wr) + np.abs(b)
    tol = (taps * cin + 2) * 2.0 ** -23 * mag + 1e-30
    assert np.all(np.abs(Z - ref) <= tol), float((np.abs(Z - ref) / tol).max())
    silu = ref / (1.0 + np.exp(-ref))
    assert np.all(np.abs(A - silu) <= 2 * tol + 4 * 2.0 ** -24 * np.abs(silu))
    # the operands really were rounded: the unrounded product differs by far more
    if taps == 27:
        exact = unet.conv3(X.astype(np.float64), N, W.astype(np.float64).reshape(27, cin, cout),
                           b.astype(np.float64))
        assert np.abs(exact - ref).max() > 100 * np.abs(Z - ref).max()


def test_tensor_core_conv_rejects_bad_arguments():
    X = torch.zeros(64, 8, device=DEV)
    W = torch.zeros(27 * 8, 200, device=DEV)          # more than 128 output channels
    with pytest.raises(pkg.OpError):
        pkg.binding.net_conv("bf16_tc", X, 4, 27, W)


@pytest.mark.parametrize("kind", ["fp32", "bf16_tc"])
@pytest.mark.parametrize("N,taps,cin,cout", [(10, 27, 4, 24), (9, 27, 24, 48), (8, 27, 144, 48),
                                             (11, 1, 24, 64), (7, 27, 96, 96), (5, 27, 6, 10)])
def test_layer_data_gradient_matches_oracle(kind, N, taps, cin, cout):
    """opnet_conv_dgrad against the oracle's adjoint (conv3_backward): on the tensor cores
    (cin <= 128) with BF16-rounded dZ and W, within the FP32 accumulation bound of
    taps x cout terms; on the FP32 CUDA cores (and for cin > 128) with the unrounded ones."""
    rng = np.random.default_rng(N * 100 + cin + 7 * cout)
    n = N ** 3
    dZ = rng.standard_normal((n, cout)).astype(np.float32)
    W = (rng.standard_normal((taps * cin, cout)) / np.sqrt(taps * cin)).astype(np.float32)
    dX = pkg.binding.net_conv_dgrad(kind, torch.from_numpy(dZ).to(DEV), N, taps,
                                    torch.from_numpy(W).to(DEV)).double().cpu().numpy()
    assert dX.shape == (n, cin)
    tc = kind == "bf16_tc" and cin <= 128
    dZr, Wr = (bf16(dZ), bf16(W)) if tc else (dZ.astype(np.float64), W.astype(np.float64))
    X0 = np.zeros((n, cin))
    if taps == 27:
        ref = unet.conv3_backward(X0, N, Wr.reshape(27, cin, cout), dZr)[0]
        mag = unet.conv3_backward(X0, N, np.abs(Wr).reshape(27, cin, cout), np.abs(dZr))[0]
    else:
        ref = dZr @ Wr.T
        mag = np.abs(dZr) @ np.abs(Wr).T
    tol = (taps * cout + 2) * 2.0 ** -23 * mag + 1e-30
    assert np.all(np.abs(dX - ref) <= tol), float((np.abs(dX - ref) / tol).max())
    if tc and taps == 27:
        # the operands really were rounded: the unrounded adjoint differs by far more
        exact = unet.conv3_backward(X0, N, W.astype(np.float64).reshape(27, cin, cout),
                                    dZ.astype(np.float64))[0]
        assert np.abs(exact - ref).max() > 100 * np.abs(dX - ref).max()


def test_layer_data_gradient_rejects_bad_arguments():
    dZ = torch.zeros(64, 8, device=DEV)
    with pytest.raises(pkg.OpError):
        pkg.binding.net_conv_dgrad("bf16_tc", dZ, 4, 9, torch.zeros(9 * 8, 8, device=DEV))


def test_tensor_core_gradient_close_to_fp32_gradient():
    """The whole network's loss gradient with the tensor-core forward and data gradients
    against the FP32 one: BF16 rounding (2^-9 per operand) through the 11 forward and up
    to 11 data-gradient layers, so agreement to a few percent per layer, not to FP32."""
    N, widths, p = 16, (8, 16, 24), 16
    net, theta, P, V = setup(N, widths, p, seed=2, conv="bf16_tc")
    Us = torch.from_numpy(target(P.n, p, 5)).to(DEV, torch.float32)
    loss_tc, g_tc = net.loss_grad(V, Us, GAMMA)
    net.set_conv("fp32")
    loss_32, g_32 = net.loss_grad(V, Us, GAMMA)
    net.close()
    assert loss_tc == pytest.approx(loss_32, rel=2e-2)
    table = unet.layer_table(*widths, p)
    for (name, *_), sl in zip(table, layer_slices(table)):
        rel = np.linalg.norm(g_tc[sl] - g_32[sl]) / np.linalg.norm(g_32[sl])
        assert 1e-6 < rel < 0.1, (name, rel)


def test_tensor_core_forward_close_to_fp32_forward():
    N, widths, p = 16, (8, 16, 24), 16
    net, theta, P, V = setup(N, widths, p, conv="bf16_tc")
    Y_tc = net.forward(V).double().cpu().numpy()
    net.set_conv("fp32")
    Y_32 = net.forward(V).double().cpu().numpy()
    net.close()
    rel = np.linalg.norm(Y_tc - Y_32) / np.linalg.norm(Y_32)
    # BF16 operand rounding (2^-9 relative) through 11 layers, not FP32-level agreement
    assert 1e-5 < rel < 3e-2, rel
