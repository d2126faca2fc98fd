"""Pins of the oracle's learned initial guess (the 4-layer periodic CNN of ``oracle/cnn.py``)
against definitions it does not share code with:

* the 3 x 3 periodic cross-correlation equals the convolution theorem evaluated with numpy's FFT
  (cross-correlation with the kernel embedded in the periodic grid: zhat = ahat conj(what));
* a kernel with a single 1 at offset (p, q) shifts the field (numpy's roll);
* every gradient of the backward pass equals a central difference of the loss (weights, biases,
  and the input through the chain rule of the last layers);
* the network commutes with periodic translations of its inputs and is homogeneous of degree
  one in the right-hand side;
* the bfloat16 rounding equals torch's float32 -> bfloat16 conversion (round to nearest, ties to
  even) and keeps representable values;
* Adam's first step moves every weight by lr times the sign of its gradient (bias correction),
  and later steps equal torch.optim.Adam on the same gradients.
"""
import numpy as np
import pytest

from oracle import cnn as C


def _params(rng, channels=C.CHANNELS, scale=0.4):
    ps = []
    for ci, co in zip(channels[:-1], channels[1:]):
        ps.append((rng.standard_normal((co, ci, 3, 3)) * scale / np.sqrt(9 * ci), 0.1 * rng.standard_normal(co)))
    return ps


def test_conv_equals_fft_cross_correlation():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 7, 10))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = C.conv3x3(a, W, b)
    ny, nx = a.shape[1:]
    ref = np.empty_like(z)
    for o in range(4):
        acc = np.zeros((ny, nx), dtype=complex)
        for c in range(3):
            emb = np.zeros((ny, nx))
            for p in (-1, 0, 1):
                for q in (-1, 0, 1):
                    emb[p % ny, q % nx] += W[o, c, p + 1, q + 1]
            acc += np.fft.fft2(a[c]) * np.conj(np.fft.fft2(emb))
        ref[o] = np.real(np.fft.ifft2(acc)) + b[o]
    assert np.abs(z - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("p,q", [(-1, 0), (0, 1), (1, -1), (0, 0)])
def test_delta_kernel_shifts(p, q):
    a = np.random.default_rng(1).standard_normal((1, 5, 6))
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, p + 1, q + 1] = 1.0
    z = C.conv3x3(a, W, np.zeros(1))
    assert np.array_equal(z, np.roll(a, shift=(-p, -q), axis=(1, 2)))


def _loss(params, samples):
    return C.loss_and_grads(params, samples)[0]


def test_gradients_equal_central_differences():
    rng = np.random.default_rng(2)
    ch = (2, 5, 4, 3, 1)   # the network's structure with fewer channels (the arithmetic is the same)
    params = _params(rng, ch, scale=1.0)
    ny, nx = 6, 7
    samples = [(rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx)))
               for _ in range(2)]
    _, grads = C.loss_and_grads(params, samples)
    h = 1e-6
    for l in range(len(params)):
        for which in (0, 1):
            arr = params[l][which]
            for _ in range(4):
                idx = tuple(rng.integers(0, n) for n in arr.shape)
                old = arr[idx]
                arr[idx] = old + h
                fp = _loss(params, samples)
                arr[idx] = old - h
                fm = _loss(params, samples)
                arr[idx] = old
                fd = (fp - fm) / (2 * h)
                g = grads[l][which][idx]
                assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3), (l, which, idx, g, fd)


def test_input_gradient_of_conv_equals_central_differences():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 5, 4))
    W = rng.standard_normal((3, 2, 3, 3))
    g = rng.standard_normal((3, 5, 4))
    da, _, _ = C.conv3x3_backward(a, W, g)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 3), (0, 2, 1), (1, 0, 3)]:
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        fd = (np.sum(g * C.conv3x3(ap, W, np.zeros(3))) - np.sum(g * C.conv3x3(am, W, np.zeros(3)))) / (2 * h)
        assert abs(da[idx] - fd) < 1e-7 * max(1.0, abs(fd))


def test_translation_equivariance_and_homogeneity():
    rng = np.random.default_rng(4)
    params = _params(rng)
    r = rng.standard_normal((12, 10))
    vs = rng.standard_normal((12, 10))
    x0 = C.forward(params, r, vs)
    sh = (5, -3)
    assert np.abs(C.forward(params, np.roll(r, sh, (0, 1)), np.roll(vs, sh, (0, 1))) - np.roll(x0, sh, (0, 1))).max() \
        < 1e-12 * np.abs(x0).max()
    assert np.abs(C.forward(params, 7.5 * r, vs) - 7.5 * x0).max() < 1e-12 * 7.5 * np.abs(x0).max()
    assert not np.any(C.forward(params, np.zeros_like(r), vs))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        [1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0, 2.0 ** -130]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = C.to_bf16(x)
    assert np.array_equal(got, ref)
    assert got[-6] == 1.0 and got[-5] == 1.0 and got[-4] == 1 + 2.0 ** -6 and got[-3] == -1.0
    assert np.array_equal(C.to_bf16(got), got)
    assert np.max(np.abs(got[:4000] - x[:4000]) / np.abs(x[:4000])) <= 2.0 ** -8 * (1 + 1e-6)


def test_adam_first_step_and_torch_agreement():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    theta = [rng.standard_normal((3, 4)), rng.standard_normal(5)]
    opt = C.Adam(lr=0.01)
    g0 = [rng.standard_normal(t.shape) for t in theta]
    t1 = opt.step(theta, g0)
    for a, b, g in zip(t1, theta, g0):
        assert np.allclose(a - b, -0.01 * np.sign(g), rtol=1e-6, atol=0)
    tp = [torch.tensor(t, requires_grad=True) for t in theta]
    topt = torch.optim.Adam(tp, lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    ours = C.Adam(lr=0.01)
    cur = [t.copy() for t in theta]
    for k in range(5):
        gs = [rng.standard_normal(t.shape) for t in theta]
        for p, g in zip(tp, gs):
            p.grad = torch.tensor(g)
        topt.step()
        cur = ours.step(cur, gs)
    for p, c in zip(tp, cur):
        assert np.abs(p.detach().numpy() - c).max() < 1e-14
