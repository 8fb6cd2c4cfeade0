"""Pins of the FP64 reference network of the learned Poisson initial guess (no GPU): the convolution
against an explicit loop over cells and taps, and every gradient against central finite differences."""
import numpy as np

from oracle import learned as NL


def test_conv_matches_explicit_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 8))
    W = rng.standard_normal((8, 27, 8))
    b = rng.standard_normal(8)
    z = NL.conv(x, W, b)
    nz, ny, nx = x.shape[:3]
    for (k, j, i) in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (1, 0, 4)]:
        ref = b.copy()
        for t, (dz, dy, dx) in enumerate(NL.TAPS):
            kk, jj, ii = k + dz, j + dy, i + dx
            if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx:
                ref += W[:, t, :] @ x[kk, jj, ii]
        assert np.allclose(z[k, j, i], ref, rtol=1e-13, atol=1e-13)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    x = np.zeros((4, 5, 6, 8))
    x[..., :3] = rng.standard_normal((4, 5, 6, 3))
    target = rng.standard_normal((4, 5, 6))
    W, B = NL.init_params(seed=2, scale=0.3)
    B = [rng.standard_normal(8) * 0.1, rng.standard_normal(8) * 0.1, rng.standard_normal(1) * 0.1]
    loss, dW, dB, _ = NL.loss_and_grads(x, target, W, B)
    h = 1e-6
    for l in range(3):
        for _ in range(6):
            co = rng.integers(W[l].shape[0]); t = rng.integers(27); ci = rng.integers(3 if l == 0 else 8)
            Wp = [w.copy() for w in W]; Wp[l][co, t, ci] += h
            Wm = [w.copy() for w in W]; Wm[l][co, t, ci] -= h
            fd = (NL.loss_and_grads(x, target, Wp, B)[0] - NL.loss_and_grads(x, target, Wm, B)[0]) / (2 * h)
            assert abs(fd - dW[l][co, t, ci]) <= 1e-6 * max(1.0, abs(fd))
        co = rng.integers(B[l].shape[0])
        Bp = [b.copy() for b in B]; Bp[l][co] += h
        Bm = [b.copy() for b in B]; Bm[l][co] -= h
        fd = (NL.loss_and_grads(x, target, W, Bp)[0] - NL.loss_and_grads(x, target, W, Bm)[0]) / (2 * h)
        assert abs(fd - dB[l][co]) <= 1e-6 * max(1.0, abs(fd))
