"""CPU: the seeded synthetic inputs have the shapes and value distributions
their recipes state (the stand-ins for the paper's data sets, Table II and
the "Random" set of Sec. IV-A), and are pure functions of their seed."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("gen,args", [
    (workloads.gaussian_mixture, (500, 16, 20)),
    (workloads.mnist_like, (300, 20)),
    (workloads.lognormal_int, (400, 32, 10)),
    (workloads.latent_factor, (300, 96, 10)),
    (workloads.unit_gaussian, (200, 40, 10)),
])
def test_shapes_dtype_and_seeding(gen, args):
    X, Q = gen(*args, seed=5)
    X2, Q2 = gen(*args, seed=5)
    X3, _ = gen(*args, seed=6)
    n, m = args[0], args[-1]
    assert X.dtype == np.float32 and Q.dtype == np.float32
    assert X.shape[0] == n and Q.shape[0] == m and X.shape[1] == Q.shape[1]
    assert X.flags["C_CONTIGUOUS"] and Q.flags["C_CONTIGUOUS"]
    assert np.array_equal(X, X2) and np.array_equal(Q, Q2), "not a pure function of the seed"
    assert not np.array_equal(X, X3), "the seed is ignored"
    assert np.isfinite(X).all() and np.isfinite(Q).all()


def test_mnist_like_recipe():
    X, Q = workloads.mnist_like(3000, 100, seed=0)
    assert X.shape[1] == 784
    A = np.concatenate([X, Q])
    assert np.array_equal(A, np.rint(A)) and A.min() == 0 and A.max() == 255, "integer pixels 0..255"
    zeros = (A == 0).mean()
    assert 0.75 < zeros < 0.90, f"zero fraction {zeros:.3f}, recipe: about 80 %"
    img = A.reshape(-1, 28, 28)
    border = np.zeros((28, 28), bool)
    border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    assert (img[:, border] > 0).any(axis=1).mean() < 0.01, "border almost always blank"
    assert (img[:, border] > 0).mean() < 1e-3, "border pixels rarely lit"
    assert (img[:, ~border] > 0).mean() > 0.1, "interior pixels often lit"
    nz = A[A > 0]
    assert (nz == 255).mean() > 0.5, "stroke cores are 255"
    assert ((nz > 0) & (nz < 255)).mean() > 0.1, "a grey ramp around the strokes"


def test_lognormal_int_recipe():
    X, _ = workloads.lognormal_int(20000, 24, 10, seed=1)
    assert np.array_equal(X, np.rint(X)) and X.min() >= 0 and X.max() <= 255
    med = np.median(X, axis=0)
    # median of exp(N(mu, s)) is exp(mu), mu ~ U(1, 4): e^1 .. e^4 before rounding
    assert ((med >= np.floor(np.e) - 1) & (med <= np.ceil(np.e ** 4) + 1)).all()
    # heavy right tail: the mean exceeds the median in (almost) every dimension
    assert (X.mean(axis=0) > med).mean() > 0.9
    assert (X == 255).any(), "clipped at 255"


def test_latent_factor_recipe():
    X, _ = workloads.latent_factor(4000, 200, 10, rank=16, seed=2)
    assert X.min() >= 0.0 and X.max() <= 1.0
    assert abs(float(X.mean()) - 0.5) < 0.02
    ev = np.linalg.eigvalsh(np.cov(X.astype(np.float64), rowvar=False))[::-1]
    # rank-16 signal (each direction ~0.15^2 d / 16) over N(0, 0.05^2) noise
    assert ev[15] > 20 * 0.05 ** 2, "the 16 factor directions stand out"
    assert ev[16] < 2 * 0.05 ** 2, "beyond the rank only noise is left"


def test_unit_gaussian_recipe():
    X, Q = workloads.unit_gaussian(3000, 64, 10, seed=3)
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, rtol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(Q, axis=1), 1.0, rtol=1e-6)
    # isotropic: no direction preferred
    assert np.abs(X.mean(axis=0)).max() < 5 / np.sqrt(3000 * 64)


def test_uneven_batches_recipe():
    b = workloads.uneven_batches(100000, seed=4)
    sizes = np.array([s for s, _, _ in b])
    assert sizes.sum() == 100000 and sizes.min() >= 1 and sizes.max() <= 4096
    assert {k for _, k, _ in b} <= {1, 10, 100} and {v for _, _, v in b} <= {2, 5, 8}
    # floor(exp(U(0, ln 4097))): median exp(ln(4097) / 2) = 64
    assert 40 <= np.median(sizes[:-1]) <= 100
    assert workloads.uneven_batches(100000, seed=4) == b
