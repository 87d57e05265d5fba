"""The seeded input recipe: the generators draw what the model and the
stated distributions say (sizes, value distributions, structure), the same
numbers for the same seed, and the device generator the same model as the
numpy one.  CPU only."""
import numpy as np
import pytest

from paper_1805_09498_gb300 import synth
from paper_1805_09498_gb300.synth import batch_lengths, cn, draw_P, make_batch, make_problem


def test_complex_gaussian_is_circular_with_unit_variance():
    z = cn(np.random.default_rng(0), 400_000)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z.real ** 2) - 0.5) < 0.01 and abs(np.mean(z.imag ** 2) - 0.5) < 0.01
    assert abs(np.mean(z * z)) < 0.01          # circular: E[z^2] = 0
    assert abs(np.mean(z.real * z.imag)) < 0.01


@pytest.mark.parametrize("I,alpha,kappa", [(3, 0.3, 10.0), (8, 0.2, 50.0)])
def test_basis_transforms_meet_the_condition_bound(I, alpha, kappa):
    P = draw_P(np.random.default_rng(1), 64, I, alpha, kappa)
    assert np.all(np.linalg.cond(P) < kappa)
    # P = I + alpha G: the off-diagonal entries have variance alpha^2
    off = P[:, ~np.eye(I, dtype=bool)]
    assert abs(np.mean(np.abs(off) ** 2) / alpha ** 2 - 1.0) < 0.25


def test_distributions_of_the_model_parameters():
    p = make_problem(3, 3, 64, 2000, seed=2)
    assert p.y.shape == (3, 64, 2000) and p.v_true.shape == (3, 64, 2000)
    assert p.lam_true.shape == (64, 3, 3) and p.P_true.shape == (64, 3, 3)
    # Gamma(shape 1/2, scale 1): mean 1/2, variance 1/2
    assert abs(p.v_true.mean() - 0.5) < 0.01 and abs(p.v_true.var() - 0.5) < 0.03
    # log-normal lambda: ln lambda ~ N(0, 1)
    ll = np.log(p.lam_true)
    assert abs(ll.mean()) < 0.15 and abs(ll.std() - 1.0) < 0.15
    # perturbed-truth initial estimate: log-ratios with standard deviation 0.3
    assert abs(np.log(p.v0 / p.v_true).std() - 0.3) < 0.01
    assert abs(np.log(p.lam0 / p.lam_true).std() - 0.3) < 0.05
    E = np.linalg.solve(p.P_true, p.P0) - np.eye(3)[None]      # P0 = P (I + 0.1 G')
    assert abs(np.mean(np.abs(E) ** 2) / 0.01 - 1.0) < 0.2


def test_mixture_covariance_is_the_model_covariance():
    """Given v and Lambda, y(n, f) ~ CN(0, sum_j v_j P^{-H} Lambda_j P^{-1}):
    whitening every point by its model covariance leaves unit-variance,
    uncorrelated entries."""
    p = make_problem(3, 3, 8, 4000, seed=3)
    # through the transformed basis: y~ = P^H y has covariance diag(sigma)
    yt = np.einsum("fai,afn->ifn", p.P_true.conj(), p.y)
    sigma = np.einsum("jfn,fji->ifn", p.v_true, p.lam_true)
    w = yt / np.sqrt(sigma)
    C = np.einsum("ifn,kfn->ik", w, w.conj()) / (8 * 4000)
    assert np.abs(C - np.eye(3)).max() < 0.03


def test_source_images_sum_to_the_mixture():
    p = make_problem(2, 3, 4, 50, seed=4, keep_images=True)
    np.testing.assert_allclose(p.x.sum(axis=0), p.y, rtol=0, atol=1e-12)


def test_same_seed_same_numbers_other_seed_other_numbers():
    a, b, c = make_problem(2, 2, 3, 20, seed=5), make_problem(2, 2, 3, 20, seed=5), make_problem(2, 2, 3, 20, seed=6)
    for f in ("y", "v_true", "lam_true", "P_true", "v0", "lam0", "P0"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(getattr(a, f), getattr(c, f))


def test_batches():
    Ns = batch_lengths(256, 200, 4000, seed=3)
    assert len(Ns) == 256 and min(Ns) >= 200 and max(Ns) <= 4000
    assert abs(np.mean(Ns) - 2100) < 150        # uniform on [200, 4000]
    probs = make_batch(2, 2, 3, [10, 17], seed=9)
    ref = make_problem(2, 2, 3, 17, seed=9 + 7919)
    assert np.array_equal(probs[1].y, ref.y) and probs[1].N == 17


def test_device_generator_draws_the_same_model():
    """make_batch_device (torch's generator, here on the CPU) draws the same
    distributions into the batch layout: padding y = 0 and v = 1, v0 with
    mean 1/2 e^{0.045} (Gamma(1/2, 1) times the log-normal perturbation)."""
    torch = pytest.importorskip("torch")
    Ns = [1001, 2002]
    y, v0, lam0, P0, Ns_, off = synth.make_batch_device(3, 2, 16, Ns, seed=7, device="cpu",
                                                        complex_dtype=torch.complex128)
    assert list(off) == [0, 1004, 3008] and lam0.shape == (2, 16, 2, 3) and P0.shape == (2, 16, 3, 3)
    yb = y.view(-1)[: 3 * 16 * 1004].view(3, 16, 1004)
    vb = v0.view(-1)[: 2 * 16 * 1004].view(2, 16, 1004)
    assert torch.all(yb[:, :, 1001:] == 0) and torch.all(vb[:, :, 1001:] == 1)
    v = vb[:, :, :1001].numpy()
    assert abs(v.mean() / (0.5 * np.exp(0.045)) - 1.0) < 0.05
    assert np.all(v > 0)
