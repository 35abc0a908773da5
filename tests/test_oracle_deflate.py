"""Pins of the oracle's projection deflation (A <- A (I - z z^T), z = x / ||x||): checked
against what the mathematics fixes, not against a retyped formula."""
import numpy as np

from paper_1212_4137_gb300 import inputs as I


def test_deflated_matrix_annihilates_z(oracle):
    A = I.gaussian_matrix(40, 60, 3)
    x = I.gaussian_matrix(1, 60, 4)[0]
    D = oracle.deflate(A, x)
    assert np.max(np.abs(D @ x)) <= 1e-12 * np.abs(A).sum(axis=1).max() * np.abs(x).max()


def test_leading_singular_vector_removed(oracle):
    # deflating by the leading right singular vector leaves the other singular values
    A = I.gaussian_matrix(30, 50, 5)
    _, sv, vt = np.linalg.svd(A, full_matrices=False)
    D = oracle.deflate(A, vt[0])
    sd = np.linalg.svd(D, compute_uv=False)
    assert np.allclose(sd[:-1], sv[1:], rtol=1e-12)
    assert sd[-1] <= 1e-10 * sv[0]


def test_rank_one_spike_removed_exactly(oracle):
    rng = np.random.default_rng(6)
    u, v = rng.standard_normal(25), rng.standard_normal(70)
    A = np.outer(u, v)
    assert np.max(np.abs(oracle.deflate(A, 3.0 * v))) <= 1e-13 * np.abs(A).max()


def test_idempotent_and_scale_free(oracle):
    A = I.gaussian_matrix(20, 35, 7)
    x = I.gaussian_matrix(1, 35, 8)[0]
    D = oracle.deflate(A, x)
    assert np.allclose(oracle.deflate(D, x), D, atol=1e-12)
    assert np.allclose(oracle.deflate(A, -2.5 * x), D, atol=1e-12)
