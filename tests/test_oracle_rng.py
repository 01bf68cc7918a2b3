"""Pins of the oracle's counter-based generator and group exponential."""
import os

import numpy as np
from scipy import stats

import helpers as H
from paper_2112_04556_gb300 import inputs


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_philox_kat():
    """(counter, key, output) triples from tests/golden/philox4x32_10_kat.txt."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_lib):
    """Philox4x32-10 known-answer vectors of its authors' reference distribution
    (Salmon, Moraes, Dror, Shaw, SC'11; Random123 kat_vectors)."""
    kat = load_philox_kat()
    assert len(kat) == 3
    for ctr, key, out in kat:
        assert oracle_lib.philox4x32_10(ctr, key).tolist() == out


def test_gaussian_field_statistics(oracle_lib):
    L = (8, 8, 8, 8)
    g = oracle_lib.gauss_field(L, seed=7, stream=3, tag=0).ravel()
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    assert stats.kstest(g, "norm").pvalue > 1e-3
    g2 = oracle_lib.gauss_field(L, seed=7, stream=4, tag=0).ravel()
    assert abs(np.corrcoef(g, g2)[0, 1]) < 5 / np.sqrt(g.size)
    u = np.array([oracle_lib.uniform(11, n) for n in range(2000)])
    assert u.min() > 0 and u.max() <= 1 and stats.kstest(u, "uniform").pvalue > 1e-3


def test_exp_matches_eigendecomposition(oracle_lib):
    """exp(i h^a T^a) against numpy's Hermitian eigensolver route; unitary, det 1."""
    rng = np.random.default_rng(3)
    h = rng.standard_normal((200, 8)) * np.array([[0.01]] * 50 + [[1.0]] * 100 + [[7.0]] * 50)
    E = oracle_lib.exp_i(h)
    M = H.to_mat(h)
    w, v = np.linalg.eigh(M)
    ref = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * w), np.conj(v))
    assert np.abs(E - ref).max() < 1e-13
    assert np.abs(H.mm(E, H.dag(E)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(E) - 1).max() < 1e-13
