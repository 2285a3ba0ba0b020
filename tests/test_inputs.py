"""The seeded input generators shared by the oracle and the GPU tests, on the CPU:
sizes and fillings of the workloads, Hermitian hopping lists (every hopping has its
conjugate partner, so H(f) is Hermitian at any f), and deterministic seeds."""
import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I


def _partner_check(m):
    """Every (i, j, R, t) has (j, i, -R, conj t) in the list (duplicates summed)."""
    acc = {}
    for i, j, R, t in zip(m.i, m.j, map(tuple, m.R), m.t):
        acc[(int(i), int(j), R)] = acc.get((int(i), int(j), R), 0.0) + complex(t)
    for (i, j, R), t in acc.items():
        u = acc.get((j, i, tuple(-x for x in R)), 0.0)
        assert abs(t - np.conj(u)) <= 1e-12 * max(1.0, abs(t)), (i, j, R)


@pytest.mark.parametrize("make, n, p", [
    (I.config_spin_hall, 4, 2),
    (I.config_bbh, 4, 2),
    (lambda: I.config_disordered(3, seed=7), 36, 18),
    (lambda: I.config_quadrupolar(2, 1.0, seed=3), 16, 8),
    (lambda: I.config_vacancy(4, 1.0), None, None),
])
def test_workloads_are_hermitian_with_documented_sizes(make, n, p):
    wl = make()
    if n is not None:
        assert wl.model.n == n and wl.p == p
    assert wl.p == wl.model.n // 2
    _partner_check(wl.model)
    rng = np.random.default_rng(0)
    for f in rng.uniform(-1, 1, (3, 3)):
        H = oracle.bloch_hamiltonian(wl.model, f)   # raises on a non-Hermitian list
        assert np.allclose(H, H.conj().T)
    if wl.spin_op is not None:
        S = np.asarray(wl.spin_op)
        assert S.shape == (wl.model.n, wl.model.n) and np.allclose(S, S.conj().T)


def test_disorder_is_seeded_and_bounded():
    a = I.supercell(I.spin_hall(1.0), 4, W=2.0, seed=11)
    b = I.supercell(I.spin_hall(1.0), 4, W=2.0, seed=11)
    c = I.supercell(I.spin_hall(1.0), 4, W=2.0, seed=12)
    clean = I.supercell(I.spin_hall(1.0), 4)
    assert np.array_equal(a.t, b.t) and np.array_equal(a.R, b.R)
    assert not np.array_equal(a.t, c.t)
    # the disorder is on-site (R = 0, i = j) and lies in [-W/2, W/2]
    f = np.zeros(3)
    d = np.diag(oracle.bloch_hamiltonian(a, f) - oracle.bloch_hamiltonian(clean, f)).real
    off = oracle.bloch_hamiltonian(a, f) - oracle.bloch_hamiltonian(clean, f)
    assert np.allclose(off - np.diag(np.diag(off)), 0.0)
    assert np.all(np.abs(d) <= 1.0 + 1e-12) and np.abs(d).max() > 0.1


def test_many_band_model_shape():
    wl = I.config_manyband(N=5)
    assert wl.model.n == 256 and wl.p == 64 and wl.nested_m == 32
    assert np.abs(wl.model.R).max() <= 3
    H = oracle.bloch_hamiltonian(wl.model, np.array([0.1, 0.2, 0.0]))
    assert np.allclose(H, H.conj().T)
    S = np.asarray(wl.spin_op)
    assert np.allclose(np.sort(np.linalg.eigvalsh(S)), np.repeat([-1.0, 1.0], 128))


def test_random_hermitian_model():
    m = I.random_hermitian_model(20, 3)
    _partner_check(m)
    assert m.n == 20
