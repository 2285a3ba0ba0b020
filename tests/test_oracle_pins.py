"""Pins of the FP64 oracle against what the paper states and the mathematics fixes.

None of these tests retypes an oracle formula: each compares the oracle with an
independent fact (a printed Bloch form, a closed-form eigenvector, a quantised
invariant, an exact identity, or an independent brute-force computation).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2312_13051_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "paper_invariants.json")))
P = I.Plane

# Independent Pauli matrices for the printed Bloch forms.
s0 = np.eye(2, dtype=complex)
s1 = np.array([[0, 1], [1, 0]], dtype=complex)
s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
s3 = np.diag([1.0 + 0j, -1.0])


def printed_forms():
    """H(k) as printed in the paper (Eqs. 4, 7, 9) or as defined for the named models."""
    k = np.kron
    return {
        "eq4": (I.chern_eq4(1.5), lambda kx, ky, kz:
                np.sin(kx) * s1 + np.sin(ky) * s2 + (np.cos(kx) + np.cos(ky) + 1.5) * s3),
        "eq7": (I.bhz_eq7(1.5), lambda kx, ky, kz:
                np.sin(kx) * k(s1, s1) + np.sin(ky) * k(s1, s2)
                + (np.cos(kx) + np.cos(ky) + 1.5) * k(s3, s0)),
        "eq9": (I.choti_eq9(1.0), lambda kx, ky, kz:
                np.sin(kx) * k(s1, s1) + np.sin(ky) * k(s1, s2) + np.sin(kz) * k(s1, s3)
                + (np.cos(kx) + np.cos(ky) + np.cos(kz) - 1.5) * k(s3, s0)
                + 1.0 * (np.cos(kx) - np.cos(ky)) * k(s2, s0)),
        "spin_hall": (I.spin_hall(1.0), lambda kx, ky, kz:
                      np.sin(kx) * k(s1, s3) + np.sin(ky) * k(s2, s0)
                      + (1.0 - np.cos(kx) - np.cos(ky)) * k(s3, s0)),
        "bbh": (I.bbh(0.5, 0.5, 1.0, 1.0), lambda kx, ky, kz:
                (0.5 + np.cos(kx)) * k(s1, s0) + np.sin(kx) * (-k(s2, s3))
                + (0.5 + np.cos(ky)) * (-k(s2, s2)) + np.sin(ky) * (-k(s2, s1))),
        # Eq. 10 with the printed s0 (x) t0 term read as s0 (x) t1 (chiral symmetry)
        "eq10": (I.quadrupolar_eq10(0.5), lambda kx, ky, kz:
                 np.sin(kx) * k(s1, s3) + np.sin(ky) * k(s2, s3)
                 + (np.cos(kx) + np.cos(ky) + 1.0) * k(s3, s3)
                 + 0.5 * (np.cos(kx) - np.cos(ky)) * k(s0, np.array([[0, 1], [1, 0]], dtype=complex))),
        "ssh": (I.ssh(0.7, 1.3), lambda kx, ky, kz:
                np.array([[0, 0.7 + 1.3 * np.exp(-1j * kx)], [0.7 + 1.3 * np.exp(1j * kx), 0]])),
    }


@pytest.mark.parametrize("name", ["eq4", "eq7", "eq9", "eq10", "spin_hall", "bbh", "ssh"])
def test_bloch_sum_matches_printed_form(name):
    """Step 1 (Bloch sum over the hopping list) equals the printed H(k), k = 2 pi f."""
    model, Hk = printed_forms()[name]
    rng = np.random.default_rng(1)
    for f in rng.uniform(-1, 1, size=(6, 3)):
        H = O.bloch_hamiltonian(model, f)
        np.testing.assert_allclose(H, Hk(*(2 * np.pi * f)), atol=1e-13)
    # periodic gauge: H(f + G) = H(f) for integer G (closure of Eq. 2)
    f = rng.uniform(size=3)
    np.testing.assert_allclose(O.bloch_hamiltonian(model, f + [1, -2, 3]),
                               O.bloch_hamiltonian(model, f), atol=1e-12)


@pytest.mark.parametrize("N", [7, 16, 40])
def test_ssh_berry_phase_quantised(N):
    """SSH chain: Berry phase 0 for v > w and pi for v < w, exactly on any mesh."""
    plane = P(N, 1, trans_dir=(0, 0, 0))
    ph, _ = O.wilson_loop(I.ssh(1.0, 0.5), plane, 1)
    assert abs(ph[0, 0]) < 1e-12
    ph, _ = O.wilson_loop(I.ssh(0.5, 1.0), plane, 1)
    assert abs(abs(ph[0, 0]) - np.pi) < 1e-12


def test_chern_eq4_winding_paper():
    """Eq. 4: WCCs interpolate from 0 to 1, C = 1 via Eq. 6."""
    ph, gap = O.wilson_loop(I.chern_eq4(1.5), P(40, 40), 1)
    assert gap.min() > 0.5
    C = O.winding(ph)
    assert abs(C - GOLDEN["chern_eq4_wcc_winding"]["value"]) < 1e-9


def _plaquette_chern(model, N, p):
    """Lattice Chern number from plaquette products of det<u_k|u_k'> (brute force)."""
    f = O.plane_points(P(N, N))
    U = [[O.occupied_states(O.bloch_hamiltonian(model, f[i, j]), p)[1] for j in range(N)]
         for i in range(N)]

    def link(a, b):
        z = np.linalg.det(a.conj().T @ b)
        return z / abs(z)

    total = 0.0
    for i in range(N):
        for j in range(N):
            u00, u10 = U[i][j], U[i][(j + 1) % N]
            u01, u11 = U[(i + 1) % N][j], U[(i + 1) % N][(j + 1) % N]
            # loop direction = j (k_x), transverse = i (k_y)
            z = link(u00, u10) * link(u10, u11) / link(u01, u11) / link(u00, u01)
            total += np.angle(z)
    return total / (2 * np.pi)


def _skyrmion_degree(d, N):
    """Degree of d/|d| on the torus: signed solid angle of the triangulated image."""
    g = np.linspace(0, 2 * np.pi, N, endpoint=False)
    D = np.array([[d(kx, ky) for kx in g] for ky in g])
    D /= np.linalg.norm(D, axis=-1, keepdims=True)

    def omega(a, b, c):
        num = np.dot(a, np.cross(b, c))
        den = 1 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
        return 2 * np.arctan2(num, den)

    tot = 0.0
    for i in range(N):
        for j in range(N):
            a, b = D[i, j], D[i, (j + 1) % N]
            c, e = D[(i + 1) % N, (j + 1) % N], D[(i + 1) % N, j]
            tot += omega(a, b, c) + omega(a, c, e)
    return tot / (4 * np.pi)


def test_chern_eq4_cross_checks():
    """The WCC winding equals the plaquette (lattice) Chern number built from the same
    states, and |C| equals the degree of d/|d|, a quantity with no eigenvectors in it."""
    model = I.chern_eq4(1.5)
    ph, _ = O.wilson_loop(model, P(24, 24), 1)
    assert abs(O.winding(ph) - _plaquette_chern(model, 24, 1)) < 1e-9
    deg = _skyrmion_degree(lambda kx, ky: np.array(
        [np.sin(kx), np.sin(ky), np.cos(kx) + np.cos(ky) + 1.5]), 48)
    assert abs(abs(deg) - 1) < 1e-9


def _covers_circle(phases, bins=16):
    """True when every phase bin of width 2pi/bins is visited by some WCC (gapless).

    The transverse grid must be fine enough that no WCC moves by more than one bin
    between neighbouring samples."""
    idx = np.floor((np.asarray(phases).ravel() + np.pi) / (2 * np.pi) * bins).astype(int) % bins
    return np.unique(idx).size == bins


def test_bhz_eq7_gapless_z2():
    """Eq. 7: fully connected WCC spectrum; the s3 (x) t3 sectors carry |C| = 1."""
    assert GOLDEN["bhz_eq7_wcc_spectrum"]["value"] == "gapless"
    model = I.bhz_eq7(1.5)
    ph, _ = O.wilson_loop(model, P(40, 128), 2)
    assert np.abs(np.diff(ph, axis=0)).max() < 2 * np.pi / 16
    assert _covers_circle(ph)
    assert abs(O.winding(ph)) < 1e-9
    S = np.kron(s3, s3)
    down, _, _, _ = O.spin_resolved_wilson_loop(model, P(30, 30), 2, S, -1)
    up, _, _, _ = O.spin_resolved_wilson_loop(model, P(30, 30), 2, S, +1)
    assert abs(abs(O.winding(down)) - 1) < 1e-9
    assert abs(O.winding(down) + O.winding(up)) < 1e-9


def test_spin_hall_windings():
    """Spin-Hall model: total winding 0; s_z-down sector -1, s_z-up sector +1.

    The s_z = +1 block sin kx tx + sin ky ty + (1 - cos kx - cos ky) tz is Eq. 4's
    d-vector shifted by (pi, pi) and rotated by pi about z (same degree, +1 by
    Eq. 4's pin); the s_z = -1 block flips the sign of d_x (degree -1).
    """
    wl = I.config_spin_hall()
    ph, gap = O.wilson_loop(wl.model, wl.plane, 2)
    assert abs(O.winding(ph)) < 1e-9
    assert abs(gap.min() - 2.0) < 1e-9      # |d| >= 1 at m = 1, so the direct gap is >= 2
    dn, pso, pgap, _ = O.spin_resolved_wilson_loop(wl.model, wl.plane, 2, wl.spin_op, -1)
    up, _, _, _ = O.spin_resolved_wilson_loop(wl.model, wl.plane, 2, wl.spin_op, +1)
    assert abs(O.winding(dn) + 1) < 1e-9 and abs(O.winding(up) - 1) < 1e-9
    np.testing.assert_allclose(np.sort(pso, axis=-1), np.broadcast_to([-1.0, 1.0], pso.shape),
                               atol=1e-12)     # s_z is conserved: PSO eigenvalues are +-1
    assert abs(pgap - 1) < 1e-12


def test_choti_eq9_paper_statements():
    """Eq. 9, Delta0 = 1: gapped WCCs at kz = 0 (Fig. 4a), |C_s| = 1 with
    s = s3 (x) t3 (Fig. 4c), nested spectrum winding once over kz (Fig. 4b)."""
    model = I.choti_eq9(1.0)
    ph, _ = O.wilson_loop(model, P(30, 30), 2)
    wgap = min(abs(np.angle(np.exp(1j * (r[1] - r[0])))) for r in ph)
    assert GOLDEN["choti_eq9_kz0_wcc_spectrum"]["value"] == "gapped"
    assert wgap > 0.5 and not _covers_circle(ph)
    S = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    dn, _, _, _ = O.spin_resolved_wilson_loop(model, P(30, 30), 2, S, -1)
    assert abs(abs(O.winding(dn)) - GOLDEN["choti_eq9_kz0_abs_spin_chern"]["value"]) < 1e-9
    assert GOLDEN["choti_eq9_nested_vs_kz"]["value"] == "gapless"
    nkz = 12
    curve = []
    for kz in np.arange(nkz) / nkz:
        _, nest, _, _ = O.nested_wilson_loop(model, P(12, 12, origin=(0, 0, kz)), 2, m=1)
        curve.append(nest[0])
    assert abs(abs(O.winding(np.array(curve))) - 1) < 1e-9
    # Delta0 = 0 at kz = 0 reduces to a BHZ-like insulator: gapless WCCs
    ph0, _ = O.wilson_loop(I.choti_eq9(0.0), P(30, 128), 2)
    assert _covers_circle(ph0)


@pytest.mark.parametrize("gamma,expected", [(0.5, np.pi), (1.5, 0.0)])
def test_bbh_nested_polarisation(gamma, expected):
    """BBH quadrupole: nested polarisation 1/2 (phase pi) for |gamma/lambda| < 1 and 0
    for |gamma/lambda| > 1, at every base point of the first loop."""
    _, nest, wgap, _ = O.nested_wilson_loop(I.bbh(gamma, gamma), P(24, 24), 2, m=1)
    err = np.abs(np.angle(np.exp(1j * (nest - expected))))
    assert err.max() < 1e-10
    assert wgap > 0.1


def _cone_phase(alpha, N):
    """Closed-form discrete Berry phase of the lower band of h_x = sin(alpha)(cos k s1 +
    sin k s2) + cos(alpha) s3 on N points.  Its lower eigenvector in the periodic gauge
    is u(k) = (sin(alpha/2), -e^{ik} cos(alpha/2)); every Eq. 2 overlap
    <u(k + 2pi/N)|u(k)> equals sin^2(alpha/2) + cos^2(alpha/2) e^{-2 pi i / N}, so the
    loop is that number to the power N."""
    z = np.sin(alpha / 2) ** 2 + np.cos(alpha / 2) ** 2 * np.exp(-2j * np.pi / N)
    return float(np.angle(z ** N))


@pytest.mark.parametrize("alpha,N", [(0.3, 7), (1.1, 24), (2.0, 24), (2.9, 40)])
def test_cone_berry_phase_closed_form(alpha, N):
    """A non-quantised Wilson-loop phase fixed in closed form (sign-sensitive, unlike the
    0 / pi of SSH): the cone (x) SSH product block along kx, at several ky."""
    model = I.cone_ssh_product(alpha, 1.0, 0.5)
    ph, _ = O.wilson_loop(model, P(N, 5), 1)
    d = np.angle(np.exp(1j * (ph[:, 0] - _cone_phase(alpha, N))))
    assert np.abs(d).max() < 1e-12


# Wannier ladder (three decoupled blocks A, B, C; inputs.wannier_ladder): Wannier centres
# xbar ~ -0.45 (A), -0.2 (B), +0.3 (C) at every ky; nested phase of each block's band
# along ky: pi (A, SSH v < w), 0 (B and C, v > w).  The sector picked by (cut, first, m)
# is listed by hand from those positions: from cut = -pi the order is A, B, C; from 0
# it is C, A, B; from -pi + 1 (past A at -0.45 * 2pi = -2.83) it is B, C, A.
LADDER_NESTED = {"A": np.pi, "B": 0.0, "C": 0.0}
LADDER_CASES = [(-np.pi, 0, 1, "A"), (-np.pi, 1, 1, "B"), (-np.pi, 2, 1, "C"),
                (-np.pi, 0, 2, "AB"), (-np.pi, 1, 2, "BC"), (0.0, 0, 1, "C"), (0.0, 1, 1, "A"),
                (0.0, 2, 1, "B"), (0.0, 0, 2, "CA"), (-np.pi + 1.0, 0, 1, "B"),
                (-np.pi + 1.0, 2, 1, "A"), (-np.pi + 1.0, 1, 2, "CA")]


def _ladder_thetas(N):
    return {b: _cone_phase(I.ladder_alpha(x), N) for b, x in zip("ABC", I.LADDER_XBAR)}


@pytest.mark.parametrize("cut,first,m,blocks", LADDER_CASES)
def test_nested_sector_choice(cut, first, m, blocks):
    """Eq. 8 on the Wannier ladder: the nested phases are those of the blocks in the
    chosen sector (at every base point), and the Wannier gap is the closed-form
    distance between the sector's centres and the others'."""
    N, Nt = 24, 20
    _, nest, wgap, _ = O.nested_wilson_loop(I.wannier_ladder(), P(N, Nt), 3, cut=cut,
                                            first=first, m=m)
    want = np.sort([LADDER_NESTED[b] for b in blocks])
    for j in range(N):
        assert O.circular_match_error(nest[j], want) < 1e-10
    th = _ladder_thetas(N)
    gaps = [abs(np.angle(np.exp(1j * (th[a] - th[b])))) for a in blocks for b in "ABC"
            if b not in blocks]
    assert abs(wgap - min(gaps)) < 1e-12


def test_ladder_first_loop_closed_form():
    """The first loop of the ladder: the three closed-form cone phases at every row."""
    N = 24
    ph, gap = O.wilson_loop(I.wannier_ladder(), P(N, 10), 3)
    want = np.sort(list(_ladder_thetas(N).values()))
    for r in range(10):
        assert O.circular_match_error(ph[r], want) < 1e-12
    # At ky = pi the SSH parts have |d_y| = |v - w| = 0.6, 0.5, 0.4; a block's levels are
    # +-1 +-|d_y|, so the three occupied ones are -1.6, -1.5, -1.4 and the next is
    # -|1 - 0.4| = -0.6: direct gap 0.8 on row 5 (t2 = 1/2).
    assert abs(gap[5] - 0.8) < 1e-12


@pytest.mark.parametrize("n,p,seed", [(6, 3, 11), (8, 4, 5)])
def test_nested_full_sector_is_transverse_loop(n, p, seed):
    """With the whole occupied space as the sector (m = p) the Wannier states span U(k),
    so the nested loop at base point t1 is the ordinary Wilson loop along the transverse
    direction at that t1 (the nested construction adds nothing).  Random models make
    the Wilson matrix non-normal, so its eigenvectors are not orthogonal and the
    orthonormalisation of the sector basis matters."""
    model = I.random_hermitian_model(n, seed)
    plane = P(9, 7)
    _, nest, _, _ = O.nested_wilson_loop(model, plane, p, m=p)
    for j in range(plane.N):
        row = P(plane.N_t, 1, origin=(j / plane.N, 0.0, 0.0), loop_dir=(0, 1, 0),
                trans_dir=(1.0, 0.0, 0.0))
        ref, _ = O.wilson_loop(model, row, p)
        assert O.circular_match_error(nest[j], ref[0]) < 1e-12


def test_grouped_bloch_sum():
    """H(f) summed per translation block equals the direct sum over the hopping list."""
    rng = np.random.default_rng(4)
    for model in (I.manyband(16), I.choti_eq9(), I.supercell(I.spin_hall(1.0), 3, W=1.0, seed=2)):
        blocks = O.translation_blocks(model)
        for _ in range(3):
            f = rng.uniform(-1, 1, 3)
            np.testing.assert_allclose(O.bloch_hamiltonian_grouped(blocks, f),
                                       O.bloch_hamiltonian(model, f), atol=1e-13)


def test_gauge_invariance():
    """Eigenphases are unchanged by a random unitary gauge U(k) -> U(k) G(k)."""
    model = I.random_hermitian_model(6, seed=3)
    rng = np.random.default_rng(7)

    def gauge(i, j, p):
        Q, _ = np.linalg.qr(rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p)))
        return Q

    plane = P(15, 5)
    a, _ = O.wilson_loop(model, plane, 3)
    b, _ = O.wilson_loop(model, plane, 3, gauge=gauge)
    for r in range(plane.N_t):
        assert O.circular_match_error(a[r], b[r]) < 1e-12


def test_two_band_closed_form_eigenvectors():
    """p = 1 loop of Eq. 4 with the closed-form lower eigenvector of d.sigma,
    u = (d_x - i d_y, -(d_z + |d|)), against the oracle's loop built on zheevd."""
    model = I.chern_eq4(1.5)
    N, Nt = 30, 9
    ph, _ = O.wilson_loop(model, P(N, Nt), 1)
    for i in range(Nt):
        ky = 2 * np.pi * i / Nt
        us = []
        for j in range(N):
            kx = 2 * np.pi * j / N
            d = np.array([np.sin(kx), np.sin(ky), np.cos(kx) + np.cos(ky) + 1.5])
            u = np.array([d[0] - 1j * d[1], -(d[2] + np.linalg.norm(d))])
            us.append(u / np.linalg.norm(u))
        z = 1.0 + 0j
        for j in range(N):
            z *= np.vdot(us[(j + 1) % N], us[j])
        assert abs(np.angle(np.exp(1j * (np.angle(z) - ph[i, 0])))) < 1e-12


def _jacobi_eigvals(A, sweeps=30):
    """Cyclic complex Jacobi in plain Python loops (independent of LAPACK)."""
    A = np.array(A, dtype=complex)
    n = A.shape[0]
    for _ in range(sweeps):
        off = sum(abs(A[p, q]) ** 2 for p in range(n) for q in range(n) if p != q)
        if off < 1e-30:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(A[p, q]) < 1e-300:
                    continue
                phase = A[p, q] / abs(A[p, q])
                tau = (A[q, q].real - A[p, p].real) / (2 * abs(A[p, q]))
                t = np.sign(tau) / (abs(tau) + np.sqrt(1 + tau * tau)) if tau != 0 else 1.0
                c = 1 / np.sqrt(1 + t * t)
                s = t * c
                J = np.eye(n, dtype=complex)
                J[p, p], J[q, q] = c, c
                J[p, q], J[q, p] = s * phase, -s * np.conj(phase)
                A = J.conj().T @ A @ J
    return np.sort(A.diagonal().real)


def test_eigh_against_independent_jacobi():
    """Step 2's eigenvalues against a hand-written Jacobi on 4 x 4 and 2 x 2 cases."""
    rng = np.random.default_rng(5)
    cases = [I.spin_hall(1.0), I.bbh(0.5, 0.5), I.choti_eq9(1.0), I.chern_eq4(1.5)]
    for model in cases:
        for f in rng.uniform(size=(4, 3)):
            H = O.bloch_hamiltonian(model, f)
            lam, _, _ = O.occupied_states(H, 1)
            np.testing.assert_allclose(lam, _jacobi_eigvals(H), atol=1e-12)


def test_eigenphases_known_spectrum():
    """Eigenphases of W = V diag(e^{i theta}) V^{-1} (non-unitary V) recover theta."""
    rng = np.random.default_rng(11)
    for p in (1, 2, 5, 8):
        th = np.sort(rng.uniform(-np.pi, np.pi, p))
        th[-1] = np.pi
        V = np.eye(p) + 0.3 * (rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p)))
        W = V @ np.diag(np.exp(1j * th)) @ np.linalg.inv(V)
        assert O.circular_match_error(O.eigenphases(W), th) < 1e-12


def test_cyclic_base_transport():
    """The loop based at k_{j+1} is M_j (loop based at k_j) M_j^{-1}: same spectrum,
    eigenvectors carried by the overlap (Eq. 8's Wannier basis along the loop)."""
    model = I.random_hermitian_model(5, seed=2)
    f = O.plane_points(P(9, 1))
    U = [O.occupied_states(O.bloch_hamiltonian(model, f[0, j]), 2)[1] for j in range(9)]
    for j in range(9):
        M = O.overlap(U[(j + 1) % 9], U[j])
        np.testing.assert_allclose(O.cyclic_wilson_matrix(U, (j + 1) % 9) @ M,
                                   M @ O.cyclic_wilson_matrix(U, j), atol=1e-13)
    np.testing.assert_allclose(O.cyclic_wilson_matrix(U, 0), O.wilson_matrix(U), atol=1e-15)


def test_supercell_band_folding():
    """Sec. II A supercells: eig H_sc(F) = union_g eig H((F + g)/L) (theta = 0 TBC)."""
    prim = I.spin_hall(1.0)
    rng = np.random.default_rng(4)
    for L in (2, 3):
        sc = I.supercell(prim, L)
        for F in rng.uniform(size=(3, 3)) * [1, 1, 0]:
            lam_sc = np.linalg.eigvalsh(O.bloch_hamiltonian(sc, F))
            lam = np.concatenate([np.linalg.eigvalsh(O.bloch_hamiltonian(
                prim, (F + [gx, gy, 0]) / [L, L, 1])) for gx in range(L) for gy in range(L)])
            np.testing.assert_allclose(lam_sc, np.sort(lam), atol=1e-12)


def test_supercell_spin_chern_unchanged():
    """A clean 2 x 2 supercell (p = 8) carries the primitive cell's spin-Chern number."""
    sc = I.supercell(I.spin_hall(1.0), 2)
    S = np.kron(np.eye(4), I.SPIN_HALL_SZ)
    dn, _, _, _ = O.spin_resolved_wilson_loop(sc, P(20, 20), 8, S, -1)
    assert abs(O.winding(dn) + 1) < 1e-9


def test_flux_plaquettes_and_hofstadter():
    """Peierls flux: every plaquette of the torus (seams included) encloses 2pi/L^2;
    the isolated lowest Hofstadter band at flux 1/4 has |C| = 1."""
    L = 3
    sc = I.supercell(I.square_lattice(1.0), L, flux=True)
    amp = {}
    for R, a, b, t in zip(map(tuple, sc.R), sc.i, sc.j, sc.t):
        amp[(int(a), int(b), R)] = t

    def site(x, y):
        sx, sy = x // L, y // L
        return (x % L) * L + (y % L), (sx, sy)

    def hop(x0, y0, x1, y1):
        a, A = site(x0, y0)
        b, B = site(x1, y1)
        return amp[(a, b, (B[0] - A[0], B[1] - A[1], 0))]

    for x in range(L):
        for y in range(L):
            z = hop(x, y, x + 1, y) * hop(x + 1, y, x + 1, y + 1) \
                * hop(x + 1, y + 1, x, y + 1) * hop(x, y + 1, x, y)
            assert abs(np.angle(z * np.exp(-2j * np.pi / L**2))) < 1e-12 \
                or abs(np.angle(z * np.exp(2j * np.pi / L**2))) < 1e-12
            assert abs(np.angle(z) - np.angle(hop(0, 0, 1, 0) * hop(1, 0, 1, 1)
                                              * hop(1, 1, 0, 1) * hop(0, 1, 0, 0))) < 1e-12
    hof = I.supercell(I.square_lattice(1.0), 2, flux=True)
    ph, gap = O.wilson_loop(hof, P(24, 24), 1)
    assert gap.min() > 0.1
    assert abs(abs(O.winding(ph)) - 1) < 1e-9


def test_disorder_recipe():
    """On-site disorder: one uniform value in [-W/2, W/2] per cell on all its orbitals."""
    W = 2.0
    sc = I.supercell(I.spin_hall(1.0), 4, W=W, seed=9)
    H0 = O.bloch_hamiltonian(sc, [0.1, 0.2, 0])
    Hc = O.bloch_hamiltonian(I.supercell(I.spin_hall(1.0), 4), [0.1, 0.2, 0])
    D = np.diag(H0 - Hc).real
    assert np.abs(np.diag(np.diag(H0 - Hc)) - (H0 - Hc)).max() < 1e-14
    cells = D.reshape(16, 4)
    assert np.allclose(cells, cells[:, :1]) and np.all(np.abs(cells) <= W / 2)
    assert np.ptp(cells[:, 0]) > 0.5


def test_error_conditions():
    """EGAP where the gap closes on the mesh; EPSOGAP / EINVAL on bad arguments."""
    with pytest.raises(O.OracleError) as e:
        O.wilson_loop(I.chern_eq4(2.0), P(8, 8), 1)       # gap closes at (pi, pi)
    assert e.value.status == "EGAP"
    wl = I.config_spin_hall()
    with pytest.raises(O.OracleError) as e:
        O.spin_resolved_wilson_loop(wl.model, P(6, 6), 2, np.eye(4, dtype=complex), -1)
    assert e.value.status == "EPSOGAP"
    with pytest.raises(O.OracleError) as e:
        O.wilson_loop(wl.model, P(6, 6, loop_dir=(0.5, 0, 0)), 2)
    assert e.value.status == "EINVAL"


def test_unitarise_option():
    """Per-overlap polar factors: identical to the raw product for an s_z-conserving
    model, unit-modulus spectrum in general."""
    wl = I.config_spin_hall()
    a, _ = O.wilson_loop(wl.model, P(12, 6), 2)
    b, _ = O.wilson_loop(wl.model, P(12, 6), 2, unitarise=True)
    for r in range(6):
        assert O.circular_match_error(a[r], b[r]) < 1e-12
    model = I.random_hermitian_model(6, seed=3)
    f = O.plane_points(P(10, 1))
    U = [O.occupied_states(O.bloch_hamiltonian(model, f[0, j]), 3)[1] for j in range(10)]
    Wu = O.wilson_matrix(U, unitarise=True)
    np.testing.assert_allclose(np.abs(np.linalg.eigvals(Wu)), 1.0, atol=1e-12)
    assert np.abs(np.abs(np.linalg.eigvals(O.wilson_matrix(U))) - 1).max() > 1e-3


# ---------------------------------------------------------------- plaquette flux
def test_plaquette_flux_chern_eq4():
    """Sec. IV A coupling-matrix flux: Eq. 4 carries C = 1 (paper, Fig. 1), equal to the
    WCC winding of the same grid and to the degree of d/|d|; m = 3.5 is trivial."""
    model = I.chern_eq4(1.5)
    flux, C = O.plaquette_flux(model, P(24, 24), 1)
    assert abs(C - GOLDEN["chern_eq4_wcc_winding"]["value"]) < 1e-9
    assert np.all(np.abs(flux) <= np.pi)
    ph, _ = O.wilson_loop(model, P(24, 24), 1)
    assert abs(C - O.winding(ph)) < 1e-9
    d = lambda kx, ky: np.array([np.sin(kx), np.sin(ky), np.cos(kx) + np.cos(ky) + 1.5])
    assert abs(abs(C) - abs(_skyrmion_degree(d, 48))) < 1e-9
    _, C0 = O.plaquette_flux(I.chern_eq4(3.5), P(16, 16), 1)
    assert abs(C0) < 1e-9


def test_plaquette_flux_spin_sectors():
    """Spin-Hall model: total flux 0, s_z-down sector -1, s_z-up sector +1 (Sec. IV);
    the same with the independent product of normalised link determinants."""
    wl = I.config_spin_hall()
    plane = P(20, 20)
    _, C = O.plaquette_flux(wl.model, plane, 2)
    _, Cd = O.plaquette_flux(wl.model, plane, 2, wl.spin_op, -1)
    _, Cu = O.plaquette_flux(wl.model, plane, 2, wl.spin_op, +1)
    assert abs(C) < 1e-9 and abs(Cd + 1) < 1e-9 and abs(Cu - 1) < 1e-9
    assert abs(C - _plaquette_chern(wl.model, 20, 2)) < 1e-9
    assert abs(O.plaquette_flux(I.chern_eq4(1.5), P(16, 16), 1)[1]
               - _plaquette_chern(I.chern_eq4(1.5), 16, 1)) < 1e-9


def test_plaquette_flux_gauge_invariant():
    """Each plaquette's flux is unchanged by a random unitary change of basis of the
    states at every corner (gauge invariance of the closed loop)."""
    rng = np.random.default_rng(9)
    model = I.random_hermitian_model(5, 3)
    f = O.plane_points(P(3, 3))
    U = [[O.occupied_states(O.bloch_hamiltonian(model, f[i, j]), 2)[1] for j in range(3)]
         for i in range(3)]
    G = [[np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))[0]
          for _ in range(3)] for _ in range(3)]
    Ug = [[U[i][j] @ G[i][j] for j in range(3)] for i in range(3)]
    for i in range(3):
        for j in range(3):
            a = np.angle(np.linalg.det(O.plaquette_matrix(O.plaquette_corners(U, i, j, 3, 3))))
            b = np.angle(np.linalg.det(O.plaquette_matrix(O.plaquette_corners(Ug, i, j, 3, 3))))
            assert abs(np.angle(np.exp(1j * (a - b)))) < 1e-12


# ----------------------------------------------------------------------------
# Z2 index from WCC connectivity (largest-gap reading; Sec. II B, II C, III)
# ----------------------------------------------------------------------------

def _lines_to_phases(lines, Nt):
    """Eigenphases of hand-drawn WCC lines x_a(t2) (t2 = i / Nt, rows 0 .. Nt - 1)."""
    t = np.arange(Nt) / Nt
    x = np.stack([f(t) for f in lines], axis=1)
    th = 2 * np.pi * (np.mod(x + 0.5, 1.0) - 0.5)
    return np.sort(th, axis=1)


def test_z2_synthetic_spectra():
    """Drawn spectra whose partner switching is known: one Kramers pair that switches
    partners between t2 = 0 and 1/2 gives 1, a pair that returns gives 0, two switching
    pairs give 0; a rigid shift, a mirror x -> -x and the order inside a row change
    nothing."""
    Nt = 400
    switch = [lambda t: t, lambda t: -t]                                   # 0 -> 1/2 and 0 -> -1/2
    stay = [lambda t: 0.2 + 0.05 * np.sin(2 * np.pi * t), lambda t: 0.2 - 0.05 * np.sin(2 * np.pi * t)]
    second = [lambda t: 0.3 + t, lambda t: 0.3 - t]
    cases = [(switch, 1), (stay, 0), (switch + second, 0), (switch + stay, 1), (stay + second, 1)]
    for lines, nu in cases:
        ph = _lines_to_phases(lines, Nt)
        assert O.z2_largest_gap(ph)[0] == nu
        shifted = _lines_to_phases([(lambda f: (lambda t: f(t) + 0.137))(f) for f in lines], Nt)
        assert O.z2_largest_gap(shifted)[0] == nu
        assert O.z2_largest_gap(np.sort(-ph, axis=1))[0] == nu
        rng = np.random.default_rng(5)
        assert O.z2_largest_gap(rng.permuted(ph, axis=1))[0] == nu
    # the widest gap of a single pair at the Kramers-degenerate row t2 = 0 is the whole cell
    nu, _, mids, widths = O.z2_largest_gap(_lines_to_phases(switch, 8))
    assert widths[0] == 1.0 and abs(mids[0] - 0.5) < 1e-15


def test_z2_paper_models():
    """Eq. 7 (m = 1.5): nu = 1 (paper); m = 3.5 (no band inversion): 0.  For the
    s_z-conserving spin-Hall model nu equals |C_down| mod 2 from the spin-resolved
    winding (the paper's nu = (C1 - C2) / 2 mod 2 with C1 = -C2), a second route."""
    ph, _ = O.wilson_loop(I.bhz_eq7(1.5), P(24, 32), 2)
    assert O.z2_largest_gap(ph)[0] == GOLDEN["bhz_eq7_z2"]["value"]
    ph, _ = O.wilson_loop(I.bhz_eq7(3.5), P(24, 32), 2)
    assert O.z2_largest_gap(ph)[0] == 0
    for m in (1.0, 3.0):
        wl = I.config_spin_hall()
        model = I.spin_hall(m)
        ph, _ = O.wilson_loop(model, P(24, 16), 2)
        dn, _, _, _ = O.spin_resolved_wilson_loop(model, P(24, 16), 2, wl.spin_op, -1)
        assert O.z2_largest_gap(ph)[0] == int(round(abs(O.winding(dn)))) % 2
        assert O.z2_largest_gap(ph)[0] == (1 if m == 1.0 else 0)


def test_z2_vacancy_supercells():
    """Sec. II C: removing the cells near the origin of an Eq. 7 supercell leaves the
    spectrum gapless and nu = 1 (Fig. 5); the conserved s3 (x) t3 sector winds -1."""
    for L, r in ((5, 0.0), (6, 1.0)):
        wl = I.config_vacancy(L, r, 12)
        removed = I.vacancy_cells(L, r).shape[0]
        assert removed == (1 if r == 0 else 5) and wl.model.n == 4 * (L * L - removed)
        ph, _ = O.wilson_loop(wl.model, P(12, 16), wl.p)
        assert O.z2_largest_gap(ph)[0] == GOLDEN["bhz_vacancy_z2"]["value"]
        dn, _, _, _ = O.spin_resolved_wilson_loop(wl.model, P(12, 16), wl.p, wl.spin_op, -1)
        assert abs(O.winding(dn) + 1) < 1e-9


def test_z2_strong_index_eq9():
    """Eq. 9 with Delta0 = 0 (strong topological insulator, Sec. III): nu = 1 on the
    kz = 0 plane and 0 on kz = pi, so the strong index nu0 = 1 and the weak indices
    vanish; the kx planes agree (nu0 is the same from every direction)."""
    assert GOLDEN["choti_eq9_delta0_zero"]["value"] == "strong"
    model = I.choti_eq9(0.0)
    z = {}
    for axis, (ld, td) in {2: ((1, 0, 0), (0, 1, 0)), 0: ((0, 1, 0), (0, 0, 1))}.items():
        for v in (0.0, 0.5):
            origin = [0.0, 0.0, 0.0]
            origin[axis] = v
            ph, _ = O.wilson_loop(model, P(24, 16, origin=tuple(origin), loop_dir=ld, trans_dir=td), 2)
            z[(axis, v)] = O.z2_largest_gap(ph)[0]
    assert (z[(2, 0.0)] + z[(2, 0.5)]) % 2 == 1 and z[(2, 0.5)] == 0
    assert (z[(0, 0.0)] + z[(0, 0.5)]) % 2 == 1 and z[(0, 0.5)] == 0


def test_z2_input_checks():
    with pytest.raises(O.OracleError):
        O.z2_largest_gap(np.zeros((7, 2)))
    with pytest.raises(O.OracleError):
        O.z2_largest_gap(np.zeros((8, 0)))


# ----------------------------------------------------------------------------
# Eq. 10, the disordered quadrupolar insulator (Sec. IV A)
# ----------------------------------------------------------------------------

def test_quadrupolar_eq10_paper_statements():
    """Eq. 10 (last term read as s0 (x) t1): chiral symmetry S^-1 H S = -H with
    S = s0 (x) t2 (stated in Sec. IV A), also for the disorder w s0 (x) t3; the
    spin-Chern number of the s = s0 (x) t3 sectors is 1 in magnitude (Fig. 6(b) at weak
    disorder), equal from the spin-resolved winding and the plaquette flux."""
    m = I.quadrupolar_eq10()
    assert GOLDEN["quadrupolar_eq10_chiral_operator"]["value"] == "sigma0 (x) tau2"
    Sc = I.EQ10_CHIRAL
    assert np.array_equal(Sc, np.kron(s0, s2))
    rng = np.random.default_rng(4)
    for f in rng.uniform(-1, 1, size=(5, 3)):
        H = O.bloch_hamiltonian(m, f)
        assert np.abs(np.linalg.inv(Sc) @ H @ Sc + H).max() < 1e-13
        lam = np.linalg.eigvalsh(H)
        assert lam[1] < 0 < lam[2]                      # insulating at half filling
    assert np.abs(np.linalg.inv(Sc) @ I.EQ10_SPIN @ Sc + I.EQ10_SPIN).max() == 0
    S = I.EQ10_SPIN
    dn, _, pg, _ = O.spin_resolved_wilson_loop(m, P(30, 30), 2, S, -1)
    up, _, _, _ = O.spin_resolved_wilson_loop(m, P(30, 30), 2, S, +1)
    expect = GOLDEN["quadrupolar_eq10_abs_spin_chern"]["value"]
    assert abs(abs(O.winding(dn)) - expect) < 1e-9 and abs(O.winding(dn) + O.winding(up)) < 1e-9
    _, C = O.plaquette_flux(m, P(20, 20), 2, S, -1)
    assert abs(C - O.winding(dn)) < 1e-9
    assert pg > 0.5


@pytest.mark.parametrize("L,seed", [(4, 1), (4, 2), (5, 1)])
def test_quadrupolar_eq10_median_split_fig6(L, seed):
    """Sec. IV A, Fig. 6(c)-(d) with the PSO sector taken as the p/2 most negative
    eigenvalues (split at the median, the alternative reading): the coupling-matrix
    flux gives |C_s| = 1 at W = 1 and C_s = 0 at W = 9, the two values the figure
    shows on either side of the disorder-driven transition."""
    g = GOLDEN["quadrupolar_eq10_spin_chern_vs_disorder"]
    for W, want in ((1.0, g["W1_abs"]), (9.0, g["W9"])):
        wl = I.config_quadrupolar(L, W, seed, nk=8)
        _, C = O.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1, pso_split="median")
        assert abs(abs(C) - want) < 1e-9, (W, C)


def test_median_split_equals_zero_split_when_sectors_are_even():
    """Where exactly p/2 PSO eigenvalues are negative at every k (the spin-Hall model,
    the clean Eq. 10 model), the median split selects the same sector as the split at
    zero: the spin-resolved phases agree."""
    for model, S in ((I.spin_hall(1.0), I.SPIN_HALL_SZ), (I.quadrupolar_eq10(), I.EQ10_SPIN)):
        for sign in (-1, 1):
            a = O.spin_resolved_wilson_loop(model, P(12, 10), 2, S, sign)[0]
            b = O.spin_resolved_wilson_loop(model, P(12, 10), 2, S, sign, pso_split="median")[0]
            for r in range(10):
                assert O.circular_match_error(a[r], b[r]) < 1e-12


def test_quadrupolar_eq10_disordered_supercells():
    """Sec. IV A, Fig. 6(c): with the chiral-preserving disorder w s0 (x) t3 per cell at
    W = 1 (below the gap closing near W = 5) the coupling-matrix flux of a supercell
    keeps |C_s| = 1.  At W = 9 the half-filled states of these small supercells no longer
    split evenly between the two s-sectors, so the fixed-size sector the method requires
    does not exist and the oracle reports EPSOGAP (the paper's C_s = 0 is not a number
    this reading produces)."""
    for L, seed in ((4, 1), (4, 2), (5, 1)):
        wl = I.config_quadrupolar(L, 1.0, seed)
        assert wl.model.n == 4 * L * L and wl.p == 2 * L * L
        _, C = O.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1)
        assert abs(abs(C) - GOLDEN["quadrupolar_eq10_abs_spin_chern"]["value"]) < 1e-9
    with pytest.raises(O.OracleError) as e:
        wl = I.config_quadrupolar(4, 9.0, 1)
        O.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1)
    assert e.value.status == "EPSOGAP"
