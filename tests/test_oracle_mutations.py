"""Planted mistakes in the oracle (on the CPU) must each fail at least one pin.

This shows that the pins in ``test_oracle_pins`` are strong enough: a dropped
closure, a conjugated or transposed overlap, a reversed product, a flipped
Fourier sign, an unprojected spin operator, the wrong bands, the wrong nested
sector (taken from the other end, or from a shifted cut) or Wannier states that
are not orthonormalised all get caught.
"""
import functools

import numpy as np
import pytest

import oracle
import oracle.wilson as W
import tests.test_oracle_pins as pins


def _all_pins():
    out = [functools.partial(pins.test_bloch_sum_matches_printed_form, n)
           for n in ("eq4", "eq7", "eq9", "spin_hall", "bbh", "ssh")]
    out += [functools.partial(pins.test_ssh_berry_phase_quantised, 7),
            pins.test_chern_eq4_winding_paper, pins.test_chern_eq4_cross_checks,
            pins.test_bhz_eq7_gapless_z2, pins.test_spin_hall_windings,
            functools.partial(pins.test_bbh_nested_polarisation, 0.5, np.pi),
            pins.test_choti_eq9_paper_statements, pins.test_eigenphases_known_spectrum,
            pins.test_two_band_closed_form_eigenvectors,
            pins.test_eigh_against_independent_jacobi, pins.test_plaquette_flux_chern_eq4,
            pins.test_plaquette_flux_spin_sectors, pins.test_z2_synthetic_spectra,
            pins.test_z2_paper_models, pins.test_ladder_first_loop_closed_form,
            functools.partial(pins.test_cone_berry_phase_closed_form, 1.1, 24)]
    out += [functools.partial(pins.test_nested_sector_choice, *case)
            for case in pins.LADDER_CASES]
    out += [functools.partial(pins.test_nested_full_sector_is_transverse_loop, 6, 3, 11)]
    return out


def _reversed_product(U_loop, unitarise=False):
    N, p = len(U_loop), U_loop[0].shape[1]
    M = np.eye(p, dtype=complex)
    for j in range(N):
        M = M @ W.overlap(U_loop[(j + 1) % N], U_loop[j])
    return M


def _reversed_cyclic(U_loop, base, unitarise=False):
    N, p = len(U_loop), U_loop[0].shape[1]
    M = np.eye(p, dtype=complex)
    for s in range(N):
        j = (base + s) % N
        M = M @ W.overlap(U_loop[(j + 1) % N], U_loop[j])
    return M


def _open_loop(U_loop, unitarise=False):
    p = U_loop[0].shape[1]
    M = np.eye(p, dtype=complex)
    for j in range(len(U_loop) - 1):
        M = W.overlap(U_loop[j + 1], U_loop[j]) @ M
    return M


def _flipped_fourier(model, f):
    f = np.asarray(f, float)
    ph = np.exp(-2j * np.pi * (model.R.astype(float) @ f))
    H = np.zeros((model.n, model.n), complex)
    np.add.at(H, (model.i, model.j), model.t * ph)
    return 0.5 * (H + H.conj().T)


def _unprojected_spin(U, S, sign, split="zero"):
    mu, V = np.linalg.eigh(U.conj().T @ U)       # forgot the spin operator
    sel = np.argsort(mu)[: U.shape[1] // 2]
    return U @ V[:, sel], mu, U.shape[1] // 2, 1.0


def _highest_bands(H, p):
    lam, V = np.linalg.eigh(H)
    return lam, V[:, -p:], (lam[p] - lam[p - 1]) if p < H.shape[0] else np.inf


def _reversed_plaquette(U, i, j, N, Nt):
    return [U[i][j], U[i][(j + 1) % N], U[(i + 1) % Nt][(j + 1) % N], U[(i + 1) % Nt][j]]


def _right_as_left_eigvecs_eigenphases(Wm):
    return np.sort(np.angle(np.linalg.eigvals(Wm.conj())))


def _smallest_gap_midpoint(x_sorted):
    x = np.asarray(x_sorted, np.float64)
    gaps = np.append(x[1:] - x[:-1], (x[0] + 1.0) - x[-1])
    m = int(np.argmin(gaps))
    return float((x[m] + 0.5 * gaps[m]) % 1.0), float(gaps[m])


def _no_wrap_gap_midpoint(x_sorted):
    x = np.asarray(x_sorted, np.float64)
    if x.size < 2:
        return float(x[0]), 0.0
    gaps = x[1:] - x[:-1]
    m = int(np.argmax(gaps))
    return float(x[m] + 0.5 * gaps[m]), float(gaps[m])


def _sector_other_end(theta, cut, first, m):
    order = np.argsort(np.mod(np.asarray(theta) - cut, 2 * np.pi), kind="stable")
    p = len(order)
    lo = p - m - first
    return order[lo:lo + m], np.concatenate([order[:lo], order[lo + m:]])


def _sector_cut_shifted(theta, cut, first, m):
    order = np.argsort(np.mod(np.asarray(theta) - (cut + 1.0), 2 * np.pi), kind="stable")
    return order[first:first + m], np.concatenate([order[:first], order[first + m:]])


def _wannier_not_orthonormalised(Uk, nu):
    return Uk @ nu


def _wannier_columns_normalised(Uk, nu):
    w = Uk @ nu
    return w / np.linalg.norm(w, axis=0)


MUTATIONS = {
    "conjugated_overlap": ("overlap", lambda a, b: b.conj().T @ a),
    "transposed_overlap": ("overlap", lambda a, b: (a.conj().T @ b).T),
    "reversed_product": ("wilson_matrix", _reversed_product),
    "reversed_cyclic_product": ("cyclic_wilson_matrix", _reversed_cyclic),
    "open_loop": ("wilson_matrix", _open_loop),
    "flipped_fourier_sign": ("bloch_hamiltonian", _flipped_fourier),
    "unprojected_spin_operator": ("projected_spin_sector", _unprojected_spin),
    "highest_bands": ("occupied_states", _highest_bands),
    "conjugated_eigenphases": ("eigenphases", _right_as_left_eigvecs_eigenphases),
    "reversed_plaquette": ("plaquette_corners", _reversed_plaquette),
    "smallest_wcc_gap": ("largest_gap_midpoint", _smallest_gap_midpoint),
    "no_circular_wcc_gap": ("largest_gap_midpoint", _no_wrap_gap_midpoint),
    "nested_sector_other_end": ("wannier_sector", _sector_other_end),
    "nested_cut_shifted": ("wannier_sector", _sector_cut_shifted),
    "nested_no_orthonormalisation": ("wannier_states", _wannier_not_orthonormalised),
    "nested_columns_only_normalised": ("wannier_states", _wannier_columns_normalised),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(W, attr, fn)
    if hasattr(oracle, attr):
        monkeypatch.setattr(oracle, attr, fn)
    caught = None
    for pin in _all_pins():
        try:
            pin()
        except (AssertionError, oracle.OracleError) as e:
            caught = e
            break
    assert caught is not None, f"no pin catches the planted mistake {name!r}"
