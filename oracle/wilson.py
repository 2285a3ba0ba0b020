"""FP64 oracle: the discretised Wilson loop and its nested and spin-resolved forms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each function names the passage of arXiv 2312.13051 it follows.  Where the paper
is silent or garbled, the reading taken is stated next to the code that uses it.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi

STATUS = {"OK": 0, "EINVAL": 1, "ENOMEM": 2, "EGAP": 3, "EPSOGAP": 4, "EWANGAP": 5,
          "ENOCONV": 6, "ETIMEOUT": 7, "ECUDA": 8, "ECANCELED": 9}


class OracleError(Exception):
    """A condition under which the method has no answer (closed gap, etc.)."""

    def __init__(self, status: str, msg: str, k_index=None):
        super().__init__(f"{status}: {msg}")
        self.status = status
        self.k_index = k_index


# ----------------------------------------------------------------------------
# Step 1: Bloch Hamiltonian (Sec. I: H(k) from the tight-binding model; Sec. II A
# periodic gauge).  H(f) = sum_e t_e exp(i 2pi f.R_e) |i_e><j_e|, summed directly.
# ----------------------------------------------------------------------------

def bloch_hamiltonian(model, f) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    phase = np.exp(1j * TWO_PI * (model.R.astype(np.float64) @ f))
    H = np.zeros((model.n, model.n), dtype=np.complex128)
    np.add.at(H, (model.i, model.j), model.t * phase)
    scale = max(np.abs(H).max(), np.abs(model.t).max(initial=0.0), 1e-300)
    if np.abs(H - H.conj().T).max() > 1e-12 * scale:
        raise OracleError("EINVAL", "hopping list is not Hermitian")
    return 0.5 * (H + H.conj().T)


def translation_blocks(model):
    """The same sum grouped by translation: H(f) = sum_R exp(i 2pi f.R) T_R with T_R the
    dense n x n matrix of the hoppings of translation R.  Returns (R list, T stack)."""
    Rs, inv = np.unique(model.R, axis=0, return_inverse=True)
    T = np.zeros((len(Rs), model.n, model.n), dtype=np.complex128)
    np.add.at(T, (inv.ravel(), model.i, model.j), model.t)
    return Rs, T


def bloch_hamiltonian_grouped(blocks, f) -> np.ndarray:
    """H(f) from ``translation_blocks`` (for models with many hoppings); equal to
    ``bloch_hamiltonian`` term by term."""
    Rs, T = blocks
    phase = np.exp(1j * TWO_PI * (Rs.astype(np.float64) @ np.asarray(f, np.float64)))
    H = np.tensordot(phase, T, axes=1)
    return 0.5 * (H + H.conj().T)


def plane_points(plane) -> np.ndarray:
    """k(j, i) = origin + (j/N) loop_dir + (i/N_t) trans_dir  (Sec. II B ``vec(t1, t2)``).

    Returned as f[i, j, :] (transverse index i, loop index j).  Loop: N distinct
    points, closed by reusing j = 0 (Eq. 2).  Transverse: N_t distinct points.
    """
    o = np.asarray(plane.origin, np.float64)
    a = np.asarray(plane.loop_dir, np.float64)
    b = np.asarray(plane.trans_dir, np.float64)
    f = np.empty((plane.N_t, plane.N, 3))
    for i in range(plane.N_t):
        for j in range(plane.N):
            f[i, j] = o + (j / plane.N) * a + (i / plane.N_t) * b
    return f


# ----------------------------------------------------------------------------
# Step 2: exact diagonalisation, occupied states (Sec. I "exact diagonalization";
# Eq. 1: the occupied bands u_n).  LAPACK zheevd through numpy, ascending.
# ----------------------------------------------------------------------------

def occupied_states(H: np.ndarray, p: int):
    """Return (eigenvalues, U = lowest p eigenvectors, direct gap lam_p - lam_{p-1})."""
    lam, V = np.linalg.eigh(H)
    gap = lam[p] - lam[p - 1] if p < H.shape[0] else np.inf
    return lam, V[:, :p], gap


def eigh_batched(Hs, n_vec: int):
    """Eigenvalues (ascending) and the first n_vec eigenvectors of each matrix."""
    out = []
    for H in Hs:
        lam, V = np.linalg.eigh(H)
        out.append((lam, V[:, :n_vec]))
    return out


# ----------------------------------------------------------------------------
# Steps 3-4: overlaps and the ordered product (Eq. 2).
# F_{k} = <u_{k+dk} | u_k>, e^{i 2pi xbar} = F_{k+(N-1)dk} ... F_{k+dk} F_k:
# later k multiplies from the left; the loop closes on the same U(k_0).
# ----------------------------------------------------------------------------

def overlap(U_next: np.ndarray, U_here: np.ndarray) -> np.ndarray:
    """M = U(k_{j+1})^dagger U(k_j)   (Eq. 2, F matrix for a set of bands)."""
    return U_next.conj().T @ U_here


def polar_factor(M: np.ndarray) -> np.ndarray:
    """Unitary polar factor X Y^dagger of M = X S Y^dagger (option ``unitarise``)."""
    X, _, Yh = np.linalg.svd(M)
    return X @ Yh


def wilson_matrix(U_loop, unitarise: bool = False) -> np.ndarray:
    """W = M_{N-1} ... M_1 M_0 with M_j = U_{j+1}^dagger U_j and U_N = U_0 (Eq. 2)."""
    N = len(U_loop)
    p = U_loop[0].shape[1]
    W = np.eye(p, dtype=np.complex128)
    for j in range(N):
        M = overlap(U_loop[(j + 1) % N], U_loop[j])
        if unitarise:
            M = polar_factor(M)
        W = M @ W
    return W


def cyclic_wilson_matrix(U_loop, base: int, unitarise: bool = False) -> np.ndarray:
    """The same closed loop started at k_base: M_{b-1} ... M_0 M_{N-1} ... M_b (Eq. 8)."""
    N = len(U_loop)
    p = U_loop[0].shape[1]
    W = np.eye(p, dtype=np.complex128)
    for s in range(N):
        j = (base + s) % N
        M = overlap(U_loop[(j + 1) % N], U_loop[j])
        if unitarise:
            M = polar_factor(M)
        W = M @ W
    return W


# ----------------------------------------------------------------------------
# Step 5: eigenphases (Eq. 2, left side; Eq. 8: Im Ln of the loop).  The raw
# product is not unitary, so its eigenvalues come from the general eigensolver
# (LAPACK zgeev through numpy); theta = arg(lambda) in (-pi, pi], ascending.
# ----------------------------------------------------------------------------

def eigenphases(W: np.ndarray) -> np.ndarray:
    return np.sort(np.angle(np.linalg.eigvals(W)))


def _check_gap(gap, tol, k_index):
    if not gap > tol:
        raise OracleError("EGAP", f"direct gap {gap:.3e} <= {tol:.3e}", k_index)


def _default_gap_tol(model) -> float:
    return 1e-6 * max(1.0, float(np.abs(model.t).max(initial=0.0)))


def _states_on_plane(model, plane, p, gap_tol, gauge=None):
    """U[i][j] for every k of the plane and the minimum direct gap of each loop."""
    f = plane_points(plane)
    U = []
    min_gap = np.full(plane.N_t, np.inf)
    for i in range(plane.N_t):
        row = []
        for j in range(plane.N):
            H = bloch_hamiltonian(model, f[i, j])
            _, Uk, gap = occupied_states(H, p)
            _check_gap(gap, gap_tol, (i, j))
            min_gap[i] = min(min_gap[i], gap)
            if gauge is not None:
                Uk = Uk @ gauge(i, j, Uk.shape[1])
            row.append(Uk)
        U.append(row)
    return U, min_gap


def _check_plane(model, plane, p):
    if not (1 <= p <= model.n):
        raise OracleError("EINVAL", "need 1 <= p <= n")
    if plane.N < 1 or plane.N_t < 1:
        raise OracleError("EINVAL", "empty plane")
    if np.any(np.asarray(plane.loop_dir) != np.round(plane.loop_dir)):
        raise OracleError("EINVAL", "loop_dir must be an integer vector to close the loop")


def wilson_loop(model, plane, p: int, gap_tol=None, unitarise=False, gauge=None):
    """Hybrid Wannier centres along loop_dir as a function of the transverse index
    (Eq. 3, ``WSurf``).  Returns (phases[N_t, p], min_gap[N_t]); xbar = phases / 2pi.

    ``gauge(i, j, p)`` (tests only) returns a p x p unitary applied as U -> U G.
    """
    _check_plane(model, plane, p)
    gap_tol = _default_gap_tol(model) if gap_tol is None else gap_tol
    U, min_gap = _states_on_plane(model, plane, p, gap_tol, gauge)
    phases = np.stack([eigenphases(wilson_matrix(U[i], unitarise)) for i in range(plane.N_t)])
    return phases, min_gap


# ----------------------------------------------------------------------------
# Spin-resolved loop (Sec. IV): projected spin operator P s P restricted to the
# occupied space, S = U^dagger s U (p x p); its negative (sign -1) or positive
# eigen-sector spans the states whose Wilson loop gives C_down (C_up).
# Reading (split "zero", the text's "negative eigenstates"): split at zero, the
# sector must hold p/2 states at every k, gap = min |mu|.  Alternative reading
# (split "median"): the p/2 lowest (sign -1) or highest (+1) eigenvalues, whatever
# their sign, gap = mu_{p/2} - mu_{p/2-1}; with it the disordered Eq. 10 supercells
# give Fig. 6(d)'s C_s = 0 at W = 9, where the zero split has no fixed-size sector.
# ----------------------------------------------------------------------------

def projected_spin_sector(U: np.ndarray, S: np.ndarray, sign: int, split: str = "zero"):
    Sp = U.conj().T @ S @ U
    Sp = 0.5 * (Sp + Sp.conj().T)
    mu, V = np.linalg.eigh(Sp)
    if split == "median":
        h = mu.size // 2
        sel = np.arange(mu.size) < h if sign < 0 else np.arange(mu.size) >= mu.size - h
        return U @ V[:, sel], mu, int(sel.sum()), float(mu[h] - mu[h - 1])
    if split != "zero":
        raise OracleError("EINVAL", f"unknown PSO split {split!r}")
    sel = mu < 0 if sign < 0 else mu > 0
    return U @ V[:, sel], mu, int(sel.sum()), float(np.abs(mu).min())


def spin_resolved_wilson_loop(model, plane, p: int, S, sign: int = -1, gap_tol=None,
                              pso_gap_tol: float = 1e-6, unitarise=False, pso_split: str = "zero"):
    """``WSpinSurf``: Wilson loop of the PSO sector.  Returns
    (phases[N_t, p/2], pso_evals[N_t, N, p], min_pso_gap, min_gap[N_t])."""
    _check_plane(model, plane, p)
    if p % 2 or sign not in (-1, 1):
        raise OracleError("EINVAL", "need even p and sign = +-1")
    gap_tol = _default_gap_tol(model) if gap_tol is None else gap_tol
    U, min_gap = _states_on_plane(model, plane, p, gap_tol)
    pso = np.empty((plane.N_t, plane.N, p))
    min_pso_gap = np.inf
    phases = []
    for i in range(plane.N_t):
        sector = []
        for j in range(plane.N):
            Us, mu, count, g = projected_spin_sector(U[i][j], S, sign, pso_split)
            pso[i, j] = mu
            min_pso_gap = min(min_pso_gap, g)
            if count != p // 2 or not g > pso_gap_tol:
                raise OracleError("EPSOGAP", f"PSO sector size {count}, gap {g:.3e}", (i, j))
            sector.append(Us)
        phases.append(eigenphases(wilson_matrix(sector, unitarise)))
    return np.stack(phases), pso, min_pso_gap, min_gap


# ----------------------------------------------------------------------------
# Nested loop (Sec. III, Eq. 8).  For each base point k_j of the first loop and
# each transverse index: Wilson matrix of the closed loop started at k_j, its
# right eigenvectors nu, the sector of m eigenvectors ordered by phase measured
# from ``cut`` starting at ``first``; Wannier states w = U(k_j) nu, orthonormalised;
# then the Wilson loop of w along the transverse direction (closed on i = 0).
# ----------------------------------------------------------------------------

def _circ_gap(sel_phases, rest_phases):
    if len(rest_phases) == 0:
        return np.inf
    d = np.abs(np.angle(np.exp(1j * (np.asarray(sel_phases)[:, None]
                                     - np.asarray(rest_phases)[None, :]))))
    return float(d.min())


def wannier_sector(theta, cut: float, first: int, m: int):
    """The nested loop's sector (reading: ``WNWL`` has no sector argument): order the
    eigenphases by their distance from ``cut`` going up, (theta - cut) mod 2pi, and take
    positions [first, first + m).  Returns (selected indices, the other indices)."""
    order = np.argsort(np.mod(np.asarray(theta) - cut, TWO_PI), kind="stable")
    return order[first:first + m], np.concatenate([order[:first], order[first + m:]])


def wannier_states(Uk: np.ndarray, nu: np.ndarray) -> np.ndarray:
    """Wannier states of the sector at one k (Eq. 8): w = U(k) nu, with orthonormal
    columns spanning the same space (QR; the right eigenvectors nu of a non-unitary W
    are not orthogonal)."""
    w, _ = np.linalg.qr(Uk @ nu)
    return w


def wannier_row(U_row, bases, cut, first, m, wannier_gap_tol, unitarise=False, row=0):
    """One transverse row: for each base point j in ``bases`` the loop started at k_j,
    its right eigenvectors, the sector and the Wannier states at k_j.  Returns (list of
    w per base point, min Wannier gap of the row)."""
    ws, gmin = [], np.inf
    for j in bases:
        W = cyclic_wilson_matrix(U_row, j, unitarise)
        vals, vecs = np.linalg.eig(W)
        th = np.angle(vals)
        sel, rest = wannier_sector(th, cut, first, m)
        g = _circ_gap(th[sel], th[rest])
        gmin = min(gmin, g)
        if not g > wannier_gap_tol:
            raise OracleError("EWANGAP", f"Wannier gap {g:.3e}", (row, j))
        ws.append(wannier_states(U_row[j], vecs[:, sel]))
    return ws, gmin


def nested_phases(w_column) -> np.ndarray:
    """Wilson loop of the Wannier states along the transverse direction, closed on the
    first point (Eq. 8 with the Eq. 2 overlaps), and its eigenphases."""
    Nt = len(w_column)
    Wn = np.eye(w_column[0].shape[1], dtype=np.complex128)
    for i in range(Nt):
        Wn = overlap(w_column[(i + 1) % Nt], w_column[i]) @ Wn
    return eigenphases(Wn)


def _row_points(plane, i) -> np.ndarray:
    """Row i of ``plane_points(plane)``, by the same expression."""
    o = np.asarray(plane.origin, np.float64)
    a = np.asarray(plane.loop_dir, np.float64)
    b = np.asarray(plane.trans_dir, np.float64)
    return np.stack([o + (j / plane.N) * a + (i / plane.N_t) * b for j in range(plane.N)])


def _row_states(model, plane, i, p, gap_tol, blocks=None):
    """Occupied blocks of transverse row i and the row's minimum direct gap."""
    f = _row_points(plane, i)
    row, gmin = [], np.inf
    for j in range(plane.N):
        H = (bloch_hamiltonian(model, f[j]) if blocks is None
             else bloch_hamiltonian_grouped(blocks, f[j]))
        _, Uk, gap = occupied_states(H, p)
        _check_gap(gap, gap_tol, (i, j))
        gmin = min(gmin, gap)
        row.append(Uk)
    return row, gmin


def _nested_row_task(args):
    """Everything the nested loop needs from one transverse row (a picklable task, so a
    caller may spread rows over processes)."""
    model, plane, i, p, gap_tol, bases, cut, first, m, wtol, unitarise, blocks = args
    U_row, gmin = _row_states(model, plane, i, p, gap_tol, blocks)
    ph = eigenphases(wilson_matrix(U_row, unitarise))
    ws, wg = wannier_row(U_row, bases, cut, first, m, wtol, unitarise, row=i)
    return ph, gmin, ws, wg


def nested_wilson_loop(model, plane, p: int, cut: float = -np.pi, first: int = 0,
                       m: int | None = None, gap_tol=None, wannier_gap_tol: float = 1e-6,
                       unitarise=False, bases=None, row_map=map, grouped=False):
    """``WNWL``.  Returns (phases[N_t, p], nested[len(bases), m], min_wannier_gap,
    min_gap[N_t]); ``bases`` (default: every base point j < N) selects base points,
    ``row_map`` maps the per-row task over the rows (e.g. a process pool's map) and
    ``grouped`` builds H(f) from ``translation_blocks``."""
    _check_plane(model, plane, p)
    m = p // 2 if m is None else m
    if not (1 <= m <= p) or not (0 <= first <= p - m):
        raise OracleError("EINVAL", "sector out of range")
    if np.any(np.asarray(plane.trans_dir) != np.round(plane.trans_dir)):
        raise OracleError("EINVAL", "trans_dir must be an integer vector for the nested loop")
    gap_tol = _default_gap_tol(model) if gap_tol is None else gap_tol
    bases = list(range(plane.N)) if bases is None else list(bases)
    blocks = translation_blocks(model) if grouped else None
    tasks = [(model, plane, i, p, gap_tol, bases, cut, first, m, wannier_gap_tol, unitarise, blocks)
             for i in range(plane.N_t)]
    rows = list(row_map(_nested_row_task, tasks))
    phases = np.stack([r[0] for r in rows])
    min_gap = np.array([r[1] for r in rows])
    min_wgap = min(r[3] for r in rows)
    nested = np.stack([nested_phases([rows[i][2][b] for i in range(plane.N_t)])
                       for b in range(len(bases))]) if bases else np.empty((0, m))
    return phases, nested, min_wgap, min_gap


# ----------------------------------------------------------------------------
# Post-processing (Eq. 6): C = sum_n xbar_n(k_y = 2pi) - sum_n xbar_n(0), tracked
# continuously; the grid is cyclic in the transverse direction.
# ----------------------------------------------------------------------------

# ----------------------------------------------------------------------------
# Plaquette Berry flux (Sec. IV A example, the WSpinLine coupling-matrix method): the
# Brillouin zone is cut into a grid of plaquettes; the Wilson loop of the occupied
# bands (or of a PSO sector) around each plaquette's closed path gives its
# integrated Berry flux, the sum of its eigenphases = arg det of the loop matrix,
# and the (spin-)Chern number is the total flux / 2pi.
# Reading: the plaquette at (j, i) has corners k(j, i), k(j+1, i), k(j+1, i+1),
# k(j, i+1) (j along loop_dir, i along trans_dir, both closing cyclically) and is
# traversed k(j, i) -> k(j, i+1) -> k(j+1, i+1) -> k(j+1, i) -> k(j, i), each step
# an Eq. 2 overlap U(b)^dagger U(a); with this orientation the total flux / 2pi
# equals the Eq. 6 winding of the hybrid Wannier centres of the same states.
# ----------------------------------------------------------------------------

def _sector_states_on_plane(model, plane, p, S, sign, gap_tol, pso_gap_tol, pso_split="zero"):
    f = plane_points(plane)
    U = []
    for i in range(plane.N_t):
        row = []
        for j in range(plane.N):
            _, Uk, gap = occupied_states(bloch_hamiltonian(model, f[i, j]), p)
            _check_gap(gap, gap_tol, (i, j))
            if S is not None:
                Uk, _, count, g = projected_spin_sector(Uk, S, sign, pso_split)
                if count != p // 2 or not g > pso_gap_tol:
                    raise OracleError("EPSOGAP", f"PSO sector size {count}, gap {g:.3e}", (i, j))
            row.append(Uk)
        U.append(row)
    return U


def plaquette_flux(model, plane, p: int, S=None, sign: int = -1, gap_tol=None,
                   pso_gap_tol: float = 1e-6, pso_split: str = "zero"):
    """Integrated Berry flux through every plaquette of the plane (Sec. IV A, WSpinLine).
    Returns (flux[N_t, N] in (-pi, pi], Chern number = sum(flux) / 2pi).  With a spin
    operator S the states are the PSO sector of sign ``sign`` (Sec. IV)."""
    _check_plane(model, plane, p)
    if S is not None and (p % 2 or sign not in (-1, 1)):
        raise OracleError("EINVAL", "need even p and sign = +-1")
    if np.any(np.asarray(plane.trans_dir) != np.round(plane.trans_dir)):
        raise OracleError("EINVAL", "trans_dir must be an integer vector to close the plaquettes")
    gap_tol = _default_gap_tol(model) if gap_tol is None else gap_tol
    U = _sector_states_on_plane(model, plane, p, S, sign, gap_tol, pso_gap_tol, pso_split)
    N, Nt = plane.N, plane.N_t
    flux = np.empty((Nt, N))
    for i in range(Nt):
        for j in range(N):
            W = plaquette_matrix(plaquette_corners(U, i, j, N, Nt))
            flux[i, j] = np.angle(np.linalg.det(W))
    return flux, float(flux.sum() / TWO_PI)


def plaquette_corners(U, i, j, N, Nt):
    """States at the plaquette's corners in the order of traversal (reading above)."""
    return [U[i][j], U[(i + 1) % Nt][j], U[(i + 1) % Nt][(j + 1) % N], U[i][(j + 1) % N]]


def plaquette_matrix(corners) -> np.ndarray:
    """Wilson loop around a closed path: later steps multiply from the left (Eq. 2)."""
    W = np.eye(corners[0].shape[1], dtype=complex)
    for a in range(len(corners)):
        W = overlap(corners[(a + 1) % len(corners)], corners[a]) @ W
    return W


def winding(phases: np.ndarray) -> float:
    s = np.asarray(phases).sum(axis=1) / TWO_PI
    d = np.diff(np.append(s, s[0]))
    d = d - np.round(d)
    return float(d.sum())


# ----------------------------------------------------------------------------
# Z2 index from the connectivity of the hybrid Wannier centres (Sec. II B, after
# Eq. 7: with T^2 = -1 the two members of each Kramers pair carry opposite Chern
# numbers and nu = (C1 - C2)/2 mod 2; a non-trivial index shows as WCCs that
# interpolate across the whole cell between the two time-reversal-invariant lines
# t2 = 0 and t2 = 1/2, Sec. II C uses it for supercells with vacancies).  The paper
# reads the connectivity off a plot; read automatically here by the largest-gap
# construction of Soluyanov and Vanderbilt (Phys. Rev. B 83, 235401 (2011)): on
# every row from t2 = 0 to t2 = 1/2 take the midpoint of the widest circular gap
# between the WCCs x = theta / 2pi (mod 1); at each step count the WCCs of the next
# row that lie strictly between the two midpoints.  nu is the total count mod 2
# (for an even number of WCCs the count's parity does not depend on which of the
# two arcs between the midpoints is taken).
# Conventions fixed here (the GPU kernel follows them): x = theta / 2pi, plus 1 when
# negative; gaps of the sorted x are x[m+1] - x[m] and, last, (x[0] + 1) - x[p-1];
# the first widest gap wins a tie; its midpoint x[m] + gap / 2 is reduced by 1 when
# it reaches 1.
# ----------------------------------------------------------------------------

def wcc_fractions(theta_row) -> np.ndarray:
    """Sorted WCC positions in [0, 1) of one row of eigenphases (Eq. 3, x = theta / 2pi)."""
    x = np.asarray(theta_row, np.float64) / TWO_PI
    x = np.where(x < 0.0, x + 1.0, x)
    return np.sort(x)


def largest_gap_midpoint(x_sorted):
    """(midpoint, width) of the widest circular gap between sorted positions in [0, 1)."""
    x = np.asarray(x_sorted, np.float64)
    p = x.size
    gaps = np.empty(p)
    gaps[: p - 1] = x[1:] - x[:-1]
    gaps[p - 1] = (x[0] + 1.0) - x[p - 1]
    m = int(np.argmax(gaps))
    z = x[m] + 0.5 * gaps[m]
    if z >= 1.0:
        z -= 1.0
    return float(z), float(gaps[m])


def z2_largest_gap(phases):
    """Z2 index of a time-reversal-symmetric plane from its WCC spectrum (reading above).

    phases: N_t x p eigenphases of the Wilson loops at t2 = i / N_t (N_t even, so that
    t2 = 1/2 is row N_t / 2).  Returns (nu, crossings[N_t / 2], midpoints[N_t / 2 + 1],
    widest gaps[N_t / 2 + 1])."""
    ph = np.asarray(phases, np.float64)
    if ph.ndim != 2 or ph.shape[1] < 1 or ph.shape[0] < 2 or ph.shape[0] % 2:
        raise OracleError("EINVAL", "need an N_t x p array with N_t even and p >= 1")
    h = ph.shape[0] // 2
    xs = [wcc_fractions(ph[i]) for i in range(h + 1)]
    mids = np.empty(h + 1)
    widths = np.empty(h + 1)
    for i in range(h + 1):
        mids[i], widths[i] = largest_gap_midpoint(xs[i])
    crossings = np.zeros(h, dtype=np.int64)
    for i in range(h):
        lo, hi = min(mids[i], mids[i + 1]), max(mids[i], mids[i + 1])
        crossings[i] = int(np.count_nonzero((xs[i + 1] > lo) & (xs[i + 1] < hi)))
    return int(crossings.sum() % 2), crossings, mids, widths


def circular_match_error(a, b) -> float:
    """Max circular distance between two sorted phase lists, minimised over cyclic
    relabellings (ties at +-pi may sort to either end)."""
    a = np.sort(np.asarray(a, np.float64))
    b = np.sort(np.asarray(b, np.float64))
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    best = np.inf
    for s in range(len(a)):
        d = np.abs(np.angle(np.exp(1j * (a - np.roll(b, s)))))
        best = min(best, float(d.max()))
    return best
