"""Seeded synthetic inputs: tight-binding hopping lists, k-planes and workloads.

This module builds *inputs* only (hopping lists of the paper's models, supercells
with disorder and Peierls flux, the reciprocal-space planes the loops run over).
It holds none of the Wilson-loop arithmetic: no Bloch sum, no eigensolve, no
overlap, no eigenphase.  Both the CUDA path and the CPU oracle consume what it
returns, so the two never disagree about their inputs.

Hopping-list convention (Sec. II A, periodic gauge used by the loops):

    H(f) = sum_e t_e exp(i 2 pi f . R_e) |i_e><j_e|,

with ``f`` in fractional coordinates of the reciprocal basis and ``R_e`` an
integer lattice translation; t_R[i, j] is the amplitude between orbital i of a
cell and orbital j of the cell displaced by R.  Lists are *full*: every
(i, j, R, t) comes with its partner (j, i, -R, conj t), so H(f) is Hermitian.
No orbital-position phases are used, hence H(f + G) = H(f) for integer G and a
loop closes on the same matrix (Eq. 2, periodic condition psi(k) = psi(k+2pi/a)).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# Pauli matrices, index 0 = identity.
PAULI = (
    np.array([[1, 0], [0, 1]], dtype=np.complex128),
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)

GLOBAL_SEED = 20231213


def kron(a: int, b: int) -> np.ndarray:
    """PAULI[a] (x) PAULI[b]; the first factor is the slow (outer) index."""
    return np.kron(PAULI[a], PAULI[b])


@dataclass
class HoppingList:
    """Full hopping list of a periodic tight-binding model (host arrays)."""
    n: int
    R: np.ndarray          # (nnz, 3) int32 lattice translations
    i: np.ndarray          # (nnz,) int32 row orbital
    j: np.ndarray          # (nnz,) int32 column orbital
    t: np.ndarray          # (nnz,) complex128 amplitude
    dim: int = 2
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.t.shape[0])

    def __post_init__(self):
        self.R = np.ascontiguousarray(self.R, dtype=np.int32).reshape(-1, 3)
        self.i = np.ascontiguousarray(self.i, dtype=np.int32)
        self.j = np.ascontiguousarray(self.j, dtype=np.int32)
        self.t = np.ascontiguousarray(self.t, dtype=np.complex128)


def from_blocks(blocks: dict, n: int, dim: int = 2, name: str = "") -> HoppingList:
    """Hopping list from dense blocks {R: t_R}.

    ``blocks`` holds t_0 (must be Hermitian) and t_R for R in one half-space;
    the partner blocks t_{-R} = t_R^dagger are added here.  Exact zeros are dropped.
    """
    full = {}
    for R, T in blocks.items():
        R = tuple(int(x) for x in R) + (0,) * (3 - len(R))
        T = np.asarray(T, dtype=np.complex128)
        if T.shape != (n, n):
            raise ValueError(f"block {R} has shape {T.shape}, expected {(n, n)}")
        if R == (0, 0, 0):
            if not np.allclose(T, T.conj().T, atol=1e-14):
                raise ValueError("t_0 must be Hermitian")
            full[R] = full.get(R, 0) + T
        else:
            mR = tuple(-x for x in R)
            if mR in blocks or mR in full and mR != R:
                raise ValueError(f"give t_R only for one of R={R} and -R")
            full[R] = full.get(R, 0) + T
            full[mR] = full.get(mR, 0) + T.conj().T
    Rs, I, J, Ts = [], [], [], []
    for R, T in sorted(full.items()):
        ii, jj = np.nonzero(T)
        Rs.append(np.tile(np.array(R, np.int32), (ii.size, 1)))
        I.append(ii)
        J.append(jj)
        Ts.append(T[ii, jj])
    return HoppingList(n=n, R=np.concatenate(Rs), i=np.concatenate(I),
                       j=np.concatenate(J), t=np.concatenate(Ts), dim=dim, name=name)


def from_bloch_terms(n: int, const, cos_terms: dict, sin_terms: dict, dim: int,
                     name: str = "") -> HoppingList:
    """Model H(k) = C + sum_d [A_d cos k_d + B_d sin k_d] as a hopping list.

    With e^{ik} t + e^{-ik} t^dagger = A cos k + B sin k one has t = A/2 - i B/2.
    ``cos_terms``/``sin_terms`` map an axis (0, 1, 2) to the Hermitian A_d / B_d.
    """
    blocks = {(0, 0, 0): np.asarray(const, np.complex128)}
    for d in sorted(set(cos_terms) | set(sin_terms)):
        A = np.asarray(cos_terms.get(d, np.zeros((n, n))), np.complex128)
        B = np.asarray(sin_terms.get(d, np.zeros((n, n))), np.complex128)
        R = [0, 0, 0]
        R[d] = 1
        blocks[tuple(R)] = 0.5 * A - 0.5j * B
    return from_blocks(blocks, n, dim=dim, name=name)


# --------------------------------------------------------------------------
# The paper's models and the named workloads
# --------------------------------------------------------------------------

def ssh(v: float, w: float) -> HoppingList:
    """Su-Schrieffer-Heeger chain: H(k) = [[0, v + w e^{-ik}], [v + w e^{ik}, 0]] (Sec. II)."""
    t0 = np.array([[0, v], [v, 0]], np.complex128)
    tx = np.array([[0, 0], [w, 0]], np.complex128)   # e^{+ik} sits in H[1, 0]
    return from_blocks({(0, 0, 0): t0, (1, 0, 0): tx}, 2, dim=1, name=f"ssh({v},{w})")


def chern_eq4(m: float = 1.5) -> HoppingList:
    """Eq. 4: sin kx s1 + sin ky s2 + (cos kx + cos ky + m) s3."""
    s = PAULI
    return from_bloch_terms(2, m * s[3], {0: s[3], 1: s[3]}, {0: s[1], 1: s[2]}, dim=2,
                            name="chern_eq4")


def bhz_eq7(m: float = 1.5) -> HoppingList:
    """Eq. 7: sin kx s1(x)t1 + sin ky s1(x)t2 + (cos kx + cos ky + m) s3(x)t0, kron(sigma, tau)."""
    return from_bloch_terms(4, m * kron(3, 0), {0: kron(3, 0), 1: kron(3, 0)},
                            {0: kron(1, 1), 1: kron(1, 2)}, dim=2, name="bhz_eq7")


def choti_eq9(delta0: float = 1.0, m: float = -1.5) -> HoppingList:
    """Eq. 9 (chiral HOTI), 3D, kron(sigma, tau):
    sin kx s1t1 + sin ky s1t2 + sin kz s1t3 + (cos kx + cos ky + cos kz + m) s3t0
    + Delta0 (cos kx - cos ky) s2t0, with m = -1.5 as printed."""
    cos_terms = {0: kron(3, 0) + delta0 * kron(2, 0),
                 1: kron(3, 0) - delta0 * kron(2, 0),
                 2: kron(3, 0)}
    sin_terms = {0: kron(1, 1), 1: kron(1, 2), 2: kron(1, 3)}
    return from_bloch_terms(4, m * kron(3, 0), cos_terms, sin_terms, dim=3, name="choti_eq9")


def quadrupolar_eq10(delta: float = 0.5) -> HoppingList:
    """Eq. 10 (spinful quadrupolar insulator, Sec. IV A), kron(sigma, tau):
    sin kx s1t3 + sin ky s2t3 + (cos kx + cos ky + 1) s3t3 + delta (cos kx - cos ky) s0t1,
    delta = 0.5.  The last term is printed with s0t0, which commutes with the chiral
    operator S = s0t2 the text names; s0t1 is the reading that makes S^-1 H S = -H hold
    and keeps the spectrum gapped (the other anticommuting choice, s0t3, closes the gap
    at (pi, 0))."""
    return from_bloch_terms(4, kron(3, 3),
                            {0: kron(3, 3) + delta * kron(0, 1), 1: kron(3, 3) - delta * kron(0, 1)},
                            {0: kron(1, 3), 1: kron(2, 3)}, dim=2, name="quadrupolar_eq10")


EQ10_SPIN = np.diag([1.0, -1.0, 1.0, -1.0]).astype(np.complex128)   # s0 (x) t3 (Sec. IV A)
EQ10_CHIRAL = np.kron(PAULI[0], PAULI[2])                            # S = s0 (x) t2


def spin_hall(m: float = 1.0) -> HoppingList:
    """4-band spin-Hall model, kron(tau, s) (orbital-major, spin-minor):
    sin kx tx(x)sz + sin ky ty(x)s0 + (m - cos kx - cos ky) tz(x)s0."""
    return from_bloch_terms(4, m * kron(3, 0), {0: -kron(3, 0), 1: -kron(3, 0)},
                            {0: kron(1, 3), 1: kron(2, 0)}, dim=2, name=f"spin_hall({m})")


SPIN_HALL_SZ = np.diag([1.0, -1.0, 1.0, -1.0]).astype(np.complex128)   # tau0 (x) s_z


def bbh(gx: float = 0.5, gy: float = 0.5, lx: float = 1.0, ly: float = 1.0) -> HoppingList:
    """Benalcazar-Bernevig-Hughes quadrupole model (the model behind Sec. III's nested loop):
    (gx + lx cos kx) G4 + lx sin kx G3 + (gy + ly cos ky) G2 + ly sin ky G1,
    G4 = t1(x)s0, G_a = -t2(x)s_a (a = 1, 2, 3), kron(tau, sigma)."""
    G4 = kron(1, 0)
    G1, G2, G3 = (-kron(2, a) for a in (1, 2, 3))
    return from_bloch_terms(4, gx * G4 + gy * G2, {0: lx * G4, 1: ly * G2},
                            {0: lx * G3, 1: ly * G1}, dim=2, name=f"bbh({gx},{gy})")


def cone_ssh_product(alpha: float, v: float, w: float) -> HoppingList:
    """Four-band product model h_x(kx) (x) 1 + 1 (x) h_y(ky), kron(x-part, y-part):
    h_x = sin(alpha) (cos kx s1 + sin kx s2) + cos(alpha) s3 (a unit vector on a cone of
    opening alpha, so the Berry phase of its lower band along kx is known in closed form)
    and h_y = (v + w cos ky) s1 + w sin ky s2 (the SSH chain of ``ssh`` along ky, Berry
    phase pi for v < w and 0 for v > w).  Its lowest band is the product of the two
    lower bands, so the two directions decouple."""
    s = PAULI
    hx_c, hx_s = np.sin(alpha) * np.kron(s[1], s[0]), np.sin(alpha) * np.kron(s[2], s[0])
    const = np.cos(alpha) * np.kron(s[3], s[0]) + v * np.kron(s[0], s[1])
    return from_bloch_terms(4, const, {0: hx_c, 1: w * np.kron(s[0], s[1])},
                            {0: hx_s, 1: w * np.kron(s[0], s[2])}, dim=2,
                            name=f"cone_ssh({alpha:.4f},{v},{w})")


def direct_sum(models, name: str = "") -> HoppingList:
    """Block-diagonal model: the orbitals of model b follow those of models 0 .. b-1 and
    no hopping couples two blocks."""
    off, R, I, J, T = 0, [], [], [], []
    for m in models:
        R.append(m.R)
        I.append(m.i + off)
        J.append(m.j + off)
        T.append(m.t)
        off += m.n
    return HoppingList(n=off, R=np.concatenate(R), i=np.concatenate(I), j=np.concatenate(J),
                       t=np.concatenate(T), dim=max(m.dim for m in models),
                       name=name or "+".join(m.name for m in models))


# Wannier ladder: three decoupled cone (x) SSH blocks.  The Wilson loop along kx has one
# Wannier centre per block, at a different position for each block and the same at
# every ky; the nested loop of a block's Wannier band along ky has the phase of that
# block's SSH chain.  Targets xbar = theta / 2pi: about -0.45, -0.2, +0.3; nested
# phases pi, 0, 0.
LADDER_XBAR = (-0.45, -0.2, 0.3)
LADDER_SSH = ((0.4, 1.0), (1.0, 0.5), (1.0, 0.6))


def ladder_alpha(xbar: float) -> float:
    """Cone opening whose lower band has Wannier centre close to xbar (-cos^2(alpha/2),
    the continuum value, taken mod 1)."""
    c2 = -xbar % 1.0
    return float(2.0 * np.arccos(np.sqrt(c2)))


def wannier_ladder() -> HoppingList:
    return direct_sum([cone_ssh_product(ladder_alpha(x), v, w)
                       for x, (v, w) in zip(LADDER_XBAR, LADDER_SSH)], name="wannier_ladder")


def square_lattice(t: float = 1.0) -> HoppingList:
    """One orbital per cell, nearest-neighbour hopping -t (used for flux pins)."""
    T = np.array([[-t]], np.complex128)
    return from_blocks({(0, 0, 0): np.zeros((1, 1)), (1, 0, 0): T, (0, 1, 0): T}, 1, dim=2,
                       name="square")


def supercell(model: HoppingList, L: int, W: float = 0.0, seed: int | None = None,
              flux: bool = False, Ly: int | None = None, onsite=None) -> HoppingList:
    """L x Ly supercell of a 2D model (Sec. II A, twisted boundary conditions with theta = 0).

    Supercell orbital index = ((x * Ly) + y) * n_cell + orbital.  A primitive hopping
    t_R from cell X to X + R becomes a supercell hopping with translation
    floor((x + R) / L).  ``W`` adds on-site Anderson disorder w ~ U[-W/2, W/2], one
    value per primitive cell times the identity on its orbitals, or times the matrix
    ``onsite`` (n_cell x n_cell; Eq. 10's chiral-preserving disorder is s0 (x) t3).  ``flux`` threads one
    flux quantum per supercell (2 pi / (L Ly) per plaquette) in a torus-periodic
    Landau gauge: a +y bond starting at column x gets phase exp(i 2 pi x / (L Ly)),
    an x bond crossing the supercell seam gets exp(-i 2 pi s y / Ly) for s seam
    crossings.  Flux requires axis-aligned bonds.
    """
    Ly = L if Ly is None else Ly
    nc = model.n
    n = nc * L * Ly
    phi = 1.0 / (L * Ly)
    rng = np.random.default_rng(seed) if W else None
    wdis = rng.uniform(-W / 2, W / 2, size=(L, Ly)) if W else None
    R_out, I_out, J_out, T_out = [], [], [], []
    for x in range(L):
        for y in range(Ly):
            cell = (x * Ly + y) * nc
            Rx, Ry = model.R[:, 0], model.R[:, 1]
            xt, yt = x + Rx, y + Ry
            sx, sy = np.floor_divide(xt, L), np.floor_divide(yt, Ly)
            xc, yc = xt - sx * L, yt - sy * Ly
            tcell = (xc * Ly + yc) * nc
            t = model.t.copy()
            if flux:
                if np.any((Rx != 0) & (Ry != 0)):
                    raise ValueError("flux needs axis-aligned bonds")
                theta = 2 * np.pi * phi * x * Ry - 2 * np.pi * sx * y / Ly
                t = t * np.exp(1j * theta)
            R_out.append(np.stack([sx, sy, model.R[:, 2]], axis=1))
            I_out.append(cell + model.i)
            J_out.append(tcell + model.j)
            T_out.append(t)
            if W:
                Md = np.eye(nc) if onsite is None else np.asarray(onsite, np.complex128)
                ii, jj = np.nonzero(Md)
                R_out.append(np.zeros((ii.size, 3), np.int64))
                I_out.append(cell + ii)
                J_out.append(cell + jj)
                T_out.append(wdis[x, y] * Md[ii, jj].astype(np.complex128))
    return HoppingList(n=n, R=np.concatenate(R_out), i=np.concatenate(I_out),
                       j=np.concatenate(J_out), t=np.concatenate(T_out), dim=2,
                       name=f"{model.name}_sc{L}x{Ly}" + (f"_W{W}" if W else "")
                       + ("_flux" if flux else ""))


def remove_orbitals(model: HoppingList, drop) -> HoppingList:
    """The model with the orbitals in ``drop`` taken out (every hopping that touches one
    is dropped) and the rest renumbered in their original order (Sec. II C: vacancies
    through PyBinding's site-state modifier)."""
    drop = np.unique(np.asarray(drop, np.int64))
    keep = np.ones(model.n, bool)
    keep[drop] = False
    new_index = np.cumsum(keep) - 1
    sel = keep[model.i] & keep[model.j]
    return HoppingList(n=int(keep.sum()), R=model.R[sel], i=new_index[model.i[sel]],
                       j=new_index[model.j[sel]], t=model.t[sel], dim=model.dim,
                       name=f"{model.name}_minus{drop.size}")


def vacancy_cells(L: int, r: float, Ly: int | None = None) -> np.ndarray:
    """Cells (x, y) of an L x Ly supercell within distance r of the origin cell, distances
    taken to the nearest periodic image (Sec. II C: sites removed inside a circle of
    radius r centred at the origin; r = 0 removes the origin cell alone)."""
    Ly = L if Ly is None else Ly
    out = []
    for x in range(L):
        for y in range(Ly):
            dx, dy = min(x, L - x), min(y, Ly - y)
            if dx * dx + dy * dy <= r * r:
                out.append((x, y))
    return np.array(out, np.int64).reshape(-1, 2)


def vacancy_supercell(model: HoppingList, L: int, r: float, Ly: int | None = None,
                      W: float = 0.0, seed: int | None = None) -> HoppingList:
    """L x Ly supercell of a 2D model with the cells within radius r of the origin removed
    (every orbital of a removed cell, Sec. II C), optionally with Anderson disorder."""
    Ly = L if Ly is None else Ly
    sc = supercell(model, L, W=W, seed=seed, Ly=Ly)
    nc = model.n
    cells = vacancy_cells(L, r, Ly)
    drop = ((cells[:, 0] * Ly + cells[:, 1])[:, None] * nc + np.arange(nc)[None, :]).ravel()
    out = remove_orbitals(sc, drop)
    out.name = f"{sc.name}_vac{cells.shape[0]}"
    return out


def manyband(norb: int = 128, seed: int = GLOBAL_SEED + 3, decay: float = 1.5,
             soc: float = 0.1, zeeman: float = 0.05, n_low: int | None = None,
             e_low: float = -4.0) -> HoppingList:
    """Synthetic Wannier-like spinful model (n = 2 norb), orbital-major, spin-minor.

    Translations: shells |R| in {0, 1, sqrt 2, 2} (13 vectors).  For R in a half-space
    t_R = exp(-|R|/decay)/sqrt(norb) [A_R (x) s0 + soc sum_a B_{R,a} (x) s_a] with
    complex Gaussian A, B; t_0 is the Hermitian part of the same form; plus
    zeeman * I (x) s_z, plus an on-site energy e_low on the first n_low = norb / 4
    orbitals (low-lying Wannier orbitals).  The offset opens a direct gap at quarter
    filling wider than the Zeeman splitting, so each spin sector holds half of the
    occupied states; the spin-independent part dominates so the projected spin
    operator keeps a gap at zero.
    """
    n_low = norb // 4 if n_low is None else n_low
    rng = np.random.default_rng(seed)
    n = 2 * norb

    def cn(shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)

    half = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 0), (0, 2)]
    blocks = {}
    for R in [(0, 0)] + half:
        amp = np.exp(-np.hypot(*R) / decay) / np.sqrt(norb)
        T = np.kron(cn((norb, norb)), PAULI[0])
        for a in (1, 2, 3):
            T = T + soc * np.kron(cn((norb, norb)), PAULI[a])
        T = amp * T
        if R == (0, 0):
            low = np.diag((np.arange(norb) < n_low).astype(float))
            T = 0.5 * (T + T.conj().T) + zeeman * np.kron(np.eye(norb), PAULI[3]) \
                + e_low * np.kron(low, PAULI[0])
        blocks[R] = T
    return from_blocks(blocks, n, dim=2, name=f"manyband({norb})")


def manyband_sz(norb: int = 128) -> np.ndarray:
    return np.kron(np.eye(norb), PAULI[3]).astype(np.complex128)


# --------------------------------------------------------------------------
# Planes (Sec. II B: vec(t1, t2) in units of the reciprocal vectors)
# --------------------------------------------------------------------------

@dataclass
class Plane:
    """k(j, i) = origin + (j/N) loop_dir + (i/N_t) trans_dir, j < N, i < N_t (fractional)."""
    N: int
    N_t: int
    origin: tuple = (0.0, 0.0, 0.0)
    loop_dir: tuple = (1, 0, 0)
    trans_dir: tuple = (0.0, 1.0, 0.0)


@dataclass
class PlaneStack:
    """N_s parallel planes (Sec. III: the nested loop against k_z; Sec. II B: weak and
    strong Z2 from the planes k_a = 0 and 1/2): plane s is ``plane`` with its origin
    moved by (s / N_s) sweep_dir, sweep_dir an integer reciprocal vector."""
    plane: Plane
    sweep_dir: tuple = (0, 0, 1)
    N_s: int = 2

    @property
    def N(self) -> int:
        return self.plane.N

    @property
    def N_t(self) -> int:
        return self.plane.N_t

    def planes(self) -> list:
        pl = self.plane
        return [Plane(pl.N, pl.N_t,
                      origin=tuple(float(o) + (s / self.N_s) * float(d)
                                   for o, d in zip(pl.origin, self.sweep_dir)),
                      loop_dir=pl.loop_dir, trans_dir=pl.trans_dir)
                for s in range(self.N_s)]


@dataclass
class Workload:
    name: str
    model: HoppingList
    plane: Plane
    p: int
    spin_op: np.ndarray | None = None
    nested_m: int | None = None
    extra: dict = field(default_factory=dict)


def config_spin_hall() -> Workload:
    """4-band spin-Hall model, m = 1, p = 2, 51 x 51 grid, loop along kx; S = tau0 (x) s_z."""
    return Workload("spin_hall_51x51", spin_hall(1.0), Plane(51, 51), 2, SPIN_HALL_SZ)


def config_bbh(gamma: float = 0.5) -> Workload:
    """BBH quadrupole, gamma = 0.5, lambda = 1, 60 x 60 grid, nested on the lower Wannier band."""
    return Workload(f"bbh_60x60_g{gamma}", bbh(gamma, gamma, 1.0, 1.0), Plane(60, 60), 2,
                    None, nested_m=1)


def config_disordered(L: int, seed: int, W: float = 2.0, nk: int = 16) -> Workload:
    """L x L supercell of the spin-Hall model with on-site Anderson disorder, half filling."""
    model = supercell(spin_hall(1.0), L, W=W, seed=seed)
    sz = np.kron(np.eye(L * L), SPIN_HALL_SZ)
    return Workload(f"disordered_L{L}_s{seed}", model, Plane(nk, nk), model.n // 2, sz)


def config_vacancy(L: int = 6, r: float = 1.0, nk: int = 16, m: float = 1.5) -> Workload:
    """Eq. 7 insulator on an L x L supercell with the cells within radius r of the origin
    removed (Sec. II C uses 21 x 21), half filling, loop along kx, S = s3 (x) t3."""
    model = vacancy_supercell(bhz_eq7(m), L, r)
    cells = model.n // 4
    sz = np.kron(np.eye(cells), np.diag([1.0, -1.0, -1.0, 1.0])).astype(np.complex128)
    return Workload(f"bhz_vacancy_L{L}_r{r:g}", model, Plane(nk, nk), model.n // 2, sz)


def config_quadrupolar(L: int, W: float, seed: int, nk: int = 6) -> Workload:
    """Eq. 10 on an L x L supercell with the chiral-preserving disorder w s0 (x) t3 per
    cell, w ~ U[-W/2, W/2] (Sec. IV A: 21 x 21, W from 0 to 9), half filling,
    S = I (x) s0 (x) t3."""
    model = supercell(quadrupolar_eq10(), L, W=W, seed=seed, onsite=EQ10_SPIN)
    sz = np.kron(np.eye(L * L), EQ10_SPIN)
    return Workload(f"quadrupolar_L{L}_W{W:g}_s{seed}", model, Plane(nk, nk), model.n // 2, sz)


def config_manyband(N: int = 101, norb: int = 128) -> Workload:
    """n = 256 spinful many-band model, 1/4 filling, 101 x 101 grid, S = I (x) s_z."""
    model = manyband(norb)
    return Workload(f"manyband_n{2 * norb}_{N}x{N}", model, Plane(N, N), norb // 2,
                    manyband_sz(norb), nested_m=norb // 4)


def serving_requests(count: int, rate: float = 200.0, seed: int = GLOBAL_SEED + 4,
                     sides=(8, 12, 16, 24, 32), nk_range=(8, 24)):
    """Poisson stream of Wilson-loop requests on flux-threaded disordered supercells.

    Yields dicts with arrival time (s), supercell side L, disorder W ~ U[0, 4], the
    k-grid side (uniform integer in nk_range) and the request seed.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += rng.exponential(1.0 / rate)
        out.append(dict(id=r, arrival=t, L=int(rng.choice(sides)), W=float(rng.uniform(0, 4)),
                        nk=int(rng.integers(nk_range[0], nk_range[1] + 1)),
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out


def serving_model(req: dict) -> HoppingList:
    return supercell(spin_hall(1.0), req["L"], W=req["W"], seed=req["seed"], flux=True)


def random_hermitian_model(n: int, seed: int, shells=((1, 0), (0, 1)), scale: float = 1.0
                           ) -> HoppingList:
    """Dense random model with nearest-neighbour translations (parity tests)."""
    rng = np.random.default_rng(seed)

    def cn(shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2 * n)

    A = cn((n, n))
    blocks = {(0, 0, 0): scale * (A + A.conj().T)}
    for R in shells:
        blocks[tuple(R) + (0,) * (3 - len(R))] = scale * cn((n, n))
    return from_blocks(blocks, n, dim=2, name=f"random{n}_s{seed}")


def random_hermitian_batch(sizes, seed: int) -> list:
    """Random dense Hermitian matrices (complex128) with the given sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
        out.append(A + A.conj().T)
    return out
