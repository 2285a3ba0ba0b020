"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: eigenphases within 1e-10 rad in FP64 and 1e-6 rad in mixed precision
(compared as sorted lists on the circle); Hamiltonians within 1e-13 relative;
eigenvalues within 1e-12 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import circ_err_rows, ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu
P = I.Plane
TOL = {"fp64": 1e-10, "mixed": 1e-6}


def _torch():
    import torch
    return torch


# ---------------------------------------------------------------- build_hk
@pytest.mark.parametrize("complex64", [False, True])
def test_build_hk_parity(lib, ctx, complex64):
    torch = _torch()
    rng = np.random.default_rng(0)
    models = [I.random_hermitian_model(7, 1, shells=((1, 0), (0, 1), (1, 1), (2, -1))),
              I.choti_eq9(1.0), I.supercell(I.spin_hall(1.0), 3, W=2.0, seed=5),
              I.supercell(I.spin_hall(1.0), 2, flux=True), I.manyband(20)]
    for model in models:
        f = rng.uniform(-2, 2, size=(37, 3))
        H = lib.build_hk(model, torch.tensor(f, device="cuda"), complex64=complex64, ctx=ctx)
        H = H.cpu().numpy()
        for k in range(f.shape[0]):
            ref = oracle.bloch_hamiltonian(model, f[k])
            scale = max(1.0, np.abs(ref).max())
            tol = 2e-7 if complex64 else 1e-13
            assert np.abs(H[k] - ref).max() <= tol * scale, model.name


# ---------------------------------------------------------------- eigh_batched
def _pack(mats):
    return np.concatenate([m.ravel() for m in mats])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eigh_batched_ragged(lib, ctx, precision):
    torch = _torch()
    # mixed precision refines the lowest n_vec block and needs n_vec < n
    sizes = ([1, 2, 3, 4, 5, 7, 8, 13, 16, 17, 31, 32, 4, 2] if precision == "fp64"
             else [4, 5, 7, 8, 13, 16, 17, 31, 32, 4, 6])
    mats = I.random_hermitian_batch(sizes, seed=3)
    n_vec = 1 if precision == "fp64" else 3
    H = torch.tensor(_pack(mats), device="cuda")
    ev, vec = lib.eigh_batched(H, sizes, n_vec, precision=precision, ctx=ctx)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    eo = vo = 0
    for A, n in zip(mats, sizes):
        ref = np.linalg.eigvalsh(A)
        got = ev[eo:eo + n]
        scale = max(1.0, np.abs(ref).max())
        tol_v = 1e-12 if precision == "fp64" else 2e-5
        assert np.abs(got - ref).max() <= tol_v * scale
        assert np.abs(got[:n_vec] - ref[:n_vec]).max(initial=0) <= 1e-12 * scale
        V = vec[vo:vo + n * n_vec].reshape(n, n_vec)
        if n_vec:
            res = A @ V - V * got[:n_vec]
            assert np.abs(res).max() <= 1e-11 * scale
            assert np.abs(V.conj().T @ V - np.eye(n_vec)).max() <= 1e-12
        eo += n
        vo += n * n_vec


def test_eigh_degenerate_spectrum(lib, ctx):
    """Exactly doubly degenerate spectra (Kramers-like pairs): the span of each pair."""
    torch = _torch()
    rng = np.random.default_rng(8)
    mats = []
    for n2 in (2, 4, 8, 16):
        A = I.random_hermitian_batch([n2], seed=n2)[0]
        Q, _ = np.linalg.qr(rng.standard_normal((2 * n2, 2 * n2)) + 1j * rng.standard_normal((2 * n2, 2 * n2)))
        mats.append(Q @ np.kron(A, np.eye(2)) @ Q.conj().T)
    sizes = [m.shape[0] for m in mats]
    H = torch.tensor(_pack(mats), device="cuda")
    ev, vec = lib.eigh_batched(H, sizes, 2, ctx=ctx)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    eo = vo = 0
    for A, n in zip(mats, sizes):
        lam, W = np.linalg.eigh(A)
        assert np.abs(ev[eo:eo + n] - lam).max() < 1e-12 * max(1, np.abs(lam).max())
        V = vec[vo:vo + 2 * n].reshape(n, 2)
        Pg, Pr = V @ V.conj().T, W[:, :2] @ W[:, :2].conj().T
        assert np.abs(Pg - Pr).max() < 1e-10
        eo += n
        vo += 2 * n


# ---------------------------------------------------------------- Wilson loops
CASES = {
    "spin_hall_51": (lambda: I.spin_hall(1.0), P(51, 51), 2),
    "chern_eq4": (lambda: I.chern_eq4(1.5), P(30, 13), 1),
    "ssh_pi": (lambda: I.ssh(0.5, 1.0), P(7, 1, trans_dir=(0, 0, 0)), 1),
    "random6_p3": (lambda: I.random_hermitian_model(6, 2), P(17, 5), 3),
    "random13_p5": (lambda: I.random_hermitian_model(13, 4, shells=((1, 0), (0, 1), (1, 1))),
                    P(11, 3, origin=(0.1, 0.2, 0.3), trans_dir=(0.5, 1, 0)), 5),
    "choti_kz": (lambda: I.choti_eq9(1.0), P(20, 9, origin=(0, 0, 0.3)), 2),
    "supercell_L2": (lambda: I.supercell(I.spin_hall(1.0), 2, W=1.0, seed=1), P(9, 6), 8),
    "one_point_loop": (lambda: I.random_hermitian_model(4, 9), P(1, 3), 2),
    "all_bands": (lambda: I.random_hermitian_model(5, 6), P(8, 2), 5),
    "single_band_model": (lambda: I.square_lattice(1.0), P(6, 4), 1),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_wilson_loop_parity(lib, ctx, case, precision):
    mk, plane, p = CASES[case]
    model = mk()
    ref, rgap = oracle.wilson_loop(model, plane, p)
    ph, gap = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    g = gap.cpu().numpy()
    fin = np.isfinite(rgap)
    assert np.all(np.isfinite(g) == fin)
    assert np.abs(g[fin] - rgap[fin]).max(initial=0) <= 1e-9 * max(1, np.abs(rgap[fin]).max(initial=1))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unitarised_loop_parity(lib, ctx, precision):
    model = I.random_hermitian_model(8, 12)
    plane = P(13, 4)
    ref, _ = oracle.wilson_loop(model, plane, 3, unitarise=True)
    ph, _ = lib.wilson_loop(model, plane, 3, precision=precision, ctx=ctx, unitarise=True)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]


# ---------------------------------------------------------------- nested
NESTED = {
    "bbh_24": (lambda: I.bbh(0.5, 0.5), P(24, 24), 2, 1),
    "bbh_trivial": (lambda: I.bbh(1.5, 1.5), P(12, 10), 2, 1),
    "choti_kz": (lambda: I.choti_eq9(1.0), P(12, 12, origin=(0, 0, 0.25)), 2, 1),
    "random8_p4_m2": (lambda: I.random_hermitian_model(8, 21), P(9, 7), 4, 2),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(NESTED))
def test_nested_parity(lib, ctx, case, precision):
    mk, plane, p, m = NESTED[case]
    model = mk()
    try:
        ref_ph, ref_n, ref_wg, _ = oracle.nested_wilson_loop(model, plane, p, m=m)
    except oracle.OracleError as e:
        pytest.skip(f"oracle: {e}")
    ph, nest, wg, _ = lib.nested_wilson_loop(model, plane, p, m=m, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= TOL[precision]
    assert circ_err_rows(nest.cpu().numpy(), ref_n) <= TOL[precision]
    assert abs(wg.cpu().numpy().min() - ref_wg) <= 10 * TOL[precision]


def test_bbh_config_full_size(lib, ctx):
    """The 60 x 60 BBH workload the benchmark times: FP64 and mixed against the oracle."""
    wl = I.config_bbh()
    ref_ph, ref_n, _, _ = oracle.nested_wilson_loop(wl.model, wl.plane, wl.p, m=1)
    for prec in ("fp64", "mixed"):
        ph, nest, _, _ = lib.nested_wilson_loop(wl.model, wl.plane, wl.p, m=1, precision=prec,
                                                ctx=ctx)
        assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= TOL[prec]
        assert circ_err_rows(nest.cpu().numpy(), ref_n) <= TOL[prec]
        assert np.all(np.abs(np.abs(nest.cpu().numpy()) - np.pi) < 1e-9)


# ---------------------------------------------------------------- spin-resolved
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sign", [-1, 1])
def test_spin_resolved_parity(lib, ctx, sign, precision):
    wl = I.config_spin_hall()
    ref, rpso, rpg, _ = oracle.spin_resolved_wilson_loop(wl.model, wl.plane, 2, wl.spin_op, sign)
    ph, pso, pg, _ = lib.spin_resolved_wilson_loop(wl.model, wl.plane, 2, wl.spin_op, sign,
                                                   precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    assert np.abs(pso.cpu().numpy() - rpso).max() <= 1e-10
    assert abs(pg.cpu().numpy().min() - rpg) <= 1e-10
    assert abs(oracle.winding(ph.cpu().numpy()) - sign) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spin_resolved_choti_and_random(lib, ctx, precision):
    model = I.choti_eq9(1.0)
    S = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    plane = P(20, 20)
    ref, rpso, _, _ = oracle.spin_resolved_wilson_loop(model, plane, 2, S, -1)
    ph, pso, _, _ = lib.spin_resolved_wilson_loop(model, plane, 2, S, -1, precision=precision,
                                                  ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    assert np.abs(pso.cpu().numpy() - rpso).max() <= 1e-9
    # a 2 x 2 disordered supercell, p = 8 -> sector of 4
    sc = I.supercell(I.spin_hall(1.0), 2, W=1.5, seed=3)
    S = np.kron(np.eye(4), I.SPIN_HALL_SZ)
    plane = P(8, 6)
    ref, _, _, _ = oracle.spin_resolved_wilson_loop(sc, plane, 8, S, -1)
    ph, _, _, _ = lib.spin_resolved_wilson_loop(sc, plane, 8, S, -1, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]


# ---------------------------------------------------------------- statuses and errors
def test_device_status_gap(lib, ctx):
    with pytest.raises(lib.BWError) as e:
        lib.wilson_loop(I.chern_eq4(2.0), P(8, 8), 1, ctx=ctx)
    assert e.value.status == "EGAP"
    # the status is cleared after being read
    ph, _ = lib.wilson_loop(I.chern_eq4(1.5), P(8, 8), 1, ctx=ctx)


def test_device_status_pso_and_wannier(lib, ctx):
    wl = I.config_spin_hall()
    with pytest.raises(lib.BWError) as e:
        lib.spin_resolved_wilson_loop(wl.model, P(6, 6), 2, np.eye(4, dtype=complex), -1, ctx=ctx)
    assert e.value.status == "EPSOGAP"
    with pytest.raises(lib.BWError) as e:      # Kramers-degenerate WCCs at ky = 0
        lib.nested_wilson_loop(wl.model, P(8, 8), 2, m=1, ctx=ctx)
    assert e.value.status == "EWANGAP"


def test_argument_errors(lib, ctx):
    wl = I.config_spin_hall()
    bad = I.HoppingList(n=2, R=np.zeros((1, 3)), i=[0], j=[1], t=[1.0 + 0j])   # no partner
    for call in (lambda: lib.wilson_loop(bad, P(4, 4), 1, ctx=ctx),
                 lambda: lib.wilson_loop(wl.model, P(4, 4), 5, ctx=ctx),
                 lambda: lib.wilson_loop(wl.model, P(0, 4), 1, ctx=ctx),
                 lambda: lib.spin_resolved_wilson_loop(wl.model, P(4, 4), 1, wl.spin_op, -1, ctx=ctx),
                 lambda: lib.spin_resolved_wilson_loop(wl.model, P(4, 4), 2, wl.spin_op, 0, ctx=ctx),
                 lambda: lib.nested_wilson_loop(wl.model, P(4, 4, trans_dir=(0, 0.5, 0)), 2, m=1, ctx=ctx),
                 lambda: lib.nested_wilson_loop(wl.model, P(4, 4), 2, first=1, m=2, ctx=ctx)):
        with pytest.raises(lib.BWError) as e:
            call()
        assert e.value.status == "EINVAL"


def test_two_streams_same_context(lib, ctx):
    """Calls on different streams through one context are ordered by the context."""
    torch = _torch()
    wl = I.config_bbh()
    ref, _ = lib.wilson_loop(wl.model, wl.plane, 2, ctx=ctx)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for s in (s1, s2, s1):
        with torch.cuda.stream(s):
            outs.append(lib.wilson_loop(wl.model, wl.plane, 2, ctx=ctx, check=False))
    torch.cuda.synchronize()
    ctx.status()
    for ph, _ in outs:
        assert torch.equal(ph, ref)


# ---------------------------------------------------------------- large n (tridiagonal path)
LARGE = {
    "random40_p10": (lambda: I.random_hermitian_model(40, 31), P(9, 5), 10),
    "clean_supercell_L3": (lambda: I.supercell(I.spin_hall(1.0), 3), P(8, 4), 18),
    "disordered_L4": (lambda: I.supercell(I.spin_hall(1.0), 4, W=2.0, seed=7), P(6, 5), 32),
    "manyband64": (lambda: I.manyband(64), P(7, 3), 32),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(LARGE))
def test_large_n_wilson_parity(lib, ctx, case, precision):
    mk, plane, p = LARGE[case]
    model = mk()
    ref, rgap = oracle.wilson_loop(model, plane, p)
    ph, gap = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    rel = np.abs(gap.cpu().numpy() - rgap) / np.maximum(1.0, np.abs(rgap))
    assert rel.max() <= (1e-9 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_n_spin_and_nested(lib, ctx, precision):
    sc = I.supercell(I.spin_hall(1.0), 4, W=1.5, seed=3)          # n = 64, p = 32
    S = np.kron(np.eye(16), I.SPIN_HALL_SZ)
    plane = P(6, 5)
    ref, rpso, _, _ = oracle.spin_resolved_wilson_loop(sc, plane, 32, S, -1)
    ph, pso, _, _ = lib.spin_resolved_wilson_loop(sc, plane, 32, S, -1, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    assert np.abs(pso.cpu().numpy() - rpso).max() <= 1e-8
    model = I.manyband(32)                                          # n = 64, p = 16, m = 8
    plane = P(6, 6)
    try:
        rph, rn, _, _ = oracle.nested_wilson_loop(model, plane, 16, m=8)
    except oracle.OracleError as e:
        pytest.skip(f"oracle: {e}")
    ph, nest, _, _ = lib.nested_wilson_loop(model, plane, 16, m=8, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), rph) <= TOL[precision]
    assert circ_err_rows(nest.cpu().numpy(), rn) <= TOL[precision]


# ---------------------------------------------------------------- many occupied bands (p > 64)
MANY = {
    "flux_L6": (lambda: I.supercell(I.spin_hall(1.0), 6, W=1.0, seed=11, flux=True), P(6, 4), 72),
    "random160_p80": (lambda: I.random_hermitian_model(160, 41), P(5, 3), 80),
    "disordered_L10": (lambda: I.supercell(I.spin_hall(1.0), 10, W=2.0, seed=5), P(4, 3), 200),
    # either side of the switch to the cluster eigenphase solver (p >= 128), with sweeps
    # whose rotation count is not a multiple of the 16-rotation chunk
    "random254_p127": (lambda: I.random_hermitian_model(254, 43), P(4, 3), 127),
    "random256_p128": (lambda: I.random_hermitian_model(256, 44), P(4, 3), 128),
    "random300_p149": (lambda: I.random_hermitian_model(300, 45), P(3, 2), 149),
    # coarse loops (8 k-points) of a disordered L = 12 supercell filled to p = 144 of
    # n = 576: a Wilson matrix far from unitary, on which the double-float QR of the
    # mixed request stalled short of deflation at a 2^-47 threshold
    "disordered_L12_p144": (lambda: I.supercell(I.spin_hall(1.0), 12, W=2.0, seed=5), P(8, 8), 144),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(MANY))
def test_many_band_wilson_parity(lib, ctx, case, precision):
    """Streamed loop (GEMM overlaps and products, global-memory eigenphases) vs the oracle."""
    mk, plane, p = MANY[case]
    model = mk()
    ref, rgap = oracle.wilson_loop(model, plane, p)
    ph, gap = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    rel = np.abs(gap.cpu().numpy() - rgap) / np.maximum(1.0, np.abs(rgap))
    assert rel.max() <= (1e-9 if precision == "fp64" else 1e-6)


def test_many_band_blocks_of_loops(lib):
    """A budget that holds a few loops and a few k-points at a time (several blocks of
    loops, several solver waves per block) gives the same phases as one block."""
    torch = pytest.importorskip("torch")
    model = I.supercell(I.spin_hall(1.0), 6, W=1.0, seed=11, flux=True)   # n = 144, p = 72
    plane = P(5, 5)
    big = lib.Context(0)
    small = lib.Context(0, 8 << 20)
    try:
        a, ga = lib.wilson_loop(model, plane, 72, precision="mixed", ctx=big)
        b, gb = lib.wilson_loop(model, plane, 72, precision="mixed", ctx=small)
        assert torch.equal(a, b) and torch.equal(ga, gb)
    finally:
        big.close()
        small.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n_vec", [0, 3])
def test_eigh_batched_large_ragged(lib, ctx, precision, n_vec):
    """Uneven sizes across the shared-memory (n <= 32) and tridiagonal (n > 32) solvers
    in one batch; the upper triangle of the large matrices is garbage (only the lower
    one is read)."""
    torch = _torch()
    sizes = [5, 40, 33, 64, 40, 100, 7, 129]
    mats = I.random_hermitian_batch(sizes, seed=17)
    packed = []
    for A, n in zip(mats, sizes):
        B = A.copy()
        if n > 32:
            B[np.triu_indices(n, 1)] = 7.0 + 3.0j
        packed.append(B.reshape(-1))
    H = torch.tensor(np.concatenate(packed), device="cuda")
    ev, vec = lib.eigh_batched(H, sizes, n_vec, precision=precision, ctx=ctx)
    ev = ev.cpu().numpy()
    vec = vec.cpu().numpy() if vec is not None else None
    eo = vo = 0
    for A, n in zip(mats, sizes):
        ref = np.linalg.eigvalsh(A)
        got = ev[eo:eo + n]
        scale = max(1.0, np.abs(ref).max())
        tol_v = 1e-12 if precision == "fp64" else 2e-5
        assert np.abs(got - ref).max() <= tol_v * scale, (n, np.abs(got - ref).max())
        assert np.abs(got[:n_vec] - ref[:n_vec]).max(initial=0) <= 1e-12 * scale
        if n_vec:
            V = vec[vo:vo + n * n_vec].reshape(n, n_vec)
            res = A @ V - V * got[:n_vec]
            assert np.abs(res).max() <= 1e-11 * scale, (n, np.abs(res).max())
            assert np.abs(V.conj().T @ V - np.eye(n_vec)).max() <= 1e-12
        eo += n
        vo += n * n_vec


# ---------------------------------------------------------------- winding (Eq. 6)
def test_winding_parity(lib, ctx):
    """bw_winding against the oracle's winding: loop outputs of the spin-Hall model
    (total 0, sectors -1 / +1), Eq. 4 (+1), and seeded random phase tables, including
    one row and one band."""
    torch = _torch()
    wl = I.config_spin_hall()
    for sign in (-1, 1):
        ph, _, _, _ = lib.spin_resolved_wilson_loop(wl.model, wl.plane, 2, wl.spin_op, sign, ctx=ctx)
        w, sums = lib.winding(ph, ctx=ctx, want_sums=True)
        ref = oracle.winding(ph.cpu().numpy())
        assert abs(w.item() - ref) < 1e-12 and abs(w.item() - sign) < 1e-6
        assert np.abs(sums.cpu().numpy() - ph.cpu().numpy().sum(axis=1) / (2 * np.pi)).max() < 1e-14
    ph, _ = lib.wilson_loop(I.chern_eq4(), P(24, 24), 1, ctx=ctx)
    assert abs(lib.winding(ph, ctx=ctx).item() - oracle.winding(ph.cpu().numpy())) < 1e-12
    assert abs(lib.winding(ph, ctx=ctx).item() - 1) < 1e-6
    rng = np.random.default_rng(11)
    for Nt, p in ((1, 1), (7, 1), (300, 3), (1000, 16)):
        th = rng.uniform(-np.pi, np.pi, size=(Nt, p))
        w = lib.winding(torch.tensor(th, device="cuda"), ctx=ctx).item()
        assert abs(w - oracle.winding(th)) < 1e-11, (Nt, p)


# ---------------------------------------------------------------- mixed, four bands
# The mixed request with n = 4 and p = 2 runs states, overlaps and loop products in
# double-float on the FP32 pipe; its phases stay within 1e-9 rad of the FP64 oracle
# (far inside the 1e-6 rad the mixed path promises) and its gaps, Ritz values of
# the refined pairs, within 1e-9 relative even with degenerate bands (Eq. 9, BBH).
# The other occupied counts take the FP64 four-lane kernel and meet the same bounds.
DF_TOL = 1e-9
DF_CASES = {
    "random4_p1": (lambda: I.random_hermitian_model(4, 31), P(13, 7, origin=(0.1, 0.2, 0.0)), 1),
    "random4_p2": (lambda: I.random_hermitian_model(4, 32), P(13, 7), 2),
    "random4_p3": (lambda: I.random_hermitian_model(4, 33, shells=((1, 0), (0, 1), (1, 1))),
                   P(11, 5, origin=(0.3, 0.0, 0.0)), 3),
    "random4_p4": (lambda: I.random_hermitian_model(4, 34), P(9, 3), 4),
    "spin_hall_51": (lambda: I.spin_hall(1.0), P(51, 51), 2),
    "choti_kz": (lambda: I.choti_eq9(1.0), P(20, 9, origin=(0, 0, 0.3)), 2),
}


@pytest.mark.parametrize("case", sorted(DF_CASES))
def test_mixed_four_band_double_float(lib, ctx, case):
    mk, plane, p = DF_CASES[case]
    model = mk()
    ref, rgap = oracle.wilson_loop(model, plane, p)
    ph, gap = lib.wilson_loop(model, plane, p, precision="mixed", ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= DF_TOL
    g = gap.cpu().numpy()
    fin = np.isfinite(rgap)
    assert np.all(np.isfinite(g) == fin)
    assert np.abs(g[fin] - rgap[fin]).max(initial=0) <= 1e-9 * max(1, np.abs(rgap[fin]).max(initial=1))


def test_mixed_four_band_nested_double_float(lib, ctx):
    for model, plane, p, m in ((I.bbh(0.5, 0.5), P(60, 60), 2, 1),
                               (I.bbh(1.5, 1.5), P(12, 10), 2, 1),
                               (I.choti_eq9(1.0), P(12, 12, origin=(0, 0, 0.25)), 2, 1)):
        ref_ph, ref_n, ref_wg, _ = oracle.nested_wilson_loop(model, plane, p, m=m)
        ph, nest, wg, _ = lib.nested_wilson_loop(model, plane, p, m=m, precision="mixed", ctx=ctx)
        assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= DF_TOL
        assert circ_err_rows(nest.cpu().numpy(), ref_n) <= DF_TOL
        assert abs(wg.cpu().numpy().min() - ref_wg) <= 1e-8


# ---------------------------------------------------------------- spin-resolved, p > 64
# Spin-resolved loop with many occupied bands: S = U^dagger s U by GEMM, its FP64
# eigensolve on the tridiagonal path, the sector states U V through the batched loop.
SPIN_MANY = {
    # disordered spin-Hall supercell (s_z conserved: PSO eigenvalues exactly +-1,
    # 36-fold degenerate), n = 144, p = 72
    "disordered_L6": (lambda: I.supercell(I.spin_hall(1.0), 6, W=2.0, seed=7),
                      lambda: np.kron(np.eye(36), I.SPIN_HALL_SZ), P(6, 5), 72),
    # Eq. 9 supercell with s3 (x) t3 (a spread PSO spectrum), n = 144, p = 72
    "choti_L6": (lambda: I.supercell(I.choti_eq9(1.0), 6),
                 lambda: np.kron(np.eye(36), np.diag([1.0, -1.0, -1.0, 1.0])), P(5, 4, origin=(0, 0, 0.1)), 72),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(SPIN_MANY))
@pytest.mark.parametrize("sign", [-1, 1])
def test_spin_resolved_many_bands(lib, ctx, case, precision, sign):
    mk, mkS, plane, p = SPIN_MANY[case]
    model, S = mk(), mkS()
    ref, rpso, rpg, _ = oracle.spin_resolved_wilson_loop(model, plane, p, S, sign)
    ph, pso, pg, _ = lib.spin_resolved_wilson_loop(model, plane, p, S, sign, precision=precision,
                                                   ctx=ctx)
    assert ph.shape == (plane.N_t, p // 2)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
    assert np.abs(pso.cpu().numpy() - rpso).max() <= 1e-9
    assert abs(pg.cpu().numpy().min() - rpg) <= 1e-9


def test_spin_resolved_many_bands_status(lib, ctx):
    """A spin operator whose projected spectrum has no gap at zero fails with EPSOGAP."""
    model = I.supercell(I.spin_hall(1.0), 6, W=2.0, seed=7)
    S = np.kron(np.eye(36), np.diag([1.0, 1.0, 1.0, 1.0]))   # every PSO eigenvalue is +1
    with pytest.raises(lib.BWError) as e:
        lib.spin_resolved_wilson_loop(model, P(4, 3), 72, S, -1, ctx=ctx)
    assert e.value.status == "EPSOGAP"


# ---------------------------------------------------------------- plaquette flux
PLAQ = {
    "chern_eq4": (lambda: I.chern_eq4(1.5), None, P(16, 16), 1, -1),
    "spin_hall_down": (lambda: I.spin_hall(1.0), I.SPIN_HALL_SZ, P(20, 20), 2, -1),
    "spin_hall_up": (lambda: I.spin_hall(1.0), I.SPIN_HALL_SZ, P(20, 20), 2, 1),
    "random6_p3": (lambda: I.random_hermitian_model(6, 2), None, P(7, 5), 3, -1),
    "supercell_L4_down": (lambda: I.supercell(I.spin_hall(1.0), 4, W=1.5, seed=3),
                          np.kron(np.eye(16), I.SPIN_HALL_SZ), P(5, 4), 32, -1),
    # Eq. 10 (Sec. IV A): clean, and a 4 x 4 supercell with chiral disorder at W = 1
    "quadrupolar_eq10": (lambda: I.quadrupolar_eq10(), I.EQ10_SPIN, P(16, 16), 2, -1),
    "quadrupolar_L4_W1": (lambda: I.config_quadrupolar(4, 1.0, 1).model,
                          np.kron(np.eye(16), I.EQ10_SPIN), P(6, 6), 32, -1),
    # more than 64 bands in the loop: link matrices by batched GEMM and determinant
    # phases by LU in global memory (Eq. 4 supercell, p = 81; Eq. 10 L = 9, sector 81),
    # and the PSO split of p = 72 feeding the shared-memory links (Eq. 10 L = 6)
    "chern_eq4_L9_p81": (lambda: I.supercell(I.chern_eq4(1.5), 9), None, P(6, 5), 81, -1),
    "quadrupolar_L6_W1_p72": (lambda: I.config_quadrupolar(6, 1.0, 2).model,
                              np.kron(np.eye(36), I.EQ10_SPIN), P(5, 5), 72, -1),
    "quadrupolar_L9_W1_p162": (lambda: I.config_quadrupolar(9, 1.0, 3).model,
                               np.kron(np.eye(81), I.EQ10_SPIN), P(4, 4), 162, -1),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(PLAQ))
def test_plaquette_flux_parity(lib, ctx, case, precision):
    """Flux of every plaquette against the oracle (circular distance) and the total."""
    mk, S, plane, p, sign = PLAQ[case]
    model = mk()
    rflux, rC = oracle.plaquette_flux(model, plane, p, S, sign)
    flux, C, gap, pg = lib.plaquette_flux(model, plane, p, S, sign, precision=precision, ctx=ctx)
    d = np.abs(np.angle(np.exp(1j * (flux.cpu().numpy() - rflux))))
    assert d.max() <= TOL[precision]
    assert abs(C.item() - rC) <= 1e-8
    assert np.all(np.isfinite(gap.cpu().numpy()))
    if S is not None:
        assert np.all(pg.cpu().numpy() > 0)


def test_plaquette_flux_many_band_invariants(lib, ctx):
    """Past 64 bands: the Eq. 4 supercell keeps C = 1 (band folding preserves the Chern
    number of the filled bands) and the Eq. 10 supercell at W = 1 keeps |C_s| = 1
    (Sec. IV A, Fig. 6(c)), on finer grids than the parity cases."""
    _, C, _, _ = lib.plaquette_flux(I.supercell(I.chern_eq4(1.5), 9), P(12, 12), 81,
                                    precision="mixed", ctx=ctx)
    assert abs(C.item() - 1) < 1e-9
    wl = I.config_quadrupolar(9, 1.0, 4)
    _, Cs, _, pg = lib.plaquette_flux(wl.model, P(8, 8), wl.p, wl.spin_op, -1, precision="mixed",
                                      ctx=ctx)
    assert abs(abs(Cs.item()) - 1) < 1e-9
    assert pg.min().item() > 1e-3


def test_plaquette_flux_invariants(lib, ctx):
    """Eq. 4 carries C = 1 (paper); the spin-Hall sectors -1 / +1, total 0."""
    _, C, _, _ = lib.plaquette_flux(I.chern_eq4(1.5), P(24, 24), 1, ctx=ctx)
    assert abs(C.item() - 1) < 1e-9
    wl = I.config_spin_hall()
    _, Ct, _, _ = lib.plaquette_flux(wl.model, wl.plane, 2, ctx=ctx)
    _, Cd, _, _ = lib.plaquette_flux(wl.model, wl.plane, 2, wl.spin_op, -1, precision="mixed", ctx=ctx)
    _, Cu, _, _ = lib.plaquette_flux(wl.model, wl.plane, 2, wl.spin_op, 1, precision="mixed", ctx=ctx)
    assert abs(Ct.item()) < 1e-9 and abs(Cd.item() + 1) < 1e-9 and abs(Cu.item() - 1) < 1e-9


def test_disordered_supercell_spin_chern(lib, ctx):
    """Disordered spin-Hall supercell at full size (L = 10, n = 400, p = 200, W = 2,
    16 x 16): the C_down / C_up windings are -1 / +1 (the clean model's values survive
    this disorder), and one transverse row matches the oracle."""
    wl = I.config_disordered(10, 5)
    for sign in (-1, 1):
        ph, _, pg, _ = lib.spin_resolved_wilson_loop(wl.model, wl.plane, wl.p, wl.spin_op, sign,
                                                     precision="mixed", ctx=ctx, want_pso=False)
        assert abs(lib.winding(ph, ctx=ctx).item() - sign) < 1e-6
        assert pg.min().item() > 0.9
    row = 7
    plr = P(wl.plane.N, 1, origin=tuple(np.array(wl.plane.trans_dir) * row / wl.plane.N_t))
    ref, _, _, _ = oracle.spin_resolved_wilson_loop(wl.model, plr, wl.p, wl.spin_op, -1)
    ph, _, _, _ = lib.spin_resolved_wilson_loop(wl.model, wl.plane, wl.p, wl.spin_op, -1,
                                                precision="mixed", ctx=ctx, want_pso=False)
    assert circ_err_rows(ph.cpu().numpy()[row:row + 1], ref) <= TOL["mixed"]


def test_mixed_four_band_launch_shapes(lib, ctx):
    """The double-float path at the edges of its launch shapes: loops of exactly 64
    points (256 threads, one CTA per loop), loops of 70 points (separate states and
    loop kernels), and a nested loop over more loops than the GPU holds at once (no
    cooperative launch: loop kernel, then the nested kernel)."""
    model = I.bbh(0.5, 0.5)
    for plane in (P(64, 5), P(70, 4, origin=(0.0, 0.1, 0.0))):
        ref, rgap = oracle.wilson_loop(model, plane, 2)
        ph, gap = lib.wilson_loop(model, plane, 2, precision="mixed", ctx=ctx)
        assert circ_err_rows(ph.cpu().numpy(), ref) <= DF_TOL
        assert np.abs(gap.cpu().numpy() - rgap).max() <= 1e-9 * np.abs(rgap).max()
    plane = P(8, 2000)
    ref_ph, ref_n, _, _ = oracle.nested_wilson_loop(model, plane, 2, m=1)
    ph, nest, _, _ = lib.nested_wilson_loop(model, plane, 2, m=1, precision="mixed", ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= DF_TOL
    assert circ_err_rows(nest.cpu().numpy(), ref_n) <= DF_TOL


# ---------------------------------------------------------------- Z2 from WCC connectivity
def _z2_phase_tables():
    """Seeded phase tables: oracle spectra of the paper's models and drawn spectra
    with exact ties (Kramers-degenerate rows, repeated values), +-pi, one band, many
    bands, and enough rows that the row and step kernels span several CTAs."""
    rng = np.random.default_rng(17)
    out = {}
    out["eq7"] = oracle.wilson_loop(I.bhz_eq7(1.5), P(16, 32), 2)[0]
    out["eq7_trivial"] = oracle.wilson_loop(I.bhz_eq7(3.5), P(16, 32), 2)[0]
    out["vacancy_L4"] = oracle.wilson_loop(I.config_vacancy(4, 0.0).model, P(10, 16), 30)[0]
    t = np.arange(64) / 64
    out["switch_pair"] = np.sort(np.stack([2 * np.pi * t, -2 * np.pi * t], 1), axis=1)
    out["degenerate"] = np.sort(np.repeat(rng.uniform(-np.pi, np.pi, (40, 3)), 2, axis=1), axis=1)
    edge = np.sort(rng.uniform(-np.pi, np.pi, (10, 5)), axis=1)
    edge[:, 0], edge[:, -1] = -np.pi, np.pi
    out["plus_minus_pi"] = edge
    out["one_band"] = rng.uniform(-np.pi, np.pi, (18, 1))
    out["many"] = np.sort(rng.uniform(-np.pi, np.pi, (300, 97)), axis=1)
    out["quantised"] = np.sort(rng.integers(-8, 9, (50, 6)) * (np.pi / 8), axis=1)
    return out


def test_z2_largest_gap_parity(lib, ctx):
    """Same phases in, bit-identical midpoints, widths, crossings and index out."""
    torch = _torch()
    for name, ph in _z2_phase_tables().items():
        nu_r, c_r, mid_r, w_r = oracle.z2_largest_gap(ph)
        nu, c, mid, w = lib.z2_largest_gap(torch.tensor(np.ascontiguousarray(ph), device="cuda"),
                                           ctx=ctx, want_detail=True)
        assert nu.item() == nu_r, name
        assert np.array_equal(c.cpu().numpy(), c_r), name
        assert np.array_equal(mid.cpu().numpy(), mid_r), name
        assert np.array_equal(w.cpu().numpy(), w_r), name


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_z2_from_gpu_loops(lib, ctx, precision):
    """The paper's statements end to end on the GPU: Eq. 7 nu = 1 (Sec. II B), nu = 0
    past the band inversion, and nu = 1 for supercells with vacancies (Sec. II C,
    p = 48 and p = 62); each equal to the oracle's index of the oracle's spectrum."""
    cases = [(I.bhz_eq7(1.5), P(24, 32), 2, 1), (I.bhz_eq7(3.5), P(24, 32), 2, 0),
             (I.config_vacancy(5, 0.0).model, P(12, 16), 48, 1),
             (I.config_vacancy(6, 1.0).model, P(12, 16), 62, 1)]
    for model, plane, p, expect in cases:
        ph, _ = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
        nu = lib.z2_largest_gap(ph, ctx=ctx).item()
        ref = oracle.z2_largest_gap(oracle.wilson_loop(model, plane, p)[0])[0]
        assert nu == ref == expect, model.name


def test_z2_rejects_bad_input(lib, ctx):
    """An unsorted row gives nu = -1 and BW_EINVAL from the device status (with the row);
    an odd N_t is refused at the call."""
    torch = _torch()
    ph = np.sort(np.random.default_rng(3).uniform(-np.pi, np.pi, (8, 4)), axis=1)
    bad = ph.copy()
    bad[3] = bad[3][::-1]
    nu = lib.z2_largest_gap(torch.tensor(bad, device="cuda"), ctx=ctx, check=False)
    assert nu.item() == -1
    with pytest.raises(lib.BWError) as e:
        ctx.status()
    assert e.value.code == 1 and e.value.k_index == 3
    with pytest.raises(lib.BWError):
        lib.z2_largest_gap(torch.tensor(ph[:7].copy(), device="cuda"), ctx=ctx)


# ---------------------------------------------------------------- stacks of planes
def _stack_ref(fn, stack, *args, **kw):
    return [fn(*args[:1], pl, *args[1:], **kw) for pl in stack.planes()]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plane_stack_parity(lib, ctx, precision):
    """Every plane of a stack against the oracle on that plane: Eq. 9 over k_z (3D, the
    tabulated four-band kernels), a many-band model (n = 40, tridiagonal path), and one
    plane (the single-plane call, bit for bit)."""
    tol = TOL[precision]
    model = I.choti_eq9(1.0)
    st = I.PlaneStack(P(12, 10, origin=(0.0, 0.05, 0.0)), (0, 0, 1), 5)
    ph, gap = lib.wilson_loop(model, st, 2, precision=precision, ctx=ctx)
    assert ph.shape == (5, 10, 2) and gap.shape == (5, 10)
    for s, pl in enumerate(st.planes()):
        rph, rgap = oracle.wilson_loop(model, pl, 2)
        assert circ_err_rows(ph[s].cpu().numpy(), rph) <= tol, s
        assert np.abs(gap[s].cpu().numpy() - rgap).max() <= 1e-9 * max(1.0, rgap.max())
    big = I.manyband(20)
    st = I.PlaneStack(P(6, 4), (0, 0, 1), 3)        # a 2D model: identical planes
    ph, _ = lib.wilson_loop(big, st, 10, precision=precision, ctx=ctx)
    rph, _ = oracle.wilson_loop(big, P(6, 4), 10)
    for s in range(3):
        assert circ_err_rows(ph[s].cpu().numpy(), rph) <= tol
        assert np.array_equal(ph[s].cpu().numpy(), ph[0].cpu().numpy())
    one = I.PlaneStack(P(12, 10, origin=(0.0, 0.0, 0.25)), (0, 0, 1), 1)
    a, _ = lib.wilson_loop(model, one, 2, precision=precision, ctx=ctx)
    b, _ = lib.wilson_loop(model, one.plane, 2, precision=precision, ctx=ctx)
    assert np.array_equal(a[0].cpu().numpy(), b.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nested_stack_over_kz(lib, ctx, precision):
    """Sec. III, Fig. 4(b): the nested spectrum of Eq. 9 (Delta0 = 1) over a k_z stack,
    every plane against the oracle; its phase winds once over k_z.  The 12 x 12 x 12
    stack runs the mixed path's fused kernel (one cooperative launch for all planes)."""
    model = I.choti_eq9(1.0)
    st = I.PlaneStack(P(12, 12), (0, 0, 1), 12)
    ph, nest, wg, gap = lib.nested_wilson_loop(model, st, 2, m=1, precision=precision, ctx=ctx)
    assert nest.shape == (12, 12, 1) and wg.shape == (12, 12)
    tol = TOL[precision]
    for s, pl in enumerate(st.planes()):
        rph, rnest, _, _ = oracle.nested_wilson_loop(model, pl, 2, m=1)
        assert circ_err_rows(ph[s].cpu().numpy(), rph) <= tol, s
        d = np.abs(np.angle(np.exp(1j * (nest[s].cpu().numpy() - rnest))))
        assert d.max() <= 10 * tol, s
    curve = nest[:, 0, :].cpu().numpy()
    assert abs(abs(oracle.winding(curve)) - 1) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spin_resolved_stack(lib, ctx, precision):
    """Spin-resolved loops of Eq. 9 on a k_z stack (s = s3 (x) t3) against the oracle."""
    model = I.choti_eq9(1.0)
    S = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    st = I.PlaneStack(P(10, 8), (0, 0, 1), 4)
    ph, pso, pg, _ = lib.spin_resolved_wilson_loop(model, st, 2, S, -1, precision=precision, ctx=ctx)
    assert ph.shape == (4, 8, 1) and pso.shape == (4, 8, 10, 2)
    for s, pl in enumerate(st.planes()):
        rph, rpso, rpg, _ = oracle.spin_resolved_wilson_loop(model, pl, 2, S, -1)
        assert circ_err_rows(ph[s].cpu().numpy(), rph) <= TOL[precision], s
        assert np.abs(np.sort(pso[s].cpu().numpy(), -1) - np.sort(rpso, -1)).max() <= 1e-9


def test_z2_weak_strong_from_planes(lib, ctx):
    """Sec. II B / Sec. III: Eq. 9 with Delta0 = 0 is a strong topological insulator.
    The stacks k_z in {0, 1/2} and k_x in {0, 1/2} give nu = (1, 0) each on the GPU,
    so nu0 = 1 and the weak indices vanish (the oracle agrees plane by plane)."""
    model = I.choti_eq9(0.0)
    stacks = [I.PlaneStack(P(24, 16), (0, 0, 1), 2),
              I.PlaneStack(P(24, 16, loop_dir=(0, 1, 0), trans_dir=(0, 0, 1)), (1, 0, 0), 2)]
    for st in stacks:
        ph, _ = lib.wilson_loop(model, st, 2, ctx=ctx)
        z = [lib.z2_largest_gap(ph[s].contiguous(), ctx=ctx).item() for s in range(2)]
        ref = [oracle.z2_largest_gap(oracle.wilson_loop(model, pl, 2)[0])[0] for pl in st.planes()]
        assert z == ref == [1, 0]


def test_plane_stack_rejections(lib, ctx):
    """A stack with N_s < 1 is refused at the call."""
    st = I.PlaneStack(P(6, 6), (0, 0, 1), 0)
    with pytest.raises(lib.BWError):
        lib.wilson_loop(I.choti_eq9(1.0), st, 2, ctx=ctx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vacancy_supercell_parity(lib, ctx, precision):
    """Sec. II C: an Eq. 7 supercell with the cells within r = 1 of the origin removed
    (6 x 6 cells less 5, n = 124, p = 62): Wannier centres and the s3 (x) t3 sector's
    centres against the oracle; the sector winds -1."""
    wl = I.config_vacancy(6, 1.0)
    plane = P(10, 8)
    ph, gap = lib.wilson_loop(wl.model, plane, wl.p, precision=precision, ctx=ctx)
    rph, rgap = oracle.wilson_loop(wl.model, plane, wl.p)
    assert circ_err_rows(ph.cpu().numpy(), rph) <= TOL[precision]
    assert np.abs(gap.cpu().numpy() - rgap).max() <= 1e-9
    dn, _, pg, _ = lib.spin_resolved_wilson_loop(wl.model, plane, wl.p, wl.spin_op, -1,
                                                 precision=precision, ctx=ctx, want_pso=False)
    rdn, _, _, _ = oracle.spin_resolved_wilson_loop(wl.model, plane, wl.p, wl.spin_op, -1)
    assert circ_err_rows(dn.cpu().numpy(), rdn) <= TOL[precision]
    assert abs(lib.winding(dn, ctx=ctx).item() + 1) < 1e-6


def test_eigh_batched_n256_n1024(lib, ctx):
    """The FP64 tridiagonal solver at n = 256 and 1024 in one batch, with a degenerate
    spectrum (each eigenvalue of a 128 x 128 block repeated four times at n = 512):
    eigenvalues against LAPACK, residual |A V - V lam| and orthonormality of the lowest
    eight vectors (a degenerate block's vectors only span the right subspace).  The
    lowest eight eigenvalues of the degenerate matrix are two clusters of four with a
    gap of 0.16 above them."""
    torch = _torch()
    rng = np.random.default_rng(23)
    mats = I.random_hermitian_batch([256, 1024], seed=29)
    B = I.random_hermitian_batch([128], seed=31)[0]
    Q, _ = np.linalg.qr(rng.standard_normal((512, 512)) + 1j * rng.standard_normal((512, 512)))
    D = Q @ np.kron(np.eye(4), B) @ Q.conj().T
    mats.append(0.5 * (D + D.conj().T))
    sizes = [m.shape[0] for m in mats]
    n_vec = 8
    H = torch.tensor(np.concatenate([m.reshape(-1) for m in mats]), device="cuda")
    ev, vec = lib.eigh_batched(H, sizes, n_vec, precision="fp64", ctx=ctx)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy()
    eo = vo = 0
    for A, n in zip(mats, sizes):
        ref = np.linalg.eigvalsh(A)
        got = ev[eo:eo + n]
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= 1e-12 * scale, n
        assert np.abs(got[:n_vec] - ref[:n_vec]).max() <= 1e-11 * scale, n
        V = vec[vo:vo + n * n_vec].reshape(n, n_vec)
        assert np.abs(A @ V - V * got[:n_vec]).max() <= 1e-10 * scale, n
        assert np.abs(V.conj().T @ V - np.eye(n_vec)).max() <= 1e-11, n
        eo += n
        vo += n * n_vec


@pytest.mark.parametrize("n,n_vec", [(256, 8), (256, 64), (1024, 8), (1024, 64)])
def test_eigh_batched_mixed_refined_block(lib, ctx, n, n_vec):
    """The mixed solver at n = 256 and 1024: FP32 tridiagonal solve, then the lowest
    n_vec vectors refined to FP64 grade.  A gap of 0.5 is opened above the refined block
    (its eigenvalues are shifted down), as the refinement needs.  The refined block is
    FP64-grade, not FP64: its residual and Ritz values are formed in compensated FP32
    arithmetic (about 48 significant bits, 2^-48 ~ 3.6e-15), which over an n = 1024
    inner product leaves ~1e-11 relative (measured 4.0e-11 absolute at |A| = 3.3); the
    bounds are ten times the FP64 solver's: eigenvalues 1e-10 |A| against LAPACK,
    residual |A V - V lam| 1e-9 |A|, orthonormality 1e-10.  The other eigenvalues are
    FP32-accurate."""
    torch = _torch()
    A = I.random_hermitian_batch([n], seed=41 + n + n_vec)[0]
    lam, V = np.linalg.eigh(A)
    A = A - 0.5 * (V[:, :n_vec] @ V[:, :n_vec].conj().T)
    A = 0.5 * (A + A.conj().T)
    H = torch.tensor(A.reshape(-1), device="cuda")
    ev, vec = lib.eigh_batched(H, [n], n_vec, precision="mixed", ctx=ctx)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy().reshape(n, n_vec)
    ref = lam.copy()      # the shift moves the lowest n_vec eigenvalues by -0.5 exactly
    ref[:n_vec] -= 0.5
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(ev[:n_vec] - ref[:n_vec]).max() <= 1e-10 * scale
    assert np.abs(A @ vec - vec * ev[:n_vec]).max() <= 1e-9 * scale
    assert np.abs(vec.conj().T @ vec - np.eye(n_vec)).max() <= 1e-10
    assert np.abs(ev[n_vec:] - ref[n_vec:]).max() <= 1e-5 * scale


LADDER_GPU = [(-np.pi, 0, 1), (-np.pi, 1, 1), (-np.pi, 2, 1), (-np.pi, 0, 2), (0.0, 1, 1),
              (0.0, 0, 2), (-np.pi + 1.0, 0, 1), (-np.pi + 1.0, 1, 2), (-np.pi, 0, 3)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cut,first,m", LADDER_GPU)
def test_nested_sector_choice_ladder(lib, ctx, precision, cut, first, m):
    """The nested sector (cut, first, m) on the three-block Wannier ladder, whose nested
    phases identify the sector (pinned in closed form on the oracle): GPU against the
    oracle, nested phases and Wannier gap."""
    model, plane = I.wannier_ladder(), P(24, 20)
    ref_ph, ref_n, ref_g, _ = oracle.nested_wilson_loop(model, plane, 3, cut=cut, first=first, m=m)
    ph, nest, wg, _ = lib.nested_wilson_loop(model, plane, 3, cut=cut, first=first, m=m,
                                             precision=precision, ctx=ctx)
    assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= TOL[precision]
    assert circ_err_rows(nest.cpu().numpy(), ref_n) <= TOL[precision]
    if np.isfinite(ref_g):
        assert abs(float(wg.min()) - ref_g) <= TOL[precision]


@pytest.mark.parametrize("case", ["bbh_60x60", "disordered_L4"])
def test_row_blocks_match_whole_plane(lib, ctx, case):
    """The row blocks a rank computes when a plane is sharded (shard.row_block), run one
    after another on this GPU, reproduce the whole-plane call row by row."""
    from paper_2312_13051_gb300 import shard
    if case == "bbh_60x60":
        model, plane, p = I.config_bbh().model, P(60, 60), 2
    else:
        model, plane, p = I.supercell(I.spin_hall(1.0), 4, W=2.0, seed=7), P(10, 9), 32
    for precision in ("fp64", "mixed"):
        full, gfull = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
        full, gfull = full.cpu().numpy(), gfull.cpu().numpy()
        compute = shard.gpu_wilson_rows(precision, ctx=ctx)
        for i0, i1 in shard.partition(plane.N_t, 3):
            ph, gap = compute(model, shard.row_block(plane, i0, i1), p)
            assert circ_err_rows(ph, full[i0:i1]) <= 1e-12
            np.testing.assert_allclose(gap, gfull[i0:i1], atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pso_median_split_fig6(lib, ctx, precision):
    """The PSO sector split at the median (bw_opts.pso_split = 1) on the Eq. 10
    supercells: flux of every plaquette against the oracle's median-split reading, and
    Fig. 6(c)-(d)'s spin-Chern numbers, |C_s| = 1 at W = 1 and C_s = 0 at W = 9 (where the
    split at zero reports EPSOGAP)."""
    for W, want in ((1.0, 1.0), (9.0, 0.0)):
        wl = I.config_quadrupolar(4, W, 1, nk=6)
        rflux, rC = oracle.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1, pso_split="median")
        flux, C, _, pg = lib.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1, precision=precision,
                                            ctx=ctx, pso_split="median")
        d = np.abs(np.angle(np.exp(1j * (flux.cpu().numpy() - rflux))))
        assert d.max() <= TOL[precision]
        assert abs(abs(C.item()) - want) < 1e-8 and abs(C.item() - rC) < 1e-8
        assert pg.min().item() > 0
    wl = I.config_quadrupolar(4, 9.0, 1, nk=6)
    with pytest.raises(lib.BWError) as e:
        lib.plaquette_flux(wl.model, wl.plane, wl.p, wl.spin_op, -1, precision=precision, ctx=ctx)
    assert e.value.status == "EPSOGAP"


@pytest.mark.parametrize("case", ["eq10_clean_n4", "eq10_L2_n16", "eq10_L4_n64"])
def test_pso_median_split_spin_resolved_parity(lib, ctx, case):
    """Spin-resolved phases with the median split against the oracle, on the one-thread
    (n = 4), shared-memory (n = 16) and tridiagonal (n = 64) paths, both signs."""
    if case == "eq10_clean_n4":
        model, S, plane, p = I.quadrupolar_eq10(), I.EQ10_SPIN, P(12, 10), 2
    elif case == "eq10_L2_n16":
        wl = I.config_quadrupolar(2, 9.0, 3, nk=6)
        model, S, plane, p = wl.model, wl.spin_op, P(8, 6), wl.p
    else:
        wl = I.config_quadrupolar(4, 9.0, 2, nk=6)
        model, S, plane, p = wl.model, wl.spin_op, P(6, 5), wl.p
    for sign in (-1, 1):
        ref, rpso, _, _ = oracle.spin_resolved_wilson_loop(model, plane, p, S, sign, pso_split="median")
        for precision in ("fp64", "mixed"):
            ph, pso, pg, _ = lib.spin_resolved_wilson_loop(model, plane, p, S, sign, precision=precision,
                                                           ctx=ctx, pso_split="median")
            assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]
            assert np.abs(pso.cpu().numpy().reshape(rpso.shape) - rpso).max() <= 1e-7


def test_eigh_batched_maximum_size(lib, ctx):
    """The largest matrix the solver takes, n = 4096 (mixed: FP32 tridiagonal solve,
    lowest eight vectors refined; a gap of 0.5 opened above them): refined eigenvalues,
    residual and orthonormality within the mixed bounds, every eigenvalue within FP32
    accuracy of LAPACK; n = 4097 is refused on the host before any device work."""
    torch = _torch()
    n, n_vec = 4096, 8
    A = I.random_hermitian_batch([n], seed=53)[0]
    lam, V = np.linalg.eigh(A)
    A = A - 0.5 * (V[:, :n_vec] @ V[:, :n_vec].conj().T)
    A = 0.5 * (A + A.conj().T)
    ev, vec = lib.eigh_batched(torch.tensor(A.reshape(-1), device="cuda"), [n], n_vec,
                               precision="mixed", ctx=ctx)
    ev, vec = ev.cpu().numpy(), vec.cpu().numpy().reshape(n, n_vec)
    ref = lam.copy()      # the shift moves the lowest n_vec eigenvalues by -0.5 exactly
    ref[:n_vec] -= 0.5
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(ev[:n_vec] - ref[:n_vec]).max() <= 1e-10 * scale
    assert np.abs(A @ vec - vec * ev[:n_vec]).max() <= 1e-9 * scale
    assert np.abs(vec.conj().T @ vec - np.eye(n_vec)).max() <= 1e-10
    assert np.abs(ev[n_vec:] - ref[n_vec:]).max() <= 1e-5 * scale
    big = torch.zeros(4097 * 4097, dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.BWError) as e:
        lib.eigh_batched(big, [4097], 1, ctx=ctx)
    assert e.value.status == "EINVAL"


def test_unit_circle_double_float_against_fp64(lib, ctx):
    """The double-float e^{2 pi i m / N}, e^{i pi t} and arg z of the four-band loop
    kernel (Taylor series after quarter-turn reduction; refined float arctangent)
    against the FP64 sincospi / atan2 of the CUDA math library: within a few units of
    the double-float resolution 2^-48 = 3.6e-15."""
    e_ratio, e_cis, e_phase = ctx.selftest_unit_circle()
    assert e_ratio <= 1e-14, e_ratio
    assert e_cis <= 1.5e-14, e_cis
    assert e_phase <= 2e-14, e_phase


def test_plan_cache_follows_in_place_edits(lib, ctx):
    """A context reuses the plan of an unchanged hopping list, and plans again when the
    caller edits the same arrays in place: halving every intra-cell amplitude of the
    BBH model (still Hermitian) changes the loop, and the result follows the oracle
    of the edited model."""
    torch = _torch()
    model = I.bbh(0.5, 0.5)
    plane = P(12, 12)
    a, _ = lib.wilson_loop(model, plane, 2, ctx=ctx)
    b, _ = lib.wilson_loop(model, plane, 2, ctx=ctx)
    assert torch.equal(a, b)
    intra = np.all(np.asarray(model.R) == 0, axis=1)
    assert intra.any()
    model.t[intra] *= 0.5
    c, _ = lib.wilson_loop(model, plane, 2, ctx=ctx)
    ref, _ = oracle.wilson_loop(model, plane, 2)
    assert circ_err_rows(c.cpu().numpy(), ref) <= TOL["fp64"]
    assert not torch.equal(a, c)
