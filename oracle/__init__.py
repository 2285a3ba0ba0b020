"""Plain, slow FP64 CPU oracle of the Wilson-loop method (Tyner, "BerryEasy", arXiv 2312.13051).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check and the
benchmark's CPU-baseline leg may import this package.  The library never calls
it: there is no CPU fallback.  It shares no code with the CUDA path; both take
their inputs from the seeded generators in ``paper_2312_13051_gb300.inputs``,
which this package does not import either (models are duck-typed: any object
with ``n, R, i, j, t``; planes: any object with ``N, N_t, origin, loop_dir,
trans_dir``).

Every function is pinned in ``tests/test_oracle_pins.py`` against values the
paper states or the mathematics fixes.  No function here is "parity unpinned".
"""
from .wilson import (  # noqa: F401
    OracleError, STATUS, bloch_hamiltonian, plane_points, occupied_states,
    overlap, polar_factor, wilson_matrix, eigenphases, wilson_loop,
    projected_spin_sector, spin_resolved_wilson_loop, nested_wilson_loop,
    wannier_sector, wannier_states, wannier_row, nested_phases,
    translation_blocks, bloch_hamiltonian_grouped,
    cyclic_wilson_matrix, winding, circular_match_error, eigh_batched,
    plaquette_flux, plaquette_corners, plaquette_matrix,
    wcc_fractions, largest_gap_midpoint, z2_largest_gap,
)
