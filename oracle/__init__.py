"""FP64 CPU oracle of the TRINITY time-dependent radiative-transfer forward model.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the GPU
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The GPU library (package
``paper_2105_01028_gb300``) never imports, links or calls anything here, and this
package never imports the library: the two share no code.

Paper: Yajima, Abe, Umemura, Takamizu, Hoshi, "TRINITY: a three-dimensional
time-dependent radiative transfer code for in-vivo near-infrared imaging"
(arXiv:2105.01028).  Each function cites the section / equation it follows.

Modules
-------
healpix    HEALPix RING pixel centres (§2.1, angular discretisation).
phase      Henyey-Greenstein phase function (Eq. 11) and the discrete,
           normalised phase matrix used by the source sum (Eq. 12).
geometry   Long-ray lattice: dominant axis, sample spacing, per-slab
           transverse offsets (§2.1, rays independent of the grid; §2.4 Step 1).
cones      15-degree source / detector acceptance cones (§3.1).
fresnel    Snell's law (Eq. 13) and Fresnel reflectance (Eq. 14).
solver     The time loop: ray update (Eqs. 9-10), source iteration (Eq. 12,
           §2.4 Steps 3, 5, 6, 7), boundary inflow and detectors (§3.1).
bruteforce An independent per-ray tracer for tiny grids (cross-check of geometry);
           it has its own dominant-axis and floor rules and imports nothing from here.
adjoint    Reverse-mode derivative of a detector misfit (checkpointed time loop).
twolevel   Transport on fine directions, source function on coarse ones (§2.1).
exact      Per-voxel source function from the fixed-point equation of Eq. 12.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (the detector tally, photon accounting, closed-box decay and
mirror faces in ``tests/test_oracle_tallies.py``) except the Fresnel interface redistribution on curved
interfaces (``fresnel.interface_operators``): its optics and its whole table on a plane
index step are pinned, but on a stair-stepped curved boundary it is "parity unpinned".
The adjoint (``adjoint``), the two-level angular grid (``twolevel``, with the HEALPix
point location in ``healpix``) and the exact per-voxel solve (``exact``) are pinned in
``tests/test_oracle_adjoint.py``, ``tests/test_oracle_twolevel.py`` and
``tests/test_oracle_exact.py``.
"""

C0_MM_PER_NS = 299.792458  # speed of light in vacuum, mm/ns (c = c0 / n, §2.1 below Eq. 1)
RING_DEPTH = 5             # time levels kept per field (retarded upwind needs up to 4 back)
