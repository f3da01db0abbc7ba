"""CPU tests of the C-ABI library: it loads, exports every symbol the header declares,
and its host-side FP64 tables agree with the oracle's (integers exactly)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2105_01028_gb300 as T
from paper_2105_01028_gb300 import _lib
from oracle.healpix import ring_directions
from oracle.phase import phase_matrix as oracle_phase
from oracle.geometry import RayLattice
from oracle.cones import cone_fractions

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "trinity.h")


def header_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(trinity_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = T.lib()
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding lacks " + name


def test_no_gpu_is_an_error_not_a_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = _lib.GridDesc(4, 4, 4, 1.0, 1, 0.5, 1.4, 0, 0, 1e-6, 10)
    h = ctypes.c_void_p()
    rc = T.lib().trinity_create_grid(ctypes.byref(d), None, ctypes.byref(h))
    assert rc < 0 and not h.value


def test_footprint_and_invalid_descriptions():
    d = _lib.GridDesc(96, 96, 64, 1.0, 4, 0.5, 1.4, 0, 1, 1e-6, 2000)
    fb = T.lib().trinity_footprint_bytes(ctypes.byref(d))
    nv, na = 96 * 96 * 64, 192
    assert fb >= 11 * na * nv * 4
    for bad in [_lib.GridDesc(1, 4, 4, 1.0, 2, 0.5, 1.4, 0, 0, 1e-6, 10),
                _lib.GridDesc(4, 4, 4, 1.0, 3, 0.5, 1.4, 0, 0, 1e-6, 10),
                _lib.GridDesc(4, 4, 4, 1.0, 2, 0.5, 1.4, 0, 0, 0.0, 10),
                _lib.GridDesc(4, 4, 4, -1.0, 2, 0.5, 1.4, 0, 0, 1e-6, 10)]:
        assert T.lib().trinity_footprint_bytes(ctypes.byref(bad)) == 0


def test_adjoint_footprint():
    # 64^3, 192 directions, 800 steps, checkpoints every 50: 17 checkpoints of 8 levels,
    # a 54-level store of I and S, 13 more levels for the reverse sweep (adjoint ring of I
    # and S, Qbar, two warm-start levels)
    d = _lib.GridDesc(64, 64, 64, 1.0, 4, 0.5, 1.4, 0, 0, 1e-6, 2000)
    fb = T.lib().trinity_adjoint_footprint_bytes(ctypes.byref(d), 800, 50, 8, 202)
    lvl = 64 ** 3 * 192 * 4
    assert (17 * 8 + 54 * 2 + 13) * lvl <= fb <= (17 * 8 + 54 * 2 + 13) * lvl + 64 * 2 ** 20
    assert T.lib().trinity_adjoint_footprint_bytes(ctypes.byref(d), 0, 50, 8, 202) == 0
    assert T.lib().trinity_adjoint_footprint_bytes(ctypes.byref(d), 800, 0, 8, 202) == 0


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_healpix_matches_oracle(nside):
    np.testing.assert_allclose(T.healpix_dirs(nside), ring_directions(nside), atol=2e-15, rtol=0)


@pytest.mark.parametrize("nside,g", [(1, 0.9), (2, 0.9), (4, 0.9), (2, 0.0), (4, 0.5)])
def test_phase_matrix_matches_oracle(nside, g):
    P, geff = T.phase_matrix(nside, g)
    Po, geo = oracle_phase(nside, g, return_geff=True)
    assert abs(geff - geo) < 1e-12
    np.testing.assert_allclose(P, Po, atol=1e-13, rtol=0)


@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("shape_xyz", [(16, 16, 16), (96, 96, 64), (128, 128, 96), (5, 7, 3)])
@pytest.mark.parametrize("periodic", [False, True])
def test_lattice_matches_oracle_exactly(nside, shape_xyz, periodic):
    nx, ny, nz = shape_xyz
    dom_sgn, ds, offs = T.lattice_tables(nside, nx, ny, nz, 1.0, periodic)
    lat = RayLattice(ring_directions(nside), (nz, ny, nx), 1.0, periodic)
    np.testing.assert_array_equal(dom_sgn[:, 0], lat.dom)
    np.testing.assert_array_equal(dom_sgn[:, 1], lat.sgn)
    np.testing.assert_allclose(ds, lat.ds, rtol=2e-16, atol=0)
    for d in range(len(ds)):
        n_dom = (nx, ny, nz)[lat.dom[d]]
        np.testing.assert_array_equal(offs[d, :, :n_dom], lat.offsets[d])


@pytest.mark.parametrize("nside", [2, 4])
@pytest.mark.parametrize("face", range(6))
@pytest.mark.parametrize("inward", [True, False])
def test_cone_weights_match_oracle_exactly(nside, face, inward):
    a = T.cone_weights(nside, face, 15.0, inward)
    np.testing.assert_array_equal(a, cone_fractions(ring_directions(nside), face, 15.0, inward))


@pytest.mark.parametrize("nside,scale,dims", [(2, 0.25, (32, 32, 12)), (4, 0.25, (24, 28, 10))])
def test_interface_table_matches_oracle(nside, scale, dims):
    """The library's FP64 interface split (voxel, j, d, weight) equals the oracle's."""
    import workloads as W
    from oracle.solver import Model
    nx, ny, nz = dims
    p = W.config_hetero(steps=1, precision="fp32", nx=nx, ny=ny, nz=nz, nside=nside, scale=scale)
    m = Model(p)
    ref = {}
    for v, cols in m.interfaces.items():
        for j, outs in cols.items():
            for d, wgt in outs:
                ref[(v, j, d)] = ref.get((v, j, d), 0.0) + wgt
    vox, jj, dd, ww = T.interface_entries(nside, p["nidx"])
    got = {}
    for v, j, d, wgt in zip(vox, jj, dd, ww):
        got[(int(v), int(j), int(d))] = got.get((int(v), int(j), int(d)), 0.0) + float(wgt)
    ref = {k: x for k, x in ref.items() if x != 0.0}
    got = {k: x for k, x in got.items() if x != 0.0}
    assert len(ref) > 0
    assert set(got) == set(ref)
    for k in ref:
        assert abs(got[k] - ref[k]) <= 1e-13


@pytest.mark.parametrize("fine,coarse", [(16, 4), (8, 4), (4, 2), (2, 1), (16, 2), (4, 4)])
def test_parent_map_matches_oracle_exactly(fine, coarse):
    from oracle.healpix import parent_map as oracle_parent
    assert np.array_equal(T.parent_map(fine, coarse), oracle_parent(fine, coarse))
