"""CPU checks of the C ABI library: it loads, exports every symbol include/hbi.h declares,
its host-side tree and lattice partition equal the oracle's bit for bit, and argument
validation rejects bad input before any device work.  No GPU compute calls."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import meshes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hbi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hbi_status|void|const char \*)\s*(hbi_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = hbi.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for s in names:
        assert hasattr(L, s), s
    assert sorted(hbi.SYMBOLS) == names


def test_status_strings():
    assert hbi.status_string(0) == "HBI_OK"
    assert hbi.status_string(-4) == "HBI_ERR_ACA_FAIL"
    assert hbi.status_string(-9) == "HBI_ERR_SINGULAR"


@pytest.mark.parametrize("mk,op,leaf,L", [
    (lambda: meshes.scaled_thrust_mesh(24, 12, seed=5), 3, 16, 0),
    (lambda: meshes.scaled_thrust_mesh(24, 12, seed=5), 0, 16, 2),
    (lambda: meshes.planar_vertical_rect(40, 13, 250.0), 1, 32, 3),
    (lambda: meshes.planar_vertical_rect(7, 3, 250.0), 0, 4, 5),     # lattice deeper than the tree
    (lambda: meshes.planar_vertical_rect(1, 1, 250.0), 0, 32, 0),    # a single element
])
def test_host_plan_equals_oracle_tree_and_partition(mk, op, leaf, L):
    m = mk()
    perm, starts, blocks = hbi.hbi_plan(m.verts, op, leaf, L)
    H = oracle.HMatrix(m, op, 1e-4, leaf, L, 32e9, 0.25)
    ex = H.export()
    assert np.array_equal(perm, ex["perm"])
    ob = ex["blocks"]
    assert np.array_equal(blocks[:, :4], ob[:, :4])
    leaves = sorted(int(c[0]) for c in ex["clusters"] if c[3] < 0)
    assert np.array_equal(starts, np.array(leaves + [m.n_elem]))


def test_invalid_arguments_rejected_on_host():
    m = meshes.planar_vertical_rect(4, 4, 250.0)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_plan(m.verts, 0, 0, 0)                      # leaf size 0
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_plan(m.verts, 7, 8, 0)                      # unknown operator
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_build(m.verts[:0], 32e9, 0.25, 0, 1e-4, 8, 0, "fp32")   # no elements
    # overlapping / incomplete tiling is rejected before any device allocation
    n = m.n_elem
    blocks = np.array([[0, n, 0, n, 0, 0], [0, n, 0, n, 0, 0]], dtype=np.int64)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_build_from_factors(m.verts, 32e9, 0.25, 0, "fp64", np.arange(n), blocks,
                                   np.array([0, 0]), np.zeros(n * n), np.array([0, n]))
    blocks = np.array([[0, n, 0, n - 1, 0, 0]], dtype=np.int64)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_build_from_factors(m.verts, 32e9, 0.25, 0, "fp64", np.arange(n), blocks,
                                   np.array([0]), np.zeros(n * n), np.array([0, n]))
    bad_perm = np.zeros(n, dtype=np.int32)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_build_from_factors(m.verts, 32e9, 0.25, 0, "fp64", bad_perm,
                                   np.array([[0, n, 0, n, 0, 0]]), np.array([0]), np.zeros(n * n),
                                   np.array([0, n]))


def test_event_list_from_step_records():
    rec = np.array([[0, 1, 1e-9, 0], [1, 1, 2e-3, 0], [2, 1, 5e-1, 0], [3, 1, 1e-4, 0],
                    [4, 1, 1e-9, 0], [5, 1, 3e-3, 1], [6, 1, 1e-5, 0]], dtype=float)
    assert hbi.events(rec) == [(1.0, 0.5), (5.0, 3e-3)]
    assert hbi.events(rec, vth=1.0) == []
