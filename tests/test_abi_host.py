"""CPU-only checks of the C ABI library: it loads, exports every symbol that
include/opf.h declares, validates arguments, and its host-side setup (mesh,
stencils, quadrature) agrees with the independently written oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.opf_oracle import fd_matrices, mesh, quadrature_weights
from paper_1705_03838_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def declared_functions():
    text = open(os.path.join(ROOT, "include", "opf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(opf_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(opf):
    names = declared_functions()
    assert len(names) >= 18
    L = ctypes.CDLL(opf.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_setup_query_rejects_bad_arguments(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(8, 4, 4, 1, 1.25, 100.0, 0.01, "r")  # N < 9
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(16, 4, 4, 1, 1.25, 100.0, 0.01, "nonsense")


@pytest.mark.parametrize("N", [9, 16, 33])
def test_host_stencils_match_oracle(opf, N):
    r = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "r")
    assert np.abs(r - mesh(N)).max() < 1e-15
    wq = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "wq")
    assert np.abs(wq - quadrature_weights(mesh(N))).max() < 1e-15
    for what, idx in (("d1", 0), ("d2", 1)):
        w = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, what).reshape(2, N, 9)
        for par, sgn in ((0, 1), (1, -1)):
            ref = fd_matrices(mesh(N), sgn)[idx]
            A = np.zeros((N, N))
            for n in range(N):
                lo = min(max(n - 4, 0), N - 9)
                A[n, lo:lo + 9] = w[par, n]
            assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("N", [12, 24])
def test_host_setup_on_a_user_mesh_matches_oracle(opf, N):
    """A user radial mesh (opf_setup_query_mesh / opf_create_mesh): points,
    quadrature and both stencils against the oracle on the same points."""
    rm = inputs.stretched_mesh(N)
    r = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "r", r=rm)
    assert np.array_equal(r, rm)
    wq = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "wq", r=rm)
    assert np.abs(wq - quadrature_weights(rm)).max() < 1e-15
    for what, idx in (("d1", 0), ("d2", 1)):
        w = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, what, r=rm).reshape(2, N, 9)
        for par, sgn in ((0, 1), (1, -1)):
            ref = fd_matrices(rm, sgn)[idx]
            A = np.zeros((N, N))
            for n in range(N):
                lo = min(max(n - 4, 0), N - 9)
                A[n, lo:lo + 9] = w[par, n]
            assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def test_user_mesh_is_validated(opf):
    rm = inputs.stretched_mesh(12)
    for bad in (rm[::-1], np.concatenate([rm[:-1], [0.99]]), np.concatenate([[0.0], rm[1:]]),
                np.concatenate([rm[:5], rm[4:5], rm[6:]])):
        with pytest.raises(opf.OpfError):
            opf.opf_setup_query(12, 4, 4, 1, 1.25, 100.0, 0.01, "r", r=bad)


def test_flux_response_is_positive_and_vanishes_at_wall(opf):
    G = opf.opf_setup_query(24, 4, 4, 1, 1.25, 2000.0, 0.01, "G")
    assert G[-1] == 0.0 and np.all(G[:-1] > 0)


def test_setup_rejects_unfactorable_sizes(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(4, 4, 4, 1, 1.25, 100.0, 0.01, "r")
