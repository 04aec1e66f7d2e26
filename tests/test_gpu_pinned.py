"""State transfers through pinned host buffers: the GPU reads (set_state)
and writes (get_state) pinned memory directly instead of copying through a
staging buffer.  The result must equal the copy path for pageable buffers
bit for bit, including the Hermitian projection of m = 0 and the rejection
of non-finite values with the previous state kept."""
import ctypes

import numpy as np
import pytest

from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def pinned_copy(U):
    t = torch.from_numpy(np.ascontiguousarray(U).view(np.float64).copy()).pin_memory()
    assert t.is_pinned()
    return t


def test_pinned_set_and_get_equal_the_copy_path(opf):
    N, K, M, m_p = 24, 5, 4, 1
    U = inputs.seeded_state(N, K, M, m_p, 1.25, 0.1, 17)
    U[:, 0] += 1e-3 * (1 + 1j)  # an m = 0 part that the projection must symmetrise
    a = opf.opf_create(N, K, M, m_p, 1.25, 1000.0, 0.01)
    b = opf.opf_create(N, K, M, m_p, 1.25, 1000.0, 0.01)
    opf.opf_set_state(a, U)  # pageable: copy path
    note = opf.lib().opf_last_error()
    assert b"not Hermitian" in note
    pin = pinned_copy(U)
    assert opf.lib().opf_set_state(b.ptr, ctypes.c_void_p(pin.data_ptr())) == 0  # pinned: read in place
    assert opf.lib().opf_last_error() == note  # the same asymmetry note
    ref = opf.opf_get_state(a)
    out = torch.empty_like(pin).pin_memory()
    assert opf.lib().opf_get_state(b.ptr, ctypes.c_void_p(out.data_ptr())) == 0  # pinned: written in place
    got = out.numpy().view(np.complex128).reshape(ref.shape)
    assert np.array_equal(got, ref)
    opf.opf_step(a, 3)
    opf.opf_step(b, 3)
    assert opf.lib().opf_get_state(b.ptr, ctypes.c_void_p(out.data_ptr())) == 0
    assert np.array_equal(out.numpy().view(np.complex128).reshape(ref.shape), opf.opf_get_state(a))


def test_pinned_non_finite_state_is_rejected(opf):
    N, K, M, m_p = 16, 4, 4, 1
    h = opf.opf_create(N, K, M, m_p, 1.25, 1000.0, 0.01)
    U = inputs.seeded_state(N, K, M, m_p, 1.25, 0.1, 18)
    opf.opf_set_state(h, U)
    before = opf.opf_get_state(h)
    bad = U.copy()
    bad[1, 2, 3, 4] = complex(np.nan, 0.0)
    pin = pinned_copy(bad)
    rc = opf.lib().opf_set_state(h.ptr, ctypes.c_void_p(pin.data_ptr()))
    assert rc == -3  # OPF_ENAN
    assert np.array_equal(opf.opf_get_state(h), before)
    bad[1, 2, 3, 4] = complex(0.0, np.inf)
    pin = pinned_copy(bad)
    assert opf.lib().opf_set_state(h.ptr, ctypes.c_void_p(pin.data_ptr())) == -3
    assert np.array_equal(opf.opf_get_state(h), before)


def test_pinned_ensemble_members(opf):
    shapes = [(16, 4, 4), (16, 4, 4), (12, 3, 5)]
    n = len(shapes)
    N, K, M = zip(*shapes)
    e = opf.opf_ens_create(N, K, M, [1] * n, [1.25] * n, [900.0, 1100.0, 1300.0], [0.01] * n)
    e2 = opf.opf_ens_create(N, K, M, [1] * n, [1.25] * n, [900.0, 1100.0, 1300.0], [0.01] * n)
    for i, (Ni, Ki, Mi) in enumerate(shapes):
        U = inputs.seeded_state(Ni, Ki, Mi, 1, 1.25, 0.05, 40 + i)
        opf.opf_ens_set_state(e, i, U)
        pin = pinned_copy(U)
        assert opf.lib().opf_ens_set_state(e2.ptr, i, ctypes.c_void_p(pin.data_ptr())) == 0
    opf.opf_ens_step(e, 2)
    opf.opf_ens_step(e2, 2)
    for i in range(n):
        assert np.array_equal(opf.opf_ens_get_state(e, i), opf.opf_ens_get_state(e2, i))
