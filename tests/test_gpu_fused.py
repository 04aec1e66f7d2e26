"""The fused mixed-precision transforms (one cluster launch per step pass for
z synthesis, theta product and z analysis, the half-physical fields kept in
distributed shared memory) against the three-kernel path they replace: the
same block FFTs on the same sequences, the same product and epilogue
arithmetic, so the results must be identical bit for bit -- for single
evaluations, whole steps (with frame rotation, a body force and the CFL
maximum), both cluster sizes and batched ensembles.  The three-kernel FP32
path itself is checked against the oracle in test_gpu_parity/test_gpu_mixed."""
import numpy as np
import pytest

from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


SHAPES = [(12, 16, 16, 1), (10, 24, 24, 1), (14, 32, 24, 2), (9, 16, 32, 1), (20, 32, 32, 1), (48, 32, 24, 2)]


@pytest.mark.parametrize("N,K,M,m_p", SHAPES)
def test_fused_nonlinear_term_equals_three_kernels(opf, N, K, M, m_p):
    alpha, Re = 1.25, 1000.0
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 55)
    out = []
    for fused in (0, 1, 2, 4, 8):  # off, chosen cluster size, forced sizes
        h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
        opf.opf_set_option(h, "precision", 1)
        opf.opf_set_option(h, "fused", fused)
        got = opf.opf_get_option(h, "fused")  # the cluster size in use (0: three kernels)
        assert got == fused if fused != 1 else got in (2, 4, 8)
        out.append(opf.opf_nonlinear(h, U0))
    for o in out[1:]:
        assert np.array_equal(out[0], o)
    want = Oracle(Params(N, K, M, m_p, alpha, Re, 0.01)).nonlinear(U0)
    assert np.abs(out[1] - want).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("opts", [{}, {"rot_z": 0.7}, {"rot_x": 0.3, "rot_y": -0.2}, {"cfl": 0.5}, {"forcing": 1}])
def test_fused_steps_equal_three_kernels(opf, opts):
    N, K, M, m_p, alpha, Re, dt = 16, 16, 16, 1, 1.25, 1500.0, 0.005
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 56)
    F = inputs.seeded_state(N, K, M, m_p, alpha, 0.01, 57, laminar=False)
    res = []
    for fused in (0, 1):
        h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
        opf.opf_set_option(h, "precision", 1)
        opf.opf_set_option(h, "fused", fused)
        for k, v in opts.items():
            if k == "forcing":
                opf.opf_set_forcing(h, F)
            else:
                opf.opf_set_option(h, k, v)
        opf.opf_set_state(h, U0)
        opf.opf_step(h, 4)
        res.append((opf.opf_get_state(h), opf.opf_get_dt(h),
                    opf.opf_get_option(h, "cfl_number") if "cfl" in opts else 0.0))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]


def test_fused_batched_ensemble_equals_three_kernels(opf):
    """A batched group (cluster size 4) and a second shape, mixed precision."""
    shapes = [(24, 16, 16)] * 20 + [(16, 24, 24)] * 3
    n = len(shapes)
    Re = [1500.0 + 30.0 * i for i in range(n)]
    N, K, M = zip(*shapes)
    outs = []
    for fused in (0, 1):
        e = opf.opf_ens_create(N, K, M, [1] * n, [1.25] * n, Re, [0.005] * n)
        opf.opf_ens_set_option(e, "precision", 1)
        opf.opf_ens_set_option(e, "fused", fused)
        for i, (Ni, Ki, Mi) in enumerate(shapes):
            opf.opf_ens_set_state(e, i, inputs.seeded_state(Ni, Ki, Mi, 1, 1.25, 0.05, 900 + i))
        opf.opf_ens_step(e, 3)
        outs.append([opf.opf_ens_get_state(e, i) for i in range(n)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
