"""Batched ensembles: trajectories stepped together in shared launches must
equal the same trajectories stepped alone (identical arithmetic per
trajectory -> bit-for-bit), for uneven shapes and per-trajectory Re/dt."""
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


def run_single(opf, N, K, M, m_p, alpha, Re, dt, U0, n, precision):
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt)
    opf.opf_set_option(h, "precision", precision)
    # a lone small grid takes the split solve (equal to round-off, checked in
    # test_gpu_fullsize); the batched groups here are too large for it, and
    # the comparison is bit for bit, so both sides use the single-chain solve
    opf.opf_set_option(h, "spike", 0)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, n)
    return opf.opf_get_state(h), opf.opf_energy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_uneven_ensemble_equals_single_runs(opf, precision):
    specs = [  # (N, K, M, m_p, alpha, Re, dt)
        (16, 4, 4, 1, 1.25, 900.0, 0.01),
        (12, 3, 6, 2, 1.25, 1200.0, 0.01),
        (16, 4, 4, 1, 1.25, 1500.0, 0.005),
        (20, 5, 3, 1, 0.8, 700.0, 0.01),
        (16, 4, 4, 1, 1.25, 900.0, 0.01),
        (12, 3, 6, 2, 1.25, 2000.0, 0.02),
    ]
    cols = list(zip(*specs))
    e = opf.opf_ens_create(*cols)
    opf.opf_ens_set_option(e, "precision", precision)
    states = []
    for i, (N, K, M, m_p, alpha, Re, dt) in enumerate(specs):
        U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.05, 500 + i)
        states.append(U0)
        opf.opf_ens_set_state(e, i, U0)
    opf.opf_ens_step(e, 4)
    for i, sp in enumerate(specs):
        U, E = run_single(opf, *sp, states[i], 4, precision)
        assert np.array_equal(opf.opf_ens_get_state(e, i), U)
        assert np.array_equal(opf.opf_ens_energy(e, i), E)
        assert abs(opf.opf_ens_get_time(e, i) - 4 * sp[6]) < 1e-15


def test_shared_setup_batch_matches_oracle(opf):
    """A batch with one shared setup (equal Re and dt), checked per member
    against the oracle."""
    N, K, M, m_p, alpha, Re, dt = 16, 4, 4, 1, 1.25, 800.0, 0.01
    e = opf.opf_ens_create([N] * 3, [K] * 3, [M] * 3, [m_p] * 3, [alpha] * 3, [Re] * 3, [dt] * 3)
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt))
    U0s = [inputs.seeded_state(N, K, M, m_p, alpha, a, 900 + i) for i, a in enumerate((1e-3, 1e-2, 0.1))]
    for i, U0 in enumerate(U0s):
        opf.opf_ens_set_state(e, i, U0)
    opf.opf_ens_step(e, 3)
    for i, U0 in enumerate(U0s):
        ref = o.step(U0, 3)
        U = opf.opf_ens_get_state(e, i)
        assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-12


def test_ensemble_workload_shapes(opf):
    """The batched-ensemble workload's three resolutions (N=32/48/64,
    |k|<16/24/32, m<16/24/32), a few members each, mixed precision, against
    single runs of the same members."""
    shapes = [(32, 16, 16)] * 3 + [(48, 24, 24)] * 3 + [(64, 32, 32)] * 2
    Re = [1800.0 + 800.0 * u for u in inputs.uniforms(1705038383, len(shapes))]
    N, K, M = zip(*shapes)
    n = len(shapes)
    e = opf.opf_ens_create(N, K, M, [1] * n, [1.25] * n, Re, [0.01] * n)
    opf.opf_ens_set_option(e, "precision", 1)
    U0s = []
    for i, (Ni, Ki, Mi) in enumerate(shapes):
        U0 = inputs.seeded_state(Ni, Ki, Mi, 1, 1.25, 1e-2, 1705038383 + i)
        U0s.append(U0)
        opf.opf_ens_set_state(e, i, U0)
    opf.opf_ens_step(e, 2)
    for i in (0, 4, 7):
        Ni, Ki, Mi = shapes[i]
        U, _ = run_single(opf, Ni, Ki, Mi, 1, 1.25, Re[i], 0.01, U0s[i], 2, 1)
        assert np.array_equal(opf.opf_ens_get_state(e, i), U)


def test_ensemble_rejects_bad_input(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_ens_create([8], [4], [4], [1], [1.25], [100.0], [0.01])
    e = opf.opf_ens_create([12], [3], [3], [1], [1.25], [100.0], [0.01])
    with pytest.raises(opf.OpfError):
        opf.opf_ens_energy(e, 5)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_shapes_give_identical_results(opf, precision):
    """Launch shapes change only how work is split across blocks, never the
    arithmetic of a mode: the autotuned run equals the default one exactly."""
    w = inputs.WORKLOADS["medium"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    U0 = inputs.workload_state("medium")
    out = []
    for tune in (0, 1):
        h = opf.opf_create(*args)
        opf.opf_set_option(h, "precision", precision)
        opf.opf_set_option(h, "autotune", tune)
        opf.opf_set_state(h, U0)
        opf.opf_step(h, 3)
        out.append(opf.opf_get_state(h))
        if tune:
            assert opf.opf_get_option(h, "autotune") == 2
            assert opf.opf_get_option(h, "tile") in (4, 8, 16)
    assert np.array_equal(out[0], out[1])


def test_rotating_ensemble_equals_single_runs(opf):
    """Frame rotation on an ensemble (every trajectory, several shape groups)
    gives each trajectory exactly what a single handle with the same
    rotation gives."""
    specs = [(16, 4, 4, 2, 1.0, 140.0, 0.01), (16, 4, 4, 2, 1.0, 150.0, 0.01), (12, 3, 5, 2, 1.0, 130.0, 0.01)]
    cols = list(zip(*specs))
    e = opf.opf_ens_create(*cols)
    opf.opf_ens_set_option(e, "rot_z", 1.0)
    U0s = [inputs.seeded_state(N, K, M, m_p, a, 0.05, 300 + i) for i, (N, K, M, m_p, a, Re, dt) in enumerate(specs)]
    for i, U in enumerate(U0s):
        opf.opf_ens_set_state(e, i, U)
    opf.opf_ens_step(e, 20)
    for i, (N, K, M, m_p, a, Re, dt) in enumerate(specs):
        h = opf.opf_create(N, K, M, m_p, a, Re, dt)
        opf.opf_set_option(h, "rot_z", 1.0)
        opf.opf_set_option(h, "spike", 0)
        opf.opf_set_state(h, U0s[i])
        opf.opf_step(h, 20)
        assert np.array_equal(opf.opf_ens_get_state(e, i), opf.opf_get_state(h))
    h = opf.opf_create(*specs[0])
    opf.opf_set_state(h, U0s[0])
    opf.opf_step(h, 20)
    assert not np.array_equal(opf.opf_ens_get_state(e, 0), opf.opf_get_state(h))  # the rotation acts
    with pytest.raises(opf.OpfError):  # a transverse axis needs m_p = 1 in every group
        opf.opf_ens_set_option(e, "rot_x", 0.5)
