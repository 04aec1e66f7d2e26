"""The allocation-free nonlinear-term entry point against opf_nonlinear.

opf_nonlinear_noalloc serves callers that must not allocate device memory
when they call (all their device memory belongs to their own pool, or an
allocation could synchronise the device at the wrong moment): they pass
device input/output buffers and the library uses a fixed device array for
everything else.  This file sorts last so that a stop-at-first-failure run
has executed every other test before it; it also passes on its own.
"""
import numpy as np
import pytest

from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1705_03838_gb300 import build, opf

    build.build()
    opf.lib()
    return torch, opf


def _device(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.float64).copy()).cuda()


def test_noalloc_matches_opf_nonlinear_twice(env):
    torch, opf = env
    N, K, M, m_p, alpha, Re = 32, 16, 16, 1, 1.25, 2000.0
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
    for seed in (11, 12):  # two calls in a row on different states
        U = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, seed)
        want = opf.opf_nonlinear(h, U)
        d_in = _device(torch, U)
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        got = d_out.cpu().numpy().view(np.complex128).reshape(want.shape)
        # same tolerance as the nonlinear-term parity tests
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_noalloc_second_shape_and_rejections(env):
    torch, opf = env
    N, K, M, m_p, alpha, Re = 12, 3, 4, 2, 1.0, 500.0
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
    U = inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 5)
    want = opf.opf_nonlinear(h, U)
    d_in = _device(torch, U)
    d_out = torch.empty_like(d_in)
    opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr())
    got = d_out.cpu().numpy().view(np.complex128).reshape(want.shape)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the medium resolution needs ~30 MB, beyond the fixed 16 MiB array
    with pytest.raises(opf.OpfError) as e:
        opf.opf_nonlinear_noalloc(48, 32, 24, 2, 1.25, 2400.0, d_in.data_ptr(), d_out.data_ptr())
    assert e.value.code == opf.OPF_EINVAL and "scratch" in str(e.value)


def test_noalloc_calls_after_the_first_take_no_device_memory(env):
    """The contract itself: once the first call on the device has placed the
    array and the kernels there, further calls leave free device memory as
    it was (torch's caching allocator holds the buffers made beforehand)."""
    torch, opf = env
    N, K, M, m_p, alpha, Re = 16, 4, 6, 1, 1.25, 800.0
    d_in = _device(torch, inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 21))
    d_out = torch.empty_like(d_in)
    st = torch.cuda.current_stream().cuda_stream
    opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr(), st)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr(), st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_a_capturing_stream_without_breaking_the_capture(env):
    """The call synchronises its stream, so under capture it must return the
    documented error before launching anything, leaving the capture valid."""
    torch, opf = env
    N, K, M, m_p, alpha, Re = 12, 3, 4, 2, 1.0, 500.0
    d_in = _device(torch, inputs.seeded_state(N, K, M, m_p, alpha, 0.1, 6))
    d_out = torch.empty_like(d_in)
    opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr())  # first call
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        y = d_in * 2.0
        with pytest.raises(opf.OpfError) as e:
            opf.opf_nonlinear_noalloc(N, K, M, m_p, alpha, Re, d_in.data_ptr(), d_out.data_ptr(),
                                      side.cuda_stream)
    assert e.value.code == opf.OPF_EINVAL and "captur" in str(e.value)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, d_in * 2.0)
