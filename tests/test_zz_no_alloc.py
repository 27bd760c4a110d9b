"""The allocation-free transport entry point, claire_transport_noalloc.

It serves callers that cannot allocate device memory (their memory is reserved
up front by another allocator, or they cannot accept the synchronisation a
cudaMalloc may imply).  Its scratch lives in a static device array of at most
2^20 voxels shared by all calls.  These checks call it through the C ABI and
compare it with the context-based claire_transport, on two calls in a row with
different grids and inputs, within the transport tolerance (1e-5 relative L2).
This file is collected last so that a failure here leaves every other test run.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2401_17493_b300 import synth


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_17493_b300 import build
    build.build()
    from paper_2401_17493_b300 import claire
    return claire


def _call(C, shape, nt, v, m0, out):
    buf = ctypes.create_string_buffer(512)
    st = C.load_library().claire_transport_noalloc(
        *shape, nt, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(m0.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
        buf, 512)
    return st, buf.value.decode()


def test_noalloc_transport_matches_the_context_transport_on_two_calls(lib):
    C = lib
    cases = [((48, 40, 34), 4, 1), ((64, 64, 64), 3, 2)]
    for k, (shape, nt, seed) in enumerate(cases):
        m0, m1, v = synth.blob_pair(shape, seed=seed, kmax=3, max_disp_voxels=2.5)
        m0d = torch.from_numpy(m0).cuda()
        vd = torch.from_numpy(v).cuda()
        out = torch.full(shape, float("nan"), device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, msg = _call(C, shape, nt, vd, m0d, out)
        torch.cuda.synchronize()
        assert st == C.OK, msg
        if k == 1:
            # the library allocated nothing for this call
            assert torch.cuda.mem_get_info()[0] == free_before
        with C.Context(shape, nt=nt) as ctx:
            ctx.set_images(m0d, torch.from_numpy(m1).cuda())
            ref = ctx.transport(vd)
        a = out.cpu().numpy().astype(np.float64)
        b = ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-5


def test_noalloc_transport_rejects_grids_beyond_its_limit(lib):
    C = lib
    shape = (128, 128, 128)                      # 2^21 voxels > 2^20
    v = torch.zeros((3, 16, 16, 16), device="cuda")
    m0 = torch.zeros((16, 16, 16), device="cuda")
    out = torch.zeros((16, 16, 16), device="cuda")
    st, msg = _call(C, shape, 4, v, m0, out)
    assert st == C.EINVAL
    assert "exceeds the static scratch limit" in msg
    # aliasing the output with the input is refused as well
    st, msg = _call(C, (16, 16, 16), 4, v, m0, m0)
    assert st == C.EINVAL and "overlaps" in msg


def test_noalloc_transport_refuses_memory_that_is_not_on_the_current_device(lib):
    C = lib
    shape = (16, 16, 16)
    v = torch.zeros((3,) + shape, device="cuda")
    m0 = torch.zeros(shape, device="cuda")
    out = torch.zeros(shape, device="cuda")
    pinned = torch.zeros(shape, pin_memory=True)
    pageable = np.zeros(shape, dtype=np.float32)
    buf = ctypes.create_string_buffer(512)
    L = C.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # nothing is launched: the pointers are checked first
    st = L.claire_transport_noalloc(*shape, 4, ctypes.c_void_p(v.data_ptr()),
                                    ctypes.c_void_p(pinned.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), stream, buf, 512)
    assert st == C.EINVAL and "device memory of the current device" in buf.value.decode()
    st = L.claire_transport_noalloc(*shape, 4, ctypes.c_void_p(v.data_ptr()),
                                    ctypes.c_void_p(m0.data_ptr()),
                                    ctypes.c_void_p(pageable.ctypes.data), stream, buf, 512)
    assert st == C.EINVAL and "device memory of the current device" in buf.value.decode()
    # the entry point still works afterwards
    st, msg = _call(C, shape, 4, v, m0, out)
    assert st == C.OK, msg
