"""The allocation-free solver entry point, foeed_inpaint_static.

Some callers cannot call cudaMalloc (code running inside another framework's
memory arena, plug-ins barred from the device heap, latency-critical paths
where an allocation may block or fail). foeed_inpaint_static serves them: its
scratch is a fixed static device array, so the caller passes only the input
and output images. These tests call it through the C ABI and check that it
returns what the workspace-based foeed_inpaint returns, twice in a row (the
shared array keeps the previous call's contents), and that it rejects images
whose scratch would not fit. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_10406_gb300 as fg  # noqa: E402

DEV = torch.device("cuda", 0)


def _static_call(fd, md, ud, params, dtype_code):
    L = fg.lib()
    fn = L.foeed_inpaint_static
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_long, C.c_int,
                   C.POINTER(fg._Params), C.c_void_p, C.POINTER(fg._Report)]
    fn.restype = C.c_int
    h, w = fd.shape
    rep = fg._Report()
    st = fn(C.c_void_p(fd.data_ptr()), C.c_void_p(md.data_ptr()), C.c_void_p(ud.data_ptr()), w, h, fd.stride(0),
            dtype_code, C.byref(params), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(rep))
    return st, rep


@pytest.mark.parametrize("dtype,tdt", [(fg.F32, torch.float32), (fg.F64, torch.float64)])
@pytest.mark.parametrize("n", [12, 1])
def test_static_entry_matches_workspace_entry_twice(dtype, tdt, n):
    """Two calls in a row (the shared array keeps the first call's contents) on two
    image sizes, with a cycle length of 12 and of 1 (the single-step cycle copies
    its result back into the cycle buffer): the same kernels run in the same order
    as in foeed_inpaint, so the results are bitwise equal."""
    for call, (h, w, seed_inst) in enumerate([(96, 130, 0), (61, 47, 1)]):
        img, mask, p = synth.workload(2, h=h, w=w, instance=seed_inst)
        fd = torch.from_numpy(img).to(DEV, tdt)
        md = torch.from_numpy(mask).to(DEV)
        ref, rrep = fg.foeed_inpaint(fd, md, 0.03, 1.0, n, 6)
        ud = torch.full_like(fd, float("nan"))
        params = fg._params(0.03, 1.0, 0.0, n, 6)
        st, rep = _static_call(fd, md, ud, params, dtype)
        assert st == 0, fg.lib().foeed_last_error()
        assert rep.cycles_run == rrep.cycles_run == 6
        assert torch.equal(ud, ref), (call, float((ud - ref).abs().max().item()))
        k = md.bool()
        assert torch.equal(ud[k], fd[k])


def test_static_entry_allocates_no_device_memory():
    """After the first call on the device (which loads the library's module and with
    it the static array), further calls leave the device's free memory unchanged."""
    img, mask, p = synth.workload(2, h=200, w=300)
    fd = torch.from_numpy(img).to(DEV, torch.float32)
    md = torch.from_numpy(mask).to(DEV)
    ud = torch.empty_like(fd)
    params = fg._params(0.03, 1.0, 0.0, 10, 3)
    st, _ = _static_call(fd, md, ud, params, fg.F32)
    assert st == 0, fg.lib().foeed_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st, _ = _static_call(fd, md, ud, params, fg.F32)
    assert st == 0, fg.lib().foeed_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_entry_rejects_images_beyond_the_scratch():
    L = fg.lib()
    L.foeed_static_scratch_bytes.restype = C.c_size_t
    limit = L.foeed_static_scratch_bytes()
    h = w = 2400
    assert fg.workspace_bytes(w, h, fg.F32) > limit
    fd = torch.zeros((h, w), dtype=torch.float32, device=DEV)
    md = torch.zeros((h, w), dtype=torch.uint8, device=DEV)
    ud = torch.zeros_like(fd)
    st, _ = _static_call(fd, md, ud, fg._params(0.03, 1.0, 0.0, 4, 1), fg.F32)
    assert st == 1
    assert b"static" in fg.lib().foeed_last_error()
