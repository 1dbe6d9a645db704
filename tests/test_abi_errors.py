"""Argument validation of the C ABI (include/foeed.h), on the host.

Every entry point checks sizes, parameters and pointers before it touches the
GPU and returns FOEED_ERR_ARG with a thread-local message. These calls pass
NULL or dummy addresses that a failed check rejects first; the module is skipped
where a GPU is present, so that no dummy address can ever reach a device.
"""
import ctypes as C
import math

import pytest

torch = pytest.importorskip("torch")
if torch.cuda.is_available():
    pytest.skip("host-only argument checks (a GPU is present)", allow_module_level=True)

import paper_2006_10406_gb300 as fg  # noqa: E402

ERR_ARG = 1
F32, F64, F32_F64U = fg.F32, fg.F64, fg.F32_F64U
FAKE = C.c_void_p(0x10000)          # 256-byte aligned dummy address (never dereferenced)
FAKE2 = C.c_void_p(0x20000)
MISALIGNED = C.c_void_p(0x10008)


def params(**kw):
    p = fg._Params(0.1, 1.0, 0.0, 4, 2, 0.0, 0, 0, 0, 8)
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def last_error():
    return fg.lib().foeed_last_error().decode()


def inpaint(w=16, h=16, pitch=16, dtype=F32, p=None, f=FAKE, mask=FAKE, u=FAKE, ws=FAKE, nbytes=1 << 30,
            entry="foeed_inpaint"):
    prm = C.byref(p) if p is not None else None
    return getattr(fg.lib(), entry)(f, mask, u, w, h, pitch, dtype, prm, ws, nbytes, None, None)


@pytest.mark.parametrize("entry", ["foeed_inpaint", "eed_inpaint"])
@pytest.mark.parametrize("kw, needle", [
    (dict(w=0), "size"),
    (dict(h=-3), "size"),
    (dict(pitch=15), "pitch"),
    (dict(dtype=7), "dtype"),
    (dict(p=None), "params"),
    (dict(p=params(lam=0.0)), "lambda"),
    (dict(p=params(lam=math.nan)), "lambda"),
    (dict(p=params(sigma=2.5)), "sigma"),
    (dict(p=params(sigma=-1.0)), "sigma"),
    (dict(p=params(tau=math.inf)), "tau"),
    (dict(p=params(diffusivity=5)), "diffusivity"),
    (dict(p=params(mu3_mode=3)), "mu3_mode"),
    (dict(p=params(cycle_len=0)), "cycle_len"),
    (dict(p=params(max_cycles=0)), "max_cycles"),
    (dict(p=params(tol=-1e-3)), "tol"),
    (dict(p=params(init_mode=2)), "init_mode"),
    (dict(p=params(), f=None), "NULL"),
    (dict(p=params(), mask=None), "NULL"),
    (dict(p=params(), ws=None), "NULL"),
    (dict(p=params(), ws=MISALIGNED), "aligned"),
    (dict(p=params(), nbytes=64), "too small"),
])
def test_solver_rejects_bad_arguments(entry, kw, needle):
    kw.setdefault("p", params())
    assert inpaint(entry=entry, **kw) == ERR_ARG
    assert needle in last_error()


def test_workspace_size_of_a_bad_image_is_zero():
    assert fg.lib().foeed_workspace_bytes(0, 16, F32) == 0
    assert fg.lib().foeed_workspace_bytes(16, 16, 9) == 0


@pytest.mark.parametrize("entry", ["foeed_step", "eed_step"])
def test_step_rejects_bad_arguments(entry):
    fn = getattr(fg.lib(), entry)
    p = params()
    assert fn(FAKE, FAKE, FAKE2, None, 0, 8, 8, F32, 1.0, C.byref(p), None) == ERR_ARG
    assert fn(FAKE, None, FAKE2, None, 8, 8, 8, F32, 1.0, C.byref(p), None) == ERR_ARG
    assert "NULL" in last_error()
    assert fn(FAKE, FAKE, FAKE, None, 8, 8, 8, F32, 1.0, C.byref(p), None) == ERR_ARG
    assert "alias" in last_error()
    assert fn(FAKE, FAKE, FAKE2, None, 8, 8, 8, F32, math.inf, C.byref(p), None) == ERR_ARG
    assert "alpha" in last_error()
    bad = params(sigma=3.0)
    assert fn(FAKE, FAKE, FAKE2, None, 8, 8, 8, F32, 1.0, C.byref(bad), None) == ERR_ARG


def test_batch_rejects_bad_arguments():
    L = fg.lib()
    inst = (fg._Instance * 2)(fg._Instance(FAKE.value, FAKE.value, FAKE2.value, 32, 32, 32, 0.1),
                              fg._Instance(FAKE.value, FAKE.value, FAKE2.value, 16, 8, 16, 0.1))
    p = params()
    assert L.foeed_inpaint_batch(inst, 0, F32, C.byref(p), FAKE, 1 << 30, None, None) == ERR_ARG
    assert L.foeed_inpaint_batch(inst, 2, F64, C.byref(p), FAKE, 1 << 30, None, None) == ERR_ARG
    assert "FOEED_F32" in last_error()
    one = params(cycle_len=1)
    assert L.eed_inpaint_batch(inst, 2, F32, C.byref(one), FAKE, 1 << 30, None, None) == ERR_ARG
    assert "cycle_len" in last_error()
    inst[1].lambda_ = -1.0
    assert L.foeed_inpaint_batch(inst, 2, F32, C.byref(p), FAKE, 1 << 30, None, None) == ERR_ARG
    assert "lambda" in last_error()
    inst[1].lambda_ = 0.1
    assert L.foeed_inpaint_batch(inst, 2, F32, C.byref(p), FAKE, 64, None, None) == ERR_ARG
    assert "too small" in last_error()
    inst[0].w = 0
    assert L.foeed_batch_workspace_bytes(inst, 2, F32) == 0


def test_adjoint_rejects_bad_arguments():
    L = fg.lib()

    def vjp(dtype=F32, p=None, K=16, f=FAKE):
        p = p or params()
        return L.foeed_inpaint_vjp(f, FAKE, FAKE, FAKE2, None, 16, 16, 16, dtype, C.byref(p), K, FAKE, 1 << 34,
                                   None)
    assert vjp(dtype=F32_F64U) == ERR_ARG
    assert vjp(p=params(tol=1e-6)) == ERR_ARG and "tol" in last_error()
    assert vjp(p=params(init_mode=1)) == ERR_ARG and "init_mode" in last_error()
    assert vjp(p=params(diffusivity=1)) == ERR_ARG and "Charbonnier" in last_error()
    assert vjp(K=0) == ERR_ARG and "checkpoint" in last_error()
    assert vjp(f=None) == ERR_ARG and "NULL" in last_error()
    assert L.foeed_vjp_workspace_bytes(16, 16, F32, C.byref(params()), 0) == 0


def test_tensor_field_rejects_bad_arguments():
    L = fg.lib()
    assert L.foeed_apply_tensor_field(FAKE, FAKE, FAKE2, 8, 8, 8, F32_F64U, None) == ERR_ARG
    assert L.foeed_apply_tensor_field(FAKE, None, FAKE2, 8, 8, 8, F32, None) == ERR_ARG
    assert "NULL" in last_error()
    assert L.foeed_apply_tensor_field(FAKE, FAKE, FAKE, 8, 8, 8, F32, None) == ERR_ARG
    assert "alias" in last_error()
    assert L.foeed_apply_tensor_field(FAKE, FAKE, FAKE2, 8, 8, 4, F64, None) == ERR_ARG


def test_static_entry_rejects_images_beyond_its_scratch():
    fn = fg.lib().foeed_inpaint_static
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_long, C.c_int,
                   C.POINTER(fg._Params), C.c_void_p, C.POINTER(fg._Report)]
    fn.restype = C.c_int
    p = params()
    side = 4096
    assert fn(FAKE, FAKE, FAKE2, side, side, side, F32, C.byref(p), None, None) == ERR_ARG
    assert "static" in last_error()


def test_messages_are_per_call():
    assert inpaint(w=0) == ERR_ARG
    first = last_error()
    assert inpaint(p=params(lam=-1.0)) == ERR_ARG
    assert last_error() != first and "lambda" in last_error()


def test_tile_policy_arguments_are_checked_on_the_host():
    """foeed_set_tile_policy accepts AUTO (0), 8, 16, 32 and 64 only; foeed_last_tile_plan
    rejects NULL. Neither touches the GPU."""
    import ctypes as C

    import paper_2006_10406_gb300 as fg
    L = fg.lib()
    try:
        for bad in (1, 4, 24, 128, -1):
            assert L.foeed_set_tile_policy(bad) == 1
            assert b"tile policy" in L.foeed_last_error()
        for good in (8, 16, 32, 64, 0):
            assert L.foeed_set_tile_policy(good) == 0
        assert L.foeed_last_tile_plan(None) == 1
        plan = fg._TilePlan()
        assert L.foeed_last_tile_plan(C.byref(plan)) == 0
        with pytest.raises(KeyError):
            fg.set_tile_policy("h128")
    finally:
        L.foeed_set_tile_policy(0)
