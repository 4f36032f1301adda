"""The C-ABI library builds, loads and exports every symbol include/ddlra.h declares
(no GPU needed: nothing is computed)."""
import os
import re

import pytest

from paper_2602_14854_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "ddlra.h")).read()
    return sorted(set(re.findall(r"\b(dd_\w+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert header_symbols() == sorted(binding.EXPORTS)


def test_library_exports_every_symbol():
    path = build.build()
    lib = binding.load(path)
    for name in header_symbols():
        assert hasattr(lib, name), name
    assert lib.dd_set_allocator(None) == 0          # a successful call clears the message
    assert lib.dd_last_error() == b""


def test_create_rejects_bad_arguments():
    """Argument checks run before any device call."""
    import ctypes as C
    lib = binding.load(build.build())
    h = C.c_void_p()
    st = lib.dd_dlra_create(None, None, None, None, None, None, None, C.byref(h))
    assert st == 1 and b"null" in lib.dd_last_error()


def test_selftest_wait_rejects_bad_arguments():
    """The wait self-test checks its arguments before any device call."""
    import ctypes as C
    lib = binding.load(build.build())
    out = C.c_int(5)
    assert lib.dd_selftest_wait(C.c_uint(0), C.byref(out)) == 1
    assert lib.dd_selftest_wait(C.c_uint((1 << 21) + 1), C.byref(out)) == 1
    assert lib.dd_selftest_wait(C.c_uint(16), None) == 1
    assert b"polls" in lib.dd_last_error() or b"null" in lib.dd_last_error()


def test_allocator_setter_checks_its_callbacks():
    """dd_set_allocator refuses an allocator with one callback missing, accepts a complete
    one and NULL (both host-only: no device memory is touched), and dd_dlra_last_error
    reports the thread's last message whatever the handle."""
    import ctypes as C
    lib = binding.load(build.build())
    half = binding.Allocator(binding._ALLOC_FN(lambda n, ctx: None), binding._RELEASE_FN(), None)
    assert lib.dd_set_allocator(C.byref(half)) == 1
    assert b"both" in lib.dd_last_error()
    assert lib.dd_dlra_last_error(None) == lib.dd_last_error()
    binding.set_allocator(lambda n: 0, lambda p: None)
    assert lib.dd_last_error() == b""
    binding.set_allocator()
    assert lib.dd_set_allocator(None) == 0
    with pytest.raises(ValueError):
        binding.set_allocator(lambda n: 0)


def test_instance_flux_rejects_bad_arguments():
    """dd_dlra_scalar_flux_instance checks its handle and output before any device call."""
    import ctypes as C
    lib = binding.load(build.build())
    out = (C.c_double * 4)()
    assert lib.dd_dlra_scalar_flux_instance(None, 0, out, 0) == 1
    assert lib.dd_dlra_scalar_flux_instance(None, 0, None, 0) == 1


@pytest.mark.parametrize("block", [0, 0x1008])
def test_allocator_failure_paths(block):
    """A caller's allocator that returns NULL, or a block off the 256-byte alignment, makes the
    create fail with DD_ERR_CUDA before anything runs on the device; a misaligned block goes
    straight back through release, and nothing else is released."""
    from paper_2602_14854_gb300 import inputs
    calls = {"alloc": [], "release": []}
    binding.set_allocator(lambda n: calls["alloc"].append(n) or block,
                          lambda p: calls["release"].append(p))
    try:
        wl = inputs.random_small_problem(3, nx=8, ny=8, tiles_x=2, tiles_y=2, n_mu=2, n_phi=8,
                                         rank=2, r_aug_max=4, nsteps=1)
        with pytest.raises(binding.DDError) as e:
            binding.Solver(wl)
    finally:
        binding.set_allocator()
    assert e.value.status == 2
    assert len(calls["alloc"]) == 1 and calls["alloc"][0] > 0
    assert calls["release"] == ([block] if block else [])


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the built CUDA library the binding raises; there is no fallback path."""
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(OSError, match="not built"):
        binding.load(str(tmp_path / "libddlra.so"))
