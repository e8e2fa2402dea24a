"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rsf.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:rsf_status|void|const char\*|int64_t)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rsf_build", "rsf_logdet", "rsf_solve", "gp_loglik_and_score", "rsf_peel_trace"):
        assert must in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_loads_and_exports_every_symbol():
    from paper_1603_08057_gb300 import build, binding
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == declared_functions()
    # options defaults are readable without a GPU
    o = binding.RsfOpts()
    lib.rsf_opts_default(ctypes.byref(o))
    assert (o.n_occ, o.n_prox, o.n_rings, o.oversample, o.q0, o.seed) == (64, 256, 8, 10, 64, 0)
    assert (o.r_near, o.r_in, o.r_out) == (1.0, 1.0, 2.0)
    assert (o.precision, o.trace_form, o.refine, o.probes) == (binding.PREC_MIXED, binding.TRACE_SYM, -1, 64)
    # sizes of the C structs (x86-64 and aarch64 alike): the field lists match rsf.h
    assert ctypes.sizeof(o) == 72 and ctypes.sizeof(binding.RsfInfo) == 80
    assert ctypes.sizeof(binding.RsfKernel) == 24 and binding.RsfKernel.anisotropic.offset == 16
    # the hook setter rejects a half-set pair without touching the GPU
    alloc = binding._ALLOC_FN(lambda n, s, c: None)
    assert binding.lib().rsf_set_allocator(alloc, binding._FREE_FN(), None) == 1
    assert binding.lib().rsf_set_allocator(binding._ALLOC_FN(), binding._FREE_FN(), None) == 0


def test_batched_offsets_are_validated():
    from paper_1603_08057_gb300 import binding
    assert list(binding._offsets([0, 3, 10], 10)) == [0, 3, 10]
    for bad in ([1, 10], [0, 9], [0]):
        with pytest.raises(ValueError):
            binding._offsets(bad, 10)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1603_08057_gb300 import binding
    monkeypatch.setattr(binding, "LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        binding.lib()


def test_argument_errors_of_the_later_entry_points_need_no_gpu():
    # NULL or out-of-range arguments are rejected with RSF_EINVAL (1) before
    # any device work, and rsf_last_error names the problem
    import ctypes
    from paper_1603_08057_gb300 import binding
    L = binding.lib()
    k = binding.RsfKernel(binding.MATERN32, 0.0, 0)
    th = (ctypes.c_double * 3)(0.1, 1.0, 0.01)
    ll = ctypes.c_double()
    assert L.gp_profile_loglik_and_score(None, None, 10, ctypes.byref(k), th, 1e-9, 1e-6, None, None,
                                         ctypes.byref(ll), None, None) == 1
    mean = (ctypes.c_double * 4)()
    assert L.gp_conditional(None, 10, None, None, 4, ctypes.byref(k), th, 1e-9, None, None, 0, mean, None, 0,
                            None) == 1
    n, nb = ctypes.c_int64(), ctypes.c_int()
    assert L.rsf_tree_export(None, ctypes.byref(n), ctypes.byref(nb), None, None) == 1
    assert L.rsf_selftest_gemm(9, 1, 1, 1, 0, 0, 1.0, None, 1, None, 1, 0.0, None, 1, None) == 1
    L.rsf_last_error.restype = ctypes.c_char_p
    assert b"engine" in L.rsf_last_error()
