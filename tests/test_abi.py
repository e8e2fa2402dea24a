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
    assert (o.n_occ, o.n_prox, o.oversample) == (64, 256, 10)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1603_08057_gb300 import binding
    monkeypatch.setattr(binding, "LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        binding.lib()
