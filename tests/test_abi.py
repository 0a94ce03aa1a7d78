"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mm.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:mm_status|void|const char \*|int64_t)\s*\**\s*(mm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1707_05333_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ("mm_tessellate", "mm_gradients", "mm_flux_step", "mm_drift", "mm_timestep",
                     "mm_mesh_velocity", "mm_step", "mm_create", "mm_destroy", "mm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1707_05333_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_functions()


def test_default_config_and_struct_layout(lib):
    from paper_1707_05333_gb300 import binding
    binding._lib = None
    cfg = binding.default_config()
    assert cfg.gamma == pytest.approx(5.0 / 3.0) and cfg.cfl == 0.3 and cfg.limiter == 1
    # 9 doubles, 8 ints, bin_scale, mach_th, entropy and integrator, clip_sort and the padding to 8 bytes
    assert ctypes.sizeof(binding.Config) == 9 * 8 + 8 * 4 + 8 + 8 + 2 * 4 + 4 + 4
    assert cfg.clip_sort == 0 and cfg.clip_warps == 2 and cfg.cand_cap == 64
    assert ctypes.sizeof(binding.MeshStruct) == 4 * 8 + 3 * 8 + 8 + 2 * 8 + 10 * 8


def test_binding_refuses_host_tensors():
    import torch
    from paper_1707_05333_gb300 import binding
    with pytest.raises(ValueError):
        binding._ptr(torch.zeros(3, dtype=torch.float64))
