"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every symbol include/mehdg.h declares (no compute calls without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mehdg.h")).read()
    return sorted(set(re.findall(r"\b(mehdg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2507_22195_gb300 import build, mehdg
    lib = ctypes.CDLL(build.build())
    names = declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(mehdg.EXPORTED)


def test_binding_loads_and_fills_defaults():
    from paper_2507_22195_gb300 import mehdg
    p = mehdg.mehdg_default_params()
    assert p.gamma == 1.4 and p.refine_tol == 1e-12 and p.prec == mehdg.MEHDG_MIXED_TF32


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2507_22195_gb300 import mehdg
    import pytest
    with pytest.raises(mehdg.MehdgError, match="ECUDA"):
        mehdg.mehdg_create(mehdg.mehdg_default_params())
