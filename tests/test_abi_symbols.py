"""The C ABI library loads and exports every entry point include/dino.h declares (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dino.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(dino_\w+)\s*\(", text, re.M)))


def _library():
    import paper_2403_08220_gb300 as dino
    from paper_2403_08220_gb300 import build as b
    if not os.path.exists(dino.LIB_PATH):
        try:
            b.build()
        except RuntimeError as e:  # no toolkit
            pytest.skip(str(e))
    return dino


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["dino_init", "dino_destroy", "dino_load_surrogate", "dino_chains_create",
                 "dino_chains_step", "dino_chains_read", "dino_surrogate_eval"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    dino = _library()
    out = subprocess.run(["nm", "-D", "--defined-only", dino.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (dino_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_symbol_and_loads_without_gpu():
    dino = _library()
    L = dino.lib()
    for n in _declared():
        assert hasattr(L, n)
        assert n in dino.exported_symbols()
    assert dino.dino_version() >= 100


def test_no_gpu_means_an_error_not_a_fallback():
    """Without a CUDA device the library refuses to create a context (ECUDA):
    there is no host fallback for any step of the path."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2403_08220_gb300 as dino
    with pytest.raises(dino.DinoError) as ei:
        dino.dino_init(0)
    assert ei.value.code == dino.DINO_ECUDA
