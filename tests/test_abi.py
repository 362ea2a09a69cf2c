"""The C-ABI library builds, loads without a GPU, and exports every symbol
that include/clue.h declares (no compute calls here)."""
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2001_09761_gb300 import build, clue
    build.build()
    return clue.load()


def _declared():
    txt = (ROOT / "include" / "clue.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(clue_\w+)\s*\(", txt)))


def test_header_declares_the_binding_names():
    from paper_2001_09761_gb300 import clue
    assert _declared() == sorted(clue.ABI_SYMBOLS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_2001_09761_gb300 import clue
    assert clue.clue_strerror(0) == "ok"
    assert "invalid argument" in clue.clue_strerror(clue.CLUE_ERR_ARG)
    assert clue.clue_version().startswith("clue-gb300")
    o = clue.clue_default_opts()
    assert (o.x_min, o.x_max, o.max_layers, o.use_graphs) == (-250.0, 250.0, 128, 1)
    assert o.expand == clue.CLUE_EXPAND_CHASE and o.chi == 0 and o.max_scratch_bytes == 0
    # null arguments are rejected before any CUDA call
    assert lib.clue_run(None, None, None, None, None, 10, 2.0, 2.0, 2.0, 4.0, None, None) == \
        clue.CLUE_ERR_ARG
    assert lib.clue_sync(None) == clue.CLUE_ERR_ARG
    assert lib.clue_create(None, None) == clue.CLUE_ERR_ARG
    from paper_2001_09761_gb300 import serve
    serve._lib()
    so = serve.ClueServerOpts()
    lib.clue_server_default_opts(so)
    assert (so.n_regions, so.max_inflight, so.max_events_per_batch) == (3, 2, 512)
    assert lib.clue_server_create(None, None, None, 2.0, 2.0, 2.0, 4.0, None) == \
        clue.CLUE_ERR_ARG
    assert lib.clue_server_submit(None, None, None, None, None, 5, None, None, None) == \
        clue.CLUE_ERR_ARG


def test_library_has_no_oracle_dependency():
    """The product never loads or names the oracle."""
    for p in (ROOT / "paper_2001_09761_gb300").rglob("*"):
        if p.suffix in (".py", ".cu", ".cuh", ".h", ".cpp"):
            text = p.read_text()
            assert "import oracle" not in text and "oracle_clue" not in text, p
