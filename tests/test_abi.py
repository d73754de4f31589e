"""The C-ABI library loads on a machine without a GPU and exports every entry point
declared in include/links.h (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

from paper_2208_14567_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "links.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"LINKS_API\s+[\w\s\*]*?\b(links_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    return ctypes.CDLL(B.build())


def test_header_declares_the_boundary():
    names = declared()
    for n in ("links_create", "links_plan_build", "links_plan_build_host", "links_simulate", "links_strerror"):
        assert n in names
    assert len(names) >= 18


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared() if not hasattr(so, n)]
    assert not missing


def test_strerror_is_host_only(so):
    so.links_strerror.restype = ctypes.c_char_p
    assert so.links_strerror(0) == b"LINKS_OK"
    assert so.links_strerror(6) == b"LINKS_ETIMEDOUT"
    assert so.links_strerror(99) == b"LINKS_UNKNOWN"


def test_binding_names_match_the_header():
    from paper_2208_14567_gb300 import links
    for n in declared():
        if n in ("links_strerror",):
            continue
        assert hasattr(links, n), n


def test_null_arguments_are_rejected_without_a_gpu(so):
    so.links_plan_free.argtypes = [ctypes.c_void_p]
    assert so.links_plan_free(None) == 1  # LINKS_EINVAL
    so.links_destroy.argtypes = [ctypes.c_void_p]
    assert so.links_destroy(None) == 1


def test_topology_source_compiles():
    """The generated source of a topology-specialised screen compiles for sm_103a (host
    side only: code generation and nvcc, no device)."""
    import shutil

    import numpy as np
    import subprocess
    import tempfile
    from paper_2208_14567_gb300 import inputs as I
    from paper_2208_14567_gb300 import links
    B.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    for n in (6, 12):
        b = I.paper_topologies(2, n, seed=n)
        src = links.links_topo_source(int(b.n_joints[0]), b.adj[0], b.jtype[0])
        assert "topo_screen" in src and src.count("fp32_dyad_core(") == int(n - 2 - (b.jtype[0] == 0).sum() + 1)
        with tempfile.TemporaryDirectory() as d:
            p = f"{d}/t.cu"
            open(p, "w").write(src)
            csrc = os.path.join(os.path.dirname(os.path.abspath(links.__file__)), "csrc")
            r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-I", csrc, "-c", p, "-o",
                                f"{d}/t.o"], capture_output=True, text=True)
            assert r.returncode == 0, r.stderr[-2000:]
    with pytest.raises(links.LinksError):
        links.links_topo_source(6, np.zeros((6, 6), np.uint8), np.array([0, 2, 1, 1, 1, 1], np.int8))


def test_embedded_headers_match_the_sources():
    """The run-time compiled screens include step.cuh and dw_core.cuh from text the build
    embeds in the library: after a build that text is the current source."""
    B.build()
    inc = open(os.path.join(B.OUT_DIR, "embedded_headers.inc")).read()
    for name in B.EMBEDDED:
        text = open(os.path.join(B.CSRC, name)).read()
        assert f'"{name}"' in inc and text in inc, name
