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
