"""Helpers for tests that call the C ABI (build on demand, seeded systems, oracle references)."""
import functools
import os
import re

import numpy as np

from tests.conftest import ROOT


@functools.lru_cache(maxsize=1)
def lib():
    from paper_1005_0088_gb300.build import build
    build()
    import paper_1005_0088_gb300 as nd
    nd.load()
    return nd


def header_functions():
    """Function names declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(ndsi_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))
