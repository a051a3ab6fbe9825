"""Helpers shared by the tests: build-on-demand of libtddft and header parsing."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_library():
    from paper_1005_5340_gb300 import build, tddft
    srcs = build.sources() + [os.path.join(ROOT, "include", "tddft.h"),
                              os.path.join(build.CSRC, "internal.h")]
    if (not os.path.exists(tddft.LIB_PATH)
            or os.path.getmtime(tddft.LIB_PATH) < max(os.path.getmtime(s) for s in srcs)):
        build.build()
    return tddft.load_library()


def header_functions():
    """Names of the functions declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(tddft_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))
