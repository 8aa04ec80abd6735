"""Helpers shared by the tests: header parsing and library build."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    """Names of every function declared in include/*.h."""
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(INCLUDE, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", txt, flags=re.M):
            head = txt[m.start():m.end()]
            if head.lstrip().startswith(("typedef", "#")):
                continue
            names.append(m.group(1))
    return names


def built_lib():
    from paper_2005_07132_gb300 import build
    return build.build()
