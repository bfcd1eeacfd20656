"""The oracle and the CUDA library share no code (CPU).

Neither side imports or includes the other; the seeded input generators are
the only module both use, and the package loads without the oracle."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_18996_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if not x.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_reaches_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*oracle)", re.M)
    for p in sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        assert not pat.search(open(p).read()), p


def test_oracle_never_reaches_the_package():
    pat = re.compile(r"^\s*(import\s+paper_2310_18996_gb300|from\s+paper_2310_18996_gb300\b|"
                     r"#\s*include\s*[<\"][^>\"]*(mockskewer|mk_[a-z_]+)\.)", re.M)
    for p in sources(ORACLE, (".py", ".c", ".h")):
        assert not pat.search(open(p).read()), p


def test_package_imports_without_loading_the_oracle():
    code = ("import sys; import paper_2310_18996_gb300 as mk; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle loaded'")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)
