"""The product path has no fallback: without the compiled library the binding
raises instead of computing anything, and no module of the package (nor the
seeded input generators it shares with the tests) imports the CPU oracle."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_raises_import_error():
    code = ("import paper_1712_00403_gb300 as fd\n"
            "try:\n"
            "    fd.load_library('/nonexistent/libfdst.so')\n"
            "except ImportError as e:\n"
            "    print('raised', 'libfdst.so' in str(e))\n"
            "else:\n"
            "    print('loaded')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "raised True"


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_product_modules_never_import_the_oracle():
    files = []
    for d in ("paper_1712_00403_gb300", "synth"):
        for base, _, names in os.walk(os.path.join(ROOT, d)):
            files += [os.path.join(base, n) for n in names if n.endswith(".py")]
    assert files
    for f in files:
        for mod in _imports(f):
            assert not mod.split(".")[0] == "oracle", f"{f} imports {mod}"
