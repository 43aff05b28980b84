"""The oracle and the CUDA path share no code (no GPU needed): no module of the product
package imports the oracle, the oracle imports nothing of the product package (it reads
network descriptions through duck typing only), and the product's CUDA sources include
nothing from the oracle.  The only committed places that may run the oracle outside the
tests are the smoke check and the bench's CPU baseline."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                out.add(node.module.split(".")[0])
    return out


def _py_files(folder):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_product_package_does_not_import_the_oracle():
    for path in _py_files("paper_2512_09502_gb300"):
        assert "oracle" not in _imports(path), path


def test_oracle_does_not_import_the_product():
    for path in _py_files("oracle"):
        assert "paper_2512_09502_gb300" not in _imports(path), path
        assert "torch" not in _imports(path), path


def test_cuda_sources_do_not_reach_the_oracle():
    csrc = os.path.join(ROOT, "paper_2512_09502_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f


def test_oracle_runs_only_from_the_allowed_places():
    for path in [os.path.join(ROOT, "__graft_entry__.py"), os.path.join(ROOT, "bench.py")]:
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.FunctionDef):
                inner = {n.module.split(".")[0] for n in ast.walk(node)
                         if isinstance(n, ast.ImportFrom) and n.level == 0 and n.module}
                if "oracle" in inner:
                    assert node.name in ("smoke", "cpu_sample"), (path, node.name)
        top = {n.module.split(".")[0] for n in tree.body if isinstance(n, ast.ImportFrom) and n.module}
        top |= {a.name.split(".")[0] for n in tree.body if isinstance(n, ast.Import) for a in n.names}
        assert "oracle" not in top, path
