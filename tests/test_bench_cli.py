"""The benchmark's command line (CPU): every documented option parses, and the
functions that run only on a GPU machine name no module they do not import."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def test_help_lists_the_documented_options():
    out = subprocess.run([sys.executable, BENCH, "--help"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT).stdout
    for opt in ["--gpus", "--steps", "--warmup", "--impl", "--storage", "--rescore", "--workload", "--psf",
                "--filter", "--stamps", "--cluster", "--swizzle", "--vorder", "--e2e-steps", "--topk",
                "--rp-steps", "--serve-sample"]:
        assert opt in out, opt


def test_functions_import_what_they_use():
    """Modules imported inside functions (torch, synth, oracle, ...) must be imported in every
    function that names them, at module level, or be passed in as an argument."""
    tree = ast.parse(open(BENCH).read())
    top = {a.asname or a.name.split(".")[0] for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))
           for a in n.names}
    local_mods = {"torch", "synth", "oracle", "kb", "replicas", "serve"}

    def check(fn, inherited):
        names = {n.id for n in ast.walk(fn) if isinstance(n, ast.Name)}
        imports = {a.asname or a.name.split(".")[0] for n in ast.walk(fn)
                   if isinstance(n, (ast.Import, ast.ImportFrom)) for a in n.names}
        params = {a.arg for a in fn.args.args + fn.args.kwonlyargs}   # a module passed in as an argument
        avail = inherited | imports | top | params
        for mod in local_mods & names:
            assert mod in avail, "%s uses %s without importing it" % (fn.name, mod)
        for sub in ast.walk(fn):
            if sub is not fn and isinstance(sub, ast.FunctionDef):
                check(sub, avail)

    for fn in tree.body:
        if isinstance(fn, ast.FunctionDef):
            check(fn, set())
