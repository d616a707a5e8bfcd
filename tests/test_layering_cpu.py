"""Layering rules checked on the sources (CPU only): the product path never uses
the oracle, and the oracle shares no code with the CUDA path."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    for dirpath, _, names in os.walk(os.path.join(ROOT, sub)):
        if "__pycache__" in dirpath or "_lib" in dirpath:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(dirpath, n)


def test_package_never_imports_the_oracle():
    for path in _files("paper_1411_2860_gb300", (".py", ".cu", ".hpp", ".cuh", ".h")):
        text = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), path
        assert "oracle.c" not in text and "liboracle" not in text, path


def test_oracle_shares_no_code_with_the_cuda_path():
    for path in _files("oracle", (".py", ".c", ".h")):
        text = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+paper_1411_2860_gb300\b", text, re.M), path
        assert "libprojgemm" not in text, path
        assert not re.search(r'#include\s+"[^"]*(common\.hpp|tc\.cuh|projgemm\.h)"', text), path


def test_bench_uses_the_oracle_only_for_the_cpu_baseline_and_reference_arm():
    text = open(os.path.join(ROOT, "bench.py")).read()
    # every use of the oracle module sits in one of the two CPU-timing functions
    funcs = re.split(r"^def ", text, flags=re.M)
    for body in funcs[1:]:
        name = body.split("(", 1)[0]
        if re.search(r"\boracle\.", body) or re.search(r"^\s*import oracle\b", body, re.M):
            assert name in ("_oracle_sample", "cpu_baseline", "run_reference"), name
