"""The library build that runs one process per GPU on several GPUs holds no
cluster-multicast form.

The one-GPU build lets the reduced GEMMs run on clusters of two CTAs that share
operand tiles through ``.multicast::cluster`` TMA loads and MMA commits.  A
process that runs one of several GPUs (``bench.py`` under torchrun) loads the
"solo" variant instead, compiled from the same sources with ``-DPJ_CTA_PAIRS=0``.
These tests preprocess every translation unit of that variant exactly as the
build compiles it and search the code that comes from this repository (the
package sources and ``include/``) for any multicast form.  No GPU is needed.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1411_2860_gb300 import _build  # noqa: E402

OWN = (os.path.join(ROOT, "paper_1411_2860_gb300"), os.path.join(ROOT, "include"))
LINE_MARK = re.compile(r'^#\s*(?:line\s+)?\d+\s+"([^"]+)"')


def _own_code(src, variant):
    """Lines of the preprocessed translation unit that come from this repository's files."""
    cmd = [_build.nvcc(), *_build.compile_flags(variant), "-E", src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    cur, out = src, []
    for line in r.stdout.splitlines():
        m = LINE_MARK.match(line)
        if m:
            cur = os.path.realpath(m.group(1))
            continue
        if any(cur.startswith(o) for o in OWN):
            out.append(line)
    return "\n".join(out)


def _all_units(variant):
    srcs = _build.sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        return dict(zip(srcs, ex.map(lambda s: _own_code(s, variant), srcs)))


@pytest.fixture(scope="module")
def solo_units():
    return _all_units("solo")


def test_solo_variant_compiles_every_source_without_pairs():
    flags = _build.compile_flags("solo")
    assert "-DPJ_CTA_PAIRS=0" in flags
    assert _build.lib_path("solo") != _build.lib_path("pairs")
    assert len(_build.sources()) >= 10


def test_no_multicast_in_the_solo_build(solo_units):
    for src, code in solo_units.items():
        hits = [ln for ln in code.splitlines() if "multicast" in ln]
        assert not hits, f"{os.path.basename(src)} (solo build) still holds: {hits[:3]}"


def test_the_pairs_build_is_where_multicast_lives():
    # the check above is not vacuous: the one-GPU build of the GEMM holds both forms
    src = os.path.join(_build.CSRC, "gemm_tc.cu")
    code = _own_code(src, "pairs")
    assert "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster" in code
    assert "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster" in code


def test_only_the_pair_header_names_multicast():
    # every multicast form sits in csrc/tc_pair.cuh, which the solo build never includes
    for name in os.listdir(_build.CSRC):
        path = os.path.join(_build.CSRC, name)
        with open(path) as f:
            text = f.read()
        forms = re.findall(r"\.multicast::cluster", text)
        if name == "tc_pair.cuh":
            assert len(forms) >= 2
        else:
            assert not forms, f"{name} names a multicast form outside tc_pair.cuh"


def test_bench_ranks_of_a_multi_gpu_run_load_the_solo_build():
    import bench
    assert bench.library_variant(1) == "pairs"
    for world in (2, 4, 8):
        assert bench.library_variant(world) == "solo"


def test_select_library_refuses_a_second_variant_once_loaded(monkeypatch):
    import paper_1411_2860_gb300 as pj
    monkeypatch.setattr(pj, "_variant", "pairs")
    monkeypatch.setattr(pj, "_lib", None)        # as if nothing were loaded yet
    pj.select_library("solo")
    assert pj.library_variant() == "solo"
    assert pj.lib_path().endswith("libprojgemm_solo.so")
    with pytest.raises(ValueError):
        pj.select_library("multicast")
    monkeypatch.setattr(pj, "_lib", object())   # as if a library were loaded
    with pytest.raises(RuntimeError):
        pj.select_library("pairs")
