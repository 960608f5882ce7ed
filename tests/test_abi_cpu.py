"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, and rejects bad arguments before any
CUDA call."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2404_17744_gb300 import build, thc
    if not os.path.exists(thc.LIB_PATH):
        build.build()
    return thc.load_library()


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[\w\s\*]+?\b(thc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "thc_sigma_init" in names and "thc_sigma_eval" in names and "thc_energy" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_init_rejects_bad_arguments_without_gpu(lib):
    from paper_2404_17744_gb300 import thc
    X = np.zeros((2, 3))
    V = np.zeros((3, 3))
    tau = np.array([1.0, 2.0])
    bad = [
        dict(n_ao=0, n_thc=3, n_tau=2, beta=3.0),
        dict(n_ao=2, n_thc=0, n_tau=2, beta=3.0),
        dict(n_ao=2, n_thc=3, n_tau=0, beta=3.0),
        dict(n_ao=2, n_thc=3, n_tau=2, beta=-1.0),
        dict(n_ao=2, n_thc=70000, n_tau=2, beta=3.0),
    ]
    for kw in bad:
        with pytest.raises(thc.ThcError) as ei:
            thc.thc_sigma_init(kw["n_ao"], kw["n_thc"], kw["n_tau"], kw["beta"], X, V, tau)
        assert ei.value.code == thc.THC_EINVAL
        assert thc.thc_last_error(None) != ""
    with pytest.raises(thc.ThcError):
        thc.thc_sigma_init(2, 3, 2, 3.0, X, V, tau, precision=7)
    with pytest.raises(thc.ThcError):
        thc.thc_sigma_init(2, 3, 2, 3.0, X, V, tau, terms=0)
    with pytest.raises(thc.ThcError):
        thc.thc_sigma_init(2, 3, 2, 3.0, None, V, tau)


def test_null_context_calls_are_rejected(lib):
    from paper_2404_17744_gb300 import thc
    with pytest.raises(thc.ThcError):
        thc.thc_sigma_eval(None, None, None, None)
    assert thc.thc_launch_count(None) == 0
    thc.thc_destroy(None)


def test_tf32_is_reported_as_not_built(lib):
    from paper_2404_17744_gb300 import thc
    X = np.zeros((2, 3))
    V = np.zeros((3, 3))
    with pytest.raises(thc.ThcError) as ei:
        thc.thc_sigma_init(2, 3, 2, 3.0, X, V, np.array([1.0, 2.0]), precision=thc.THC_TF32)
    assert ei.value.code == thc.THC_ENOTSUP
    assert "TF32" in thc.thc_last_error(None)


def test_wait_selftest_rejects_bad_limits_without_gpu(lib):
    from paper_2404_17744_gb300 import thc
    for bad in (0, 999, 10 ** 10):
        with pytest.raises(thc.ThcError) as ei:
            thc.thc_wait_selftest(bad)
        assert ei.value.code == thc.THC_EINVAL


def test_autotune_cache_round_trip_and_validation(lib, tmp_path):
    """The tile-table cache is host logic: a load keeps only the choices the kernels can
    take (tile widths 128 / 256; fused B C/D cluster shapes 11, 12, 22), stops at a line
    it cannot parse, and a save writes back what the table holds; a missing file is
    THC_EINVAL."""
    from paper_2404_17744_gb300 import thc
    bcd = thc.THC_KCLASS_SOX_BCD
    src = tmp_path / "tiles.txt"
    src.write_text(
        f"3 1000 1000 200 4 256\n"        # a contraction class, BN 256: kept
        f"3 1000 1000 200 8 128\n"        # BN 128: kept
        f"3 1000 1000 200 16 64\n"        # BN 64: no such tile, dropped
        f"{bcd} 1000 1000 200 0 12\n"     # 1 x 2 cluster: kept
        f"{bcd} 1000 1000 200 512 22\n"   # 2 x 2 cluster: kept
        f"{bcd} 1000 1000 200 256 13\n"   # 1 x 3: not a shape of the kernel, dropped
        f"{bcd} 1000 1000 200 768 128\n"  # a tile width for the cluster class, dropped
        "garbage line\n"
        f"3 1000 1000 200 32 256\n")      # after the unparsable line: not read
    before = thc.thc_autotune_entries()
    thc.thc_autotune_load(src)
    assert thc.thc_autotune_entries() == before + 4
    out = tmp_path / "saved.txt"
    thc.thc_autotune_save(out)
    saved = {tuple(int(x) for x in line.split()) for line in out.read_text().splitlines()}
    for row in ((3, 1000, 1000, 200, 4, 256), (3, 1000, 1000, 200, 8, 128), (bcd, 1000, 1000, 200, 0, 12),
                (bcd, 1000, 1000, 200, 512, 22)):
        assert row in saved
    for key in ((3, 1000, 1000, 200, 16), (bcd, 1000, 1000, 200, 256), (bcd, 1000, 1000, 200, 768),
                (3, 1000, 1000, 200, 32)):
        assert not any(r[:5] == key for r in saved)
    with pytest.raises(thc.ThcError) as ei:
        thc.thc_autotune_load(tmp_path / "missing.txt")
    assert ei.value.code == thc.THC_EINVAL
