"""The C-ABI library builds, loads and exports every entry point of
include/lbm.h; argument validation happens before any device work, so it is
checked here without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1609_09685_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_every_declared_entry_point_has_a_binding_of_the_same_name():
    missing = [n for n in sorted(_declared()) if not hasattr(lbm, n)]
    assert missing == []
    assert lbm.lbm_status_string(lbm.LBM_ERR_ARG) == "invalid argument"
    assert lbm.lbm_options_default().k_tol == pytest.approx(1e-5)


def test_binding_names_match_header():
    names = _declared()
    for n in ("lbm_qsgs", "lbm_create_domain", "lbm_create_domain_3d", "lbm_batch_create",
              "lbm_run_to_steady", "lbm_permeability", "lbm_step", "lbm_get_fields",
              "lbm_get_populations", "lbm_set_populations", "lbm_set_fields", "lbm_save",
              "lbm_load"):
        assert n in names
        assert hasattr(lbm, n)


def test_version_and_status_strings(lib):
    assert re.match(r"\d+\.\d+\.\d+", lbm.lbm_version())
    assert lib.lbm_status_string(lbm.LBM_ERR_ARG).decode() == "invalid argument"


def _create_status(mask, tau=0.8, drho=1e-3):
    o = lbm.make_options()
    h = C.c_void_p()
    m = np.ascontiguousarray(mask, np.uint8)
    return lbm.load().lbm_create_domain(m.ctypes.data, m.shape[1], m.shape[0], tau, drho,
                                        C.byref(o), C.byref(h)), h


@pytest.mark.parametrize("kw,shape", [
    (dict(tau=0.5), (8, 8)),          # tau must exceed 1/2
    (dict(tau=float("nan")), (8, 8)),
    (dict(drho=float("inf")), (8, 8)),
    (dict(), (8, 2)),                 # nx < 3
])
def test_create_rejects_bad_arguments(lib, kw, shape):
    st, h = _create_status(np.zeros(shape), **kw)
    assert st == lbm.LBM_ERR_ARG
    assert h.value is None
    assert lib.lbm_last_error(None).decode()


def test_create_rejects_non_binary_mask(lib):
    m = np.zeros((6, 9), np.uint8)
    m[2, 3] = 7
    st, _ = _create_status(m)
    assert st == lbm.LBM_ERR_ARG
    assert "0 (fluid) or 1 (solid)" in lib.lbm_last_error(None).decode()


def test_create_rejects_bad_in_place_pairs_option(lib):
    o = lbm.make_options()
    o.in_place_pairs = 2
    h = C.c_void_p()
    m = np.zeros((6, 9), np.uint8)
    assert lib.lbm_create_domain(m.ctypes.data, 9, 6, 0.8, 1e-3, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG
    assert h.value is None


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    t = np.zeros(4)
    c = np.zeros(4, np.int64)
    assert lib.lbm_profile_steps(None, 2, t.ctypes.data, c.ctypes.data) == lbm.LBM_ERR_ARG
    assert lib.lbm_run_to_steady(None, 1e-9, 10, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_permeability(None, None, None) == lbm.LBM_ERR_ARG


def test_qsgs_rejects_bad_arguments(lib):
    out = np.zeros(16, np.uint8)
    assert lib.lbm_qsgs(1, 4, 4, 1, 0.02, 1.5, 0.2, None, out.ctypes.data, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_qsgs(1, 0, 4, 1, 0.02, 0.5, 0.2, None, out.ctypes.data, None) == lbm.LBM_ERR_ARG


def test_load_rejects_missing_and_corrupt_files(lib, tmp_path):
    h = C.c_void_p()
    o = lbm.make_options()
    assert lib.lbm_load(str(tmp_path / "nope").encode(), C.byref(o), C.byref(h)) == lbm.LBM_ERR_IO
    p = tmp_path / "bad.ckpt"
    p.write_bytes(b"LBMGB300" + b"\x00" * 7)
    assert lib.lbm_load(str(p).encode(), C.byref(o), C.byref(h)) == lbm.LBM_ERR_IO


def test_forced_create_rejects_bad_arguments(lib):
    m = np.zeros((6, 9), np.uint8)
    desc = (lbm.lbm_domain_desc * 1)()
    desc[0] = lbm.lbm_domain_desc(m.ctypes.data, 9, 6, 1, 0.8, 0.0)
    h = C.c_void_p()
    o = lbm.make_options()
    assert lib.lbm_batch_create_forced(1, desc, None, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG
    g = np.array([np.nan])
    assert lib.lbm_batch_create_forced(1, desc, g.ctypes.data, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG
    g = np.array([1e-5])
    t = lbm.make_options(collision=lbm.LBM_COLL_TRT, trt_lambda=-1.0)
    assert lib.lbm_batch_create_forced(1, desc, g.ctypes.data, C.byref(t), C.byref(h)) == lbm.LBM_ERR_ARG
    assert h.value is None


def test_trt_options_are_validated(lib):
    m = np.zeros((6, 9), np.uint8)
    h = C.c_void_p()
    for kw in (dict(collision=2), dict(collision=1, trt_lambda=0.0), dict(collision=1, trt_lambda=float("inf"))):
        o = lbm.make_options(**kw)
        assert lib.lbm_create_domain(m.ctypes.data, 9, 6, 0.8, 1e-3, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG


def test_local_knudsen_rejects_null_handle(lib):
    assert lib.lbm_local_knudsen(None, 0, None, None, None) == lbm.LBM_ERR_ARG


def test_batch_calls_reject_a_null_batch(lib):
    st = np.zeros(1, np.int32)
    k = np.zeros(1)
    assert lib.lbm_batch_run_to_steady(None, 1e-9, 10, st.ctypes.data) == lbm.LBM_ERR_ARG
    assert lib.lbm_batch_permeability(None, k.ctypes.data) == lbm.LBM_ERR_ARG
    lib.lbm_batch_destroy(None)  # a no-op, like lbm_destroy(NULL)


def test_lattice_tables(lib):
    """The kernels' direction tables: opposite and mirrored directions are
    involutions with the right velocities, and the weights make the second
    moment isotropic with c_s^2 = 1/3."""
    for q in (9, 19):
        c, w, opp, fy, fz = lbm.lbm_lattice(q)
        assert c.shape == (q, 3) and abs(w.sum() - 1.0) < 1e-15
        assert np.array_equal(c[opp], -c) and np.array_equal(opp[opp], np.arange(q))
        assert np.array_equal(c[fy], c * [1, -1, 1]) and np.array_equal(c[fz], c * [1, 1, -1])
        second = np.einsum("i,ia,ib->ab", w, c, c)
        d = 2 if q == 9 else 3
        assert np.allclose(second[:d, :d], np.eye(d) / 3.0, atol=1e-15)
    out = np.zeros(57, np.int32)
    assert lib.lbm_lattice(7, out.ctypes.data, None, None, None, None) == lbm.LBM_ERR_ARG


def test_readme_c_example_compiles(lib, tmp_path):
    """The C example of the README compiles against include/lbm.h and links
    against the library (it is not run: it needs a GPU)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    txt = open(os.path.join(ROOT, "README.md")).read()
    m = re.search(r"```c\n(.*?)```", txt, flags=re.S)
    assert m, "README has no C example"
    src = tmp_path / "example.c"
    src.write_text(m.group(1))
    libdir = os.path.dirname(lbm.library_path())
    r = subprocess.run([cc, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(tmp_path / "example"), "-L", libdir, "-llbm_gb300", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_tile_rows_option_is_validated(lib):
    m = np.zeros((6, 9), np.uint8)
    h = C.c_void_p()
    for rows in (-2, 5):
        o = lbm.make_options(tile_rows=rows)
        assert lib.lbm_create_domain(m.ctypes.data, 9, 6, 0.8, 1e-3, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG


def test_band_rows_option_is_validated(lib):
    """band_rows in -1..64, and not together with a staged tile height."""
    m = np.zeros((6, 9), np.uint8)
    h = C.c_void_p()
    for kw in (dict(band_rows=-2), dict(band_rows=65), dict(band_rows=8, tile_rows=2), dict(pair_block_mb=-2),
               dict(pair_block_mb=4097)):
        o = lbm.make_options(**kw)
        assert lib.lbm_create_domain(m.ctypes.data, 9, 6, 0.8, 1e-3, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG


def test_tune_key_format(lib):
    """Key = device (spaces -> '_') | Q | floor(log2 fluid nodes) | equilibrium |
    collision | hash of the kernel sources."""
    h = build.kernel_hash()
    assert lbm.lbm_tune_key_for("NVIDIA GB300", 9, 23228319, 0, 0) == f"NVIDIA_GB300|q9|n2^24|eq0|coll0|{h}"
    assert lbm.lbm_tune_key_for("x", 19, 1 << 24, 1, 1) == f"x|q19|n2^24|eq1|coll1|{h}"
    assert lbm.lbm_tune_key_for("x", 19, (1 << 24) - 1, 1, 1) == f"x|q19|n2^23|eq1|coll1|{h}"
    assert lbm.lbm_tune_key_for("x", 9, 1, 0, 0).split("|")[2] == "n2^0"
    small = C.create_string_buffer(8)
    assert lib.lbm_tune_key_for(b"NVIDIA GB300", 9, 100, 0, 0, small, 8) == lbm.LBM_ERR_ARG


def test_tune_cache_round_trip(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    assert lbm.lbm_tune_cache_get(path, "k1") is None  # missing file = empty cache
    a = dict(block_threads=64, strip_rows=16, gather_batch=2, tile_rows=0, band_rows=32, pair_block_mb=0)
    b = dict(block_threads=256, strip_rows=4, gather_batch=4, tile_rows=3, band_rows=0, pair_block_mb=24)
    lbm.lbm_tune_cache_put(path, "k1", a, 301.25)
    lbm.lbm_tune_cache_put(path, "GPU A|q9|n2^20|eq0|coll0|abc", b, 12.5)
    assert lbm.lbm_tune_cache_get(path, "k1") == (a, 301.25)
    assert lbm.lbm_tune_cache_get(path, "GPU A|q9|n2^20|eq0|coll0|abc") == (b, 12.5)
    lbm.lbm_tune_cache_put(path, "k1", b, 99.0)  # replace
    assert lbm.lbm_tune_cache_get(path, "k1") == (b, 99.0)
    import json
    doc = json.load(open(path))  # the file is valid JSON
    assert set(doc) == {"k1", "GPU A|q9|n2^20|eq0|coll0|abc"} and doc["k1"]["strip_rows"] == 4
    with open(path, "a") as fh:  # garbage lines are ignored
        fh.write("not json at all\n\"k2\": {\"block_threads\": \n")
    assert lbm.lbm_tune_cache_get(path, "k2") is None
    assert lbm.lbm_tune_cache_get(path, "k1") == (b, 99.0)
    with open(path, "a") as fh:  # an entry without band_rows reads as 0
        fh.write('"k3": {"block_threads": 64, "strip_rows": 8, "gather_batch": 4, "tile_rows": 0, '
                 '"us_per_step": 5.0}\n')
    assert lbm.lbm_tune_cache_get(path, "k3") == (dict(a, strip_rows=8, gather_batch=4, band_rows=0), 5.0)
    # an entry without band_rows / pair_block_mb reads them as 0
    cfg = lbm.lbm_launch(128, 8, 4, 0)
    assert lib.lbm_tune_cache_put(path.encode(), b'bad"key', C.byref(cfg), 1.0) == lbm.LBM_ERR_ARG
    assert lib.lbm_tune_cache_put(str(tmp_path / "no" / "dir.json").encode(), b"k", C.byref(cfg), 1.0) == lbm.LBM_ERR_IO


def test_autotune_option_is_validated(lib):
    m = np.zeros((6, 9), np.uint8)
    h = C.c_void_p()
    o = lbm.make_options()
    o.autotune = 2
    assert lib.lbm_create_domain(m.ctypes.data, 9, 6, 0.8, 1e-3, C.byref(o), C.byref(h)) == lbm.LBM_ERR_ARG
    assert lib.lbm_autotune(None, None, 0, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_time_steps(None, 2, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_set_launch(None, None) == lbm.LBM_ERR_ARG
