"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/thin.h declares, rejects bad arguments on the host, and its point
table matches the oracle on all 256 masks.  No compute call reaches a GPU."""
import ctypes
import os
import re

import pytest

import oracle
from paper_1603_09180_gb300 import build as thin_build
from paper_1603_09180_gb300 import thin

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    thin_build.build()
    return thin.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "thin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(thin_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) >= {"thin_run", "thin_batch", "thin_point_table", "thin_serve_create",
                          "thin_serve_submit", "thin_serve_poll", "thin_serve_destroy"}
    for n in names:
        assert hasattr(lib, n), n
    assert set(thin.EXPORTS) <= set(names)
    assert "sm_103a" in thin.version()


@pytest.mark.parametrize("adj", [thin.ADJ_8_4, thin.ADJ_4_8])
def test_point_table_matches_oracle(adj):
    tab = thin.point_table(adj)
    if adj == thin.ADJ_8_4:
        assert tab == thin.point_table()
    for m in range(256):
        e = tab[m]
        tp, tm, lab = oracle.mask_numbers(m, adj=adj)
        assert (e & 7, (e >> 3) & 7) == (tp, tm), m
        assert bool(e >> 30 & 1) == (tp == 1 and tm == 1)
        assert bool(e >> 31 & 1) == (tm >= 2)
        got = [((e >> (6 + 3 * i)) & 7) - 1 for i in range(8)]
        # same partition (component numbering may differ)
        pairs_g = {(i, j) for i in range(8) for j in range(8) if got[i] >= 0 and got[i] == got[j]}
        pairs_o = {(i, j) for i in range(8) for j in range(8) if lab[i] >= 0 and lab[i] == lab[j]}
        assert pairs_g == pairs_o, m
        assert [g >= 0 for g in got] == [l >= 0 for l in lab]


def test_host_side_argument_errors(lib):
    o = thin.options()
    st = thin.Stats()
    run = lambda *a: lib.thin_run(*a, ctypes.byref(o), ctypes.byref(st))
    assert run(None, 10, 10, 10, thin.U8, 0, thin.ADJ_8_4, None) == thin.THIN_ERR_ARG
    assert run(ctypes.c_void_p(4096), -1, 10, 10, thin.U8, 0, thin.ADJ_8_4, None) == thin.THIN_ERR_ARG
    assert run(ctypes.c_void_p(4096), 10, 10, 9, thin.U8, 0, thin.ADJ_8_4, None) == thin.THIN_ERR_ARG
    assert run(ctypes.c_void_p(4096), 10, 10, 20, 7, 0, thin.ADJ_8_4, None) == thin.THIN_ERR_ARG
    assert run(ctypes.c_void_p(4097), 10, 10, 20, thin.U16, 0, thin.ADJ_8_4, None) == thin.THIN_ERR_ARG
    assert run(ctypes.c_void_p(4096), 10, 10, 10, thin.U8, 0, 7, None) == thin.THIN_ERR_ARG  # no such adjacency pair
    assert run(ctypes.c_void_p(4096), 10, 10, 10, thin.U8, 0, 9, None) == thin.THIN_ERR_ARG
    # empty and interior-free images are valid no-ops that touch no memory
    assert run(None, 0, 0, 0, thin.U8, 0, thin.ADJ_8_4, None) == thin.THIN_OK
    assert st.converged == 1 and st.phases == 0
    assert run(ctypes.c_void_p(4096), 2, 50, 2, thin.U8, 0, thin.ADJ_8_4, None) == thin.THIN_OK
    bad = thin.options(rule=5)
    assert lib.thin_run(ctypes.c_void_p(4096), 10, 10, 10, thin.U8, 0, thin.ADJ_8_4, None, ctypes.byref(bad),
                        None) == thin.THIN_ERR_ARG
    bad = thin.options(start_phase=-1)
    assert lib.thin_run(ctypes.c_void_p(4096), 10, 10, 10, thin.U8, 0, thin.ADJ_8_4, None, ctypes.byref(bad),
                        None) == thin.THIN_ERR_ARG
    assert lib.thin_batch(None, 3, thin.ADJ_8_4, None, None, None) == thin.THIN_ERR_ARG
    assert lib.thin_batch(None, 0, thin.ADJ_8_4, None, None, None) == thin.THIN_OK


def test_product_path_has_no_oracle_dependency():
    """The library and its binding never load the oracle; no CPU fallback."""
    pkg = os.path.join(ROOT, "paper_1603_09180_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f
                assert "thin_oracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path):
    import importlib
    mod = importlib.import_module("paper_1603_09180_gb300.thin")
    with pytest.raises(RuntimeError):
        saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "nope.so"))
        finally:
            mod._lib = saved


def test_serve_host_side_errors(lib):
    h = ctypes.c_void_p()
    assert lib.thin_serve_create(0, 4, 4, ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_serve_create(1 << 20, 0, 4, ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_serve_create(1 << 20, 4, 0, ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_serve_create(1 << 20, 4, 4, None) == thin.THIN_ERR_ARG
    t = ctypes.c_uint64()
    done = ctypes.c_int()
    assert lib.thin_serve_submit(None, None, 4, 4, 4, thin.U8, 0, ctypes.byref(t)) == thin.THIN_ERR_ARG
    assert lib.thin_serve_poll(None, 1, None, 0, ctypes.byref(done), None) == thin.THIN_ERR_ARG
    assert lib.thin_serve_wait_any(None, 0, ctypes.byref(t)) == thin.THIN_ERR_ARG
    assert lib.thin_serve_destroy(None) == thin.THIN_ERR_ARG


def test_plan_host_side_errors(lib):
    h = ctypes.c_void_p()
    o = thin.options()
    assert lib.thin_plan_create(None, -1, thin.ADJ_8_4, ctypes.byref(o), ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_plan_create(None, 0, 5, ctypes.byref(o), ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_plan_create(None, 0, thin.ADJ_8_4, ctypes.byref(o), None) == thin.THIN_ERR_ARG
    naive = thin.options(kernel="naive")
    assert lib.thin_plan_create(None, 0, thin.ADJ_8_4, ctypes.byref(naive), ctypes.byref(h)) == thin.THIN_ERR_UNSUPPORTED
    jobs = (thin.Job * 1)()
    jobs[0].img_dev, jobs[0].w, jobs[0].h, jobs[0].pitch, jobs[0].dtype = 4096, 8, 8, 8, 7
    assert lib.thin_plan_create(jobs, 1, thin.ADJ_8_4, ctypes.byref(o), ctypes.byref(h)) == thin.THIN_ERR_ARG
    assert lib.thin_plan_launch(None, None) == thin.THIN_ERR_ARG
    assert lib.thin_plan_destroy(None) == thin.THIN_ERR_ARG


def test_calls_without_work_need_no_device(lib):
    """Zero images, empty images and images without interior points finish on
    the host: converged stats, nothing launched (this machine may have no GPU)."""
    o = thin.options()
    st = thin.Stats()
    assert lib.thin_batch(None, 0, thin.ADJ_8_4, None, ctypes.byref(o), None) == thin.THIN_OK
    assert lib.thin_run(None, 0, 0, 0, thin.U8, 0, thin.ADJ_8_4, None, ctypes.byref(o), ctypes.byref(st)) == thin.THIN_OK
    assert st.converged == 1 and st.phases == 0 and st.last_change_phase == -1
    st = thin.Stats()
    assert lib.thin_run(ctypes.c_void_p(4096), 9, 2, 9, thin.U8, 0, thin.ADJ_4_8, None, ctypes.byref(o),
                        ctypes.byref(st)) == thin.THIN_OK
    assert st.converged == 1
    assert lib.thin_run_noalloc(None, 0, 0, 0, thin.U8, 0, thin.ADJ_8_4, None, None, ctypes.byref(st)) == thin.THIN_OK
    h = ctypes.c_void_p()
    assert lib.thin_plan_create(None, 0, thin.ADJ_8_4, ctypes.byref(o), ctypes.byref(h)) == thin.THIN_OK
    assert lib.thin_plan_launch(h, None) == thin.THIN_OK
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.thin_plan_tiling(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == thin.THIN_OK
    assert (a.value, b.value, c.value) == (0, 0, 0)
    assert lib.thin_plan_destroy(h) == thin.THIN_OK


def test_option_checks(lib):
    img = ctypes.c_void_p(4096)
    for field, bad in (("rule", 2), ("op", 7), ("kernel", 9), ("start_phase", -1), ("tile_w", -16), ("halo", -1)):
        o = thin.options()
        setattr(o, field, bad)
        assert lib.thin_run(img, 9, 9, 9, thin.U8, 0, thin.ADJ_8_4, None, ctypes.byref(o), None) == thin.THIN_ERR_ARG, field
    o = thin.options()
    assert lib.thin_run(img, 9, 9, 9, thin.U16, 0, thin.ADJ_8_4, None, ctypes.byref(o), None) == thin.THIN_ERR_ARG  # odd pitch
    assert lib.thin_run(ctypes.c_void_p(4097), 9, 9, 18, thin.U16, 0, thin.ADJ_8_4, None, ctypes.byref(o),
                        None) == thin.THIN_ERR_ARG  # odd address for u16
    assert lib.thin_run(img, 9, 9, 8, thin.U8, 0, thin.ADJ_8_4, None, ctypes.byref(o), None) == thin.THIN_ERR_ARG  # pitch < w


def test_binding_rejects_host_tensors():
    """The binding marshals CUDA tensors only: a host tensor, a 3-D tensor or a
    strided column is refused before anything reaches the library."""
    torch = pytest.importorskip("torch")
    host = torch.zeros(8, 8, dtype=torch.uint8)
    with pytest.raises(ValueError):
        thin.run(host, 0)
    with pytest.raises(ValueError):
        thin.autotune(host, 0)
    with pytest.raises(ValueError):
        thin.batch([host], [0])
    with pytest.raises(ValueError):
        thin.BatchPlan([host], [0])
    with pytest.raises(ValueError):
        thin.batch([host, host], [0])  # one lambda per image
