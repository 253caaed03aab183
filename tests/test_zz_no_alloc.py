"""The allocation-free entry point, thin_run_noalloc, against thin_run.

thin_run_noalloc exists for callers that cannot allocate device memory when
they call in (an application whose device memory is all handed to its own
allocator at start-up, or a loop with a fixed time budget that may not call
into the allocator).  It must give exactly what thin_run gives, call after
call, although every call reuses one fixed scratch array, and it must leave
the device's free memory as it found it.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import ctypes

import numpy as np
import pytest

from paper_1603_09180_gb300 import synth, thin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(fn, t, lam, opts=None):
    h, w = t.shape
    st = thin.Stats()
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(ctypes.c_void_p(t.data_ptr()), w, h, t.stride(0) * t.element_size(),
            thin.U16 if t.dtype == torch.uint16 else thin.U8, lam, thin.ADJ_8_4, ctypes.c_void_p(stream),
            ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    torch.cuda.synchronize()
    return rc, st.as_dict()


def _host(t):
    return t.view(torch.int16).cpu().numpy() if t.dtype == torch.uint16 else t.cpu().numpy()


def test_noalloc_matches_thin_run_on_two_calls_in_a_row():
    lib = thin.load()
    cases = [(synth.value_noise_image(300, 420, "u8", seed=21), 7),
             (synth.value_noise_image(260, 333, "u16", seed=22), 120)]
    for img, lam in cases:
        ref = torch.from_numpy(img.view(np.int16) if img.dtype == np.uint16 else img).cuda()
        if img.dtype == np.uint16:
            ref = ref.view(torch.uint16)
        base = ref.clone()
        # thin_run_noalloc is the tiled engine: compare with thin_run on that engine
        rc0, st0 = _call(lib.thin_run, ref, lam, thin.options(kernel="tiled"))
        assert rc0 == thin.THIN_OK
        for _ in range(2):  # the second call finds the first call's leftovers in the scratch array
            t = base.clone()
            rc, st = _call(lib.thin_run_noalloc, t, lam)
            assert rc == thin.THIN_OK
            assert np.array_equal(_host(t), _host(ref))  # integer work: bit-exact
            for k in ("lowered", "last_change_phase", "converged", "tiles_visited", "steps"):
                assert st[k] == st0[k], k


def test_noalloc_unaligned_rows_and_cap():
    lib = thin.load()
    img = synth.value_noise_image(100, 130, "u8", seed=5)
    big = torch.zeros((110, 141), dtype=torch.uint8, device="cuda")
    big[4:104, 3:133] = torch.from_numpy(img).cuda()
    ref = big.clone()
    o = thin.options(max_phases=13, kernel="tiled")
    rc0, st0 = _call(lib.thin_run, ref[4:104, 3:133], 9, o)
    rc, st = _call(lib.thin_run_noalloc, big[4:104, 3:133], 9, o)
    assert rc == rc0 and st["end_phase"] == st0["end_phase"] == 13
    assert torch.equal(big, ref)


def test_noalloc_allocates_nothing():
    lib = thin.load()
    img = synth.value_noise_image(700, 900, "u8", seed=31)
    t = torch.from_numpy(img).cuda()
    rc, _ = _call(lib.thin_run_noalloc, t.clone(), 12)  # first call: the module and its array are in place after it
    assert rc == thin.THIN_OK
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rc, st = _call(lib.thin_run_noalloc, t, 12)
        assert rc == thin.THIN_OK and st["converged"] == 1
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0  # the driver's free bytes: no allocation by any route


def test_noalloc_rejects_images_beyond_its_scratch():
    lib = thin.load()
    img = synth.value_noise_image(4096, 4096, "u8", seed=32)
    t = torch.from_numpy(img).cuda()
    before = t.clone()
    rc, _ = _call(lib.thin_run_noalloc, t, 0)
    assert rc == thin.THIN_ERR_TOO_LARGE
    assert torch.equal(t, before)  # rejected: the image is left untouched
