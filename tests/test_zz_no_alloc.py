"""The allocation-free scan entry point against the regular one.

pm_scan_device_noalloc serves callers that cannot allocate device memory
while they scan (an application that owns the GPU allocator, or a loop that
reserved all its memory up front). It must give exactly what pm_scan_device
gives -- occurrence list, per-pattern counts and total -- including on a
second call right after the first, which finds the first call's leftovers
in the library's shared scratch array.
"""
import numpy as np
import pytest

from paper_1407_2889_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1407_2889_gb300 import pmscan as pm  # noqa: E402


def _regular(s, d_text, n, flags, d, cap):
    ws = torch.zeros(s.workspace_bytes(n, counts_only=bool(flags & pm.PM_COUNTS_ONLY)),
                     dtype=torch.uint8, device="cuda")
    counts = torch.zeros(d, dtype=torch.int64, device="cuda")
    occ = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    pm.pm_scan_device(s.h, d_text, n, flags, counts, occ, cap, nocc, ws, ws.numel())
    assert pm.pm_scan_status(ws) == pm.PM_OK
    k = int(nocc.item())
    return occ[: min(k, cap)].cpu().numpy(), counts.cpu().numpy(), k


def _noalloc(s, d_text, n, flags, d, cap):
    counts = torch.full((d,), -1, dtype=torch.int64, device="cuda")
    occ = torch.full((max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    nocc = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    pm.pm_scan_device_noalloc(s.h, d_text, n, flags, counts, occ, cap, nocc)
    # the kernel's status word lives in the library's array, not in a
    # caller's workspace: read it through the allocation-free reader
    assert pm.pm_noalloc_scan_status() == pm.PM_OK
    torch.cuda.synchronize()
    k = int(nocc.item())
    return occ[: min(k, cap)].cpu().numpy(), counts.cpu().numpy(), k


@pytest.mark.parametrize("flags", [0, pm.PM_COUNTS_ONLY])
def test_noalloc_matches_regular_scan_on_two_calls(flags):
    T = synth.est_text(12 << 20, 31)  # list mode: 4 bytes of the array per text byte
    P = synth.mixed_patterns(T, 3000, 8, 31)
    P = np.concatenate([P, P[:20]])  # duplicates exercise the group path
    d = P.shape[0]
    s = pm.PatternSet.ac(P)
    d_text = torch.from_numpy(T).cuda()
    cap = T.size // 4
    want = _regular(s, d_text, T.size, flags, d, cap)
    assert want[2] > 0
    for call in range(2):
        got = _noalloc(s, d_text, T.size, flags, d, cap)
        assert got[2] == want[2], f"call {call}: total"
        assert np.array_equal(got[1], want[1]), f"call {call}: counts"
        if not flags & pm.PM_COUNTS_ONLY:
            assert np.array_equal(got[0], want[0]), f"call {call}: occurrences"
    s.close()


def test_noalloc_on_a_set_tuned_to_two_characters_per_lookup():
    """A set whose plan takes two characters per lookup: the allocation-free
    call always walks one character at a time, with the same results."""
    T = synth.est_text(4 << 20, 37)
    P = synth.mixed_patterns(T, 300, 10, 37)
    d = P.shape[0]
    s = pm.PatternSet.ac(P, {"stride": 2})
    assert s.info()["stride"] == 2
    d_text = torch.from_numpy(T).cuda()
    cap = T.size // 4
    want = _regular(s, d_text, T.size, 0, d, cap)
    assert want[2] > 0
    for call in range(2):
        got = _noalloc(s, d_text, T.size, 0, d, cap)
        assert got[2] == want[2], f"call {call}: total"
        assert np.array_equal(got[1], want[1]), f"call {call}: counts"
        assert np.array_equal(got[0], want[0]), f"call {call}: occurrences"
    s.close()


@pytest.mark.parametrize("flags", [0, pm.PM_COUNTS_ONLY])
def test_noalloc_on_a_late_ids_plan(flags):
    """A plan with late terminal ids (the expand kernel maps ids to codes and
    counts them, with its own finished-CTA counter in the array's header):
    two calls in a row equal the regular scan."""
    T = synth.est_text(8 << 20, 41)
    P = synth.mixed_patterns(T, 2000, 8, 41)
    P = np.concatenate([P, P[:9], P[:3]])  # groups of two and three
    d = P.shape[0]
    s = pm.PatternSet.ac(P, {"ids_place": 3})
    d_text = torch.from_numpy(T).cuda()
    cap = T.size // 4
    want = _regular(s, d_text, T.size, flags, d, cap)
    assert want[2] > 0
    for call in range(2):
        got = _noalloc(s, d_text, T.size, flags, d, cap)
        assert got[2] == want[2], f"call {call}: total"
        assert np.array_equal(got[1], want[1]), f"call {call}: counts"
        if not flags & pm.PM_COUNTS_ONLY:
            assert np.array_equal(got[0], want[0]), f"call {call}: occurrences"
    s.close()


def test_noalloc_rejects_a_scan_larger_than_its_scratch():
    P = synth.random_patterns(100, 8, 5)
    s = pm.PatternSet.ac(P)
    n = (1 << 32) - 1              # a real buffer, so nothing could read past it
    d_text = torch.zeros(n, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(100, dtype=torch.int64, device="cuda")
    occ = torch.zeros(16, dtype=torch.int64, device="cuda")
    nocc = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pm.PmError) as e:
        pm.pm_scan_device_noalloc(s.h, d_text, n, 0, counts, occ, 16, nocc)
    assert e.value.code == pm.PM_ETOOBIG
    assert pm.pm_noalloc_scratch_bytes() == 64 << 20
    del d_text
    s.close()
