"""The allocation-free Morton sort against the regular evaluation's tree export.

gbfmm_sort_static serves callers that may not allocate device memory (their host framework
owns the device memory, or they only receive the buffers they read and write); it keeps its
scratch in a static device array.  Its outputs must equal, bit for bit, the sorted keys,
permutation and particles that gbfmm_evaluate builds with the same parameters, on two calls
in a row (the second call reuses the scratch the first one left behind).  The cases cover
every buffer parity of the radix sort: depth 0 (no key bits, identity order), 1 pass
(depth 2), 2 passes (depths 3 and 4) and 3 passes (depth 6).  This file is collected last so
that a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1010_1482_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(G, ctx, x, prm):
    """Tree of the existing entry point: gbfmm_evaluate, then gbfmm_export_tree."""
    L, ws = G.gbfmm_plan(prm, len(x))
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    wsb = torch.empty(ws, dtype=torch.uint8, device="cuda")
    G.gbfmm_evaluate(ctx, prm, xd, out, wsb)
    G.gbfmm_sync_status(ctx)
    t = G.gbfmm_export_tree(ctx, len(x), G.level_offset(L + 1))
    return t["sorted_leaf_keys"], t["perm"]


def _static(G, x, prm):
    n = len(x)
    xd = torch.from_numpy(x).cuda()
    sx = torch.full_like(xd, -1.0)
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    G.gbfmm_sort_static(prm, xd, sx, perm, keys, status)
    torch.cuda.synchronize()
    return (keys.cpu().numpy().view(np.uint32), perm.cpu().numpy().view(np.uint32), sx.cpu().numpy(),
            int(status.item()))


# (n, leaf, depth L): 3L key bits in ceil(3L / 8) radix passes of 8 bits
CASES = [(50, 64, 0), (4096, 64, 2), (4096, 8, 3), (200000, 64, 4), (1 << 20, 4, 6)]


@pytest.mark.parametrize("n,leaf,depth", CASES)
def test_sort_static_matches_evaluate_twice(n, leaf, depth):
    from paper_1010_1482_gb300 import gbfmm as G

    prm = G.gbfmm_default_params(p=4, leaf_size=leaf)
    assert G.gbfmm_plan(prm, n)[0] == depth
    ctx = G.gbfmm_create(0)
    try:
        for call, seed in enumerate((11, 12)):  # two calls in a row, different particles
            x = inputs.uniform_cube(n, seed) if call == 0 else inputs.plummer(n, seed)
            ref_keys, ref_perm = _reference(G, ctx, x, prm)
            keys, perm, sx, status = _static(G, x, prm)
            assert status == 0, call
            assert np.array_equal(keys, ref_keys), call
            assert np.array_equal(perm, ref_perm), call
            assert np.array_equal(sx, x[perm.astype(np.int64)]), call
    finally:
        G.gbfmm_destroy(ctx)


def test_sort_static_reports_nonfinite_input():
    """A non-finite coordinate is clamped into a boundary cell and reported in the status word."""
    from paper_1010_1482_gb300 import gbfmm as G

    prm = G.gbfmm_default_params(p=4, leaf_size=64)
    x = inputs.uniform_cube(5000, 3)
    x[17, 1] = np.nan
    keys, perm, sx, status = _static(G, x, prm)
    assert status == 1
    assert np.array_equal(np.sort(perm), np.arange(len(x), dtype=np.uint32))


def test_sort_static_rejects_oversize_and_adaptive():
    from paper_1010_1482_gb300 import gbfmm as G

    prm = G.gbfmm_default_params(p=4, leaf_size=64)
    n = (1 << 20) + 1
    x = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_sort_static(prm, x, torch.empty_like(x), torch.empty(n, dtype=torch.int32, device="cuda"),
                            torch.empty(n, dtype=torch.int32, device="cuda"))
    assert ei.value.code == G.GBFMM_EUNSUPPORTED
    n = 4096
    x = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    prm = G.gbfmm_default_params(p=4, leaf_size=64, tree=G.TREE_ADAPTIVE)
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_sort_static(prm, x, torch.empty_like(x), torch.empty(n, dtype=torch.int32, device="cuda"),
                            torch.empty(n, dtype=torch.int32, device="cuda"))
    assert ei.value.code == G.GBFMM_EUNSUPPORTED
