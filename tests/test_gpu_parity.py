"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP32 path vs FP64 oracle):
  * tree keys, sort permutation, cell ranges, interaction lists: bit-exact;
  * potentials and gradients vs the oracle FMM (same tree, same p): relative L2 <= 1e-5;
  * vs the FP64 direct sum: within the truncation error the oracle itself has, plus 1e-5;
  * expansions: per-degree relative L2 of the scaled coefficients <= 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FMM = 1e-5


@pytest.fixture(scope="module")
def G():
    from paper_1010_1482_gb300 import gbfmm

    gbfmm.lib()
    return gbfmm


@pytest.fixture(scope="module")
def ctx(G):
    c = G.gbfmm_create(0)
    yield c
    G.gbfmm_destroy(c)


def run(G, ctx, x, **kw):
    prm = G.gbfmm_default_params(**kw)
    L, ws = G.gbfmm_plan(prm, len(x))
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    out = torch.empty_like(xd)
    wsb = torch.empty(max(ws, 256), dtype=torch.uint8, device="cuda")
    G.gbfmm_evaluate(ctx, prm, xd, out, wsb)
    G.gbfmm_sync_status(ctx)
    return out.cpu().numpy().astype(np.float64), L


def degenerate(kind):
    if kind == "duplicates":
        base = inputs.uniform_cube(5, 3)
        x = np.repeat(base, 40, axis=0)
        x[:, 3] = 0.01
        return x.astype(np.float32), 8
    if kind == "one":
        return np.array([[0.3, 0.2, 0.1, 1.0]], dtype=np.float32), 64
    if kind == "two":
        return np.array([[0.3, 0.2, 0.1, 1.0], [0.7, 0.1, 0.9, 2.0]], dtype=np.float32), 64
    if kind == "below_leaf":
        return inputs.uniform_cube(50, 4), 64
    if kind == "line":  # all on a line: flat box extents
        x = inputs.uniform_cube(3000, 6)
        x[:, 1] = 0.5
        x[:, 2] = 0.25
        return x, 8
    raise KeyError(kind)


TREE_CASES = [("uniform", 4096, 64), ("uniform", 20000, 16), ("uniform", 50000, 8), ("plummer", 30000, 32)]


@pytest.mark.parametrize("dist,n,leaf", TREE_CASES)
def test_tree_and_lists_bit_exact(G, ctx, dist, n, leaf):
    x = inputs.make_particles(n, dist, 1000 + n)
    _, L = run(G, ctx, x, p=4, leaf_size=leaf)
    t = O.build_tree(x, leaf)
    assert L == t["L"]
    C = O.level_offset(L + 1)
    g = G.gbfmm_export_tree(ctx, n, C)
    assert np.array_equal(g["origin"], t["origin"]) and g["side"] == t["side"]
    assert np.array_equal(g["sorted_leaf_keys"].astype(np.uint64), t["sorted_leaf_keys"])
    assert np.array_equal(g["perm"].astype(np.int64), t["perm"])
    assert np.array_equal(g["count"], t["count"])
    assert np.array_equal(g["begin"], t["begin"])
    ls = O.build_lists(t)
    offs, ids = G.gbfmm_export_lists(ctx, G.LIST_P2P, 8 ** L)
    assert np.array_equal(offs, ls["p2p_offs"]) and np.array_equal(ids, ls["p2p_ids"])
    offs, ids = G.gbfmm_export_lists(ctx, G.LIST_M2L, C)
    assert np.array_equal(offs, ls["m2l_offs"]) and np.array_equal(ids, ls["m2l_ids"])


def test_sort_of_large_inputs_bit_exact(G, ctx):
    # 5,000,000 particles at leaf 8: depth 7, 21-bit keys in 3 radix passes of the
    # reduce-then-scan form (inputs of 2^22 particles and more)
    n, leaf = 5_000_000, 8
    x = inputs.uniform_cube(n, 4242)
    _, L = run(G, ctx, x, p=4, leaf_size=leaf)
    assert L == 7
    origin, side, _ = O.root_box(x)
    keys = O.morton_keys(x, origin, side) >> np.uint64(3 * (O.ADAPTIVE_MAX_LEVEL - L))
    perm = np.lexsort((np.arange(n), keys))
    g = G.gbfmm_export_tree(ctx, n, O.level_offset(L + 1))
    assert np.array_equal(g["perm"].astype(np.int64), perm)
    assert np.array_equal(g["sorted_leaf_keys"].astype(np.uint64), keys[perm])


def test_keys_on_leaf_cell_faces(G, ctx):
    """Coordinates exactly on leaf-cell faces (j / 32 in the unit box, depth 5) and one float step
    to either side: the key kernel's FP32 estimate cannot decide these and takes the FP64 steps;
    keys, permutation and cells must still equal the oracle's bit for bit."""
    g = np.arange(33, dtype=np.float64) / 32.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)
    lo = np.nextafter(pts, np.float32(-1)).astype(np.float32)
    hi = np.nextafter(pts, np.float32(2)).astype(np.float32)
    xyz = np.concatenate([pts, np.clip(lo, 0, 1), np.clip(hi, 0, 1)])
    q = inputs.uniform_cube(len(xyz), 12)[:, 3:4]
    x = np.concatenate([xyz, q], axis=1).astype(np.float32)
    leaf = 16
    _, L = run(G, ctx, x, p=4, leaf_size=leaf)
    t = O.build_tree(x, leaf)
    assert L == t["L"] == 5
    g_ = G.gbfmm_export_tree(ctx, len(x), O.level_offset(L + 1))
    assert np.array_equal(g_["sorted_leaf_keys"].astype(np.uint64), t["sorted_leaf_keys"])
    assert np.array_equal(g_["perm"].astype(np.int64), t["perm"])
    assert np.array_equal(g_["count"], t["count"])


@pytest.mark.parametrize("kind", ["duplicates", "one", "two", "below_leaf", "line"])
def test_degenerate_inputs(G, ctx, kind):
    x, leaf = degenerate(kind)
    out, L = run(G, ctx, x, p=4, leaf_size=leaf)
    t = O.build_tree(x, leaf)
    g = G.gbfmm_export_tree(ctx, len(x), O.level_offset(L + 1))
    assert np.array_equal(g["perm"].astype(np.int64), t["perm"])
    assert np.array_equal(g["count"], t["count"])
    ref = O.fmm(x, 4, leaf)["out"]
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.max(np.abs(out - ref)) <= 2e-5 * scale
    if kind == "one":
        assert np.all(out == 0.0)


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_expansions_match_oracle(G, ctx, p):
    n, leaf = 20000, 16
    x = inputs.uniform_cube(n, 77)
    run(G, ctx, x, p=p, leaf_size=leaf)
    r = O.fmm(x, p, leaf, keep=True)
    L = r["L"]
    C = O.level_offset(L + 1)
    Mg = G.gbfmm_export_expansions(ctx, 0, C, p)
    Lg = G.gbfmm_export_expansions(ctx, 1, C, p)
    side = r["tree"]["side"]
    for l in range(2, L + 1):
        sl = slice(O.level_offset(l), O.level_offset(l + 1))
        h = side / 2**l
        for n in range(p):
            cols = slice(n * (n + 1) // 2, (n + 1) * (n + 2) // 2)
            for A, B, sc in ((Mg, r["M"], h ** (-n)), (Lg, r["Lc"], h ** (n + 1))):
                num = np.linalg.norm((A[sl, cols] - B[sl, cols]) * sc)
                den = np.linalg.norm(B[sl, cols] * sc)
                assert num <= 1e-4 * den, (l, n, num / den)


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_fmm_matches_oracle(G, ctx, p):
    n, leaf = 20000, 48
    x = inputs.uniform_cube(n, 99)
    out, L = run(G, ctx, x, p=p, leaf_size=leaf)
    assert L == 3
    ref = O.fmm(x, p, leaf)["out"]
    assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM
    d = O.direct(x)
    e_or = O.rel_l2(ref[:, 1:], d[:, 1:])
    assert O.rel_l2(out[:, 1:], d[:, 1:]) <= e_or + TOL_FMM


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_m2l_tensor_cores_and_cuda_cores_agree(G, ctx, p):
    """The three M2L forms compute Eq. 4 over the same admissible pairs: the block form (one
    GEMM per parent offset on the tensor cores, the default; at this size the offsets are split
    over several CTAs per tile), the list-based tensor-core kernel (FLAG_M2L_GATHERED) and the
    FP32 CUDA-core kernel.  All match the oracle, and each other to rounding."""
    n, leaf = 30000, 16
    x = inputs.uniform_cube(n, 123 + p)
    blk, L = run(G, ctx, x, p=p, leaf_size=leaf)
    gat, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_GATHERED)
    cc, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_CUDA_CORES)
    assert L == 4
    ref = O.fmm(x, p, leaf)["out"]
    for out in (blk, gat, cc):
        assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
        assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM
    assert O.rel_l2(blk, cc) <= 5e-6
    assert O.rel_l2(gat, cc) <= 5e-6


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_m2l_rotation_matches(G, ctx, p):
    """The M2L by rotation to the translation axis (FLAG_M2L_ROTATION: rotate, coaxial
    translation, rotate back; O(p^3) per pair) computes the same Eq. 4 as the dense operators:
    outputs match the oracle and the FP32 CUDA-core M2L, local expansions per level match the
    CUDA-core ones (scaled coefficients)."""
    n, leaf = 30000, 16
    x = inputs.uniform_cube(n, 321 + p)
    rot, L = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_ROTATION)
    C = O.level_offset(L + 1)
    Lr = G.gbfmm_export_expansions(ctx, 1, C, p)
    cc, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_CUDA_CORES)
    Lcc = G.gbfmm_export_expansions(ctx, 1, C, p)
    ref = O.fmm(x, p, leaf)["out"]
    assert O.rel_l2(rot[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(rot[:, 1:], ref[:, 1:]) <= TOL_FMM
    assert O.rel_l2(rot, cc) <= 5e-6
    side = float(np.max(x[:, :3].max(0).astype(np.float64) - x[:, :3].min(0)))
    deg = np.concatenate([np.full(k + 1, k) for k in range(p)])
    for l in range(2, L + 1):
        sl = slice(O.level_offset(l), O.level_offset(l + 1))
        sc = (side / 2**l) ** (deg + 1.0)
        assert np.linalg.norm((Lr[sl] - Lcc[sl]) * sc) <= 1e-5 * np.linalg.norm(Lcc[sl] * sc), l


@pytest.mark.parametrize("p,n,leaf", [(8, 40000, 8), (10, 30000, 16), (4, 5000, 64), (6, 300000, 64)])
def test_m2l_block_local_expansions(G, ctx, p, n, leaf):
    """Local expansions after the M2L and L2L of the block form against the FP32 CUDA-core M2L,
    level by level (relative L2 of the scaled coefficients).  The cases split the 26 parent
    offsets over 4 (depth 5) and 13 or 26 (depths 3 and 4) CTAs per tile; every tree has level 2
    (one 2 x 2 x 2 parent box, 8 of the 128 MMA rows used) and level 3 (a 4 x 4 x 4 box)."""
    x = inputs.uniform_cube(n, 4242 + p)
    _, L = run(G, ctx, x, p=p, leaf_size=leaf)
    C = O.level_offset(L + 1)
    Lb = G.gbfmm_export_expansions(ctx, 1, C, p)
    _, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_CUDA_CORES)
    Lcc = G.gbfmm_export_expansions(ctx, 1, C, p)
    side = float(np.max(x[:, :3].max(0).astype(np.float64) - x[:, :3].min(0)))
    deg = np.concatenate([np.full(k + 1, k) for k in range(p)])  # degree of each complex coefficient
    for l in range(2, L + 1):
        sl = slice(O.level_offset(l), O.level_offset(l + 1))
        sc = (side / 2**l) ** (deg + 1.0)  # the scaled coefficients h^(n+1) L_n^m
        num = np.linalg.norm((Lb[sl] - Lcc[sl]) * sc)
        den = np.linalg.norm(Lcc[sl] * sc)
        assert num <= 1e-5 * den, (l, num / den)


def test_fmm_clustered_input(G, ctx):
    x = inputs.plummer(30000, 5)
    out, _ = run(G, ctx, x, p=6, leaf_size=32)
    ref = O.fmm(x, 6, 32)["out"]
    assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM


@pytest.mark.parametrize("p", [4, 8])
def test_treecode_matches_oracle(G, ctx, p):
    n, leaf = 12000, 16
    x = inputs.uniform_cube(n, 31)
    out, _ = run(G, ctx, x, p=p, leaf_size=leaf, method=G.METHOD_TREECODE)
    ref = O.fmm(x, p, leaf, method=O.TREECODE)["out"]
    assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM


def test_treecode_1m_sampled(G, ctx):
    # the treecode at full size (1,048,576 uniform particles, p = 8, leaf 64): 256 seeded targets
    # against the oracle treecode on the same tree
    n, p, leaf = 1 << 20, 8, 64
    x = inputs.uniform_cube(n, 5150)
    out, L = run(G, ctx, x, p=p, leaf_size=leaf, method=G.METHOD_TREECODE)
    assert L == 5 and np.all(np.isfinite(out))
    tg = inputs.sample_indices(n, 256, 5151)
    ref = O.fmm(x, p, leaf, method=O.TREECODE, targets=tg)["out"]
    assert O.rel_l2(out[tg, 0], ref[tg, 0]) <= TOL_FMM
    assert O.rel_l2(out[tg, 1:], ref[tg, 1:]) <= TOL_FMM


def test_small_config_p4(G, ctx):
    w = inputs.workload("uniform_4k_p4")
    x = inputs.make_particles(w["n"], w["dist"], w["seed"])
    out, L = run(G, ctx, x, p=w["p"], leaf_size=w["leaf_size"])
    assert L == 2
    ref = O.fmm(x, w["p"], w["leaf_size"])["out"]
    assert O.rel_l2(out, ref) <= TOL_FMM
    d = O.direct(x)
    assert abs(O.rel_l2(out[:, 1:], d[:, 1:]) - O.rel_l2(ref[:, 1:], d[:, 1:])) <= TOL_FMM


def test_softening_and_direct_kernel(G, ctx):
    x = inputs.uniform_cube(3000, 8)
    out, _ = run(G, ctx, x, p=6, leaf_size=64, eps2=1e-4)
    ref = O.fmm(x, 6, 64, eps2=1e-4)["out"]
    assert O.rel_l2(out, ref) <= TOL_FMM
    xd = torch.from_numpy(x).cuda()
    od = torch.empty_like(xd)
    G.gbfmm_direct(ctx, xd, xd, od, 0.0)
    torch.cuda.synchronize()
    d = O.direct(x)
    assert O.rel_l2(od.cpu().numpy(), d) <= 1e-6


def test_nonfinite_input_is_rejected(G, ctx):
    x = inputs.uniform_cube(2000, 9)
    x[17, 1] = np.nan
    prm = G.gbfmm_default_params(p=4, leaf_size=16)
    _, ws = G.gbfmm_plan(prm, len(x))
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    wsb = torch.empty(ws, dtype=torch.uint8, device="cuda")
    G.gbfmm_evaluate(ctx, prm, xd, out, wsb)
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_sync_status(ctx)
    assert ei.value.code == G.GBFMM_EINVAL
    # the context stays usable
    good, _ = run(G, ctx, inputs.uniform_cube(2000, 9), p=4, leaf_size=16)
    assert np.all(np.isfinite(good))


def test_empty_input_and_small_workspace(G, ctx):
    prm = G.gbfmm_default_params(p=4)
    e = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    G.gbfmm_evaluate(ctx, prm, e, torch.empty_like(e), torch.empty(256, dtype=torch.uint8, device="cuda"))
    x = torch.from_numpy(inputs.uniform_cube(5000, 1)).cuda()
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_evaluate(ctx, prm, x, torch.empty_like(x), torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert ei.value.code == G.GBFMM_ENOMEM


def test_host_path_and_determinism(G, ctx):
    x = inputs.uniform_cube(30000, 13)
    a, _ = run(G, ctx, x, p=8, leaf_size=32)
    b, _ = run(G, ctx, x, p=8, leaf_size=32)
    assert np.array_equal(a, b)
    prm = G.gbfmm_default_params(p=8, leaf_size=32)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    G.gbfmm_evaluate_host(ctx, prm, hin, hout)
    assert np.array_equal(hout.numpy().astype(np.float64), a)


@pytest.mark.parametrize("p,leaf", [(8, 32), (10, 64)])
def test_concurrent_near_field_equals_serial(G, ctx, p, leaf):
    """The default FMM evaluation runs P2P on a second stream beside M2L / L2L; its output is
    the serial one (all stages on the caller's stream, and the timed evaluation) bit for bit,
    and both agree with the oracle."""
    x = inputs.uniform_cube(60000, 21)
    a, _ = run(G, ctx, x, p=p, leaf_size=leaf)
    b, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_SERIAL)
    c, _ = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_STAGE_TIMING)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    for _ in range(3):  # back-to-back evaluations reuse the workspace: each waits for the last
        d, _ = run(G, ctx, x, p=p, leaf_size=leaf)
        assert np.array_equal(a, d)
    if p == 8:
        ref = O.fmm(x, p, leaf)["out"]
        assert O.rel_l2(a, ref) <= TOL_FMM


def test_stage_timing(G, ctx):
    x = inputs.uniform_cube(40000, 2)
    run(G, ctx, x, p=6, leaf_size=32, flags=G.FLAG_STAGE_TIMING)
    st = G.gbfmm_stage_times(ctx)
    assert list(st)[:9] == G.STAGES[:9]
    assert all(v >= 0 for v in st.values()) and st["P2P"] > 0


def test_large_uniform_p10_sampled(G, ctx):
    """1,048,576 uniform particles, p = 10, leaf 64 (depth 5), in the bench's launch shape:
    4096 seeded targets against the FP64 direct sum over all sources and the FP64 FMM."""
    w = inputs.workload("uniform_1m_p10")
    x = inputs.make_particles(w["n"], w["dist"], w["seed"])
    out, L = run(G, ctx, x, p=w["p"], leaf_size=w["leaf_size"])
    assert L == 5
    tg = inputs.sample_indices(w["n"], 4096, w["seed"])
    d = O.direct(x, targets=tg)
    e_phi = O.rel_l2(out[tg, 0], d[:, 0])
    e_grad = O.rel_l2(out[tg, 1:], d[:, 1:])
    assert e_grad <= 1e-4 and e_phi <= 1e-4, (e_phi, e_grad)
    sub = tg[:512]
    f = O.fmm(x, w["p"], w["leaf_size"], targets=sub)["out"]
    assert O.rel_l2(out[sub], f[sub]) <= TOL_FMM


def test_bounded_wait_reports_timeout_and_context_survives(G, ctx):
    # a wait on an mbarrier that nothing arrives on gives up after 50 ms and raises ETIMEOUT
    G.gbfmm_selftest_wait(ctx, 50.0)
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_sync_status(ctx)
    assert ei.value.code == G.GBFMM_ETIMEOUT
    G.gbfmm_sync_status(ctx)  # the status word was cleared
    x = inputs.uniform_cube(5000, 3)
    out, _ = run(G, ctx, x, p=4, leaf_size=32)
    ref = O.fmm(x, 4, 32)["out"]
    assert O.rel_l2(out, ref) <= TOL_FMM
