"""Pins of the whole oracle evaluation: direct-sum invariants and FMM/treecode convergence."""
import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs


def test_direct_two_particles_closed_form():
    x = np.array([[0, 0, 0, 2.0], [3, 4, 0, 5.0]], dtype=np.float32)
    out = O.direct(x)
    assert out[0, 0] == 5.0 / 5.0 and out[1, 0] == 2.0 / 5.0
    # grad_0 = -q_1 (x_0 - x_1) / r^3
    assert np.allclose(out[0, 1:], -5.0 * np.array([-3, -4, 0]) / 125.0, rtol=1e-15)


def test_direct_newtons_third_law():
    x = inputs.uniform_cube(1500, 21)
    out = O.direct(x)
    q = x[:, 3].astype(np.float64)
    net = (q[:, None] * out[:, 1:]).sum(axis=0)
    scale = np.abs(q[:, None] * out[:, 1:]).sum()
    assert np.all(np.abs(net) < 1e-14 * scale)
    # sum_i q_i phi_i is the same in i-major and j-major order
    xs = x.astype(np.float64)
    d = np.linalg.norm(xs[:, None, :3] - xs[None, :, :3], axis=2)
    np.fill_diagonal(d, np.inf)
    assert np.sum(q * out[:, 0]) == pytest.approx(np.sum(q[None, :] * q[:, None] / d), rel=1e-13)


def test_duplicate_points_and_softening():
    x = np.array([[0.5, 0.5, 0.5, 1.0], [0.5, 0.5, 0.5, 2.0], [0.5, 0.5, 1.5, 3.0]], dtype=np.float32)
    out = O.direct(x)
    assert out[0, 0] == 3.0 and out[1, 0] == 3.0  # coincident pair skipped
    soft = O.direct(x, eps2=3.0)
    assert soft[0, 0] == pytest.approx(3.0 / 2.0)


def test_power_of_two_scaling_is_exact():
    x = inputs.uniform_cube(700, 4)
    y = x.copy()
    y[:, :3] *= 4.0
    a, b = O.direct(x), O.direct(y)
    assert np.array_equal(b[:, 0], a[:, 0] / 4.0)
    assert np.array_equal(b[:, 1:], a[:, 1:] / 16.0)
    ta, tb = O.build_tree(x, 8), O.build_tree(y, 8)
    assert np.array_equal(ta["keys"], tb["keys"])
    fa, fb = O.fmm(x, 6, 8)["out"], O.fmm(y, 6, 8)["out"]
    assert np.allclose(fb[:, 0], fa[:, 0] / 4.0, rtol=1e-12)
    assert np.allclose(fb[:, 1:], fa[:, 1:] / 16.0, rtol=1e-11, atol=1e-12 * np.abs(fa[:, 1:]).max() / 16)


@pytest.mark.parametrize("method", [O.FMM, O.TREECODE])
@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_error_falls_with_p(method, dist):
    x = inputs.make_particles(1800, dist, 17)
    ref = O.direct(x)
    errs = []
    for p in (2, 4, 6, 8, 10):
        out = O.fmm(x, p, 8, method=method)["out"]
        assert O.fmm(x, p, 8, method=method)["L"] == 3
        errs.append(O.rel_l2(out[:, 1:], ref[:, 1:]))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    if dist == "uniform":
        assert errs[-1] < 1e-4


def test_shallow_tree_is_the_direct_sum():
    # L < 2: no well-separated cells, so the evaluation is pure P2P
    x = inputs.uniform_cube(400, 9)
    r = O.fmm(x, 4, 64)
    assert r["L"] == 1
    ref = O.direct(x)
    assert np.allclose(r["out"], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_target_subset_matches_full_evaluation():
    x = inputs.uniform_cube(3000, 12)
    tg = inputs.sample_indices(3000, 100, 5)
    full = O.fmm(x, 6, 16)["out"]
    part = O.fmm(x, 6, 16, targets=tg)["out"]
    assert np.array_equal(full[tg], part[tg])


def test_small_config_p4_vs_direct():
    # the 4,096-particle p=4 workload (L=2): error level fixed by the truncation
    w = inputs.workload("uniform_4k_p4")
    x = inputs.make_particles(w["n"], w["dist"], w["seed"])
    ref = O.direct(x)
    r = O.fmm(x, w["p"], w["leaf_size"])
    assert r["L"] == 2
    e_phi = O.rel_l2(r["out"][:, 0], ref[:, 0])
    e_grad = O.rel_l2(r["out"][:, 1:], ref[:, 1:])
    assert e_phi < 1e-3 and e_grad < 1e-2
