"""CPU oracle pinned to the paper and to mathematics (no GPU).

Sec. III-A of the paper defines membership by the crossing-number test
(ray to +x, odd = inside, concave and multiply-connected polygons allowed);
Appendix A's findCensusBlock lets the first containing polygon claim a point.
The checks live in oracle_pins.py; this file runs them on the oracle and on
copies of the oracle with a planted mistake, each of which must be caught.
"""
import os

import numpy as np
import pytest

import oracle
from tests import oracle_pins as pins

HERE = os.path.dirname(os.path.abspath(__file__))


def test_quantize_exact_rationals():
    pins.check_quantize(oracle, np.random.default_rng(7))


def test_crossing_rule_matches_perturbed_textbook_test():
    pins.check_perturbation(oracle, np.random.default_rng(8))


def test_fan_and_shared_edges_one_owner():
    pins.check_fans(oracle)


def test_rectangle_closed_form():
    pins.check_rectangles(oracle, np.random.default_rng(9))


def test_unit_square_grid():
    pins.check_unit_grid(oracle)


def test_convex_half_planes():
    pins.check_convex(oracle, np.random.default_rng(10))


def check_overlap(orc):
    """Appendix A: the first (lowest-index) containing polygon claims the
    point; overlapping squares -> the lower id wins in the overlap."""
    a = [[(0, 0), (6, 0), (6, 6), (0, 6)]]
    b = [[(3, 3), (9, 3), (9, 9), (3, 9)]]
    for order, ids in (([a, b], (0, 1)), ([b, a], (1, 0))):
        ps = pins.poly_set(order)
        X, Y = np.meshgrid(np.arange(-1, 11), np.arange(-1, 11), indexing="ij")
        X, Y = X.ravel(), Y.ravel()
        got = orc.join_bruteforce_q(ps, X, Y)
        in_a = (X >= 0) & (X < 6) & (Y >= 0) & (Y < 6)
        in_b = (X >= 3) & (X < 9) & (Y >= 3) & (Y < 9)
        ia, ib = ids
        want = np.full(X.shape, -1)
        want[in_b] = ib
        want[in_a & (~in_b | (ia < ib))] = ia
        assert (got == want).all()
        lon, lat = X / 1e7, Y / 1e7
        assert (orc.join_hier(ps, lon, lat) == want).all()


def test_overlap_lowest_index_claims():
    check_overlap(oracle)


def test_tiny_partition_invariant(tiny_set):
    pins.check_partition(oracle, tiny_set, 20000, np.random.default_rng(11))


def test_partition_with_holes(tiny_set_holes):
    ps = tiny_set_holes
    assert ps.meta["n_islands"] > 10
    pins.check_partition(oracle, ps, 20000, np.random.default_rng(12))
    # points at the hole vertices belong to exactly one of host / island
    hosts = np.nonzero(np.diff(ps.poly_ring_off) == 2)[0]
    assert len(hosts) == ps.meta["n_islands"]


def test_o0_equals_o1_tiny(tiny_set):
    from synth import configs, degenerate_lattice, lattice_to_degrees
    lon, lat = configs.tiny_points(tiny_set, n=30000)
    pins.check_o0_o1(oracle, tiny_set, lon, lat)
    qx, qy = degenerate_lattice(tiny_set, 6000, np.random.default_rng(13))
    pins.check_o0_o1(oracle, tiny_set, lattice_to_degrees(qx), lattice_to_degrees(qy))


def test_o0_equals_o1_holes(tiny_set_holes):
    from synth import degenerate_lattice, lattice_to_degrees
    qx, qy = degenerate_lattice(tiny_set_holes, 6000, np.random.default_rng(14))
    pins.check_o0_o1(oracle, tiny_set_holes, lattice_to_degrees(qx), lattice_to_degrees(qy))


def read_paper_bboxes():
    rows = {}
    with open(os.path.join(HERE, "golden", "paper_bboxes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals[:4]] + [int(vals[4])]
    return rows


def test_paper_bboxes_fit_lattice_and_nest():
    """Sec. III-B prints MA, Middlesex County and an MIT block group with
    boxes [x_min x_max y_min y_max]; on the 1e-7 degree lattice they are exact
    integers, nest (block in county in state) and are filters that keep the
    box's own lower-left corner."""
    rows = read_paper_bboxes()
    q = {}
    for name, (x0, x1, y0, y1, nv) in rows.items():
        qq, ok = oracle.quantize([x0, x1, y0, y1])
        assert ok.all()
        assert [int(v) for v in qq] == [round(v * 10000) * 1000 for v in (x0, x1, y0, y1)]
        assert qq[0] < qq[1] and qq[2] < qq[3]
        q[name] = [int(v) for v in qq]
    ma, mx, mit = q["massachusetts"], q["middlesex_county"], q["mit_block_group"]
    for outer, inner in ((ma, mx), (mx, mit)):
        assert outer[0] <= inner[0] and inner[1] <= outer[1]
        assert outer[2] <= inner[2] and inner[3] <= outer[3]
    # the three boxes as rectangles in a 3-level hierarchy: the MIT box's
    # lower-left corner is in all three; the lowest index claims it.
    rect = lambda b: [[(b[0], b[2]), (b[1], b[2]), (b[1], b[3]), (b[0], b[3])]]
    ps = pins.poly_set([rect(mit), rect(mx), rect(ma)])
    lon = np.array([mit[0], mit[1], ma[0], ma[1]]) / 1e7
    lat = np.array([mit[2], mit[2], ma[2], ma[3]]) / 1e7
    got = oracle.join_hier(ps, lon, lat)
    assert list(got) == [0, 1, 2, -1]


MUTANTS = {
    "on_edge_counts": ("if (s == 0) return 0;", "if (s == 0) return 1;"),
    "sign_flip": ("return (s > 0) == (by > ay);", "return (s < 0) == (by > ay);"),
    "right_early_out_closed": ("if (std::min(ax, bx) > px) return 1;",
                               "if (std::min(ax, bx) >= px) return 1;"),
    "closed_y_rule": ("if ((ay > py) == (by > py)) return 0;",
                      "if ((ay >= py) == (by >= py)) return 0;"),
    "no_closing_edge": ("const int64_t j = (i == last) ? first : i + 1;",
                        "if (i == last) break;\n      const int64_t j = i + 1;"),
    "first_ring_only": ("for (int64_t r = s.poly_ring_off[p]; r < s.poly_ring_off[p + 1]; ++r) {",
                        "for (int64_t r = s.poly_ring_off[p]; r < s.poly_ring_off[p] + 1; ++r) {"),
    "q_ties_away": ("if (rest > half || (rest == half && (whole & 1))) whole += 1;",
                    "if (rest >= half) whole += 1;"),
    "q_range_off_by_one": ("if (whole > (u128)INT32_MAX) return 0;",
                           "if (whole > (u128)INT32_MAX + 1) return 0;"),
    "strict_filter_box": ("return x_min <= px && px <= x_max && y_min <= py && py <= y_max;",
                          "return x_min < px && px < x_max && y_min < py && py < y_max;"),
    "highest_index_claims": ("std::sort(cand.begin(), cand.end());",
                             "std::sort(cand.rbegin(), cand.rend());"),
    "parity_or": ("parity ^= edge_crossing(s.vx[i], s.vy[i], s.vx[j], s.vy[j], px, py);",
                  "parity |= edge_crossing(s.vx[i], s.vy[i], s.vx[j], s.vy[j], px, py);"),
    "transposed_orientation": ("const i128 s = (i128)(bx - ax) * (py - ay) - (i128)(by - ay) * (px - ax);",
                               "const i128 s = (i128)(bx - ax) * (px - ax) - (i128)(by - ay) * (py - ay);"),
    "q_truncates": ("if (rest > half || (rest == half && (whole & 1))) whole += 1;",
                    "(void)rest;"),
    "last_vertex_skipped": ("for (int64_t i = first; i <= last; ++i) {",
                            "for (int64_t i = first; i < last; ++i) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tiny_set_holes):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    mut = oracle.load_variant(src.replace(old, new), name)
    from synth import degenerate_lattice, lattice_to_degrees
    qx, qy = degenerate_lattice(tiny_set_holes, 3000, np.random.default_rng(15))
    checks = [
        lambda: pins.check_quantize(mut, np.random.default_rng(7)),
        lambda: pins.check_perturbation(mut, np.random.default_rng(8), n_poly=60),
        lambda: pins.check_rectangles(mut, np.random.default_rng(9), n=20),
        lambda: pins.check_unit_grid(mut),
        lambda: check_overlap(mut),
        lambda: pins.check_o0_o1(mut, tiny_set_holes, lattice_to_degrees(qx), lattice_to_degrees(qy)),
    ]
    caught = 0
    for c in checks:
        try:
            c()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"mutant {name} passed every pin"
