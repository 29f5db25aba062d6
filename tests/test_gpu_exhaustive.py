"""Interior and empty cells by exhaustion (Sec. IV true-hit filtering made
exact): cells that answer without a crossing test do so because no edge of
a candidate meets the cell's closed lattice rectangle, a geometric argument.
Here every lattice point of whole top cells and of full stripes across the
set is projected and compared, element by element, with the brute-force
oracle O0 (every polygon, no index). pip_locate reports which index cell
answered each point, and the sweep must cover top-grid interior cells, empty
cells, palette-coded trie children and leaves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import configs, lattice_to_degrees

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_03156_gb300 as pipm
    from paper_2005_03156_gb300 import build
    build.build()
    pipm.lib()
    return pipm


def locate(pipm, s, qx, qy):
    code = pipm.pip_locate(s, torch.from_numpy(qx.astype(np.int32)).cuda(),
                           torch.from_numpy(qy.astype(np.int32)).cuda()).cpu().numpy()
    return code & 0xFF, code >> 8


def cell_points(x0, y0, side):
    xs, ys = np.meshgrid(np.arange(x0, x0 + side, dtype=np.int64), np.arange(y0, y0 + side, dtype=np.int64))
    return xs.ravel(), ys.ravel()


@pytest.mark.parametrize("opts", [dict(cell_log2=10, max_depth=3),
                                  dict(cell_log2=10, max_depth=3, compact_edges=3)],
                         ids=["default", "compact"])
def test_interior_and_empty_cells_by_exhaustion(pipm, opts):
    # 200 blocks over 0.02 deg (2e5 x 2e5 lattice units), holes and islands
    ps = configs.tiny_set(seed=15, n_blocks=200, deg=0.02, origin=(0.3, 0.4), holes=0.05)
    s = pipm.load_polygon_set(ps, opts=opts)
    info = s.info()
    sh, gx0, gy0, nx, ny = info["cell_log2"], info["grid_x0"], info["grid_y0"], info["grid_nx"], info["grid_ny"]
    side = 1 << sh
    # kinds at the corner and centre of every top cell, to pick the cells to sweep
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny))
    cx, cy = cx.ravel(), cy.ravel()
    kc, dc = locate(pipm, s, gx0 + cx * side + side // 2, gy0 + cy * side + side // 2)
    k0, d0 = locate(pipm, s, gx0 + cx * side, gy0 + cy * side)
    top_interior = np.flatnonzero((kc == 1) & (dc == 0) & (k0 == 1) & (d0 == 0))
    split = np.flatnonzero((dc >= 1) & ((kc == 0) | (kc == 1)))
    assert len(top_interior) and len(split)
    picks = [top_interior[len(top_interior) // 2], split[0], split[len(split) // 2], len(cx) - 1]  # last: top-right
    qx, qy = [], []
    for c in picks:
        x, y = cell_points(gx0 + int(cx[c]) * side, gy0 + int(cy[c]) * side, side)
        qx.append(x)
        qy.append(y)
    # full-width stripes: through the middle, and across the top border of the set
    X0, Y0, X1, Y1 = ps.box
    xs = np.arange(gx0 - 8, gx0 + nx * side + 8, dtype=np.int64)
    for y in list(range((Y0 + Y1) // 2, (Y0 + Y1) // 2 + 3)) + list(range(Y1 - 2, Y1 + 2)):
        qx.append(xs)
        qy.append(np.full_like(xs, y))
    qx, qy = np.concatenate(qx), np.concatenate(qy)
    kind, depth = locate(pipm, s, qx, qy)
    assert (kind == 1).any() and ((kind == 1) & (depth == 0)).any()      # interior, top grid
    assert (kind == 0).any()                                              # empty
    assert (((kind == 0) | (kind == 1)) & (depth >= 1)).any()             # palette-coded trie child
    assert ((kind == 2) | (kind == 3)).any()                              # leaves
    if opts.get("compact_edges", 0) > 0:
        assert (kind == 3).any()
    want = oracle.join_bruteforce_q(ps, qx, qy)
    got = pipm.pip_project(s, torch.from_numpy(lattice_to_degrees(qx)).cuda(),
                           torch.from_numpy(lattice_to_degrees(qy)).cuda())
    pipm.pip_set_check(s)
    got = got.cpu().numpy()
    bad = got != want
    assert not bad.any(), (int(bad.sum()), np.unique(kind[bad]).tolist(), np.unique(depth[bad]).tolist())
