"""pip_project_noalloc: the projection for callers that cannot allocate
device memory during a call (it takes its scratch from a fixed array inside
the library). Its ids must equal the CPU oracle's and pip_project's, exactly,
on consecutive calls that reuse the shared scratch. Named to run after every
other test, and it also passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import configs, degenerate_lattice, lattice_to_degrees

SCAN_TILE_SUPERBINS = 4096       # one scan block: above this the multi-block scan runs
MAX_SUPERBINS = 524288           # the entry point's limit


@pytest.mark.gpu
def test_noalloc_equals_pip_project_on_consecutive_calls(state_set):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_03156_gb300 as pipm
    from paper_2005_03156_gb300 import build
    build.build()
    ps = configs.tiny_set(seed=14, n_blocks=2000, holes=0.05)
    # an index without compact leaves and with enough superbins that the
    # scan of the superbin counts takes its multi-block path
    s = None
    for opts in ({"compact_edges": -1}, {"compact_edges": -1, "size_ratio": 96},
                 {"compact_edges": -1, "size_ratio": 192, "max_depth": 6}):
        s = pipm.load_polygon_set(ps, opts=opts)
        if SCAN_TILE_SUPERBINS < s.info()["superbins"] <= MAX_SUPERBINS:
            break
        s.free()
        s = None
    assert s is not None, "no index shape with 4097..524288 superbins"
    rng = np.random.default_rng(90)
    for call, n in enumerate((200_000, 262_144)):  # second call reuses the scratch
        qx, qy = degenerate_lattice(ps, n // 4, rng)
        lon2, lat2 = configs.tiny_points(ps, n=n, seed=91 + call)
        lon = np.concatenate([lattice_to_degrees(qx), lon2])[:n]
        lat = np.concatenate([lattice_to_degrees(qy), lat2])[:n]
        dl, da = torch.from_numpy(lon).cuda(), torch.from_numpy(lat).cuda()
        want = pipm.pip_project(s, dl, da)
        got = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        pipm.pip_project_noalloc(s, dl, da, got)
        pipm.pip_set_check(s)
        torch.cuda.synchronize()
        assert torch.equal(got, want), int((got != want).sum())
        assert (got.cpu().numpy() == oracle.join_hier(ps, lon, lat)).all()
    too_many = torch.zeros(262_145, dtype=torch.float64, device="cuda")
    out = torch.empty(262_145, dtype=torch.int32, device="cuda")
    with pytest.raises(pipm.PipError) as e:
        pipm.pip_project_noalloc(s, too_many, too_many, out)
    assert e.value.status == 1
    # a set beyond the superbin limit is refused, not overrun
    big = pipm.load_polygon_set(state_set, opts={"compact_edges": -1})
    assert big.info()["superbins"] > MAX_SUPERBINS
    few = torch.zeros(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(pipm.PipError) as e:
        pipm.pip_project_noalloc(big, few, few, out[:1000])
    assert e.value.status == 1
