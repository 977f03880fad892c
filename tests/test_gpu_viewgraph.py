"""Viewgraph estimation on the GPU (Section 3, Eq. 2; Algorithm 1 BuildViewgraph) against the
oracle: the round-trip fractions of every ordered pair are ratios of integer counts taken
with the same FP64 arithmetic in the same order, so they are compared exactly, as are the
kept pairs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402


@pytest.mark.parametrize("preset,stride,which", [("RING8_128x96", 1, "T_gt"), ("RING8_128x96", 3, "T_init"),
                                                 ("RING32_518x392", 6, "T_init")])
def test_viewgraph_matches_oracle(preset, stride, which):
    sc = synth.make_scene(getattr(synth, preset), keep_depth=True)
    T = getattr(sc, which)
    frac, pairs = epo.build_viewgraph(sc.W, sc.H, sc.K, T, [torch.from_numpy(d).cuda() for d in sc.depth],
                                      stride=stride, tau=3.0, min_frac=0.125)
    want = oracle.viewgraph(sc.W, sc.H, sc.K, T, sc.depth, stride=stride, tau=3.0)
    assert np.array_equal(frac, want)
    assert np.array_equal(pairs, oracle.viewgraph_pairs(want, 0.125))
    assert 0 < len(pairs) <= sc.n_views * (sc.n_views - 1)


def test_viewgraph_argument_checks():
    d = torch.zeros(16, device="cuda")
    with pytest.raises(epo.EpoError):
        epo.build_viewgraph([4], [4], [[0.0, 1.0, 1.5, 1.5]], np.eye(4)[:3].reshape(1, 12), d)
