"""Video denoising (spatio-temporal grouping, reading R16) through the C ABI against the oracle:
global group indices bit-exact, pixels within 1e-3, per-frame sigma estimates within 1e-9."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, max_abs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


def _clip(F, Hh, Ww, C, seed, sigma):
    """Synthetic clip: one clean frame drifting by a pixel per frame, fresh noise in every frame."""
    clean = synth.clean_image(Hh, Ww + F, C, seed)
    return np.stack([synth.add_gaussian(np.ascontiguousarray(clean[:, t:t + Ww]), sigma, seed + 31 * t)
                     for t in range(F)])


@pytest.mark.parametrize("F,shape,prm,T,sigma", [
    (3, (48, 40, 3), dict(ps=8, stride=3, window=11, K=8), 1, 20.0),
    (4, (40, 36, 1), dict(ps=8, stride=2, window=9, K=8), 2, 25.0),
    (3, (44, 52, 3), dict(ps=8, stride=3, window=9, K=16, match_mode="full"), 1, 15.0),
    (2, (40, 40, 3), dict(ps=8, stride=3, window=13, K=32), 1, 30.0),
    # sigma estimated per frame (18 x 19 = 342 references: a full-rank 192 x 192 covariance)
    (3, (57, 62, 3), dict(ps=8, stride=3, window=9, K=8), 1, None),
])
def test_video_matches_oracle(F, shape, prm, T, sigma):
    clip = _clip(F, *shape, seed=500 + F, sigma=20.0 if sigma is None else sigma)
    ref, res = O.denoise_video(clip, sigma, prm, T=T)
    out, info = H.denoise_video(torch.from_numpy(clip).cuda(), sigma, prm, T=T, return_info=True)
    torch.cuda.synchronize()
    idx = info["idx"].cpu().numpy()
    for t in range(F):
        np.testing.assert_array_equal(idx[t].astype(np.int64), res[t].idx)
        if sigma is None:
            assert info["sigmas"][t] == pytest.approx(res[t].extra["sigma"], rel=1e-9, abs=1e-9)
    err = max_abs(out.cpu().numpy(), ref)
    assert err <= PIX_TOL, f"max abs pixel error {err}"


def test_video_without_temporal_search_equals_per_frame_calls():
    clip = _clip(3, 40, 48, 3, seed=77, sigma=20.0)
    prm = dict(ps=8, stride=3, window=11, K=16)
    v = torch.from_numpy(clip).cuda()
    out = H.denoise_video(v, 20.0, prm, T=0)
    for t in range(3):
        single = H.denoise(v[t], 20.0, prm)
        assert torch.equal(out[t], single)
