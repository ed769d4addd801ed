"""GPU parity of the recursive (Deriche) variant, BF_FP32_RECURSIVE, against
the oracle's Algorithm 1 with the recursive blur (orc_mcsf_deriche) on the
same seeded inputs and sampled frequencies.

Tolerance, derived from the arithmetic: the FP32 recursions leave an absolute
error of ~3e-4 x (kernel weight Sum w) on the 0..255 scale in P and Z (a
float32 emulation of the same two-section recursion reproduces the GPU's
errors; in float64 it matches the oracle to 5e-9), and S = P / Z scales it by
Sum w / Re Z (measured: |error| Re Z / Sum w <= 2.7e-4).  So:
|error| <= 1e-3 max(1, 0.5 Sum w / Re Z), i.e. max-abs <= 1e-3 where
Re Z >= 0.5 Sum w; pixels with Re Z < 1e-2 Sum w (near-zero normaliser) are
excluded and counted, as for the windowed paths."""
import numpy as np
import pytest

import oracle as O
from paper_1605_02164_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def bf():
    from paper_1605_02164_gb300 import bf as _bf
    from paper_1605_02164_gb300 import build
    build.build()
    _bf.lib()
    return _bf


def _case(d, H, W, s, K, seed, sr=35.0, N=10):
    f = synth.voronoi_image(H, W, d, 6, 8.0, seed=seed)
    C = synth.spd_cond(d, seed=seed, lam_min_range=(sr ** 2, (1.2 * sr) ** 2), cond=3) if d > 1 else np.array([[sr * sr]])
    return f, C, N


def _check(bf, f, C, s, N, K, seed, tol=1e-3):
    d, H, W = f.shape
    p = bf.bf_plan(d, C, s, N, K, seed)
    x = bf.to_pitched(f)
    y = bf.filter_tensor(p, x, bf.BF_FP32_RECURSIVE)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    pl = O.plan(d, C, s, N, K, seed)
    res = O.mcsf_deriche(f.astype(np.float64), s, pl["W"], N, pl["Y"])
    one = O.deriche_blur(np.ones((H, W)), s)  # total kernel weight per pixel (Z with all phases equal)
    zr = res["Zre"] / one
    mask = zr >= 1e-2
    err = np.abs(got - res["S"])
    bound = tol * np.maximum(1.0, 0.5 / np.maximum(zr, 1e-2))
    print(f"recursive d={d} {H}x{W} s={s} K={K}: max-abs {err[:, zr >= 0.5].max():.3e} (Re Z >= 0.5 Sum w), "
          f"max err x Re Z / Sum w {(err * zr)[:, mask].max():.3e}, low-Z {(~mask).sum()}")
    assert (~mask).mean() <= 0.005
    assert np.isfinite(got[:, mask]).all()
    assert (err[:, mask] <= bound[mask]).all()
    assert bf.bf_last_status(0) == bf.BF_OK
    return got


@pytest.mark.parametrize("d,H,W,s,K", [(3, 37, 53, 2.0, 16), (3, 70, 45, 5.0, 24), (1, 33, 31, 1.5, 12),
                                       (6, 41, 29, 3.0, 12), (8, 19, 40, 4.0, 8), (3, 64, 64, 8.0, 32),
                                       (2, 1, 77, 3.0, 8), (3, 90, 1, 3.0, 8)])
def test_recursive_matches_oracle(bf, d, H, W, s, K):
    f, C, N = _case(d, H, W, s, K, seed=H * 100 + W)
    _check(bf, f, C, s, N, K, seed=991 + d)


def test_recursive_beyond_the_window_limit(bf):
    """sigma_s = 15 (r = 45 > BF_MAX_RADIUS): the plan is accepted, the windowed
    variants refuse it, the recursive one filters it (its cost does not grow)."""
    f, C, N = _case(3, 60, 75, 15.0, 16, seed=5)
    p = bf.bf_plan(3, C, 15.0, N, 16, 7)
    assert p.r == 45
    x = bf.to_pitched(f)
    for v in (bf.BF_FP32, bf.BF_FP16TC):
        with pytest.raises(bf.BFError) as e:
            bf.filter_tensor(p, x, v)
        assert e.value.code == bf.BF_ERR_UNSUPPORTED
    _check(bf, f, C, 15.0, N, 16, seed=7)


def test_recursive_batch_equals_single_and_is_deterministic(bf):
    items, outs, keep = [], [], []
    for i, (H, W, s) in enumerate([(40, 33, 2.0), (25, 64, 6.0), (50, 50, 3.5)]):
        f, C, N = _case(3, H, W, s, 8, seed=40 + i)
        p = bf.bf_plan(3, C, s, N, 8, 100 + i)
        x = bf.to_pitched(f)
        y1 = bf.filter_tensor(p, x, bf.BF_FP32_RECURSIVE)
        y2 = bf.pitched_empty(3, H, W)
        items.append((p, x.data_ptr(), y2.data_ptr(), H, W, x.stride(1)))
        outs.append((y1, y2))
        keep.append(x)
    bf.bf_filter_batch(items, bf.BF_FP32_RECURSIVE, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for y1, y2 in outs:
        assert torch.equal(y1, y2)
    assert bf.bf_last_status(0) == bf.BF_OK
