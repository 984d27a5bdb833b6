"""The FP32 form's offset-to-cell renormalization, bit for bit.

After the move (Eq. coordscheme, Appendix step 2c) the FP32 form stores each
position as an int32 cell and a float offset.  The library's rule: moving
offset o by d gives the shift k = floor(o + d) and the offset nearest (in
float, ties to even) to the exact o + d - k, with an offset that rounds to 1
becoming offset 0 of the next cell.  A double-precision renormalization of the
same float inputs, rounded once to float, gives the same pair; the GPU's
single-precision evaluation (two error-free sums and one rounding) must equal
both, through pic_renormalize_f32, which runs the device function of the FP32
particle kernels.  Cases: random moves, offsets within a few ulps of 0 and 1,
moves that land within ulps of a face from either side, exact ties, and face
crossings in both directions."""
import math
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic, torch


def nearest_f32(x):
    """The float32 nearest to the rational x, ties to the even significand."""
    f = np.float32(float(x))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = None
    for c in cands:
        err = abs(Fraction(float(c)) - x)
        key = (err, int(np.array(c, dtype=np.float32).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def exact_rule(o, d):
    v = Fraction(float(o)) + Fraction(float(d))
    k = math.floor(v)
    r = nearest_f32(v - k)
    if r == np.float32(1.0):
        k, r = k + 1, np.float32(0.0)
    return k, r


def fp64_rule(o, d):
    s = np.float64(o) + np.float64(d)
    k = math.floor(s)
    r = np.float32(s - k)
    if r == np.float32(1.0):
        k, r = k + 1, np.float32(0.0)
    return k, r


def cases():
    rng = np.random.default_rng(20110110)
    f = np.float32
    o_rand = rng.random(20000).astype(np.float32)
    d_rand = rng.uniform(-0.95, 0.95, 20000).astype(np.float32)
    one_minus = [np.nextafter(f(1.0), f(0.0))]
    for _ in range(3):
        one_minus.append(np.nextafter(one_minus[-1], f(0.0)))
    tiny = [f(0.0), f(2.0 ** -149), f(2.0 ** -126), f(2.0 ** -30), f(2.0 ** -24), f(2.0 ** -23), f(3 * 2.0 ** -24)]
    o_special = tiny + one_minus + [f(0.5), np.nextafter(f(0.5), f(0.0)), f(0.25), f(0.75)]
    d_special = [f(0.0), f(2.0 ** -25), f(-2.0 ** -25), f(2.0 ** -24), f(-2.0 ** -24), f(2.0 ** -40), f(-2.0 ** -40),
                 f(1e-7), f(-1e-7), f(0.3), f(-0.3), f(0.9), f(-0.9), np.nextafter(f(1.0), f(0.0)),
                 -np.nextafter(f(1.0), f(0.0))]
    os_, ds = list(o_rand), list(d_rand)
    for o in o_special:
        for d in d_special:
            os_.append(o)
            ds.append(d)
        # moves that land on the faces and a few ulps either side of them
        for target in (f(0.0), f(1.0), f(-1.0 + 2.0 ** -23), f(2.0 - 2.0 ** -23)):
            d0 = np.float32(np.float64(target) - np.float64(o))
            for step in range(-3, 4):
                d = d0
                for _ in range(abs(step)):
                    d = np.nextafter(d, f(np.inf) if step > 0 else f(-np.inf))
                if abs(float(d)) < 1.0:
                    os_.append(o)
                    ds.append(d)
    # face crossings of random particles, both directions
    for _ in range(2000):
        o = f(rng.random())
        d = f((1.0 - float(o)) + rng.uniform(0, 0.5)) if rng.random() < 0.5 else f(-float(o) - rng.uniform(1e-6, 0.5))
        if abs(float(d)) < 1.0:
            os_.append(o)
            ds.append(d)
    return np.array(os_, dtype=np.float32), np.array(ds, dtype=np.float32)


def test_fp32_renormalization_equals_fp64_renormalization_rounded_once(env):
    P, torch = env
    o, d = cases()
    assert np.all((o >= 0) & (o < 1)) and np.all(np.abs(d) < 1)
    dev = torch.device("cuda", 0)
    to = torch.from_numpy(o).to(dev)
    td = torch.from_numpy(d).to(dev)
    shift = torch.empty(o.size, dtype=torch.int32, device=dev)
    out = torch.empty(o.size, dtype=torch.float32, device=dev)
    P.pic_renormalize_f32(to, td, shift, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    k_gpu = shift.cpu().numpy()
    r_gpu = out.cpu().numpy()
    crossings = 0
    for p in range(o.size):
        k, r = exact_rule(o[p], d[p])
        k64, r64 = fp64_rule(o[p], d[p])
        assert (k64, r64.view(np.uint32)) == (k, r.view(np.uint32)), (o[p], d[p])
        assert k_gpu[p] == k and r_gpu[p].view(np.uint32) == r.view(np.uint32), \
            f"o={o[p]!r} d={d[p]!r}: GPU ({k_gpu[p]}, {r_gpu[p]!r}), FP64 rounded once ({k}, {r!r})"
        assert 0.0 <= r_gpu[p] < 1.0
        crossings += k != 0
    assert crossings > 2000
