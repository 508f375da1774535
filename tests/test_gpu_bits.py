"""The integer-pipe helpers of the stage kernel, on the GPU, against plain
definitions evaluated with numpy: halving and quartering on the exponent field,
half the MC-limited slope from the two differences, the sign test and the
bit-pattern min / max (gbh_bits_selftest).  Inputs cover both signs, zeros of
both signs, subnormals, ties of magnitude and the whole exponent range."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TINY = 2.0 ** -1020     # below this the exponent-field scalings shift the bit pattern


@pytest.fixture(scope="module")
def gb():
    import paper_2401_03378_gb300 as gb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gb


def inputs():
    rng = np.random.default_rng(31)
    n = 200000
    sx = rng.choice([-1.0, 1.0], n)
    sy = rng.choice([-1.0, 1.0], n)
    x = sx * 10.0 ** rng.uniform(-300, 300, n)
    y = sy * 10.0 ** rng.uniform(-300, 300, n)
    # differences of comparable size (where the MC limiter's three candidates compete)
    m = 100000
    a = rng.uniform(-1.0, 1.0, m)
    b = a * rng.uniform(-4.0, 4.0, m)
    ties = np.array([1.0, 1.0, 2.0, -3.0, -3.0, 0.5, 4.0, 0.25])
    tie_y = np.array([1.0, -1.0, 0.5, -0.75, 3.0, 0.5, 1.0, 1.0])
    special_x = np.array([0.0, -0.0, 0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308,
                          -2.2250738585072014e-308, 1e-310, 3.0 * 2.0 ** -1022, 1.0, -1.0, 1e300, -1e300])
    special_y = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, 1e-310, 1.0, -1.0, -1e-310, 2.0 ** -1021,
                          0.0, -0.0, 1e299, -1e299])
    return (np.concatenate([x, a, ties, special_x]), np.concatenate([y, b, tie_y, special_y]))


def test_integer_pipe_helpers(gb):
    x, y = inputs()
    n = len(x)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    out = torch.empty(6 * n, dtype=torch.float64, device="cuda")
    lib = gb.load()
    assert lib.gbh_bits_selftest(xd.data_ptr(), yd.data_ptr(), out.data_ptr(), n,
                                 torch.cuda.current_stream().cuda_stream) == 0
    o = out.cpu().numpy().reshape(6, n)

    # x / 2 and x / 4: exact where the result is normal (>= 2^-1022 in magnitude),
    # else within one unit of the smallest subnormal
    for row, f in ((0, 0.5), (1, 0.25)):
        ref = x * f
        normal = np.abs(ref) >= 2.0 ** -1022
        assert np.array_equal(o[row][normal], ref[normal])
        assert np.all(np.abs(o[row][~normal] - ref[~normal]) <= 2.0 ** -1022)
        assert np.array_equal(np.signbit(o[row][x != 0]), np.signbit(x[x != 0]))

    # half the MC slope: sign(dp) min(|dm+dp|/4, |dm|, |dp|) for dm, dp of the same
    # strict sign, else 0; exact away from the subnormal range
    dm, dp = x, y
    with np.errstate(over="ignore"):
        s = dm + dp
        cand = np.minimum(np.minimum(np.abs(s) / 4.0, np.abs(dm)), np.abs(dp))
    same = (np.sign(dm) * np.sign(dp)) > 0
    ref = np.where(same, np.copysign(cand, dp), 0.0)
    finite = np.isfinite(s) & (np.abs(dm) < 1e300) & (np.abs(dp) < 1e300)
    exact = finite & ((cand >= TINY) | ~same)
    assert np.array_equal(o[2][exact], ref[exact])
    near = finite & ~exact
    assert np.all(np.abs(o[2][near] - ref[near]) <= 2.0 ** -1020)
    assert np.all(o[2][~same] == 0.0)

    # x >= 0, with -0 counted as >= 0
    assert np.array_equal(o[3], (x >= 0).astype(np.float64))

    # min / max in numeric order (values; the order of -0 and +0 is unspecified)
    assert np.all(o[4] == np.minimum(x, y)) and np.all(o[5] == np.maximum(x, y))
