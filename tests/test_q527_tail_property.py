"""Property behind the Q5.27 kernels' 32-bit tail (CPU, exact integers).

For an interior cell the fixed-point update is V_c + floor((sum_d W_d (u_d -
V_c) + 2^29) / 2^30), then the BRT min with V0 and saturation to int32.
When the non-negative weights sum to at most 2^30 the kernels keep only the
low 32 bits of the shifted sum and add it to V_c modulo 2^32.  That equals the
exact result because the exact value lies between the smallest and the largest
of V_c and the u_d.  Checked here with Python integers on random and extreme
codes.
"""
import numpy as np
import pytest

I32_MIN, I32_MAX = -(2 ** 31), 2 ** 31 - 1


def exact(vc, v0, u, w):
    acc = sum(wd * (ud - vc) for wd, ud in zip(w, u)) + 2 ** 29
    vn = vc + (acc >> 30)  # Python >> on ints is floor division by 2^30
    vn = min(vn, v0)
    return max(vn, I32_MIN)


def tail32(vc, v0, u, w):
    acc = -sum(w) * vc + 2 ** 29 + sum(wd * ud for wd, ud in zip(w, u))
    inc = ((acc & (2 ** 64 - 1)) >> 30) & (2 ** 32 - 1)  # low 32 bits of the 64-bit shift
    vn = (vc + inc) & (2 ** 32 - 1)
    vn = vn - 2 ** 32 if vn >= 2 ** 31 else vn
    return min(vn, v0)


def weights(rng, total):
    cuts = np.sort(rng.integers(0, total + 1, 3))
    return [int(cuts[0]), int(cuts[1] - cuts[0]), int(cuts[2] - cuts[1]), int(total - cuts[2])]


@pytest.mark.parametrize("seed", range(4))
def test_tail32_equals_exact_update(seed):
    rng = np.random.default_rng(seed)
    extremes = [I32_MIN, I32_MIN + 1, -1, 0, 1, I32_MAX - 1, I32_MAX]
    for _ in range(4000):
        if rng.random() < 0.3:
            vals = [int(rng.choice(extremes)) for _ in range(6)]
        else:
            vals = [int(x) for x in rng.integers(I32_MIN, I32_MAX, 6, endpoint=True)]
        vc, v0, u = vals[0], vals[1], vals[2:]
        total = int(rng.choice([2 ** 30, 2 ** 30 - 1, int(rng.integers(0, 2 ** 30))]))
        w = weights(rng, total)
        assert tail32(vc, v0, u, w) == exact(vc, v0, u, w), (vc, v0, u, w)


def test_tail32_needs_the_bound():
    """Above 2^30 the exact value can leave the int32 range, so the kernels
    route such cells to the 64-bit form."""
    vc, v0, u = I32_MAX, I32_MAX, [I32_MIN] * 4
    w = [2 ** 29, 2 ** 29, 2 ** 29, 0]  # sum 1.5 * 2^30
    assert exact(vc, v0, u, w) == I32_MIN  # saturated
    assert tail32(vc, v0, u, w) != exact(vc, v0, u, w)
