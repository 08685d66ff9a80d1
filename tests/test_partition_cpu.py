"""The work partition of the small-state and per-IVP batch kernels, checked
on the host: the steps [0, n) of one solve (or one IVP) are dealt out to T
threads by work weight, a regular step (index < sfill) weighing kw fill
steps, each thread one contiguous range [k0, k1) split at kreg into its
regular and fill parts.  The kernels derive every range from (n, sfill, T)
alone, so the ranges must tile [0, n) in thread order, the regular parts
[0, sfill) and the fill parts [sfill, n), with no thread's weight above the
per-thread share (csrc/batch.cu, csrc/newton_small.cuh)."""
import pytest


def ranges(n, sfill, T, kw):
    wreg = kw * sfill
    wtot = wreg + (n - sfill)
    per = (wtot + T - 1) // T
    out = []
    for t in range(T):
        w0, w1 = t * per, t * per + per
        k0 = min(n, (w0 + kw - 1) // kw if w0 <= wreg else sfill + (w0 - wreg))
        k1 = min(n, (w1 + kw - 1) // kw if w1 <= wreg else sfill + (w1 - wreg))
        kreg = min(k1, max(k0, sfill))
        out.append((k0, kreg, k1))
    return out, per


@pytest.mark.parametrize("kw", [4, 16, 64])
@pytest.mark.parametrize("T", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 257, 1000, 8191, 65536])
def test_partition_tiles_the_steps(n, T, kw):
    for sfill in sorted({1, 2, n // 3 or 1, n - 1 if n > 1 else 1, n}):
        rs, per = ranges(n, sfill, T, kw)
        pos = 0
        for k0, kreg, k1 in rs:
            assert k0 == pos and k0 <= kreg <= k1 <= n
            assert kreg == k0 or kreg <= sfill         # regular part below sfill
            assert kreg == k1 or kreg >= sfill         # fill part from sfill on
            # a thread's weight stays within one share (up to the rounding
            # of the range boundary to a whole regular step)
            assert kw * (kreg - k0) + (k1 - kreg) <= per + kw
            pos = k1
        assert pos == n
