"""ooc_heat7_steps_noalloc: heat7 steps without a caller-supplied scratch
field, for callers that cannot hand the library device memory (their
allocations belong to a host application's allocator, or they run in a loop
that must not allocate).  Its second field is a fixed array inside the
library.  Checked here through the C ABI against ooc_heat7_steps, which
takes the scratch field from the caller, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

from synth import sine_modes_field, smooth_random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ooc():
    import paper_2109_05410_gb300 as m
    m.build()
    m.lib()
    return m


def with_scratch(ooc, u0, nsteps):
    d = torch.from_numpy(u0).cuda()
    ooc.ooc_heat7_steps(d, torch.empty_like(d), nsteps)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def without_scratch(ooc, u0, nsteps):
    d = torch.from_numpy(u0).cuda()
    ooc.ooc_heat7_steps_noalloc(d, nsteps)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_two_calls_match_the_scratch_version(ooc):
    # First call: odd step count (result copied back from the fixed array);
    # second call right after, other shape and data, even step count.  The
    # parity tolerance of the in-core kernels against each other is exact.
    u1, _ = sine_modes_field((64, 48, 40), seed=0)
    u2 = smooth_random_field((96, 64, 128), 8.0, seed=5)
    for u0, nsteps in ((u1, 7), (u2, 4)):
        got = without_scratch(ooc, u0, nsteps)
        ref = with_scratch(ooc, u0, nsteps)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_largest_grid_and_refusal(ooc):
    n = ooc.OOC_NOALLOC_MAX_POINTS
    u0 = smooth_random_field((64, 256, 256), 16.0, seed=6)  # exactly the limit
    assert u0.size == n
    assert np.array_equal(without_scratch(ooc, u0, 3).view(np.uint32), with_scratch(ooc, u0, 3).view(np.uint32))
    too_big = torch.zeros((68, 256, 256), device="cuda")
    with pytest.raises(ooc.OocError):
        ooc.ooc_heat7_steps_noalloc(too_big, 1)
