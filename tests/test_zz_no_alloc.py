"""tds_find_pair_contacts_noalloc against the contact search of tds_step.

The entry point serves callers that cannot let a library allocate device
memory (a simulator stepping in a fixed-rate real-time loop, where an
allocation can synchronize the device and miss the frame, or an application
whose device memory belongs to its own fixed-budget pool): it works on the
caller's buffers and keeps its scratch in a fixed device array inside the
library. Two calls in a row on the same buffers, through the C ABI, must
return the same key array element by element, and exactly the
particle-pair contact keys that a tds_step on the same positions finds (the
bit-exact contract all contact-set tests use). Covered: the largest input the
scratch holds, a far outlier that forces the grid to coarsen (thousands of
particles per cell), and an output buffer smaller than the pair count. This
file is collected last.
"""
import ctypes

import numpy as np
import pytest

from tests.parity_cases import packed_scene

pytestmark = pytest.mark.gpu

MAX_N = 65536  # TDS_NOALLOC_MAX_PARTICLES


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    L = tds.lib()
    vp = ctypes.c_void_p
    L.tds_find_pair_contacts_noalloc.restype = ctypes.c_int32
    L.tds_find_pair_contacts_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_int32,
                                                 vp, ctypes.c_uint32, vp, vp]
    return torch, tds, L


def step_pair_keys(tds, scene):
    g = tds.Scene(scene)
    g.step(1)
    keys = g.read_contacts()["keys"]
    g.close()
    return keys[(keys & np.uint64(tds.STATIC_BIT)) == 0]


class Inputs:
    """Device copies of the positions and radii, and output buffers."""

    def __init__(self, torch, x, r, cap):
        x = np.asarray(x, np.float32)
        self.cols = [torch.tensor(np.ascontiguousarray(x[:, k]), device="cuda") for k in range(3)]
        self.r = torch.tensor(np.asarray(r, np.float32), device="cuda")
        self.keys = torch.zeros(cap, dtype=torch.int64, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.n, self.cap = len(r), cap

    def call(self, torch, L, cohesive):
        """One call; returns the raw key array (in the call's order) and the
        reported count."""
        self.keys.fill_(-1)
        stream = torch.cuda.current_stream()
        st = L.tds_find_pair_contacts_noalloc(self.cols[0].data_ptr(), self.cols[1].data_ptr(),
                                              self.cols[2].data_ptr(), self.r.data_ptr(), self.n,
                                              int(cohesive), self.keys.data_ptr(), self.cap,
                                              self.count.data_ptr(), stream.cuda_stream)
        assert st == 0, L.tds_last_error()
        torch.cuda.synchronize()
        m = int(self.count.item())
        return self.keys[:min(m, self.cap)].cpu().numpy().view(np.uint64).copy(), m


def check_two_calls(torch, L, x, r, cohesive, ref, cap):
    buf = Inputs(torch, x, r, cap)
    first, m1 = buf.call(torch, L, cohesive)
    second, m2 = buf.call(torch, L, cohesive)
    assert m1 == m2 == len(ref)
    assert np.array_equal(first, second)  # element by element, in the call's order
    assert np.array_equal(np.sort(first), ref)
    return first


@pytest.mark.parametrize("seed,cohesion", [(21, 1000.0), (22, 0.0)])
def test_two_calls_in_a_row_match_the_step(env, seed, cohesion):
    torch, tds, L = env
    scene = packed_scene(3000, seed, cohesion=cohesion, iters=5)
    ref = step_pair_keys(tds, scene)
    assert len(ref) > 3000
    check_two_calls(torch, L, scene["x"], scene["r"], cohesion > 0, ref, 16 * 3000)


def test_largest_input_the_scratch_holds(env):
    torch, tds, L = env
    scene = packed_scene(MAX_N, 23, cohesion=1000.0, iters=5)
    ref = step_pair_keys(tds, scene)
    assert len(ref) > MAX_N
    check_two_calls(torch, L, scene["x"], scene["r"], True, ref, 8 * MAX_N)


def test_far_outlier_coarsens_the_grid(env):
    """One particle 1 km away makes the fixed cell budget cover a huge box:
    the packed block then sits in a few cells of tens of thousands of
    particles each, which are sorted like small ones, so the output order is
    still fixed and the pairs are still the step's."""
    torch, tds, L = env
    scene = packed_scene(MAX_N - 1, 24, cohesion=0.0, iters=5)
    ref = step_pair_keys(tds, scene)  # the outlier touches nothing
    x = np.concatenate([scene["x"], [[1000.0, 1000.0, 1000.0]]]).astype(np.float32)
    r = np.concatenate([scene["r"], [0.025]]).astype(np.float32)
    check_two_calls(torch, L, x, r, False, ref, 8 * MAX_N)


def test_output_smaller_than_the_pair_count(env):
    """count reports every pair; the cap keys written are the first cap of
    the full call's order."""
    torch, tds, L = env
    scene = packed_scene(3000, 25, cohesion=1000.0, iters=5)
    ref = step_pair_keys(tds, scene)
    full = check_two_calls(torch, L, scene["x"], scene["r"], True, ref, 16 * 3000)
    cap = len(ref) // 3
    part = Inputs(torch, scene["x"], scene["r"], cap)
    got, m = part.call(torch, L, True)
    assert m == len(ref)
    assert len(got) == cap
    assert np.array_equal(got, full[:cap])


def test_rejects_more_particles_than_its_scratch_holds(env):
    torch, tds, L = env
    buf = torch.zeros(4, device="cuda")
    p = buf.data_ptr()
    st = L.tds_find_pair_contacts_noalloc(p, p, p, p, MAX_N + 1, 0, p, 1, p, None)
    assert st == -4
    assert b"65536" in L.tds_last_error()
