"""tds_find_pair_contacts_noalloc against the contact search of tds_step.

The entry point serves callers that cannot let a library allocate device
memory (a simulator stepping in a fixed-rate real-time loop, where an
allocation can synchronize the device and miss the frame, or an application
whose device memory belongs to its own fixed-budget pool): it works on the
caller's buffers and keeps its scratch in a fixed device array inside the
library. Two calls in a row, through the C ABI, must each return exactly the
particle-pair contact keys that a tds_step on the same positions finds (the
bit-exact contract all contact-set tests use). This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from tests.parity_cases import packed_scene

pytestmark = pytest.mark.gpu


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


def noalloc_pair_keys(torch, L, scene, cap):
    x = np.asarray(scene["x"], np.float32)
    cols = [torch.tensor(np.ascontiguousarray(x[:, k]), device="cuda") for k in range(3)]
    r = torch.tensor(np.asarray(scene["r"], np.float32), device="cuda")
    keys = torch.zeros(cap, dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = L.tds_find_pair_contacts_noalloc(cols[0].data_ptr(), cols[1].data_ptr(), cols[2].data_ptr(),
                                          r.data_ptr(), len(scene["r"]), int(scene["cohesion"] > 0),
                                          keys.data_ptr(), cap, count.data_ptr(), stream.cuda_stream)
    assert st == 0, L.tds_last_error()
    torch.cuda.synchronize()
    m = int(count.item())
    assert m <= cap
    return np.sort(keys[:m].cpu().numpy().view(np.uint64))


def test_two_calls_in_a_row_match_the_step(env):
    torch, tds, L = env
    for seed, cohesion in ((21, 1000.0), (22, 0.0)):
        scene = packed_scene(3000, seed, cohesion=cohesion, iters=5)
        ref = step_pair_keys(tds, scene)
        got = noalloc_pair_keys(torch, L, scene, cap=16 * 3000)
        assert len(ref) > 3000
        assert np.array_equal(got, ref)


def test_rejects_more_particles_than_its_scratch_holds(env):
    torch, tds, L = env
    buf = torch.zeros(4, device="cuda")
    p = buf.data_ptr()
    st = L.tds_find_pair_contacts_noalloc(p, p, p, p, 65537, 0, p, 1, p, None)
    assert st == -4
    assert b"65536" in L.tds_last_error()
