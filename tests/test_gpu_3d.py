"""GPU parity of lpf_full_3d (the 3D extension) against the oracle's 3D
lineal path function on synthetic Boolean-sphere volumes (stand-ins for the
CT volumes of Sec. 6.3): every count, bit-exact, on ragged sizes and windows
up to the full domain; sampled vectors on a larger volume."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("spheres 16^3 r=5", (16, 16, 16), (5, 5, 5), 2.5, 25),
    ("ragged 7x21x37", (7, 21, 37), (9, 6, 3), 3.0, 12),
    ("full domain 6x7x9", (6, 7, 9), (8, 6, 5), 1.8, 6),
    ("one slice 1x30x40", (1, 30, 40), (12, 10, 0), 4.0, 5),
    ("tall 40x9x33", (40, 9, 33), (4, 3, 12), 3.0, 30),
]


@pytest.mark.parametrize("name,shape,window,R,n", CASES, ids=[c[0] for c in CASES])
def test_full_3d_matches_oracle(gpu_lib, name, shape, window, R, n):
    vol = synth.boolean_spheres(*shape, R, n, seed=sum(shape))
    rx, ry, rz = window
    p = gpu_lib.lpf_build_paths_3d(rx, ry, rz)
    got = gpu_lib.lpf_full_3d(torch.from_numpy(vol).cuda(), p)
    assert gpu_lib.lpf_paths_status(p) == 0
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.lpf_full3(vol, rx, ry, rz))
    # the walk's work counters cover the volume walk too: some of the program
    # walked, at most all of it
    executed, nominal = gpu_lib.lpf_paths_work(p)
    assert 0 < executed <= nominal


def test_full_3d_launch_shapes_and_sampled_large_volume(gpu_lib):
    # 64^3, window 16: every launch shape gives the same counts; sampled
    # vectors against the oracle; symmetry and L(0) at full size.
    vol = synth.boolean_spheres(64, 64, 64, 5.0, 120, seed=6)
    r = 16
    d = torch.from_numpy(vol).cuda()
    p = gpu_lib.lpf_build_paths_3d(r, r, r)
    ref = gpu_lib.lpf_full_3d(d, p).cpu().numpy()
    for T in (1, 2):
        q = gpu_lib.lpf_build_paths_3d(r, r, r)
        gpu_lib.lpf_set_launch_shape(q, 64, 64, T, 1)
        np.testing.assert_array_equal(gpu_lib.lpf_full_3d(d, q).cpu().numpy(), ref)
    rng = np.random.default_rng(2)
    vecs = [(0, 0, 0), (16, 0, 0), (0, 16, 0), (0, 0, 16), (16, -16, 16), (-5, 11, -3)]
    vecs += [tuple(int(x) for x in rng.integers(-r, r + 1, 3)) for _ in range(6)]
    for dx, dy, dz in vecs:
        k = oracle.full_index3(dx, dy, dz, r, r, r)
        for ph in (0, 1):
            assert ref[ph, k] == oracle.count3(vol, dx, dy, dz, ph), (dx, dy, dz, ph)
    np.testing.assert_array_equal(ref, ref[:, ::-1])
    _, _, base = oracle.window_sizes3(r, r, r)
    assert ref[1, base] == int(vol.sum())


def test_volume_and_image_handles_are_not_interchangeable(gpu_lib):
    p3 = gpu_lib.lpf_build_paths_3d(2, 2, 2)
    p2 = gpu_lib.lpf_build_paths(2, 2)
    img = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    vol = torch.zeros((4, 8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu_lib.LpfError):
        gpu_lib.lpf_full(img, p3)
    with pytest.raises(gpu_lib.LpfError):
        gpu_lib.lpf_full_3d(vol, p2)
