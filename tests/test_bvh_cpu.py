"""The scene builder's wide BVHs checked on the host: tests/bvh_check.cpp is
compiled with the builder (g++, no GPU) and decodes the 4- and 8-wide nodes
on its own.  Every triangle must lie in exactly one leaf of each tree, every
quantized child box (origin + code * scale per axis, in double) must contain
the exact bounds of the triangles below it, and 4-wide empty slots must hold
inverted boxes.  Meshes:
a small procedural room, the 61k-triangle benchmark room, a flat grid (zero
extent on one axis), the same grid at coordinates near 1e26, a random
triangle soup, and one and two triangles."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1903_07145_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("bvh") / "bvh_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1903_07145_gb300", "csrc"), "-I", CUDA_INC,
                    os.path.join(ROOT, "tests", "bvh_check.cpp"),
                    os.path.join(ROOT, "paper_1903_07145_gb300", "csrc", "scene_build.cpp"), "-o", exe],
                   check=True)
    return exe


def grid(n=32, scale=1.0):
    xs, ys = np.meshgrid(np.arange(n + 1), np.arange(n + 1))
    pos = np.stack([xs.ravel(), ys.ravel(), np.zeros((n + 1) ** 2)], 1) * scale
    idx = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            idx += [[a, a + 1, a + n + 1], [a + 1, a + n + 2, a + n + 1]]
    return pos, np.array(idx)


def soup(n=3000, seed=4):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-5, 5, (n, 1, 3))
    pos = (c + rng.normal(0, 0.3, (n, 3, 3))).reshape(-1, 3)
    return pos, np.arange(3 * n).reshape(n, 3)


def meshes():
    small = scenes.indoor_room(7, n_cuboids=6, cuboid_sub=3, room_sub=4, n_lights=2, n_views=1,
                               width=16, height=12)
    room = scenes.room_60k()
    return {
        "room_small": (small.positions, small.indices),
        "room_61k": (room.positions, room.indices),
        "flat_grid": grid(),
        "grid_1e26": grid(scale=1e24),
        "soup": soup(),
        "one": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]]), np.array([[0, 1, 2]])),
        "two": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]]), np.array([[0, 1, 2], [1, 3, 2]])),
    }


@pytest.mark.parametrize("name", list(meshes().keys()))
def test_bvh_covers_every_triangle_with_conservative_boxes(checker, tmp_path, name):
    pos, idx = meshes()[name]
    pf, xf = tmp_path / "pos.bin", tmp_path / "idx.bin"
    np.ascontiguousarray(pos, np.float32).tofile(pf)
    np.ascontiguousarray(idx, np.uint32).tofile(xf)
    out = subprocess.run([checker, str(pf), str(xf), str(len(pos)), str(len(idx))], capture_output=True,
                         text=True, check=True).stdout.split()
    once4, violations4, once8, violations8, nodes4, depth = (int(v) for v in out)
    assert once4 == len(idx) and once8 == len(idx), (once4, once8, len(idx))
    assert violations4 == 0 and violations8 == 0
    assert nodes4 >= 1 and depth <= 48
