"""The host scan of the solid mask that lbm_init runs (csrc/maskscan.cpp): wall nodes and the per-tile
solid flags, against a direct numpy statement of their definitions, on random and ball
masks in 2D and 3D, with the row split over one and several threads.

Definitions checked: a wall node is a solid node with at least one fluid node among its lattice
neighbours x + e_a (D2Q9: the 8 around it; D3Q19: the 18 of the velocity set), periodic in every
axis, listed in ascending linear index; a tile (t0 x t1 x t2, ragged at the
far edges) is flagged when a solid node lies in its box: the cells it covers, wrapped, plus 3 cells
on each side (no z halo in 2D), wrapped."""
import ctypes as C
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

E2 = [(dx, dy, 0) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]
E3 = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0), (1, -1, 0),
      (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("maskscan") / "libmaskscan_test.so")
    cmd = [cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", out,
           os.path.join(HERE, "native", "maskscan_shim.cpp"),
           os.path.join(ROOT, "paper_1908_04443_gb300", "csrc", "maskscan.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    so = C.CDLL(out)
    so.maskscan_run.restype = C.c_longlong
    return so


def run(lib, mask, D, t, threads):
    nz, ny, nx = mask.shape
    N = mask.size
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    tt = (C.c_int * 3)(*t)
    nfluid, ntiles = C.c_longlong(), C.c_longlong()
    walls = np.zeros(N, np.int64)
    cap = 1 << 20
    tiles = np.zeros(cap, np.uint8)
    nw = lib.maskscan_run(m.ctypes.data_as(C.c_void_p), nx, ny, nz, D, tt, threads, C.byref(nfluid),
                          walls.ctypes.data_as(C.c_void_p), tiles.ctypes.data_as(C.c_void_p), C.c_longlong(cap),
                          C.byref(ntiles))
    return nfluid.value, walls[:nw], tiles[:ntiles.value]


def reference(mask, D, t):
    """The definitions in the module docstring, written with numpy rolls."""
    solid = mask != 0
    fluid_nb = np.zeros_like(solid)
    for ex, ey, ez in (E2 if D == 2 else E3):
        # fluid_nb[x] |= fluid[x + e]
        fluid_nb |= np.roll(~solid, shift=(-ez, -ey, -ex), axis=(0, 1, 2))
    wall = solid & fluid_nb
    walls = np.flatnonzero(wall.reshape(-1))
    nz, ny, nx = mask.shape
    n = (nx, ny, nz)
    halo = (3, 3, 3 if D == 3 else 0)
    tiles = [(n[k] + t[k] - 1) // t[k] for k in range(3)]
    flags = np.zeros((tiles[2], tiles[1], tiles[0]), np.uint8)
    for kz, ky, kx in itertools.product(range(tiles[2]), range(tiles[1]), range(tiles[0])):
        k = (kx, ky, kz)
        idx = [np.unique([(k[d] * t[d] + o) % n[d] for o in range(-halo[d], t[d] + halo[d])]) for d in range(3)]
        flags[kz, ky, kx] = solid[np.ix_(idx[2], idx[1], idx[0])].any()
    return int((~solid).sum()), walls, flags.reshape(-1)


def masks():
    rng = np.random.default_rng(11)
    out = []
    for shape, D in [((1, 1, 1), 2), ((1, 5, 1), 2), ((1, 1, 7), 2), ((1, 9, 37), 2), ((1, 64, 96), 2),
                     ((3, 3, 3), 3), ((2, 5, 7), 3), ((11, 21, 37), 3), ((16, 16, 40), 3)]:
        for fill in (0.0, 0.07, 0.5, 1.0):
            out.append((f"random{fill}_{shape}", (rng.random(shape) < fill).astype(np.uint8) * rng.integers(1, 256, shape, dtype=np.uint8), D))
        zz, yy, xx = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]]
        ball = ((xx - 0.4 * shape[2]) ** 2 + (yy - 0.6 * shape[1]) ** 2 + (zz - 0.5 * shape[0]) ** 2
                < 0.3 * shape[1] * shape[2]).astype(np.uint8)
        out.append((f"ball_{shape}", ball, D))
    return out


@pytest.mark.parametrize("name,mask,D", masks(), ids=[m[0] for m in masks()])
@pytest.mark.parametrize("threads", [1, 3])
def test_mask_scan_matches_definitions(lib, name, mask, D, threads):
    t = (32, 16, 1) if D == 2 else (32, 4, 8)
    nf, walls, tiles = run(lib, mask, D, t, threads)
    rf, rwalls, rtiles = reference(mask, D, t)
    assert nf == rf
    assert np.array_equal(walls, rwalls)
    assert np.array_equal(tiles, rtiles)
    if D == 2:   # a second tile shape, with ragged tiles on a narrow grid
        _, _, tiles2 = run(lib, mask, D, (3, 2, 1), threads)
        assert np.array_equal(tiles2, reference(mask, D, (3, 2, 1))[2])
