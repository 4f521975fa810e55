"""The work list of the TMA-staged D3Q19 z-march (lbm_d3q19_work_list, host code of the library; no
GPU needed), checked against the definitions it is built from, restated here with numpy.

A column is a 32 x 8 block of cells (bx, by); it is boxed when it lies inside the grid (32 bx + 32 <=
nx, 8 by + 8 <= ny) on a grid of at least 64 x 16 x 4 nodes.  A plane z of a boxed column needs the
solid path when some plane within 3 planes of z (periodic) holds a solid node within 3 nodes of the
column in x or y (periodic).  Checked on every column:

* its items partition the planes [0, nz) exactly once;
* every plane that needs the solid path lies in a solid item (bounce-back and virtual densities are
  never skipped);
* a plane on the solid path that does not need it lies in a run of planes not needing it shorter
  than 8 (short bulk runs join the solid path; long ones stay on the bulk path);
* interior item boundaries fall on multiples of 32 planes or where the path changes, and items hold
  at most 39 planes (32 + 7: a piece of fewer than 8 planes joins its neighbour);
* a column cut by the grid's edge takes 32-plane chunks, all on the z-pair march (solid = 1);
* items come in ascending (z0, by, bx).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from paper_1908_04443_gb300 import lbmwet as L

TX, TY, CH, HALO, MIN_RUN = 32, 8, 32, 3, 8


def _boxed(bx, by, nx, ny, nz):
    return bx * TX + TX <= nx and by * TY + TY <= ny and nx >= 64 and ny >= 16 and nz >= 4


def _need(mask, bx, by):
    nz, ny, nx = mask.shape
    xs = np.arange(bx * TX - HALO, bx * TX + TX + HALO) % nx
    ys = np.arange(by * TY - HALO, by * TY + TY + HALO) % ny
    near = mask[:, ys][:, :, xs].reshape(nz, -1).any(axis=1)
    return np.array([near[(z + np.arange(-HALO, HALO + 1)) % nz].any() for z in range(nz)])


def _runs(flags):
    """Lengths of the maximal runs of equal values, per plane."""
    out = np.zeros(len(flags), int)
    z0 = 0
    for z in range(1, len(flags) + 1):
        if z == len(flags) or flags[z] != flags[z0]:
            out[z0:z] = z - z0
            z0 = z
    return out


def check_work_list(mask):
    nz, ny, nx = mask.shape
    items = L.lbm_d3q19_work_list(mask)
    gx, gy = -(-nx // TX), -(-ny // TY)
    assert items.shape[1] == 5 and len(items) > 0
    keys = [(int(z0), int(by), int(bx)) for bx, by, z0, z1, s in items]
    assert keys == sorted(keys)
    assert items[:, 0].min() >= 0 and items[:, 0].max() < gx and items[:, 1].min() >= 0 and items[:, 1].max() < gy
    cols = {}
    for bx, by, z0, z1, s in items:
        assert 0 <= z0 < z1 <= nz and s in (0, 1)
        cols.setdefault((int(bx), int(by)), []).append((int(z0), int(z1), int(s)))
    assert len(cols) == gx * gy
    stats = {"items": len(items), "solid": int(items[:, 4].sum())}
    for (bx, by), its in cols.items():
        its.sort()
        assert its[0][0] == 0 and its[-1][1] == nz
        for a, b in zip(its, its[1:]):
            assert a[1] == b[0], (bx, by, a, b)           # no gap, no overlap
        if not _boxed(bx, by, nx, ny, nz):
            assert [(z0, z1) for z0, z1, _ in its] == [(z, min(z + CH, nz)) for z in range(0, nz, CH)]
            assert all(s == 1 for *_, s in its)
            continue
        need = _need(mask, bx, by)
        path = np.zeros(nz, bool)
        for z0, z1, s in its:
            path[z0:z1] = s == 1
            assert z1 - z0 <= CH + MIN_RUN - 1
        assert not (need & ~path).any(), (bx, by)         # every plane that needs the solid path has it
        extra = path & ~need
        if extra.any():
            assert (_runs(need)[extra] < MIN_RUN).all(), (bx, by)
        for (z0, z1, s), (n0, n1, t) in zip(its, its[1:]):
            assert z1 % CH == 0 or s != t, (bx, by, z1)
    return stats


def test_all_fluid_boxed_columns_are_bulk_chunks():
    mask = np.zeros((70, 16, 64), np.uint8)
    items = L.lbm_d3q19_work_list(mask)
    assert items[:, 4].sum() == 0
    # 70 planes per column: 0-32, 32-70 (the last piece of 6 planes joins the one before)
    for bx in range(2):
        for by in range(2):
            col = items[(items[:, 0] == bx) & (items[:, 1] == by)]
            assert [tuple(r[2:4]) for r in col] == [(0, 32), (32, 70)]
    check_work_list(mask)


def test_shallow_grid_single_bulk_item():
    mask = np.zeros((5, 16, 64), np.uint8)
    items = L.lbm_d3q19_work_list(mask)
    assert [tuple(r) for r in items] == [(0, 0, 0, 5, 0), (1, 0, 0, 5, 0), (0, 1, 0, 5, 0), (1, 1, 0, 5, 0)]
    check_work_list(mask)


@pytest.mark.parametrize("plate", [(0, 2), (35, 37), (68, 70)])
def test_plate_band_wraps(plate):
    """A plate filling whole planes: every column needs the solid path on the plate and 3 planes
    around it (wrapping across z = 0 for a plate at the bottom or top), and no other plane takes it
    (the bulk runs beside the band are long)."""
    mask = np.zeros((70, 16, 64), np.uint8)
    mask[plate[0]:plate[1]] = 1
    check_work_list(mask)
    items = L.lbm_d3q19_work_list(mask)
    on = np.zeros(70, int)
    for bx, by, z0, z1, s in items:
        on[z0:z1] += s
    band = [min(min(abs(z - p), 70 - abs(z - p)) for p in range(*plate)) <= HALO for z in range(70)]
    assert list(on) == [4 if b else 0 for b in band]      # all 4 columns, on the band only


@pytest.mark.parametrize("shape", [(37, 21, 100), (40, 24, 96), (33, 16, 64), (9, 12, 40), (64, 64, 64)])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_specks(shape, seed):
    rng = np.random.default_rng(seed)
    mask = (rng.random(shape) < 2e-4).astype(np.uint8)
    check_work_list(mask)


@pytest.mark.parametrize("grid", ["edges", "ragged", "corner"])
def test_spheres_of_the_gpu_cases(grid):
    shapes = {"edges": ((40, 24, 96), (48.0, 12.0, 14.0), 4.0), "ragged": ((37, 21, 100), (70.0, 10.0, 30.0), 3.5),
              "corner": ((33, 16, 64), (10.0, 3.0, 30.0), 2.5)}
    shape, c, r = shapes[grid]
    check_work_list(W.ball_mask(shape, c, r))


def test_sphere_drop_64_and_256_cube():
    """The 64^3 anchor and the 256^3 sphere workload: 2085 items, 96 of them on the solid path, for
    the 256^3 sphere (the launch of the 3D bench line)."""
    check_work_list(W.sphere_drop_64().mask())
    st = check_work_list(W.c3_sphere_256().mask())
    assert st == {"items": 2085, "solid": 96}


def test_errors():
    with pytest.raises(L.LbmError):
        L.lbm_d3q19_work_list(np.zeros((0, 16, 64), np.uint8))
    with pytest.raises(ValueError):
        L.lbm_d3q19_work_list(np.zeros((16, 64), np.uint8))
    lib = L.library()
    mask = np.zeros((40, 16, 64), np.uint8)
    n = C.c_int64(-1)
    mp = mask.ctypes.data_as(C.c_void_p)
    assert lib.lbm_d3q19_work_list(None, 64, 16, 40, None, 0, C.byref(n)) == L.LBM_ERR_ARG
    assert lib.lbm_d3q19_work_list(mp, 64, 16, 40, None, 0, None) == L.LBM_ERR_ARG
    # 4 columns of two items (planes 0-32 and 32-40: a last piece of 8 planes stands alone)
    assert lib.lbm_d3q19_work_list(mp, 64, 16, 40, None, 0, C.byref(n)) == L.LBM_OK and n.value == 8
    buf = (C.c_int32 * 40)(*([-7] * 40))
    assert lib.lbm_d3q19_work_list(mp, 64, 16, 40, buf, 7, C.byref(n)) == L.LBM_ERR_ARG
    assert list(buf) == [-7] * 40                          # nothing written
    assert lib.lbm_d3q19_work_list(mp, 64, 16, 40, buf, 8, C.byref(n)) == L.LBM_OK
    assert sorted(tuple(buf[5 * i + 2:5 * i + 4]) for i in range(8)) == [(0, 32)] * 4 + [(32, 40)] * 4
