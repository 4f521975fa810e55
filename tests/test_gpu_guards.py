"""Memory safety of every step kernel without a memory checker: the distribution buffers and the
observable fields sit between guard zones of a known byte, and the padding nodes of the D2Q9 rows
are zero at init and written by no kernel.  After steps, observables, batched steps and an adjoint
pass on grids with ragged tiles, lbm_check_guards must find every guard byte and padding byte
untouched."""
import numpy as np
import pytest

from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu

# (ny, nx) grids: a ragged 37-wide row (27 padding nodes), a full 64-wide row (no padding), a
# narrow 30-wide grid, and a 98-wide grid with a ragged last tile in both directions.
GRIDS_2D = [((53, 37), (20.3, 17.1), 9.5, (21.0, 30.0), 10.0),
            ((48, 64), (30.0, 14.0), 7.0, (30.0, 27.0), 8.0),
            ((36, 30), (15.0, 10.0), 5.0, (15.0, 20.0), 6.0),
            ((45, 98), (50.0, 13.0), 8.0, (50.0, 28.0), 9.0)]


def _untouched(sim_or_h):
    from paper_1908_04443_gb300 import lbmwet as L
    g, p = L.lbm_check_guards(sim_or_h)
    assert (g, p) == (0, 0), f"{g} guard bytes and {p} padding bytes overwritten"


@pytest.mark.parametrize("precision,kernel", [("fp64", "tile"), ("fp64", "ymarch"), ("fp32", "tile"),
                                               ("fp32", "ymarch"), ("fp32", "pair")])
@pytest.mark.parametrize("grid", range(len(GRIDS_2D)))
@pytest.mark.parametrize("wall", ["IVD", "SF"])
def test_2d_step_kernels_stay_in_bounds(precision, kernel, grid, wall):
    shape, c, R, dc, r = GRIDS_2D[grid]
    case = drop_on_cylinder(shape, c, R, dc, r, kappa=0.1, wall=wall, Gw=-0.2 if wall == "SF" else 0.0)
    case.step_kernel = kernel
    with case.gpu(precision) as sim:
        assert sim.step_kernel() == kernel
        sim.step(19)                     # one CUDA-graph chunk of 16 and 3 single launches
        sim.observables(fields=True)     # fills the guarded density and velocity fields
        sim.check()
        _untouched(sim.h)


@pytest.mark.parametrize("precision,kernel", [("fp64", "auto"), ("fp32", "tile"), ("fp32", "pair"),
                                               ("fp32", "ztma")])
@pytest.mark.parametrize("wall", ["IVD", "SF"])
@pytest.mark.parametrize("grid", [0, 1])
def test_3d_step_kernels_stay_in_bounds(precision, kernel, wall, grid):
    # (nz, ny, nx) = (22, 20, 26): ragged in every direction of the z-march and z-pair tiles;
    # (37, 21, 100): TMA-staged columns on the x and y edges next to ragged ones, a partial chunk
    g3 = [((22, 20, 26), (13.0, 10.0, 8.0), 4.5, (13.0, 10.0, 16.0), 6.0),
          ((37, 21, 100), (70.0, 10.0, 30.0), 3.5, (70.0, 10.0, 20.0), 5.0)][grid]
    case = drop_on_cylinder(*g3, lattice="D3Q19", kappa=0.1, wall=wall, Gw=-0.2 if wall == "SF" else 0.0,
                            step_kernel=kernel)
    if precision == "fp32":
        case.rho_ref = case.bounds()[0]
    with case.gpu(precision) as sim:
        sim.step(19)
        sim.observables(fields=True)
        sim.check()
        _untouched(sim.h)


@pytest.mark.parametrize("precision,kernel", [("fp64", "tile"), ("fp32", "ymarch"), ("fp32", "pair")])
def test_batched_steps_stay_in_bounds(precision, kernel):
    from paper_1908_04443_gb300 import lbmwet as L
    cases = [drop_on_cylinder(*g, kappa=0.1) for g in GRIDS_2D]
    sims = []
    for cs in cases:
        cs.step_kernel = kernel
        sims.append(cs.gpu(precision))
    cfgs = [s.cfg for s in sims]
    for s in sims:
        s.close()
    b = L.lbm_batch_init(cfgs, [cs.mask for cs in cases], [cs.rho0 for cs in cases], [None] * len(cases))
    try:
        assert L.lbm_batch_step_kernel_used(b) == kernel
        L.lbm_batch_step(b, 19)
        L.lbm_batch_observables(b)
        for i in range(len(cases)):
            _untouched(L.lbm_batch_handle(b, i))
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_pass_stays_in_bounds(precision):
    import torch
    from paper_1908_04443_gb300 import lbmwet as L
    shape, c, R, dc, r = GRIDS_2D[0]
    case = drop_on_cylinder(shape, c, R, dc, r, kappa=0.1)
    if precision == "fp32":
        case.rho_ref = case.bounds()[0]
    with case.gpu(precision, stream=torch.cuda.current_stream()) as sim:
        nw = len(sim.wall_nodes())
        L.lbm_record(sim.h, 12, 4)
        drho = torch.ones(sim.n, dtype=torch.float64, device="cuda")
        g = L.lbm_adjoint(sim.h, drho.data_ptr(), nw)
        assert np.all(np.isfinite(g))
        _untouched(sim.h)


def test_check_finds_a_planted_padding_byte():
    # a state whose padding holds one non-zero byte, loaded through the checkpoint path (which
    # copies whole rows, padding included): the check must count exactly that byte
    from paper_1908_04443_gb300 import lbmwet as L
    shape, c, R, dc, r = GRIDS_2D[0]
    ny, nx = shape
    fp = (nx + 31) // 32 * 32
    case = drop_on_cylinder(shape, c, R, dc, r, kappa=0.1)
    with case.gpu("fp32") as sim:
        sim.step(3)
        blob = bytearray(L.lbm_save_state(sim.h))
        assert len(blob) == 9 * fp * ny * 4 + 8
        at = (3 * fp * ny + 5 * fp + nx + 4) * 4 + 1    # direction 3, row 5, 5th padding node
        assert blob[at] == 0
        blob[at] = 1
        L.lbm_load_state(sim.h, bytes(blob))
        assert L.lbm_check_guards(sim.h) == (0, 1)
