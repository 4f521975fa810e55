"""Batched stepping (one persistent kernel launch per time step over all instances): each instance
of an uneven batch evolves exactly as the same grid stepped alone, and one batched step agrees with
the FP64 oracle on every instance."""
import numpy as np
import pytest

from oracle import lbm
from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def _cases(kernel="ymarch"):
    a = drop_on_cylinder((40, 48), (24.0, 14.0), 7.0, (24.0, 27.0), 8.0, kappa=0.2)
    b = drop_on_cylinder((37, 53), (20.3, 17.1), 9.5, (21.0, 30.0), 10.0, kappa=-0.02)
    c = drop_on_cylinder((64, 70), (35.0, 20.0), 10.0, (35.0, 38.0), 12.0, kappa=0.1)
    # wider than one y-march column block (124 own columns): two blocks, the second ragged
    d = drop_on_cylinder((50, 150), (70.0, 20.0), 9.0, (70.0, 38.0), 10.0, kappa=0.05)
    geo = lbm.Geometry(c.mask, "D2Q9")
    c.kappa = np.random.default_rng(4).uniform(-0.02, 0.3, len(geo.wall_flat))
    cases = [a, b, c, d]
    for cs in cases:
        cs.step_kernel = kernel   # the batch takes instance 0's choice; single runs use the same kernel
    return cases


def _batch(cases, precision):
    from paper_1908_04443_gb300 import lbmwet as L
    sims = [cs.gpu(precision) for cs in cases]      # configs built exactly as for single runs
    cfgs = [s.cfg for s in sims]
    for s in sims:
        s.close()
    masks = [cs.mask for cs in cases]
    rho0s = [cs.rho0 for cs in cases]
    kpw = [None if np.ndim(cs.kappa) == 0 else np.asarray(cs.kappa) for cs in cases]
    return L.lbm_batch_init(cfgs, masks, rho0s, kpw)


@pytest.mark.parametrize("precision,kernel", [("fp64", "tile"), ("fp64", "ymarch"), ("fp32", "tile"),
                                               ("fp32", "ymarch"), ("fp32", "pair")])
def test_batch_equals_single_runs(precision, kernel):
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases(kernel)
    b = _batch(cases, precision)
    try:
        assert L.lbm_batch_step_kernel_used(b) == kernel
        L.lbm_batch_step(b, 37)          # 2 graph chunks of 16 + 5 single launches
        assert L.lbm_batch_kernel_launches(b) == 37
        for i, cs in enumerate(cases):
            h = L.lbm_batch_handle(b, i)
            q, n = 9, cs.mask.size
            fb = L.lbm_get_state(h, q, n)
            with cs.gpu(precision) as sim:
                assert sim.step_kernel() == kernel
                sim.step(37)
                fs = sim.get_state().reshape(-1)
            assert np.max(np.abs(fb - fs)) == 0.0
        obs = L.lbm_batch_observables(b)
        assert len(obs) == len(cases) and all(o.step == 37 for o in obs)
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("kernel", ["ymarch", "tile"])
def test_batched_step_matches_oracle(kernel):
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases(kernel)
    b = _batch(cases, "fp64")
    try:
        L.lbm_batch_step(b, 3)
        before = [L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size) for i, cs in enumerate(cases)]
        L.lbm_batch_step(b, 1)
        for i, cs in enumerate(cases):
            geo, p, _ = cs.oracle()
            ref = lbm.step(before[i].reshape((9,) + cs.shape), geo, p)
            got = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size).reshape((9,) + cs.shape)
            assert np.max(np.abs(got - ref)) < 1e-13
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_observables_report_an_unstable_instance(precision):
    """An instance whose state has lost positivity (written from the host: every population -0.1,
    so every fluid node's density is negative) makes the batched observables fail with its index:
    the fields pass raises the instance's own flag on rho <= 0, and the flag reaches the host through
    the one-launch reduction of all instances.  The other instances' flags stay clear."""
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases("pair" if precision == "fp32" else "tile")
    b = _batch(cases, precision)
    try:
        L.lbm_batch_step(b, 2)
        assert len(L.lbm_batch_observables(b)) == len(cases)
        L.lbm_set_state(L.lbm_batch_handle(b, 1), np.full(9 * cases[1].mask.size, -0.1), step=2)
        for call in (lambda: L.lbm_batch_observables(b), lambda: L.lbm_batch_observables_fields(b)):
            with pytest.raises(L.LbmError) as ei:
                call()
            assert ei.value.status == L.LBM_ERR_UNSTABLE
            assert "instance 1:" in str(ei.value)
        assert L.lbm_observables(L.lbm_batch_handle(b, 0)).step == 2
    finally:
        L.lbm_batch_destroy(b)


def test_batch_member_rules():
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases()
    b = _batch(cases, "fp32")
    try:
        h = L.lbm_batch_handle(b, 1)
        with pytest.raises(L.LbmError) as ei:
            L.lbm_step(h, 1)
        assert ei.value.status == L.LBM_ERR_STATE
        L.lbm_destroy(h)                   # ignored for batch members
        L.lbm_batch_step(b, 2)
        assert L.lbm_observables(h).step == 2
        with pytest.raises(IndexError):
            L.lbm_batch_handle(b, 4)
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("kernel", ["tile", "pair"])
def test_batch_wide_grids_equal_single_runs(kernel):
    """FP32 batches of grids with interior tiles (no periodic wrap) as well as edge and wall tiles:
    every instance evolves exactly as the grid stepped alone.  The pair kernel pulls the interior
    tiles of every grid from a TMA box in shared memory and edge tiles and grids narrower than a box
    from global memory; the grid stepped alone pulls from global memory."""
    from paper_1908_04443_gb300 import lbmwet as L
    a = drop_on_cylinder((96, 256), (128.0, 30.0), 14.0, (128.0, 58.0), 15.0, kappa=0.15, step_kernel=kernel)
    b = drop_on_cylinder((120, 200), (60.0, 50.0), 18.0, (60.0, 86.0), 19.0, kappa=-0.02, step_kernel=kernel)
    c = drop_on_cylinder((30, 36), (18.0, 10.0), 5.0, (18.0, 22.0), 6.5, kappa=0.1, step_kernel=kernel)
    d = drop_on_cylinder((50, 98), (3.0, 25.0), 9.0, (3.0, 40.0), 9.0, kappa=0.05, step_kernel=kernel)
    cases = [a, b, c, d]
    for cs in cases:
        cs.rho_ref = cs.bounds()[0]
    bt = _batch(cases, "fp32")
    try:
        L.lbm_batch_step(bt, 35)
        for i, cs in enumerate(cases):
            fb = L.lbm_get_state(L.lbm_batch_handle(bt, i), 9, cs.mask.size)
            with cs.gpu("fp32") as sim:
                sim.step(35)
                fs = sim.get_state().reshape(-1)
            assert np.array_equal(fb, fs), i
    finally:
        L.lbm_batch_destroy(bt)


def test_batch_row_padding_residues():
    """Grid widths of every residue mod 4 (81, 82, 83, 84 columns): the distributions' rows are padded
    to a multiple of 32 nodes, so every grid has TMA tensor maps and its interior tiles pull from a
    box.  Each instance evolves exactly as the grid stepped alone, and one batched step agrees with
    the FP64 oracle."""
    from paper_1908_04443_gb300 import lbmwet as L
    cases = [drop_on_cylinder((56, nx), (nx / 2.0, 20.0), 9.0, (nx / 2.0, 38.0), 10.0, kappa=0.1, step_kernel="pair")
             for nx in (81, 82, 83, 84)]
    for cs in cases:
        cs.rho_ref = cs.bounds()[0]
    bt = _batch(cases, "fp32")
    try:
        assert L.lbm_batch_step_kernel_used(bt) == "pair"
        L.lbm_batch_step(bt, 23)
        before = [L.lbm_get_state(L.lbm_batch_handle(bt, i), 9, cs.mask.size) for i, cs in enumerate(cases)]
        for i, cs in enumerate(cases):
            with cs.gpu("fp32") as sim:
                sim.step(23)
                fs = sim.get_state().reshape(-1)
            assert np.array_equal(before[i], fs), i
        L.lbm_batch_step(bt, 1)
        for i, cs in enumerate(cases):
            geo, p, _ = cs.oracle()
            ref = lbm.step(before[i].reshape((9,) + cs.shape), geo, p)
            got = L.lbm_get_state(L.lbm_batch_handle(bt, i), 9, cs.mask.size).reshape((9,) + cs.shape)
            assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref)), i
    finally:
        L.lbm_batch_destroy(bt)


def test_batch_sf_scheme():
    """A batch with the solid-fluid interaction scheme (Eq. 8): every instance evolves exactly as the
    grid stepped alone, and one batched step agrees with the FP64 oracle."""
    from paper_1908_04443_gb300 import lbmwet as L
    cases = [drop_on_cylinder((96, 256), (128.0, 30.0), 14.0, (128.0, 58.0), 15.0, wall="SF", Gw=-0.2),
             drop_on_cylinder((50, 98), (3.0, 25.0), 9.0, (3.0, 40.0), 9.0, wall="SF", Gw=-0.2)]
    for cs in cases:
        cs.rho_ref = cs.bounds()[0]
    bt = _batch(cases, "fp32")
    try:
        assert L.lbm_batch_step_kernel_used(bt) == "pair"
        L.lbm_batch_step(bt, 17)
        before = [L.lbm_get_state(L.lbm_batch_handle(bt, i), 9, cs.mask.size) for i, cs in enumerate(cases)]
        for i, cs in enumerate(cases):
            with cs.gpu("fp32") as sim:
                sim.step(17)
                assert np.array_equal(before[i], sim.get_state().reshape(-1)), i
        L.lbm_batch_step(bt, 1)
        for i, cs in enumerate(cases):
            geo, p, _ = cs.oracle()
            ref = lbm.step(before[i].reshape((9,) + cs.shape), geo, p)
            got = L.lbm_get_state(L.lbm_batch_handle(bt, i), 9, cs.mask.size).reshape((9,) + cs.shape)
            assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref)), i
    finally:
        L.lbm_batch_destroy(bt)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_observables_fields_equal_per_instance_calls(precision):
    """lbm_batch_observables_fields (one synchronisation for the batch) gives every instance the same
    observables and fields as lbm_observables called on that instance, with pinned and pageable host
    arrays and with some entries left out."""
    import torch
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases("pair" if precision == "fp32" else "tile")
    b = _batch(cases, precision)
    try:
        L.lbm_batch_step(b, 12)
        n = [cs.mask.size for cs in cases]
        pinned = lambda k: torch.zeros(k, dtype=torch.float64).pin_memory().numpy()
        rho = [pinned(n[0]), np.zeros(n[1]), None, np.zeros(n[3])]
        u = [pinned(2 * n[0]), None, np.zeros(2 * n[2]), np.zeros(2 * n[3])]
        obs = L.lbm_batch_observables_fields(b, rho, u)
        assert [o.mass for o in L.lbm_batch_observables(b)] == [o.mass for o in obs]
        for i in range(len(cases)):
            r_ref, u_ref = np.zeros(n[i]), np.zeros(2 * n[i])
            ref = L.lbm_observables(L.lbm_batch_handle(b, i), r_ref, u_ref)
            for f in ("mass", "rho_max", "rho_min", "u_max", "n_interface", "step"):
                assert getattr(obs[i], f) == getattr(ref, f), (i, f)
            assert obs[i].theta_deg == ref.theta_deg or (np.isnan(obs[i].theta_deg) and np.isnan(ref.theta_deg))
            if rho[i] is not None:
                assert np.array_equal(rho[i], r_ref)
            if u[i] is not None:
                assert np.array_equal(u[i], u_ref)
    finally:
        L.lbm_batch_destroy(b)


def test_binding_checks_host_array_sizes():
    """The binding refuses host arrays whose size is not the grid's before the library writes or reads
    N (or q*N, d*N, one per wall node) values through them."""
    from paper_1908_04443_gb300 import lbmwet as L
    cs = _cases("tile")[1]
    with cs.gpu("fp64") as sim:
        n = cs.mask.size
        assert L.lbm_grid_shape(sim.h) == (cs.shape[1], cs.shape[0], 1, 2)
        with pytest.raises(ValueError):
            L.lbm_observables(sim.h, np.zeros(n - 1))
        with pytest.raises(ValueError):
            L.lbm_observables(sim.h, None, np.zeros(n))             # u holds 2 * n values
        with pytest.raises(ValueError):
            L.lbm_get_state(sim.h, 19, n)
        with pytest.raises(ValueError):
            L.lbm_set_state(sim.h, np.zeros(9 * n - 9))
        nw = len(L.lbm_wall_nodes(sim.h))
        with pytest.raises(ValueError):
            L.lbm_set_kappa(sim.h, np.zeros(nw + 1))
        f = L.lbm_get_state(sim.h)                                     # q and n from the handle
        assert f.size == 9 * n
        L.lbm_set_state(sim.h, f)
        L.lbm_set_kappa(sim.h, np.full(nw, 0.1))
