"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

* The 600 x 400 cylinder workload over its 24-point wall-parameter sweep, stepped as one batch (FP32
  deviation storage): one batched step from an evolved state, compared with one FP64 oracle step on
  every node of three instances.
* The same sweep over 21 steps: every instance equals its grid stepped alone, bit for bit.
* The 96-instance batch of 128^2..512^2 grids: the same on four instances.
* The 256^3 sphere workload (D3Q19 z-march, FP32): one step compared at sampled nodes.  The oracle
  steps a 15^3 window around each sampled node taken from the GPU state: one step's output at a node
  depends on the state within 3 nodes (pull, psi of neighbours, virtual densities of neighbouring
  wall nodes), so the window's centre is exact although its edges wrap.
* The 600 x 400 workload run for its configured 20000 steps in FP32 deviation storage and in FP64,
  against each other and against the FP64 oracle's stored result (tests/golden): the contact angle
  within 0.5 degrees (FP32) and the split FP32 density bounds.
* A 64^3 drop on a sphere run for 1000 steps by the default D3Q19 steps (FP32 TMA z-march, FP64
  scalar z-march) against the FP64 oracle's stored result, with the same bounds.

FP32 single-step tolerances: the stored deviations carry float rounding (relative 6e-8 of the
distributions) through one collision; 2e-6 of the largest distribution bounds it with margin.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import eos as E, lbm
from tests.fp32_bounds import split_errors

pytestmark = pytest.mark.gpu


def _eos(t_over_tc):
    e = E.cs_config().at_reduced_temperature(t_over_tc)
    g, l = E.maxwell(e)
    return e, g, l


def _cfg(L, wl, precision, g, l):
    e = L.make_eos("CS", 0.25, 4.0, 1.0, 0.0)
    e.T = wl.t_over_tc * L.lbm_critical_temperature(e)
    return L.make_config(wl.lattice, precision, wl.shape, e, sigma=0.12, rho_l=l, rho_g=g, kappa=wl.kappa,
                         rho_ref=g, body=("ball", wl.body_center, wl.body_radius), drop_hint=wl.drop_center)


def _oracle_params(wl, eos, g, l):
    return lbm.Params(wl.lattice, eos, sigma=0.12, rho_l=l, rho_g=g, kappa=wl.kappa)


def _batch_one_step(wls, check_idx, t_over_tc, warm=40):
    from paper_1908_04443_gb300 import lbmwet as L
    eos, g, l = _eos(t_over_tc)
    cfgs = [_cfg(L, wl, "fp32", g, l) for wl in wls]
    b = L.lbm_batch_init(cfgs, [wl.mask() for wl in wls], [wl.rho0(l, g) for wl in wls])
    try:
        L.lbm_batch_step(b, warm)
        before = {i: L.lbm_get_state(L.lbm_batch_handle(b, i), 9, wls[i].nodes) for i in check_idx}
        L.lbm_batch_step(b, 1)
        for i in check_idx:
            wl = wls[i]
            after = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, wl.nodes).reshape((9,) + wl.shape)
            geo = lbm.Geometry(wl.mask(), "D2Q9")
            ref = lbm.step(before[i].reshape((9,) + wl.shape), geo, _oracle_params(wl, eos, g, l))
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(after - ref)) <= 2e-6 * scale, f"instance {i}"
    finally:
        L.lbm_batch_destroy(b)


def test_c2_sweep_batch_one_step_full_size():
    _, g, l = _eos(0.6)
    wls = [W.c2_cylinder_600x400(kappa=k) for k in W.c2_cylinder_sweep_kappas(l, g)]
    _batch_one_step(wls, [0, 11, 23], 0.6)


def test_c2_sweep_batch_equals_single_runs():
    """The 24-grid sweep (11,400 tiles, most of them claimed dynamically by the persistent CTAs) over
    several launches: every instance equals the grid stepped alone, bit for bit, so no tile is
    skipped or stepped twice in any launch."""
    from paper_1908_04443_gb300 import lbmwet as L
    eos, g, l = _eos(0.6)
    wls = [W.c2_cylinder_600x400(kappa=k) for k in W.c2_cylinder_sweep_kappas(l, g)]
    cfgs = [_cfg(L, wl, "fp32", g, l) for wl in wls]
    b = L.lbm_batch_init(cfgs, [wl.mask() for wl in wls], [wl.rho0(l, g) for wl in wls])
    try:
        assert L.lbm_batch_step_kernel_used(b) == "pair"
        L.lbm_batch_step(b, 21)
        for i, wl in enumerate(wls):
            fb = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, wl.nodes)
            with L.Simulation(cfgs[i], wl.mask(), wl.rho0(l, g)) as sim:
                sim.step(21)
                fs = sim.get_state().reshape(-1)
            assert np.array_equal(fb, fs), f"instance {i}"
    finally:
        L.lbm_batch_destroy(b)


def test_c4_batch_one_step_full_size():
    _, g, l = _eos(0.7)
    wls = W.c4_batch(96)
    for wl in wls:
        if wl.kappa < 0:
            wl.kappa *= (l - g)
    _batch_one_step(wls, [0, 17, 58, 95], 0.7, warm=20)


def test_c3_sphere_one_step_sampled():
    from paper_1908_04443_gb300 import lbmwet as L
    wl = W.c3_sphere_256()
    eos, g, l = _eos(wl.t_over_tc)
    mask = wl.mask()
    with L.Simulation(_cfg(L, wl, "fp32", g, l), mask, wl.rho0(l, g)) as sim:
        sim.step(3)
        before = sim.get_state()
        sim.step(1)
        after = sim.get_state()
    geo_full = lbm.Geometry(mask, "D3Q19")
    rng = np.random.default_rng(3)
    fluid = np.argwhere(mask == 0)
    # sampled nodes: random fluid nodes, plus fluid nodes next to the sphere and at grid edges
    near = np.argwhere((mask == 0) & np.roll(geo_full.wall, 1, axis=0))
    picks = list(fluid[rng.choice(len(fluid), 40, replace=False)]) + list(near[rng.choice(len(near), 20, replace=False)])
    picks += [np.array([0, 0, 0]), np.array([255, 255, 255]), np.array([0, 128, 255])]
    p = _oracle_params(wl, eos, g, l)
    r = 7
    for z, y, x in picks:
        zs = np.arange(z - r, z + r + 1) % 256
        ys = np.arange(y - r, y + r + 1) % 256
        xs = np.arange(x - r, x + r + 1) % 256
        win = np.ix_(zs, ys, xs)
        m = mask[win]
        if m[r, r, r]:
            continue
        geo = lbm.Geometry(m, "D3Q19")
        f0 = before[(slice(None),) + win]
        ref = lbm.step(f0, geo, p)[:, r, r, r]
        got = after[:, z, y, x]
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref)), (z, y, x)


def test_c2_20000_steps_fp32_against_fp64():
    from paper_1908_04443_gb300 import lbmwet as L
    eos, g, l = _eos(0.6)
    wl = W.c2_cylinder_600x400(kappa=0.15)
    out = {}
    for prec in ("fp64", "fp32"):
        with L.Simulation(_cfg(L, wl, prec, g, l), wl.mask(), wl.rho0(l, g)) as sim:
            sim.step(wl.steps)
            out[prec] = sim.observables(fields=True)
    o64, r64, _ = out["fp64"]
    o32, r32, _ = out["fp32"]
    bulk, band, nb, ni = split_errors(r32, r64, wl.mask(), l, g)
    print(f"C2 FP32 vs FP64 after 20000 steps: bulk max |drho|/rho = {bulk:.3e} over {nb} nodes, "
          f"interface band max |drho|/rho_l = {band:.3e} over {ni} nodes")
    assert bulk <= 1e-4
    assert band <= 1e-4
    assert abs(o32.theta_deg - o64.theta_deg) <= 0.5
    assert abs(o32.mass / o64.mass - 1) <= 1e-4


GOLDEN_C2 = os.path.join(os.path.dirname(__file__), "golden", "c2_600x400_kappa0.15_20000.npz")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_c2_20000_steps_against_oracle_golden(prec):
    """The 600 x 400 workload after its 20000 steps against the FP64 oracle's result (written by
    tests/golden/make_c2_golden.py, which calls only the oracle).  FP32: the split density bounds
    (1e-4 relative at bulk nodes, 1e-4 of rho_l in the interface band) and the contact angle within
    0.5 degrees.  FP64: the contact angle within 1e-6 degrees, the density within 1e-8 and the mass
    within 1e-11.  One step agrees with the oracle to 1e-16 (the same arithmetic in another order);
    over 20000 steps of the still-spreading drop those differences grow to 2.3e-9 in density
    (measured on GB300), so the 1e-10 of the 1000-step parity case is out of reach here and 1e-8 is
    the bound.  The total mass drifts by rounding on both sides (at most a few ulps of the sum per
    step, about 2e-12 relative after 20000 steps each)."""
    from paper_1908_04443_gb300 import lbmwet as L
    ref = np.load(GOLDEN_C2)
    eos, g, l = _eos(0.6)
    assert abs(float(ref["rho_l"]) - l) < 1e-14 and abs(float(ref["rho_g"]) - g) < 1e-14
    wl = W.c2_cylinder_600x400(kappa=float(ref["kappa"]))
    with L.Simulation(_cfg(L, wl, prec, g, l), wl.mask(), wl.rho0(l, g)) as sim:
        sim.step(int(ref["steps"]))
        o, rho, _ = sim.observables(fields=True)
    rho_ref = ref["rho"]
    fl = wl.mask() == 0
    d = np.abs(rho - rho_ref)[fl]
    bulk, band, nb, ni = split_errors(rho, rho_ref, wl.mask(), l, g)
    print(f"C2 {prec} vs oracle after 20000 steps: max |drho| = {d.max():.3e}, bulk max |drho|/rho = {bulk:.3e}, "
          f"band max |drho|/rho_l = {band:.3e}, theta {o.theta_deg:.6f} vs {float(ref['theta_deg']):.6f} deg")
    if prec == "fp32":
        assert bulk <= 1e-4
        assert band <= 1e-4
        assert abs(o.theta_deg - float(ref["theta_deg"])) <= 0.5
    else:
        assert d.max() <= 1e-8
        assert abs(o.theta_deg - float(ref["theta_deg"])) <= 1e-6
        assert abs(o.mass / float(ref["mass"]) - 1) <= 1e-11


GOLDEN_D3 = os.path.join(os.path.dirname(__file__), "golden", "d3q19_sphere64_1000.npz")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_d3q19_sphere64_1000_steps_against_oracle_golden(prec):
    """A 64^3 drop on a sphere (the 256^3 workload's sphere scaled by 1/4, drop radius 16) after 1000
    steps, while the drop is still spreading, against the FP64 oracle's stored result (written by
    tests/golden/make_d3q19_sphere64_golden.py, which calls only the oracle).  FP32 runs the default
    D3Q19 step, the TMA-staged z-march (64 nodes is the narrowest grid it boxes), and is held to the
    split density bounds and 0.5 degrees; FP64 (the scalar z-march) to 1e-9 in density, 1e-6
    degrees and 1e-12 in mass."""
    from paper_1908_04443_gb300 import lbmwet as L
    ref = np.load(GOLDEN_D3)
    wl = W.sphere_drop_64(int(ref["steps"]))
    assert wl.shape[0] == int(ref["n"])
    eos, g, l = _eos(wl.t_over_tc)
    assert abs(float(ref["rho_l"]) - l) < 1e-14 and abs(float(ref["rho_g"]) - g) < 1e-14
    with L.Simulation(_cfg(L, wl, prec, g, l), wl.mask(), wl.rho0(l, g)) as sim:
        if prec == "fp32":
            assert sim.step_kernel() == "ztma"
        sim.step(int(ref["steps"]))
        o, rho, _ = sim.observables(fields=True)
    rho_ref = ref["rho"]
    d = np.abs(rho - rho_ref)[wl.mask() == 0]
    bulk, band, nb, ni = split_errors(rho, rho_ref, wl.mask(), l, g)
    print(f"D3Q19 64^3 {prec} vs oracle after {int(ref['steps'])} steps: max |drho| = {d.max():.3e}, "
          f"bulk max |drho|/rho = {bulk:.3e}, band max |drho|/rho_l = {band:.3e}, "
          f"theta {o.theta_deg:.6f} vs {float(ref['theta_deg']):.6f} deg")
    if prec == "fp32":
        assert bulk <= 1e-4
        assert band <= 1e-4
        assert abs(o.theta_deg - float(ref["theta_deg"])) <= 0.5
    else:
        assert d.max() <= 1e-9       # measured 3.4e-10: rounding-order differences grown by the moving contact line
        assert abs(o.theta_deg - float(ref["theta_deg"])) <= 1e-6
        assert abs(o.mass / float(ref["mass"]) - 1) <= 1e-12
