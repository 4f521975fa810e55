"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point that
include/lbmwet.h declares, its host-only thermodynamics agree with the oracle, and invalid
configurations are rejected with LBM_ERR_ARG before any device work."""
import os
import re

import numpy as np
import pytest

from paper_1908_04443_gb300 import lbmwet as L
from oracle import eos as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lbmwet.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lbm_status|void|int64_t|int32_t|lbm_handle\*|const char\*)\s+(lbm_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 19
    lib = L.library()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTED)


def test_struct_layout_matches_header_order():
    # the ctypes mirror must list the C struct members in declaration order
    text = open(os.path.join(ROOT, "include", "lbmwet.h")).read()
    body = re.search(r"typedef struct \{((?:(?!typedef).)*?)\} lbm_config;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    members = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        for nm in names.split(","):
            members.append(nm.strip().split("[")[0])
    assert members == [f[0] for f in L.lbm_config._fields_]


@pytest.mark.parametrize("kind,tr", [("PR", 0.86), ("CS", 0.7), ("CS", 0.6)])
def test_coexistence_matches_oracle(kind, tr):
    o = E.pr_paper() if kind == "PR" else E.cs_config()
    tc_o = o.tc()
    e = L.make_eos(kind, o.a, o.b, o.R, 0.0, o.omega)
    tc = L.lbm_critical_temperature(e)
    assert abs(tc / tc_o - 1) < 1e-9
    o = o.at_reduced_temperature(tr)
    e.T = tr * tc
    g, l = L.lbm_coexistence(e)
    go, lo = E.maxwell(o)
    assert abs(g / go - 1) < 1e-8
    assert abs(l / lo - 1) < 1e-10


def test_coexistence_rejects_supercritical():
    e = L.make_eos("CS", 0.25, 4.0, 1.0, 1.0)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_coexistence(e)
    assert ei.value.status == L.LBM_ERR_ARG


def _cfg(**kw):
    e = L.make_eos("CS", 0.25, 4.0, 1.0, 0.0)
    e.T = 0.7 * L.lbm_critical_temperature(e)
    return L.make_config("D2Q9", "fp64", (8, 8), e, **kw)


@pytest.mark.parametrize("bad", [dict(s_e=0.0), dict(s_nu=2.0), dict(s_q=-1.0), dict(G=0.0), dict(wall="VD")])
def test_init_rejects_bad_config(bad):
    wall_ok = bad.pop("wall", None)
    cfg = _cfg(**bad)
    if wall_ok:
        cfg.wall_kind = 7
    with pytest.raises(L.LbmError) as ei:
        L.lbm_init(cfg, np.zeros((8, 8), np.uint8))
    assert ei.value.status == L.LBM_ERR_ARG


def test_init_rejects_bad_grid():
    cfg = _cfg()
    cfg.nz = 2          # D2Q9 with nz != 1
    with pytest.raises(L.LbmError):
        L.lbm_init(cfg, np.zeros(128, np.uint8))
    cfg = _cfg()
    cfg.eos.T = 10.0    # above the critical temperature
    with pytest.raises(L.LbmError) as ei:
        L.lbm_init(cfg, np.zeros((8, 8), np.uint8))
    assert ei.value.status == L.LBM_ERR_ARG


def test_batch_rejects_mixed_physics_before_device_work():
    a = _cfg()
    b = _cfg(sigma=0.2)
    m = np.zeros((8, 8), np.uint8)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_init([a, b], [m, m])
    assert ei.value.status == L.LBM_ERR_ARG
    assert "differs" in str(ei.value)


def test_batch_checks_every_instance_before_its_host_scans():
    """lbm_batch_init checks every configuration and mask before it scans any mask (the scans run on
    several host threads) or touches the device: a bad grid or a missing mask of a later instance is
    rejected with LBM_ERR_ARG and the instance named."""
    m = np.zeros((8, 8), np.uint8)
    bad = _cfg()
    bad.nz = 2                  # D2Q9 with nz != 1
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_init([_cfg(), _cfg(), bad], [m, m, np.zeros(128, np.uint8)])
    assert ei.value.status == L.LBM_ERR_ARG
    assert "instance 2" in str(ei.value)
    neg = _cfg()
    neg.nx = -5
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_init([_cfg(), neg], [m, m])
    assert ei.value.status == L.LBM_ERR_ARG
    assert "instance 1" in str(ei.value)
    # a null mask pointer through the C ABI itself (the binding refuses None before the call)
    cfgs = (L.lbm_config * 2)(_cfg(), _cfg())
    masks = (L.C.c_void_p * 2)(m.ctypes.data, None)
    b = L.C.c_void_p()
    assert L._lib.lbm_batch_init(2, cfgs, masks, None, None, None, L.C.byref(b)) == L.LBM_ERR_ARG
    assert not b.value
    assert "instance 1" in L._lib.lbm_batch_last_error(None).decode()


@pytest.mark.parametrize("which", ["none", "short_mask", "long_rho0", "count"])
def test_binding_checks_batch_array_sizes(which):
    """The binding refuses arrays whose size is not the grid's, since the library reads exactly
    nx * ny * nz values from every pointer it is given."""
    m = np.zeros((8, 8), np.uint8)
    masks, rho0s = [m, m], None
    if which == "none":
        masks = [m, None]
    elif which == "short_mask":
        masks = [m, np.zeros(63, np.uint8)]
    elif which == "long_rho0":
        rho0s = [None, np.ones(65)]
    else:
        masks = [m]
    with pytest.raises(ValueError):
        L.lbm_batch_init([_cfg(), _cfg()], masks, rho0s)


def test_sf_scheme_rejects_non_finite_gw_and_mixed_gw_batches():
    """The solid-fluid interaction scheme needs a finite G_w, and a batch shares one G_w: both are
    rejected with LBM_ERR_ARG before any device work."""
    cfg = _cfg(wall="SF", Gw=float("nan"))
    with pytest.raises(L.LbmError) as ei:
        L.lbm_init(cfg, np.zeros((8, 8), np.uint8))
    assert ei.value.status == L.LBM_ERR_ARG
    m = np.zeros((8, 8), np.uint8)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_init([_cfg(wall="SF", Gw=-0.1), _cfg(wall="SF", Gw=0.2)], [m, m])
    assert ei.value.status == L.LBM_ERR_ARG


def test_bounded_wait_selftest_rejects_zero_polls_before_device_work():
    with pytest.raises(L.LbmError) as ei:
        L.lbm_selftest_bounded_wait(0)
    assert ei.value.status == L.LBM_ERR_ARG


@pytest.mark.parametrize("case", ["3d", "theta0", "theta180", "thetanan", "kappa", "thin"])
def test_gf_scheme_rejections(case):
    """The geometric-formulation scheme is two-dimensional, needs 0 < theta_a < 180, takes no
    per-wall-node kappa, and cannot give a normal to a wall node whose Eq. 13 sum vanishes (a solid
    line one node thick): each is rejected with LBM_ERR_ARG before any device work."""
    e = L.make_eos("CS", 0.25, 4.0, 1.0, 0.0)
    e.T = 0.7 * L.lbm_critical_temperature(e)
    shape, kw, mask, kpw = (8, 10), dict(wall="GF", theta_a=60.0), None, None
    if case == "3d":
        shape = (6, 8, 10)
    elif case.startswith("theta"):
        kw["theta_a"] = {"theta0": 0.0, "theta180": 180.0, "thetanan": float("nan")}[case]
    mask = np.zeros(shape, np.uint8)
    if case == "thin":
        mask[4, :] = 1                                  # a one-node-thick plate, periodic in x
    else:
        mask[..., :2, :] = 1
    if case == "kappa":
        kpw = np.full(int(mask.sum()), 0.1)
    cfg = L.make_config("D3Q19" if case == "3d" else "D2Q9", "fp64", shape, e, **kw)
    with pytest.raises(L.LbmError) as ei:
        L.lbm_init(cfg, mask, kappa_per_wall=kpw)
    assert ei.value.status == L.LBM_ERR_ARG
    if case == "thin":
        assert "normal" in str(ei.value)


def test_batch_rejects_mixed_wall_schemes():
    """A batch shares one wall scheme (instances may differ in its per-grid parameter, such as the
    geometric formulation's theta_a): a geometric-formulation grid with an IVD grid is rejected with
    LBM_ERR_ARG before any device work."""
    m = np.zeros((8, 8), np.uint8)
    m[:2, :] = 1
    with pytest.raises(L.LbmError) as ei:
        L.lbm_batch_init([_cfg(wall="GF", theta_a=60.0), _cfg(kappa=0.1)], [m, m])
    assert ei.value.status == L.LBM_ERR_ARG
