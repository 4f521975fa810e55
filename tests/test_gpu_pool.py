"""The device memory pool behind handles and batches: memory freed by lbm_destroy returns to the
pool (its in-use bytes fall back), a later grid reuses it (no new reservation) and steps bit for bit
as on fresh memory, and lbm_release_cached_memory hands the unused part back to the driver."""
import numpy as np
import pytest

from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def _case(shape=(96, 128)):
    return drop_on_cylinder(shape, (40.0, 64.0), 14.0, (62.0, 64.0), 16.0, kappa=0.05)


def _run(case, steps, precision="fp32"):
    with case.gpu(precision) as sim:
        sim.step(steps)
        return sim.get_state().copy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pool_reuse_is_bit_identical(precision):
    from paper_1908_04443_gb300 import lbmwet as L
    a, b = _case(), _case((160, 200))
    L.lbm_release_cached_memory()
    ref = _run(a, 12, precision)
    _run(b, 5, precision)          # another grid on the same (now cached) memory
    again = _run(a, 12, precision)
    assert np.array_equal(ref, again)


def test_pool_accounting_and_release():
    from paper_1908_04443_gb300 import lbmwet as L
    L.lbm_release_cached_memory()
    r0, u0 = L.lbm_memory_stats()
    case = _case((200, 256))
    sim = case.gpu("fp32")
    r1, u1 = L.lbm_memory_stats()
    # two distribution buffers of 9 x (ny x padded nx) floats at least
    assert u1 - u0 >= 2 * 9 * 200 * 256 * 4
    assert r1 >= u1
    sim.step(3)
    sim.close()
    r2, u2 = L.lbm_memory_stats()
    assert u2 == u0                 # everything the handle held is back in the pool
    assert r2 >= u1 - u0            # and stays reserved
    sim = case.gpu("fp32")          # the same grid again: served from the reserve
    r3, _ = L.lbm_memory_stats()
    assert r3 == r2
    sim.close()
    L.lbm_release_cached_memory()
    r4, u4 = L.lbm_memory_stats()
    assert u4 == u0 and r4 <= r2 - (u1 - u0) // 2


def test_batch_memory_returns_to_pool():
    from paper_1908_04443_gb300 import lbmwet as L
    import workloads as W
    from oracle import eos as E
    e = E.cs_config().at_reduced_temperature(0.7)
    g, l = E.maxwell(e)
    wls = W.c4_batch(6)
    ee = L.make_eos("CS", 0.25, 4.0, 1.0, 0.0)
    ee.T = 0.7 * L.lbm_critical_temperature(ee)
    cfgs = [L.make_config("D2Q9", "fp32", wl.shape, ee, sigma=0.12, rho_l=l, rho_g=g, kappa=0.05, rho_ref=g)
            for wl in wls]
    L.lbm_release_cached_memory()
    _, u0 = L.lbm_memory_stats()
    b = L.lbm_batch_init(cfgs, [wl.mask() for wl in wls], [wl.rho0(l, g) for wl in wls])
    L.lbm_batch_step(b, 4)
    for i in range(len(wls)):
        L.lbm_observables(L.lbm_batch_handle(b, i))
    L.lbm_batch_destroy(b)
    _, u1 = L.lbm_memory_stats()
    assert u1 == u0
