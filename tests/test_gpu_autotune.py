"""The batch autotuner and batches whose instances step with different kernels.

* Mixed kernels (lbm_batch_set_kernels): each group steps as its own branch of the captured steps;
  every instance equals the same grid stepped alone with its kernel, bit for bit, over graph chunks
  and single launches.
* lbm_batch_autotune: times the candidates per size class from the current state and restores it
  (the state after tuning equals the state before, bit for bit); afterwards every instance equals
  its grid stepped alone with the kernel chosen for it, and one batched step agrees with the FP64
  oracle on sampled instances; a later batch with the automatic choice reuses the chosen kernels.
"""
import numpy as np
import pytest

from oracle import lbm
from tests.harness import drop_on_cylinder

pytestmark = pytest.mark.gpu


def _cases():
    # three size classes: 2^10 (40 x 48, 37 x 53), 2^14 (128 x 160), 2^16 (256 x 300)
    return [drop_on_cylinder((40, 48), (24.0, 14.0), 7.0, (24.0, 27.0), 8.0, kappa=0.2),
            drop_on_cylinder((37, 53), (20.3, 17.1), 9.5, (21.0, 30.0), 10.0, kappa=-0.02),
            drop_on_cylinder((128, 160), (80.0, 40.0), 16.0, (80.0, 74.0), 18.0, kappa=0.1),
            drop_on_cylinder((256, 300), (150.0, 80.0), 30.0, (150.0, 142.0), 32.0, kappa=0.05)]


def _batch(cases, precision):
    from paper_1908_04443_gb300 import lbmwet as L
    for cs in cases:
        cs.rho_ref = cs.bounds()[0] if precision == "fp32" else 0.0
    sims = [cs.gpu(precision) for cs in cases]
    cfgs = [s.cfg for s in sims]
    for s in sims:
        s.close()
    return L.lbm_batch_init(cfgs, [cs.mask for cs in cases], [cs.rho0 for cs in cases], None)


def _single(cs, precision, kernel, steps):
    cs.step_kernel = kernel
    with cs.gpu(precision) as sim:
        sim.step(steps)
        return sim.get_state().reshape(-1)


@pytest.mark.parametrize("precision,kinds", [("fp32", ["pair", "tile", "ymarch", "pair"]),
                                             ("fp64", ["ymarch", "tile", "tile", "ymarch"])])
def test_mixed_kernel_groups_equal_single_runs(precision, kinds):
    from paper_1908_04443_gb300 import lbmwet as L
    cases = _cases()
    b = _batch(cases, precision)
    try:
        L.lbm_batch_set_kernels(b, kinds)
        assert [L.lbm_batch_instance_kernel(b, i) for i in range(len(cases))] == kinds
        assert L.lbm_batch_step_kernel_used(b) == "auto"          # mixed
        L.lbm_batch_step(b, 37)                                     # 2 graph chunks of 16 + 5 single steps
        assert L.lbm_batch_kernel_launches(b) == 37 * len(set(kinds))
        for i, cs in enumerate(cases):
            fb = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size)
            assert np.array_equal(fb, _single(cs, precision, kinds[i], 37)), f"instance {i} ({kinds[i]})"
    finally:
        L.lbm_batch_destroy(b)


def test_autotune_keeps_the_state_and_steps_with_its_choice():
    from paper_1908_04443_gb300 import lbmwet as L
    L.lbm_batch_autotune_forget()
    cases = _cases()
    b = _batch(cases, "fp32")
    try:
        before = [L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size) for i, cs in enumerate(cases)]
        report = L.lbm_batch_autotune(b, 6)
        print(report)
        assert report.count("chosen") == 3                          # one choice per size class
        for i, cs in enumerate(cases):
            assert np.array_equal(L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size), before[i])
        kinds = [L.lbm_batch_instance_kernel(b, i) for i in range(len(cases))]
        assert kinds[0] == kinds[1]                                 # same class, same choice
        L.lbm_batch_step(b, 20)
        for i, cs in enumerate(cases):
            fb = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size)
            assert np.array_equal(fb, _single(cs, "fp32", kinds[i], 20)), f"instance {i} ({kinds[i]})"
        # one tuned batched step against the FP64 oracle on two instances
        state = {i: L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cases[i].mask.size) for i in (0, 3)}
        L.lbm_batch_step(b, 1)
        for i in (0, 3):
            cs = cases[i]
            geo, p, _ = cs.oracle()
            ref = lbm.step(state[i].reshape((9,) + cs.shape), geo, p)
            got = L.lbm_get_state(L.lbm_batch_handle(b, i), 9, cs.mask.size).reshape((9,) + cs.shape)
            assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
        # a new batch with the automatic choice takes the tuned kernels
        b2 = _batch(_cases(), "fp32")
        try:
            assert [L.lbm_batch_instance_kernel(b2, i) for i in range(len(cases))] == kinds
        finally:
            L.lbm_batch_destroy(b2)
    finally:
        L.lbm_batch_destroy(b)
        L.lbm_batch_autotune_forget()


def test_autotune_rejects_too_few_trial_steps():
    from paper_1908_04443_gb300 import lbmwet as L
    b = _batch(_cases()[:1], "fp32")
    try:
        with pytest.raises(L.LbmError):
            L.lbm_batch_autotune(b, 1)
    finally:
        L.lbm_batch_destroy(b)
