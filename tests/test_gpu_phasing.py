"""Phasing (Sec. II-D) on the GPU against the FP64 oracle: the magnitudes of a
merged model (c2 and c5 grids), ER / HIO iterates and their Fourier errors,
the shrinkwrap support, and recovery of a known object on the GPU alone."""
import numpy as np
import pytest

import synth
from oracle import phasing as oph
from tests.gpu_util import f32, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _blobs(N, centres, widths, weights):
    M = (N - 1) // 2
    d = np.arange(-M, M + 1, dtype=np.float64)
    z, y, x = np.meshgrid(d, d, d, indexing="ij")
    rho = np.zeros((N, N, N))
    for (cx, cy, cz), w, a in zip(centres, widths, weights):
        rho += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * w * w))
    return rho


@pytest.fixture(scope="module")
def known():
    N = 25
    rho_true = _blobs(N, [(-3, 1, 0), (1, -2, 1), (2, 2, -1)], [1.0, 1.3, 0.9], [1.0, 0.6, 0.8])
    support = rho_true > 1e-2 * rho_true.max()
    rho_true *= support
    amp = np.abs(oph.dft3(rho_true)).astype(np.float32)
    rho0 = (np.random.default_rng(4).uniform(0, 1, (N, N, N)) * support).astype(np.float32)
    return N, rho_true, support, amp, rho0


def _phaser(N, amp, rho0, support):
    import torch
    from paper_2109_05339_gb300 import Phaser
    ph = Phaser(N)
    ph.set_amplitudes(to_dev(amp))
    ph.set_state(to_dev(rho0), torch.as_tensor(support.astype(np.uint8)).cuda())
    return ph


@pytest.mark.parametrize("name", ["c2", "c5"])
def test_amplitudes_of_the_merged_model(name):
    """sqrt(max(Re DFT(x), 0)) of the model on the 81^3 and 151^3 grids."""
    from paper_2109_05339_gb300 import Phaser
    cfg = synth.CONFIGS[name]
    rng = np.random.default_rng(61)
    centres, sigmas, weights = synth.gaussian_density(rng, 40)
    _, A = synth.model_grid(cfg.N, cfg.qmax, centres, sigmas, weights)
    ph = Phaser(cfg.N)
    ph.amplitudes_from_model(to_dev(A.astype(np.float32)))
    _, _, amp = ph.get()
    ref = oph.amplitudes_from_model(f32(A.astype(np.float32)))
    assert rel_l2(amp.cpu().numpy(), ref) < 1e-5, rel_l2(amp.cpu().numpy(), ref)
    ph.close()


def test_er_and_hio_iterates_match_the_oracle(known):
    """From the same seed: 20 ER steps with positivity, and 30 HIO then 10 ER
    steps with the support alone, against the FP64 oracle (iterates and
    every Fourier error). HIO with positivity is left to the recovery test:
    its update jumps between rho - beta P_M rho and P_M rho where P_M rho
    crosses zero, so FP32 and FP64 trajectories part once such a voxel
    flips. ER's projections do not expand differences, so its iterates stay
    within 1e-4; HIO's steps outside the support can, and 40 steps amplify
    the transforms' FP32 rounding (about 1e-6 relative per step) to about
    2e-4 (measured), bounded here by 1e-3."""
    import torch
    N, rho_true, support, amp, rho0 = known
    for sched, pos, tol in (([("er", 20)], True, 1e-4), ([("hio", 30, 0.9), ("er", 10)], False, 1e-3)):
        ph = _phaser(N, amp, rho0, support)
        errs = ph.run(sched, positivity=pos)
        rho, _, _ = ph.get()
        torch.cuda.synchronize()
        ref_rho, _, ref_errs = oph.run(f32(amp), f32(rho0), support, sched, positivity=pos)
        assert rel_l2(rho.cpu().numpy(), ref_rho) < tol, (sched, rel_l2(rho.cpu().numpy(), ref_rho))
        np.testing.assert_allclose(errs.cpu().numpy(), ref_errs, rtol=tol)
        ph.close()


def test_iterations_at_the_c5_grid():
    """Two HIO and two ER steps on the 151^3 grid (magnitudes of a merged
    model, a box support, no positivity) against the oracle."""
    import torch
    from paper_2109_05339_gb300 import Phaser
    cfg = synth.CONFIGS["c5"]
    N, M = cfg.N, (cfg.N - 1) // 2
    rng = np.random.default_rng(62)
    centres, sigmas, weights = synth.gaussian_density(rng, 60)
    _, A = synth.model_grid(N, cfg.qmax, centres, sigmas, weights)
    amp = oph.amplitudes_from_model(A).astype(np.float32)
    d = np.arange(-M, M + 1)
    z, y, x = np.meshgrid(d, d, d, indexing="ij")
    support = (np.abs(x) <= 30) & (np.abs(y + 3) <= 25) & (np.abs(z - 2) <= 35)
    rho0 = (rng.uniform(0, 1, (N, N, N)) * support).astype(np.float32)
    ph = Phaser(N)
    ph.set_amplitudes(to_dev(amp))
    ph.set_state(to_dev(rho0), torch.as_tensor(support.astype(np.uint8)).cuda())
    sched = [("hio", 2, 0.8), ("er", 2)]
    errs = ph.run(sched, positivity=False)
    rho, _, _ = ph.get()
    ref_rho, _, ref_errs = oph.run(f32(amp), f32(rho0), support, sched, positivity=False)
    assert rel_l2(rho.cpu().numpy(), ref_rho) < 1e-4, rel_l2(rho.cpu().numpy(), ref_rho)
    np.testing.assert_allclose(errs.cpu().numpy(), ref_errs, rtol=1e-4)
    ph.close()


def test_shrinkwrap_support_matches_the_oracle(known):
    """The support from the blurred |rho| equals the oracle's except where the
    blur lies within FP32 rounding of the threshold."""
    import torch
    N, rho_true, support, amp, _ = known
    rng = np.random.default_rng(63)
    rho = (rho_true + 0.05 * rng.standard_normal((N, N, N))).astype(np.float32)
    ph = _phaser(N, amp, rho, support)
    ph.shrinkwrap(1.7, 0.3)
    _, sup, _ = ph.get()
    torch.cuda.synchronize()
    b = oph.blur(f32(rho), 1.7)
    ref = b > 0.3 * b.max()
    near = np.abs(b - 0.3 * b.max()) < 1e-5 * b.max()
    got = sup.cpu().numpy().astype(bool)
    np.testing.assert_array_equal(got[~near], ref[~near])
    assert ref.sum() > 100 and (~ref).sum() > 100
    ph.close()


def test_known_object_recovered_on_the_gpu(known):
    """The recovery the oracle is pinned on -- 1000 HIO and 200 ER steps from
    the magnitudes and the object's support -- run on the GPU alone."""
    N, rho_true, support, amp, rho0 = known
    ph = _phaser(N, amp, rho0, support)
    errs = ph.run([("hio", 1000, 0.9), ("er", 200)])
    rho, _, _ = ph.get()
    e = errs.cpu().numpy()
    assert e[-1] < 5e-4, e[-1]
    assert rel_l2(rho.cpu().numpy(), rho_true) < 1e-2
    ph.close()
