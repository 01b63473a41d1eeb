"""The learned warm start end to end on a small mosaic: training pairs from the plain solver,
U-Net training with the library's own kernels, and the gain it brings: from the network's
initial sky the solver reaches the cold start's final cost (within 1e-4) in fewer iterations
than the cold start needed. The cold start remains the judge of the final cost."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_warm_start_reaches_cold_final_cost_in_fewer_iterations():
    from paper_2609_17636_b300 import UNet, warmstart
    desc = synth.small_mosaic(501, n=128, nb=64, nchan=1, npoint=3, ndump=24, n_ant=30,
                              cell_arcsec=15.0, lambda_r=1e-2, lambda_s=0.0, ragged=False)
    desc.sigma_vis = 1e-3
    for p in desc.pairs:
        p.weight = np.full(p.m, 1e6, np.float32)
    prob = warmstart.sky_problem(desc, lambda_r=1e-2)
    rng = np.random.default_rng(9)
    train_skies = [synth.lognormal_sky(synth.make_rng(10_000 + i), 128)[None] for i in range(48)]
    ts = warmstart.make_pairs(prob, train_skies, crop=64, crops_per_sky=4, maxiter=300, rng=rng)
    net = UNet(8, max_batch=8, max_hw=128 * 128)
    net.set_params(synth.unet_init(8, 0))
    hist = warmstart.train(net, ts, epochs=25, batch=8, lr=2e-3, rng=rng)
    assert hist[-1] < 0.5 * hist[0], hist
    gains = []
    for i in range(3):
        sky = synth.lognormal_sky(synth.make_rng(100_000 + i), 128)[None]
        r = warmstart.compare_solves(net, prob, sky, rng, maxiter=300)
        assert r["warm_reached"], r
        gains.append(r["cold_iters"] - r["warm_iters"])
    assert np.mean(gains) > 0, gains
    net.close()
    prob.plan.close()
