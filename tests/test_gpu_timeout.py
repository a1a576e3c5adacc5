"""Device-side failure reporting: a bounded wait that runs out is reported by
inrct_device_status as INRCT_ERR_TIMEOUT, and the context stays usable.

The wait is made to run out without any fault: the library's test hook keeps the tile
kernel's producer from issuing weight loads, so nothing is in flight when the MMA issuer's
first wait on a weight chunk gives up (after a 5 ms limit); the kernel's roles then stop,
release tensor memory and return.  The next normal call on the same process gives the same
result as before the stall."""
import numpy as np
import pytest
import torch

from paper_2604_09884_gb300 import inrct, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["siren", "ffn"])
def test_a_wait_that_runs_out_is_reported_and_the_next_call_succeeds(kind):
    dev = torch.device("cuda")
    if kind == "siren":
        spec, B = synth.ArchSpec("siren", 2, 128, 3, omega0=30.0), None
    else:
        spec = synth.ArchSpec("ffn", 2, 256, 3, n_feat=256, sigma=4.0)
        B = synth.fourier_matrix(spec.n_feat, 2, spec.sigma, 1).astype(np.float32)
    N = 64
    mlp = inrct.mlp_desc(spec, inrct.BF16, B, device=dev)
    theta = torch.tensor(synth.init_theta(spec, 2).astype(np.float32), device=dev)
    v = torch.tensor(np.random.default_rng(3).normal(size=N * N).astype(np.float32), device=dev)
    idx = torch.from_numpy(synth.index_set(N * N, 1500, 4)).to(dev)
    inrct.device_status()                                   # nothing pending from earlier tests
    img0 = inrct.inr_eval_grid(mlp, theta, N)
    g0 = inrct.inr_weighted_vjp(mlp, theta, N, idx, v, 2.0)
    inrct.device_status()
    try:
        inrct.set_wait_limit(5_000_000)
        inrct.debug_stall_weight_loads(True)
        inrct.inr_eval_grid(mlp, theta, N)                  # returns OK: launches are asynchronous
        with pytest.raises(inrct.InrctError) as e:
            inrct.device_status()
        # the MMA issuer's wait for the first weight chunk (303) or, when the first stage streams
        # more than four input panels, the epilogue's wait for a free panel buffer (401) runs
        # out first: both wait on the loads that never come
        assert e.value.code == 5 and ("code 303" in str(e.value) or "code 401" in str(e.value)), str(e.value)
        inrct.inr_weighted_vjp(mlp, theta, N, idx, v, 2.0)
        with pytest.raises(inrct.InrctError) as e:
            inrct.device_status()
        assert e.value.code == 5, str(e.value)
    finally:
        inrct.debug_stall_weight_loads(False)
        inrct.set_wait_limit(0)
    inrct.device_status()                                   # cleared by the reads above
    img1 = inrct.inr_eval_grid(mlp, theta, N)
    g1 = inrct.inr_weighted_vjp(mlp, theta, N, idx, v, 2.0)
    inrct.device_status()
    assert torch.equal(img1, img0)
    assert torch.equal(g1, g0)
