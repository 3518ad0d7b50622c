"""Failure detection without a GPU fault: every tensor-core pipeline wait is
bounded (cc_model_config.wait_limit_ns); a wait that runs out records
TIMEOUT in the model's device error word, lets the copies already issued
land, frees its tensor memory and returns.  The test hook
cc_model_test_withhold_copy leaves one K slice's window rows unrequested in
one launch, so the waits on it run out after 1 ms.  The model must report it
and then stream correctly again (the TMEM of the launch that gave up was
released, or the next launches could not allocate theirs)."""
import numpy as np
import pytest

from oracle import metrics
from oracle import model as M
from oracle import pqmf
from paper_2204_07064_gb300 import api
from paper_2204_07064_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _bf16_decoder():
    nodes = W.rave_decoder(latent=16, capacity=64, ratios=(4, 2), dilations=(1, 3), bands=8, pqmf_taps=32)
    p = W.init_params(nodes, 1)
    _, g, _, _ = pqmf.design(8, 32)
    p[W.pqmf_node_index(nodes)] = (pqmf.synthesis_weights(g), None)
    return nodes, p


def _run(model, stream, z, cuda):
    import torch

    ops = model.io["out_per_step"]
    outs = []
    for t in range(0, len(z), 2):
        x = torch.tensor(z[t:t + 2], dtype=torch.float32, device=cuda)
        y = torch.empty((2 * ops, 1), dtype=torch.float32, device=cuda)
        stream.process(x, y)
        outs.append(y.cpu().numpy())
    return np.concatenate(outs).astype(np.float64)


@pytest.mark.parametrize("launches", [1, 3])
def test_bounded_wait_runs_out_then_model_recovers(cclib, cuda, launches):
    import torch

    nodes, p = _bf16_decoder()
    model = api.Model(nodes, p, dtype="bf16", max_streams=2, max_steps_per_call=2, wait_limit_ns=1_000_000)
    s = model.stream(seed=21)
    z = W.signal(6, 6, 16)
    model.test_withhold_copy(launches)
    _run(model, s, z[:2], cuda)
    torch.cuda.synchronize()
    status, code = model.device_status_code()
    assert status == -6  # CC_ERR_TIMEOUT
    assert code & 4  # the MMA issuer gave up waiting for the withheld slice
    assert code & ~7 == 0
    assert model.device_status_code() == (0, 0)  # the record was cleared
    # the launches that gave up released their tensor memory: the model streams
    # correctly again from a reset, at the BF16 bar against the oracle
    s.reset()
    out = _run(model, s, z, cuda)
    ref = M.run_causal(nodes, p, z, seed=21)
    snr = metrics.snr_db(ref, out)
    assert snr >= 35.0 and metrics.max_abs(ref, out) <= 2e-2 * np.max(np.abs(ref)), f"SNR {snr:.1f} dB"
    assert model.device_status() == 0
