"""Which rounding of the 16-bit precision variants moves the flows, in FP64 (CPU).

The precision variants are held to EPE <= 0.05 px against the FP32 flows.  The FP64 oracle
network with only the weights, or only the stored activations, rounded to a 16-bit format
(oracle.quant.flow_pair_16) attributes the deviation: on the He-init 5-level network
bfloat16 weights alone move the flows by more than 0.05 px, so no BF16 kernel can meet the
bar with these weights, while IEEE half weights and activations together stay well inside
it.  The GPU tests hold TC_FP16 to the bar and TC_BF16 to its representation bound."""
import numpy as np
import pytest

import oracle
import synth
from oracle import quant


def test_round16_matches_library_conversions():
    torch = pytest.importorskip("torch")
    g = synth.rng(90)
    a = np.concatenate([g.normal(0, 1, 20000), g.normal(0, 1e-5, 2000), g.uniform(-7e4, 7e4, 2000)]).astype(np.float32)
    bf = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(quant.round16(a, "bf16"), bf)
    h = torch.from_numpy(a).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(quant.round16(a, "fp16"), h, equal_nan=True)
    # hand-worked ties: 1 + 2^-8 lies halfway between two bfloat16 values and goes to even (1)
    assert quant.round16(np.float32(1 + 2.0 ** -8), "bf16") == 1.0
    assert quant.round16(np.float32(1 + 3 * 2.0 ** -8), "bf16") == 1 + 2.0 ** -6
    assert quant.round16(np.float32(1 + 2.0 ** -11), "fp16") == 1.0


@pytest.fixture(scope="module")
def net5():
    spec = synth.NetSpec()
    layers = synth.he_weights(spec, seed=0)
    net = oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)
    seq = synth.Sequence(width=200, height=136, seed=1)
    Ia, Ib = seq.frame(1), seq.frame(0)
    return net, Ia, Ib, oracle.flow_pair(net, Ia, Ib)


def _epe(net5, fmt, weights, activations):
    net, Ia, Ib, (fab, fba) = net5
    gab, gba = quant.flow_pair_16(net, Ia, Ib, fmt, weights, activations)
    return max(oracle.epe(gab, fab), oracle.epe(gba, fba))


def test_no_rounding_is_the_oracle_network(net5):
    assert _epe(net5, "bf16", False, False) < 1e-9


def test_bf16_weights_alone_exceed_the_fixed_epe_bar(net5):
    # measured 0.077 px (0.12 px at 1080p, where the mean flow is 21 px)
    assert _epe(net5, "bf16", True, False) > 0.05


def test_fp16_meets_the_fixed_epe_bar_with_margin(net5):
    # measured 0.015 px with weights and activations rounded (0.019 px at 1080p)
    assert _epe(net5, "fp16", True, True) < 0.03
    # each rounding alone is below the combined one's bar too
    assert _epe(net5, "fp16", True, False) < 0.03 and _epe(net5, "fp16", False, True) < 0.03
