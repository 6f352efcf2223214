"""Host-side logic of the learned warm start (no GPU): the output-scale fold
that turns a network trained on a multiple of the dual a back into one that
predicts a."""
import numpy as np

from paper_1909_00149_gb300 import unet_layer_specs
from paper_1909_00149_gb300 import warmstart as WS


class _FakeNet:
    def __init__(self, base):
        self.base = base
        n = sum(co * ci * k * k + co for _, ci, co, k in unet_layer_specs(base))
        self.p = np.arange(n, dtype=np.float32) + 1.0

    def get_params(self):
        return self.p.copy()

    def set_params(self, flat):
        self.p = np.asarray(flat, np.float32).copy()


def test_fold_scales_exactly_the_head_channel():
    """The head is the last layer, a 1x1 convolution C -> 4 with weights
    [4, C] and biases [4]: folding channel c touches its C weights and its
    bias and nothing else."""
    for base in (8, 32):
        net = _FakeNet(base)
        before = net.get_params()
        WS.fold_output_scale(net, WS.STATE_CHANNELS.index("a"), 0.25)
        after = net.get_params()
        changed = np.flatnonzero(after != before)
        head = before.size - (4 * base + 4)
        c = WS.STATE_CHANNELS.index("a")
        expect = np.concatenate([np.arange(head + c * base, head + (c + 1) * base), [head + 4 * base + c]])
        assert np.array_equal(changed, expect)
        assert np.array_equal(after[changed], before[changed] * np.float32(0.25))
