"""The read-bandwidth probe (ft_read_probe) reads every word of its buffer.

It is the measured denominator of the text Flowtree's L2 roofline in
bench.py; the check is that each pass loads every 32-bit word exactly once
(the XOR folded into the sink), including a ragged tail, and that invalid
sizes are rejected before any launch.
"""
import numpy as np
import pytest
import torch

from paper_1910_04126_gb300 import api
from paper_1910_04126_gb300._ffi import FlowtreeError

pytestmark = pytest.mark.gpu


def test_read_probe_reads_every_word_once_per_pass():
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    x = torch.randint(0, 2 ** 31 - 1, ((1 << 20) + 12,), dtype=torch.int32, device="cuda", generator=g)
    want = np.bitwise_xor.reduce(x.cpu().numpy().view(np.uint32))
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    api.read_probe(x, 1, sink)
    assert sink.cpu().numpy().view(np.uint32)[0] == want
    api.read_probe(x, 2, sink)  # two more passes leave the fold unchanged
    assert sink.cpu().numpy().view(np.uint32)[0] == want
    api.read_probe(x, 3, sink)  # three more flip it back to zero
    assert sink.cpu().numpy().view(np.uint32)[0] == 0


def test_read_probe_rejects_bad_sizes():
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(FlowtreeError):
        api.read_probe(x[:3], 1, sink)  # 12 bytes
    with pytest.raises(FlowtreeError):
        api.read_probe(x[:5], 1, sink)  # 20 bytes: not a multiple of 16
    with pytest.raises(FlowtreeError):
        api.read_probe(x, 0, sink)
